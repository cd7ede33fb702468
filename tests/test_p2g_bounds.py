"""Pins of the bounds behind the P2G fixed-point scale.

The CUDA P2G accumulates in 32-bit fixed point with a scale derived from a
bound on every contribution w (m v + A d) a particle can make: the largest
node weight, the largest weight times node offset, and the largest row
abs-sum of D^-1 (Sec. 4.4) of each stencil.  Those three numbers are
constants in the kernel source.  Here they are read from the source as text
and checked against the FP64 oracle's stencils over a dense lattice of
particle positions: each constant must cover the oracle's maximum (else a
node sum could overflow) and stay within a few percent of it (else precision
is thrown away).
"""
import os
import re

import pytest
import torch

from oracle import ckmpm_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
F64 = torch.float64


def _constants():
    src = open(os.path.join(ROOT, "paper_2412_10399_gb300", "csrc", "transfer.cu")).read()
    out = {}
    for kind in (0, 1):
        m = re.search(r"struct P2GBound<%d> \{(.*?)\};" % kind, src, re.S)
        assert m, f"P2GBound<{kind}> not found"
        out[kind] = {k: float(v) for k, v in re.findall(r"(\w+) = ([0-9.]+)f;", m.group(1))}
    return out


def _oracle_maxima(kernel):
    """Largest weight, largest |w d_a| (d in cells) and largest row abs-sum of
    D^-1 (cells^-2) over particles at fractions i/40 of a cell per axis."""
    dx = 1.0 / 64
    f = torch.arange(40, dtype=F64) / 40.0
    fx, fy, fz = torch.meshgrid(f, f, f, indexing="ij")
    x = (10.0 + torch.stack([fx, fy, fz], -1).reshape(-1, 3)) * dx
    wmax = wd = 0.0
    for k in O.grid_ids(kernel):
        _, w, d = O.stencil(x, dx, kernel, k)
        wmax = max(wmax, float(w.max()))
        wd = max(wd, float((w[..., None] * (d / dx).abs()).max()))
    prm = O.Params(res=64, dx=dx, dt=1e-4, materials=[], kernel=kernel)
    Dinv = torch.linalg.inv(O.apic_D(x, prm)) * dx * dx
    dinv = float(Dinv.abs().sum(-1).max())
    return {"wmax": wmax, "wd": wd, "dinv": dinv}


@pytest.mark.parametrize("kernel", [O.KERNEL_CK, O.KERNEL_QUADRATIC])
def test_p2g_bound_constants_cover_oracle_maxima(kernel):
    const = _constants()[0 if kernel == O.KERNEL_CK else 1]
    found = _oracle_maxima(kernel)
    for name in ("wmax", "wd", "dinv"):
        assert const[name] >= found[name] * (1.0 - 1e-9), (name, const[name], found[name])
        assert const[name] <= found[name] * 1.04, (name, const[name], found[name])
    # the two terms of the bound keep at least 0.2% for float rounding
    assert const["wmax"] >= found["wmax"] * 1.002
    assert const["wd"] * const["dinv"] >= found["wd"] * found["dinv"] * 1.002


def test_oracle_maxima_match_closed_forms():
    """The quadratic maxima have closed forms: w <= (3/4)^3, |w d| <= 1/4 *
    (3/4)^2 (at |d| = 1/2 on one axis, 0 on the others), D^-1 = 4 I.  CK: w
    <= K1(0) = 1 and max_t t K1(t) = 0.27751 at t = 0.394."""
    q = _oracle_maxima(O.KERNEL_QUADRATIC)
    assert q["wmax"] == pytest.approx(0.421875, rel=1e-12)
    assert q["wd"] == pytest.approx(0.140625, rel=1e-12)
    assert q["dinv"] == pytest.approx(4.0, rel=1e-9)
    c = _oracle_maxima(O.KERNEL_CK)
    assert c["wmax"] == pytest.approx(1.0, rel=1e-12)
    t = torch.linspace(0.0, 1.0, 200001, dtype=F64)
    assert float((t * O.K1(t)).max()) == pytest.approx(0.27751, abs=1e-5)
    assert c["wd"] <= 0.27751 + 1e-5 and c["wd"] >= 0.2765
    assert 13.9 <= c["dinv"] <= 14.05


def _fixed_constants():
    src = open(os.path.join(ROOT, "paper_2412_10399_gb300", "csrc", "transfer.cu")).read()
    count = int(re.search(r"constexpr uint32_t kP2GFmaCount = (\d+);", src).group(1))
    m = re.search(r"fmaf\(w, val, ([0-9.]+)f\)\) - (0x[0-9A-Fa-f]+);", src)
    assert m, "the fused-multiply-add rounding of p2g_fixed was not found"
    return count, float(m.group(1)), int(m.group(2), 16)


def test_fma_rounding_is_round_to_nearest_within_its_range():
    """p2g_fixed<true> rounds w * val by one float32 fused multiply-add with
    1.5 * 2^23 and subtracts that constant's bits.  The FMA rounds the exact
    value 1.5 * 2^23 + w val once; while |w val| <= 2^22 that value lies in
    [2^23, 2^24], where the float32 numbers are exactly the integers, so the
    result is w val rounded to the nearest integer (ties to even) plus
    1.5 * 2^23, and its bits minus the constant's are that integer.  Checked
    here with exact rational arithmetic on random float32 pairs and on ties
    and the ends of the range."""
    from fractions import Fraction

    import numpy as np
    count, magic, bits = _fixed_constants()
    assert magic == 1.5 * 2.0 ** 23
    assert bits == int(np.float32(magic).view(np.uint32))
    # the scale maps count x bound to 2^30, so a block of `count` particles
    # or more keeps every contribution within 2^22
    assert 2.0 ** 30 / count <= 2.0 ** 22
    rng = np.random.default_rng(0)
    n = 20_000
    w = rng.uniform(0.0, 1.003, n).astype(np.float32)
    mag = 2.0 ** rng.uniform(-30.0, 22.0, n)
    val = (np.where(rng.random(n) < 0.5, -1.0, 1.0) * mag).astype(np.float32)
    pairs = [(float(a), float(b)) for a, b in zip(w, val)]
    pairs += [(1.0, 2.0 ** 22), (1.0, -2.0 ** 22), (1.0, 0.5), (1.0, 1.5), (1.0, -2.5), (1.0, 0.0), (0.5, 3.0),
              (1.0, 2.0 ** 22 - 0.5), (1.0, -(2.0 ** 22 - 0.5))]
    two23, two24 = Fraction(2) ** 23, Fraction(2) ** 24
    checked = 0
    for a, b in pairs:
        prod = Fraction(a) * Fraction(b)
        if abs(prod) > Fraction(2) ** 22:
            continue
        exact = Fraction(magic) + prod
        assert two23 <= exact <= two24
        fma = round(exact)  # float32 rounding in [2^23, 2^24]: to the nearest integer, ties to even
        assert fma == Fraction(int(np.float32(fma)))  # an integer there is a float32
        got = int(np.float32(fma).view(np.int32)) - bits
        assert got == round(prod), (a, b)
        checked += 1
    assert checked > n // 2
