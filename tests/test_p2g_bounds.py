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
