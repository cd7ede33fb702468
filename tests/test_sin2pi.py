"""Error bound of the float32 sin(2 pi f) polynomial used by the CUDA weights
(Taylor series through x^11 after exact folding), checked by emulating its
float32 Horner evaluation with fused multiply-adds in float64-rounded-to-float32
steps against float64 sin."""
import math

import numpy as np

COEF = [6.283185307179586, -41.341702240399755, 81.60524927607504, -76.70585975306136,
        42.058693944897634, -15.094642576822984]


def test_coefficients_are_the_taylor_series_of_sin_2pi_t():
    for k, c in enumerate(COEF):
        want = (-1) ** k * (2 * math.pi) ** (2 * k + 1) / math.factorial(2 * k + 1)
        assert abs(c - want) <= 1e-15 * abs(want)


def test_float32_evaluation_error_bound():
    f = np.linspace(0.0, 1.0, 400001, endpoint=False).astype(np.float32)
    t = f - np.rint(f)
    h = np.copysign(np.float32(0.5), t) - t
    t = np.where(np.abs(t) > 0.25, h, t).astype(np.float32)
    t2 = (t * t).astype(np.float32)
    p = np.float32(COEF[5])
    for c in COEF[4::-1]:
        p = (p.astype(np.float64) * t2 + np.float32(c)).astype(np.float32)  # one rounding per fma
    s = (t * p).astype(np.float32)
    err = np.abs(s.astype(np.float64) - np.sin(2 * np.pi * f.astype(np.float64)))
    assert err.max() < 2.5e-7


def _cos_coefficients_from_source():
    """The cos_2pi Horner constants as written in the CUDA source (highest
    degree first)."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2412_10399_gb300", "csrc",
                            "transfer.cu")).read()
    body = src[src.index("float cos_2pi(float f)"):]
    body = body[:body.index("return")]
    return [float(c) for c in re.findall(r"(-?\d+\.\d+)f", body) if abs(float(c)) not in (0.5, 0.25)]


def test_cos_coefficients_are_the_taylor_series_of_cos_2pi_t():
    coef = _cos_coefficients_from_source()[::-1]  # ascending degree in t^2
    assert len(coef) == 7
    for k, c in enumerate(coef):
        want = (-1) ** k * (2 * math.pi) ** (2 * k) / math.factorial(2 * k)
        assert abs(c - want) <= 1e-15 * abs(want)


def test_cos_float32_evaluation_error_bound():
    coef = [np.float32(c) for c in _cos_coefficients_from_source()]
    f = np.linspace(0.0, 1.0, 400001, endpoint=False).astype(np.float32)
    t = f - np.rint(f)
    h = np.copysign(np.float32(0.5), t) - t
    fold = np.abs(t) > 0.25
    t = np.where(fold, h, t).astype(np.float32)
    t2 = (t * t).astype(np.float32)
    p = np.full_like(t2, coef[0])
    for c in coef[1:]:
        p = (p.astype(np.float64) * t2 + c).astype(np.float32)  # one rounding per fma
    c = np.where(fold, -p, p)
    err = np.abs(c.astype(np.float64) - np.cos(2 * np.pi * f.astype(np.float64)))
    assert err.max() < 2.5e-7
