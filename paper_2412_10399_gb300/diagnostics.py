"""Conserved quantities of a particle state, for monitoring runs (host side,
from read-back fields, float64): total mass, linear momentum, angular momentum
including APIC's particle spin (the Supplement's eq. 3:
sum x_p x m_p v_p + sum m_p eps : B_p) and kinetic energy.  Without gravity or
walls the CK-MPM step conserves the first three exactly (Supplement Thm 1.1,
2.1, 2.2), so their drift over a run measures rounding."""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import numpy as np


def conserved(x: np.ndarray, v: np.ndarray, mat: np.ndarray, materials: Sequence, dx: float, ppc: int,
              B: Optional[np.ndarray] = None) -> Dict[str, object]:
    """x, v (n, 3); mat (n,) indices into materials (objects with .rho); B
    (n, 3, 3) or None (no particle spin, e.g. under the PIC transfer)."""
    x = np.asarray(x, np.float64)
    v = np.asarray(v, np.float64)
    rho = np.array([m.rho for m in materials], np.float64)[np.asarray(mat, np.int64)]
    m = rho * (dx ** 3 / ppc)
    mv = m[:, None] * v
    L = np.cross(x, mv).sum(0)
    if B is not None:
        B = np.asarray(B, np.float64)
        spin = np.stack([B[:, 2, 1] - B[:, 1, 2], B[:, 0, 2] - B[:, 2, 0], B[:, 1, 0] - B[:, 0, 1]], -1)
        L = L + (m[:, None] * spin).sum(0)
    return {"mass": float(m.sum()), "momentum": mv.sum(0), "angular_momentum": L,
            "kinetic_energy": float(0.5 * (m * (v * v).sum(1)).sum())}
