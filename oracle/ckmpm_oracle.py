"""FP64 CPU oracle for one compact-kernel MPM (CK-MPM) time step.

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA path; the
product never calls it.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import it.  It shares no code with the CUDA
path: every quantity is computed here from the paper's definitions, in float64,
with plain PyTorch CPU tensor operations (scatter-add via ``index_add_``, 3x3
inverse, LAPACK SVD) and no blocking, fusion or closed-form shortcuts.

Paper: "CK-MPM: A Compact-Kernel Material Point Method" (arXiv 2412.10399).
Passages followed (section / equation names of the paper):
  * Sec. 4.1 final kernel equation  K1(x) = 1 - |x| + sin(2 pi |x|) / (2 pi)
  * Sec. 4.2 tensor-product kernel, dual grid G-/G+ and its coordinate map
  * Sec. 4.3.1 transfer to grid, Sec. 4.3.2 force, Sec. 4.3.3 grid update,
    Sec. 4.3.4 transfer to particles, Sec. 4.3.5 deformation-gradient update
  * Sec. 4.4 APIC on the dual grid (D_p, B_p, momentum transfer)
  * Sec. 4.5 MLS shape functions (linear basis => grad w = w D^-1 (x_i - x_p))
  * Sec. 3.2 pipeline order (P2G, grid update, G2P, F update + return mapping,
    advection) and Eq. traditional-grid-update (force sign, V_p0)
  * Supplement Thm 1.1, 2.1, 2.2 (what the tests check it against).

Readings where the paper is silent or garbled (each one is a named choice):
  R1 node i of grid k sits at (i - k/4) dx, k in {-1, +1}  (G- at +dx/4,
     G+ at -dx/4 relative to the conceptual grid G0).
  R4 force f_ik = - sum_p V0 tau_p grad w_ipk with tau = P F^T (Kirchhoff)
     and grad w the MLS gradient w D^-1 (x_i - x_p).
  R5 G2P velocity v_p = 1/2 sum_k sum_i w v~_i (no m_i / m_p factor).
  R6 the state stores B; P2G forms B D(x^n)^-1 with D at the P2G position;
     the F update uses grad v = B' D(x^n)^-1 with the gather position.
  R7 F^{n+1} = (I + dt grad v) F^n.
  R8 gravity added on nodes with m > 0; nodes with m = 0 get v~ = 0; sticky
     walls: v~ = 0 where any coordinate of the node lies below bc*dx or above
     L - bc*dx.
  R9 fixed-corotated psi = mu |F-R|^2 + lam/2 (J-1)^2; Drucker-Prager with
     Hencky elasticity and the klar2016 return mapping (cohesion 0, no
     hardening), alpha = sqrt(2/3) * 2 sin(phi) / (3 - sin(phi)).
  R10 step order: tau(F^n) -> P2G -> grid update -> G2P -> F -> return map
     -> x^{n+1}.
  R15 J-based fluid (the dam-break scenes of the performance section, an
     equation of state after monaghan1994 / tampubolon2017, both only cited):
     pressure p = B (J^-gamma - 1), Kirchhoff stress tau = -J p I, and the
     particle keeps only its volume ratio, F <- J^(1/3) I after each F update
     (the shear part of F carries no stress in a fluid).  The paper lists a
     viscosity 0.1 without its discretisation; it is not modelled.
  R16 PIC transfer (Sec. 4.3 as written, the scheme of the paper's Taichi
     comparison): P2G carries m v only, the force is f_i = -sum_p V0 tau_p
     grad w_ip (R4's sign) with the gradient of the kernel itself,
     grad w_ip = d w_ip / d x_p; G2P gives v_p (R5) and grad v_p = 1/2
     sum_k sum_i v~_i (grad w_ip)^T for the F update; B stays 0.
  R17 APIC with the kernel gradient (Sec. 4.4 taken literally: its momentum
     transfer and B update, "the rest as in the PIC scheme"): P2G carries
     w m (v + B D^-1 (x_i - x_p)) and the force of R16; G2P gives v and B as
     for APIC and the R16 grad v for the F update.
  Quadratic comparison path: hu2018 MLS-MPM on one grid with the quadratic
  B-spline, D = dx^2/4 I.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import torch

F64 = torch.float64
TWO_PI = 2.0 * math.pi

FIXED_COROTATED = 0
DRUCKER_PRAGER = 1
J_FLUID = 2
KERNEL_CK = 0
KERNEL_QUADRATIC = 1
TRANSFER_APIC_MLS = 0   # APIC momentum with the MLS force (Sec. 4.4, 4.5): the default
TRANSFER_PIC = 1        # the PIC scheme of Sec. 4.3 with the kernel gradient
TRANSFER_APIC_GRAD = 2  # APIC momentum (Sec. 4.4) with the kernel-gradient force and grad v of Sec. 4.3


# -----------------------------------------------------------------------------
# kernels (Sec. 4.1, Sec. 4.2; quadratic B-spline for the comparison path)
# -----------------------------------------------------------------------------

def K1(x: torch.Tensor) -> torch.Tensor:
    """Sec. 4.1 final 1-D kernel: 1 - |x| + sin(2 pi |x|)/(2 pi) on |x| < 1."""
    ax = x.abs()
    val = 1.0 - ax + torch.sin(TWO_PI * ax) / TWO_PI
    return torch.where(ax < 1.0, val, torch.zeros_like(val))


def K1_prime(x: torch.Tensor) -> torch.Tensor:
    """d K1 / dx = sgn(x) (cos(2 pi |x|) - 1) on |x| < 1; K1 is C^2, so K1' is 0 at 0 and at |x| = 1."""
    ax = x.abs()
    val = torch.sign(x) * (torch.cos(TWO_PI * ax) - 1.0)
    return torch.where(ax < 1.0, val, torch.zeros_like(val))


def quadratic_bspline_prime(x: torch.Tensor) -> torch.Tensor:
    """d N / dx of the quadratic B-spline: -2x on |x| < 1/2, (|x| - 3/2) sgn(x) on |x| < 3/2."""
    ax = x.abs()
    inner = -2.0 * x
    outer = (ax - 1.5) * torch.sign(x)
    return torch.where(ax < 0.5, inner, torch.where(ax < 1.5, outer, torch.zeros_like(ax)))


def quadratic_bspline(x: torch.Tensor) -> torch.Tensor:
    """Quadratic B-spline N(x): 3/4 - x^2 on |x|<1/2, (3/2-|x|)^2/2 on |x|<3/2."""
    ax = x.abs()
    inner = 0.75 - ax * ax
    outer = 0.5 * (1.5 - ax) ** 2
    return torch.where(ax < 0.5, inner, torch.where(ax < 1.5, outer, torch.zeros_like(ax)))


def grid_ids(kernel: int) -> List[int]:
    """Grid labels k: {-1, +1} for the dual grid, {0} for the quadratic grid."""
    return [-1, 1] if kernel == KERNEL_CK else [0]


def node_position(idx: torch.Tensor, k: int, dx: float) -> torch.Tensor:
    """Reading R1: node idx of grid k is at (idx - k/4) dx (Sec. 4.2 map)."""
    return (idx.to(F64) - 0.25 * k) * dx


def stencil(x: torch.Tensor, dx: float, kernel: int, k: int):
    """Nodes touched by each particle on grid k.

    Returns (idx (N,S,3) int64, w (N,S) float64, d (N,S,3) float64) with
    d = x_i - x_p and w the tensor-product kernel of Sec. 4.2 evaluated from
    the node and particle positions (no shared 1-D factors)."""
    if kernel == KERNEL_CK:
        base = torch.floor(x / dx + 0.25 * k).to(torch.int64)
        rng = [0, 1]
        kern = K1
    else:
        base = torch.floor(x / dx - 0.5).to(torch.int64)
        rng = [0, 1, 2]
        kern = quadratic_bspline
    offs = torch.tensor([[a, b, c] for c in rng for b in rng for a in rng], dtype=torch.int64)
    idx = base[:, None, :] + offs[None, :, :]
    xi = node_position(idx, k, dx)
    d = xi - x[:, None, :]
    w = torch.prod(kern(d / dx), dim=-1)
    return idx, w, d


# -----------------------------------------------------------------------------
# parameters and state
# -----------------------------------------------------------------------------

@dataclasses.dataclass
class Mat:
    model: int
    E: float            # Young's modulus; for the fluid, the equation-of-state constant B
    nu: float
    rho: float
    friction_deg: float = 0.0
    gamma: float = 7.15  # fluid equation-of-state exponent


@dataclasses.dataclass
class Params:
    res: int
    dx: float
    dt: float
    materials: List[Mat]
    gravity: Tuple[float, float, float] = (0.0, -9.8, 0.0)
    bc_cells: float = 3.0
    ppc: int = 8
    kernel: int = KERNEL_CK
    transfer: int = TRANSFER_APIC_MLS

    @property
    def V0(self) -> float:
        return self.dx ** 3 / self.ppc

    @property
    def n_nodes(self) -> int:
        """Nodes per axis on every grid: indices 0..res."""
        return self.res + 1


@dataclasses.dataclass
class State:
    x: torch.Tensor        # (N,3)
    v: torch.Tensor        # (N,3)
    B: torch.Tensor        # (N,3,3) APIC affine matrix (Sec. 4.4)
    F: torch.Tensor        # (N,3,3) (elastic) deformation gradient
    mat: torch.Tensor      # (N,) int64 material index
    E: Optional[torch.Tensor] = None  # (N,) per-particle Young's modulus override

    def clone(self) -> "State":
        return State(self.x.clone(), self.v.clone(), self.B.clone(), self.F.clone(),
                     self.mat.clone(), None if self.E is None else self.E.clone())


def make_state(x, v, B=None, F=None, mat=None, E=None) -> State:
    x = torch.as_tensor(x, dtype=F64)
    n = x.shape[0]
    v = torch.as_tensor(v, dtype=F64)
    B = torch.zeros(n, 3, 3, dtype=F64) if B is None else torch.as_tensor(B, dtype=F64).reshape(n, 3, 3)
    F = torch.eye(3, dtype=F64).expand(n, 3, 3).clone() if F is None else torch.as_tensor(F, dtype=F64).reshape(n, 3, 3)
    mat = torch.zeros(n, dtype=torch.int64) if mat is None else torch.as_tensor(mat).to(torch.int64)
    E = None if E is None else torch.as_tensor(E, dtype=F64)
    return State(x, v, B, F, mat, E)


def lame(E, nu):
    """Lame parameters from Young's modulus and Poisson's ratio."""
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def particle_lame(st: State, prm: Params):
    n = st.x.shape[0]
    E = torch.tensor([m.E for m in prm.materials], dtype=F64)[st.mat]
    if st.E is not None:
        E = st.E
    nu = torch.tensor([m.nu for m in prm.materials], dtype=F64)[st.mat]
    return lame(E, nu)


def particle_mass(st: State, prm: Params) -> torch.Tensor:
    rho = torch.tensor([m.rho for m in prm.materials], dtype=F64)[st.mat]
    return rho * prm.V0


# -----------------------------------------------------------------------------
# 3x3 decompositions (library routines: LAPACK SVD; Newton polar for autograd)
# -----------------------------------------------------------------------------

def svd_rv(F: torch.Tensor):
    """Rotation-variant SVD F = U diag(s) V^T with det U = det V = +1; the sign
    of a reflection is carried by the smallest singular value."""
    U, s, Vh = torch.linalg.svd(F)
    V = Vh.transpose(-1, -2)
    s = s.clone()
    U = U.clone()
    V = V.clone()
    du = torch.det(U) < 0
    dv = torch.det(V) < 0
    U[du, :, 2] = -U[du, :, 2]
    s[du, 2] = -s[du, 2]
    V[dv, :, 2] = -V[dv, :, 2]
    s[dv, 2] = -s[dv, 2]
    return U, s, V


def polar_rotation(F: torch.Tensor, newton: bool = False, iters: int = 14) -> torch.Tensor:
    """Rotation R of the polar decomposition F = R S.

    Default: R = U V^T from the rotation-variant SVD.  With newton=True the
    Higham (1986) iteration X <- (X + X^-T)/2 from X0 = F is used instead; it
    has the same fixed point for det F > 0 and is differentiable by autograd
    when singular values coincide (e.g. F = I)."""
    if not newton:
        U, _, V = svd_rv(F)
        return U @ V.transpose(-1, -2)
    X = F
    for _ in range(iters):
        X = 0.5 * (X + torch.linalg.inv(X).transpose(-1, -2))
    return X


# -----------------------------------------------------------------------------
# constitutive models (reading R9)
# -----------------------------------------------------------------------------

def fc_energy(F, mu, lam, newton=False):
    """Fixed-corotated energy density psi(F) = mu |F - R|^2 + lam/2 (J - 1)^2."""
    R = polar_rotation(F, newton)
    J = torch.det(F)
    return mu * ((F - R) ** 2).sum(dim=(-1, -2)) + 0.5 * lam * (J - 1.0) ** 2


def fc_piola(F, mu, lam, newton=False):
    """First Piola-Kirchhoff stress P = 2 mu (F - R) + lam (J - 1) J F^-T."""
    R = polar_rotation(F, newton)
    J = torch.det(F)
    FinvT = torch.linalg.inv(F).transpose(-1, -2)
    return 2.0 * mu[..., None, None] * (F - R) + (lam * (J - 1.0) * J)[..., None, None] * FinvT


def fc_kirchhoff(F, mu, lam, newton=False):
    """Kirchhoff stress tau = P F^T = 2 mu (F - R) F^T + lam J (J - 1) I."""
    R = polar_rotation(F, newton)
    J = torch.det(F)
    I = torch.eye(3, dtype=F.dtype).expand_as(F)
    return (2.0 * mu[..., None, None] * (F - R) @ F.transpose(-1, -2)
            + (lam * J * (J - 1.0))[..., None, None] * I)


SIGMA_FLOOR = 1e-6


def hencky_kirchhoff(F, mu, lam):
    """Hencky (StVK on log strain) Kirchhoff stress U (2 mu eps + lam tr eps I) U^T."""
    U, s, _ = svd_rv(F)
    eps = torch.log(torch.clamp(s, min=SIGMA_FLOOR))
    tr = eps.sum(-1, keepdim=True)
    d = 2.0 * mu[..., None] * eps + lam[..., None] * tr
    return U @ torch.diag_embed(d) @ U.transpose(-1, -2)


def dp_alpha(friction_deg):
    s = math.sin(math.radians(friction_deg))
    return math.sqrt(2.0 / 3.0) * 2.0 * s / (3.0 - s)


def dp_return_map(F, mu, lam, alpha):
    """klar2016 Drucker-Prager projection of the log principal strains.

    eps = ln sigma; tension (tr eps >= 0) maps to the cone tip (sigma = 1);
    otherwise dgamma = |eps_hat| + (3 lam + 2 mu)/(2 mu) tr(eps) alpha, and
    the deviatoric part shrinks by dgamma when it is positive.  dgamma <= 0
    means the state lies inside the cone and is left unchanged: a purely
    volumetric compression (eps_hat = 0, tr eps < 0) is such a state.
    dgamma > 0 with tr eps < 0 implies |eps_hat| > 0, so the division by
    |eps_hat| only happens where it is defined."""
    U, s, V = svd_rv(F)
    eps = torch.log(torch.clamp(s, min=SIGMA_FLOOR))
    tr = eps.sum(-1, keepdim=True)
    eps_hat = eps - tr / 3.0
    nrm = torch.linalg.vector_norm(eps_hat, dim=-1, keepdim=True)
    dgamma = nrm + (3.0 * lam[..., None] + 2.0 * mu[..., None]) / (2.0 * mu[..., None]) * tr * alpha
    tip = tr >= 0.0
    safe = torch.where(nrm > 0.0, nrm, torch.ones_like(nrm))
    proj = eps - dgamma * eps_hat / safe
    new_eps = torch.where(tip, torch.zeros_like(eps), torch.where(dgamma > 0.0, proj, eps))
    s_new = torch.exp(new_eps)
    unchanged = (~tip) & (dgamma <= 0.0)
    Fn = U @ torch.diag_embed(s_new) @ V.transpose(-1, -2)
    return torch.where(unchanged[..., None], F, Fn)


def fluid_pressure(J, Bk, gamma):
    """Reading R15: equation of state p = B (J^-gamma - 1)."""
    return Bk * (J ** (-gamma) - 1.0)


def fluid_kirchhoff(F, Bk, gamma):
    """Reading R15: tau = J sigma = -J p I for the J-based fluid, J = det F."""
    J = torch.det(F)
    I = torch.eye(3, dtype=F.dtype).expand_as(F)
    return (-J * fluid_pressure(J, Bk, gamma))[..., None, None] * I


def fluid_energy(J, Bk, gamma):
    """Stored energy per reference volume whose Kirchhoff stress is R15's:
    tau = J psi'(J) I with psi'(J) = -p(J), psi(1) = 0."""
    return -Bk * ((J ** (1.0 - gamma) - 1.0) / (1.0 - gamma) - (J - 1.0))


def kirchhoff_stress(st: State, prm: Params, newton=False) -> torch.Tensor:
    mu, lam = particle_lame(st, prm)
    models = torch.tensor([m.model for m in prm.materials])[st.mat]
    tau = torch.zeros_like(st.F)
    fc = models == FIXED_COROTATED
    if fc.any():
        tau_fc = fc_kirchhoff(st.F, mu, lam, newton)
        tau = torch.where(fc[:, None, None], tau_fc, tau)
    dp = models == DRUCKER_PRAGER
    if dp.any():
        tau_dp = hencky_kirchhoff(st.F, mu, lam)
        tau = torch.where(dp[:, None, None], tau_dp, tau)
    fl = models == J_FLUID
    if fl.any():
        Bk = torch.tensor([m.E for m in prm.materials], dtype=F64)[st.mat]
        gam = torch.tensor([m.gamma for m in prm.materials], dtype=F64)[st.mat]
        tau = torch.where(fl[:, None, None], fluid_kirchhoff(st.F, Bk, gam), tau)
    return tau


def plasticity(F: torch.Tensor, st: State, prm: Params) -> torch.Tensor:
    """Return mapping (Sec. 3.2 step 4) for plastic materials, the volumetric
    projection F <- J^(1/3) I for the fluid (reading R15); identity otherwise."""
    models = torch.tensor([m.model for m in prm.materials])[st.mat]
    fl = models == J_FLUID
    if fl.any():
        J = torch.det(F)
        c = torch.sign(J) * torch.abs(J) ** (1.0 / 3.0)
        F = torch.where(fl[:, None, None], c[:, None, None] * torch.eye(3, dtype=F64), F)
    dp = models == DRUCKER_PRAGER
    if not dp.any():
        return F
    mu, lam = particle_lame(st, prm)
    alpha = torch.tensor([dp_alpha(m.friction_deg) for m in prm.materials], dtype=F64)[st.mat]
    Fr = dp_return_map(F, mu, lam, alpha[:, None])
    return torch.where(dp[:, None, None], Fr, F)


# -----------------------------------------------------------------------------
# transfers
# -----------------------------------------------------------------------------

def stencil_grad(x: torch.Tensor, dx: float, kernel: int, k: int):
    """Kernel gradient grad w_ip = d w_ip / d x_p for the stencil of `stencil`
    (same node order), shape (N,S,3): with w = prod_a K((x_i - x_p)_a / dx),
    d w / d x_p,a = -K'((x_i - x_p)_a / dx) / dx * prod_{b != a} K((x_i - x_p)_b / dx)."""
    idx, w, d = stencil(x, dx, kernel, k)
    kern, kprime = (K1, K1_prime) if kernel == KERNEL_CK else (quadratic_bspline, quadratic_bspline_prime)
    t = d / dx
    kv = kern(t)
    kp = kprime(t)
    g = torch.stack([-kp[..., 0] * kv[..., 1] * kv[..., 2], -kv[..., 0] * kp[..., 1] * kv[..., 2],
                     -kv[..., 0] * kv[..., 1] * kp[..., 2]], -1) / dx
    return idx, w, d, g


def _check_domain(x: torch.Tensor, prm: Params):
    u = x / prm.dx
    if bool((u < 0.5).any()) or bool((u >= prm.res - 0.5).any()):
        raise ValueError("particle outside the valid interior [0.5 dx, (res-0.5) dx)")


def apic_D(x: torch.Tensor, prm: Params) -> torch.Tensor:
    """Sec. 4.4: D_p = 1/2 sum_k sum_i w (x_i - x_p)(x_i - x_p)^T (one grid and
    no 1/2 for the quadratic path), by explicit summation."""
    ks = grid_ids(prm.kernel)
    D = torch.zeros(x.shape[0], 3, 3, dtype=F64)
    for k in ks:
        _, w, d = stencil(x, prm.dx, prm.kernel, k)
        D = D + torch.einsum("ns,nsa,nsb->nab", w, d, d)
    return D / len(ks)


def _lin(idx: torch.Tensor, n: int) -> torch.Tensor:
    return (idx[..., 2] * n + idx[..., 1]) * n + idx[..., 0]


def p2g(st: State, prm: Params, newton=False, stress=True) -> Dict[int, Tuple[torch.Tensor, torch.Tensor]]:
    """Transfer to grid with APIC momentum and MLS force (Sec. 4.3.1-4.3.2,
    Sec. 4.4, Sec. 4.5, readings R4/R6).

    Returns {k: (m (n^3,), p (n^3,3))} where p already contains dt * f, i.e.
    m_i v_i + dt f_i, on the node range 0..res of each grid."""
    _check_domain(st.x, prm)
    n = prm.n_nodes
    mp = particle_mass(st, prm)
    if prm.transfer in (TRANSFER_PIC, TRANSFER_APIC_GRAD):
        return _p2g_pic(st, prm, mp, newton, stress)
    D = apic_D(st.x, prm)
    Dinv = torch.linalg.inv(D)
    tau = kirchhoff_stress(st, prm, newton) if stress else torch.zeros_like(st.F)
    A = (mp[:, None, None] * st.B - prm.dt * prm.V0 * tau) @ Dinv
    out = {}
    for k in grid_ids(prm.kernel):
        idx, w, d = stencil(st.x, prm.dx, prm.kernel, k)
        lin = _lin(idx, n).reshape(-1)
        m_contrib = (w * mp[:, None]).reshape(-1)
        p_contrib = w[..., None] * (mp[:, None, None] * st.v[:, None, :]
                                    + torch.einsum("nab,nsb->nsa", A, d))
        m = torch.zeros(n ** 3, dtype=F64).index_add(0, lin, m_contrib)
        p = torch.zeros(n ** 3, 3, dtype=F64).index_add(0, lin, p_contrib.reshape(-1, 3))
        out[k] = (m, p)
    return out


def _p2g_pic(st: State, prm: Params, mp, newton, stress):
    """Reading R16: m_i = sum w m_p, m_i v_i + dt f_i = sum w m_p v_p - dt sum V0 tau grad w;
    reading R17 adds the APIC term w m_p B D^-1 (x_i - x_p) to the momentum."""
    n = prm.n_nodes
    tau = kirchhoff_stress(st, prm, newton) if stress else torch.zeros_like(st.F)
    if prm.transfer == TRANSFER_APIC_GRAD:
        A = (mp[:, None, None] * st.B) @ torch.linalg.inv(apic_D(st.x, prm))
    out = {}
    for k in grid_ids(prm.kernel):
        idx, w, d, g = stencil_grad(st.x, prm.dx, prm.kernel, k)
        lin = _lin(idx, n).reshape(-1)
        m_contrib = (w * mp[:, None]).reshape(-1)
        p_contrib = (w[..., None] * mp[:, None, None] * st.v[:, None, :]
                     - prm.dt * prm.V0 * torch.einsum("nab,nsb->nsa", tau, g))
        if prm.transfer == TRANSFER_APIC_GRAD:
            p_contrib = p_contrib + w[..., None] * torch.einsum("nab,nsb->nsa", A, d)
        m = torch.zeros(n ** 3, dtype=F64).index_add(0, lin, m_contrib)
        p = torch.zeros(n ** 3, 3, dtype=F64).index_add(0, lin, p_contrib.reshape(-1, 3))
        out[k] = (m, p)
    return out


def grid_update(grids, prm: Params, gravity=None, bc=True):
    """Sec. 4.3.3 per grid, plus gravity and sticky walls (reading R8).
    Returns {k: v~ (n^3,3)}."""
    n = prm.n_nodes
    g = torch.tensor(prm.gravity if gravity is None else gravity, dtype=F64)
    ar = torch.arange(n, dtype=torch.int64)
    iz, iy, ix = torch.meshgrid(ar, ar, ar, indexing="ij")
    idx = torch.stack([ix, iy, iz], -1).reshape(-1, 3)
    L = prm.res * prm.dx
    out = {}
    for k, (m, p) in grids.items():
        has = m > 0
        safe = torch.where(has, m, torch.ones_like(m))
        v = torch.where(has[:, None], p / safe[:, None] + prm.dt * g, torch.zeros_like(p))
        if bc:
            xi = node_position(idx, k, prm.dx)
            wall = ((xi < prm.bc_cells * prm.dx) | (xi > L - prm.bc_cells * prm.dx)).any(-1)
            v = torch.where(wall[:, None], torch.zeros_like(v), v)
        out[k] = v
    return out


def g2p(st: State, vgrid, prm: Params):
    """Sec. 4.3.4 / Sec. 4.4 gather with reading R5: returns (v', B', grad v)."""
    n = prm.n_nodes
    ks = grid_ids(prm.kernel)
    N = st.x.shape[0]
    v = torch.zeros(N, 3, dtype=F64)
    B = torch.zeros(N, 3, 3, dtype=F64)
    for k in ks:
        idx, w, d = stencil(st.x, prm.dx, prm.kernel, k)
        vi = vgrid[k][_lin(idx, n)]
        v = v + torch.einsum("ns,nsa->na", w, vi)
        B = B + torch.einsum("ns,nsa,nsb->nab", w, vi, d)
    v = v / len(ks)
    B = B / len(ks)
    if prm.transfer in (TRANSFER_PIC, TRANSFER_APIC_GRAD):
        # readings R16, R17: grad v = 1/2 sum_k sum_i v~_i grad w_ip^T; PIC keeps B = 0
        C = torch.zeros(N, 3, 3, dtype=F64)
        for k in ks:
            idx, _, _, g = stencil_grad(st.x, prm.dx, prm.kernel, k)
            vi = vgrid[k][_lin(idx, n)]
            C = C + torch.einsum("nsa,nsb->nab", vi, g)
        return v, (torch.zeros_like(B) if prm.transfer == TRANSFER_PIC else B), C / len(ks)
    Dinv = torch.linalg.inv(apic_D(st.x, prm))
    return v, B, B @ Dinv


def step(st: State, prm: Params, newton=False, gravity=None, bc=True, return_grids=False):
    """One full time step in the order of reading R10."""
    grids = p2g(st, prm, newton)
    vg = grid_update(grids, prm, gravity, bc)
    v, B, C = g2p(st, vg, prm)
    I = torch.eye(3, dtype=F64)
    F = (I + prm.dt * C) @ st.F
    F = plasticity(F, st, prm)
    x = st.x + prm.dt * v
    new = State(x, v, B, F, st.mat, st.E)
    if return_grids:
        return new, grids, vg
    return new


def run(st: State, prm: Params, steps: int, **kw) -> State:
    for _ in range(steps):
        st = step(st, prm, **kw)
    return st


# -----------------------------------------------------------------------------
# diagnostics used by the tests (Supplement eq. 1-3)
# -----------------------------------------------------------------------------

def particle_momentum(st: State, prm: Params):
    return (particle_mass(st, prm)[:, None] * st.v).sum(0)


def particle_angular_momentum(st: State, prm: Params):
    """Supplement eq. 3: sum x_p x m_p v_p + sum m_p eps : B_p."""
    mp = particle_mass(st, prm)
    L = torch.cross(st.x, mp[:, None] * st.v, dim=-1).sum(0)
    B = st.B
    spin = torch.stack([B[:, 2, 1] - B[:, 1, 2], B[:, 0, 2] - B[:, 2, 0], B[:, 1, 0] - B[:, 0, 1]], -1)
    return L + (mp[:, None] * spin).sum(0)


def grid_nodes(prm: Params, k: int) -> torch.Tensor:
    n = prm.n_nodes
    ar = torch.arange(n, dtype=torch.int64)
    iz, iy, ix = torch.meshgrid(ar, ar, ar, indexing="ij")
    return node_position(torch.stack([ix, iy, iz], -1).reshape(-1, 3), k, prm.dx)


def grid_momentum(grids, prm: Params):
    """Supplement eq. 1: (1/|K|) sum_k sum_i m_i v_i."""
    return sum(p.sum(0) for (_, p) in grids.values()) / len(grids)


def grid_angular_momentum(grids, prm: Params):
    """Supplement eq. 2: (1/|K|) sum_k sum_i x_i x m_i v_i."""
    tot = torch.zeros(3, dtype=F64)
    for k, (_, p) in grids.items():
        tot = tot + torch.cross(grid_nodes(prm, k), p, dim=-1).sum(0)
    return tot / len(grids)


def params_from_scene(sc) -> Params:
    """Build oracle parameters from a scene description (duck-typed)."""
    mats = [Mat(m.model, m.E, m.nu, m.rho, m.friction_deg, getattr(m, "gamma", 7.15)) for m in sc.materials]
    return Params(res=sc.res, dx=sc.dx, dt=sc.dt, materials=mats, gravity=tuple(sc.gravity),
                  bc_cells=sc.bc_cells, ppc=sc.ppc, kernel=sc.kernel, transfer=getattr(sc, "transfer", 0))


def state_from_scene(sc, x32=True) -> State:
    """Initial state of a scene (B = 0, F = I); positions and velocities are
    rounded through float32 when x32 so both sides start from the same values."""
    import numpy as np
    x = sc.x.astype(np.float32).astype(np.float64) if x32 else sc.x
    v = sc.v.astype(np.float32).astype(np.float64) if x32 else sc.v
    return make_state(torch.from_numpy(x), torch.from_numpy(v), mat=torch.from_numpy(sc.mat.astype(np.int64)))
