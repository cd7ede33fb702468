"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests re-types an oracle formula: each checks a closed form, an
identity the paper proves (Sec. 4.2, Supplement Thm 1.1/2.1/2.2), a textbook
special case, a brute-force evaluation, or a physical law (free fall,
variational force, Young's modulus, Mohr-Coulomb) that a plausible slip in
the oracle (dropped term, sign, index, transpose, factor 1/2) would break.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import ckmpm_oracle as O
from paper_2412_10399_gb300 import scenes as S

F64 = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _prm(res=16, kernel=O.KERNEL_CK, dt=1e-4, mats=None, **kw):
    mats = mats or [O.Mat(O.FIXED_COROTATED, 1e5, 0.3, 1000.0)]
    return O.Params(res=res, dx=1.0 / res, dt=dt, materials=mats, kernel=kernel, **kw)


def _rand_state(n, res, seed, **kw):
    x, v, B, F = S.random_state(n, res, seed, **kw)
    return O.make_state(torch.from_numpy(x), torch.from_numpy(v), torch.from_numpy(B), torch.from_numpy(F))


# ----------------------------------------------------------------------------- K1

def test_k1_golden_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "k1_closed_values.txt")) if l.strip() and not l.startswith("#")]
    x = torch.tensor([float(r[0]) for r in rows], dtype=F64)
    want = torch.tensor([float(r[1]) for r in rows], dtype=F64)
    got = O.K1(x)
    assert torch.allclose(got, want, atol=1e-15, rtol=0)


def test_k1_normalisation_and_positivity():
    from scipy.integrate import quad
    val, err = quad(lambda t: float(O.K1(torch.tensor(t, dtype=F64))), -1.0, 1.0, points=[0.0], limit=200)
    assert abs(val - 1.0) < 1e-12
    x = torch.linspace(-1.2, 1.2, 4801, dtype=F64)
    assert bool((O.K1(x) >= 0).all())


def test_k1_partition_of_unity():
    x = torch.rand(10000, dtype=F64)
    assert torch.allclose(O.K1(x) + O.K1(1.0 - x), torch.ones_like(x), atol=1e-15, rtol=0)


def test_k1_monotone_on_unit_interval():
    x = torch.linspace(0, 1, 20001, dtype=F64)
    y = O.K1(x)
    assert bool((y[1:] < y[:-1]).all())


def _d1(f, x, h):
    return (f(x + h) - f(x - h)) / (2 * h)


def _d2(f, x, h):
    return (f(x + h) - 2 * f(x) + f(x - h)) / (h * h)


@pytest.mark.parametrize("knot", [0.0, 1.0, -1.0])
def test_k1_is_c2_but_not_c3_at_knots(knot):
    f = lambda t: O.K1(torch.tensor(t, dtype=F64)).item()
    # first and second derivative one-sided values -> 0 at the knot (both sides)
    for side in (-1.0, 1.0):
        prev = None
        for e in (1e-2, 1e-3):
            x0 = knot + side * e
            h = e / 10
            d1, d2 = _d1(f, x0, h), _d2(f, x0, h)
            assert abs(d1) < 25 * e * e + 1e-9
            assert abs(d2) < 45 * e + 1e-5
    # one-sided third derivatives differ (|jump| = 4 pi^2 at 0 and at +-1)
    e = 1e-3
    right = (_d2(f, knot + 2 * e, e / 10) - _d2(f, knot + e, e / 10)) / e
    left = (_d2(f, knot - e, e / 10) - _d2(f, knot - 2 * e, e / 10)) / e
    assert abs(right - left) > 0.5 * 4 * math.pi ** 2


# ----------------------------------------------------------------------------- dual grid

def test_dual_grid_weights_sum_and_position_reconstruction():
    prm = _prm(res=32)
    x = (4 + 24 * torch.rand(500, 3, dtype=F64)) * prm.dx
    recon = torch.zeros_like(x)
    for k in (-1, 1):
        idx, w, d = O.stencil(x, prm.dx, prm.kernel, k)
        assert torch.allclose(w.sum(1), torch.ones(500, dtype=F64), atol=1e-14)
        xi = O.node_position(idx, k, prm.dx)
        recon = recon + 0.5 * torch.einsum("ns,nsa->na", w, xi)
    # Sec. 4.2 eq. new-reconstruction-of-position
    assert torch.allclose(recon, x, atol=1e-15, rtol=0)


def test_single_grid_does_not_reconstruct_position():
    # the reason for the dual grid: one CK grid alone violates first-order accuracy
    prm = _prm(res=32)
    x = (4 + 24 * torch.rand(500, 3, dtype=F64)) * prm.dx
    idx, w, d = O.stencil(x, prm.dx, prm.kernel, 1)
    err = (torch.einsum("ns,nsa->na", w, O.node_position(idx, 1, prm.dx)) - x).abs().max()
    assert err > 1e-3 * prm.dx


def test_per_grid_first_moment_closed_form():
    """Per axis, sum_i K1(.)(x_i - x_p) over the 2 nodes of grid k equals
    -dx sin(2 pi f_k)/(2 pi), f_k = frac(x/dx + k/4); the two grids' moments are
    opposite (sin(2 pi (f + 1/2)) = -sin(2 pi f))."""
    prm = _prm(res=32)
    x = (4 + 24 * torch.rand(300, 3, dtype=F64)) * prm.dx
    for k in (-1, 1):
        idx, w, d = O.stencil(x, prm.dx, prm.kernel, k)
        m1 = torch.einsum("ns,nsa->na", w, d)
        u = x / prm.dx + 0.25 * k
        f = u - torch.floor(u)
        want = -prm.dx * torch.sin(2 * math.pi * f) / (2 * math.pi)
        assert torch.allclose(m1, want, atol=1e-16, rtol=0)


def test_apic_D_closed_form_and_spectrum():
    """D = diag(s - a^2) + a a^T with a = -dx sin(2 pi f+)/(2 pi) and
    s = mean over the two grids of dx^2 [f(1-f) - sin(2 pi f)/(2 pi) (1-2f)],
    derived by hand from K1; eigenvalues lie in ~[0.083, 0.153] dx^2."""
    prm = _prm(res=32)
    x = (4 + 24 * torch.rand(400, 3, dtype=F64)) * prm.dx
    D = O.apic_D(x, prm)
    u = x / prm.dx
    fp = (u + 0.25) - torch.floor(u + 0.25)
    fm = (u - 0.25) - torch.floor(u - 0.25)
    sig = lambda f: torch.sin(2 * math.pi * f) / (2 * math.pi)
    m2 = lambda f: f * (1 - f) - sig(f) * (1 - 2 * f)
    a = -prm.dx * sig(fp)
    s = 0.5 * prm.dx ** 2 * (m2(fp) + m2(fm))
    want = torch.diag_embed(s - a * a) + a[:, :, None] * a[:, None, :]
    assert torch.allclose(D, want, atol=1e-14 * prm.dx ** 2, rtol=0)
    ev = torch.linalg.eigvalsh(D) / prm.dx ** 2
    assert float(ev.min()) > 0.08 and float(ev.max()) < 0.16


def test_quadratic_D_is_quarter_dx2_identity():
    prm = _prm(res=32, kernel=O.KERNEL_QUADRATIC)
    x = (4 + 24 * torch.rand(300, 3, dtype=F64)) * prm.dx
    D = O.apic_D(x, prm)
    assert torch.allclose(D, (prm.dx ** 2 / 4) * torch.eye(3, dtype=F64).expand_as(D), atol=1e-14 * prm.dx ** 2, rtol=0)


def test_quadratic_bspline_textbook_values():
    x = torch.tensor([0.0, 0.5, 1.0, 1.5, -1.0, 0.25], dtype=F64)
    want = torch.tensor([0.75, 0.5, 0.125, 0.0, 0.125, 0.6875], dtype=F64)
    assert torch.allclose(O.quadratic_bspline(x), want, atol=1e-16, rtol=0)
    prm = _prm(res=32, kernel=O.KERNEL_QUADRATIC)
    xp = (4 + 24 * torch.rand(300, 3, dtype=F64)) * prm.dx
    idx, w, d = O.stencil(xp, prm.dx, prm.kernel, 0)
    assert torch.allclose(w.sum(1), torch.ones(300, dtype=F64), atol=1e-14)
    assert torch.allclose(torch.einsum("ns,nsa->na", w, d), torch.zeros_like(xp), atol=1e-17)


# ----------------------------------------------------------------------------- transfers

@pytest.mark.parametrize("kernel", [O.KERNEL_CK, O.KERNEL_QUADRATIC])
def test_affine_velocity_field_is_reproduced(kernel):
    prm = _prm(res=16, kernel=kernel)
    st = _rand_state(200, 16, seed=3)
    b = torch.tensor([0.3, -0.2, 0.7], dtype=F64)
    A = torch.tensor([[0.1, 2.0, -0.5], [0.3, -1.2, 0.8], [-0.9, 0.4, 0.6]], dtype=F64)
    vg = {k: b + O.grid_nodes(prm, k) @ A.T for k in O.grid_ids(kernel)}
    v, B, C = O.g2p(st, vg, prm)
    assert torch.allclose(v, b + st.x @ A.T, atol=1e-13, rtol=0)
    assert torch.allclose(C, A.expand_as(C), atol=1e-11, rtol=0)


@pytest.mark.parametrize("kernel", [O.KERNEL_CK, O.KERNEL_QUADRATIC])
def test_p2g_conserves_linear_and_angular_momentum(kernel):
    """Supplement Thm 1.1 / 2.1 / 2.2 (P2G part, with the symmetric-stress force)."""
    prm = _prm(res=16, kernel=kernel, dt=1e-3)
    st = _rand_state(300, 16, seed=5, f_scale=0.2)
    grids = O.p2g(st, prm)
    P = O.particle_momentum(st, prm)
    L = O.particle_angular_momentum(st, prm)
    assert torch.allclose(O.grid_momentum(grids, prm), P, atol=1e-13 * float(P.abs().max()) + 1e-18)
    Lg = O.grid_angular_momentum(grids, prm)
    assert torch.allclose(Lg, L, rtol=0, atol=1e-12 * float(L.abs().max()))
    # the force alone must carry no net torque: stress off changes nothing in L
    g0 = O.p2g(st, prm, stress=False)
    assert torch.allclose(O.grid_angular_momentum(g0, prm), Lg, atol=1e-12 * float(L.abs().max()))
    assert not torch.allclose(g0[O.grid_ids(kernel)[0]][1], grids[O.grid_ids(kernel)[0]][1])


@pytest.mark.parametrize("kernel", [O.KERNEL_CK, O.KERNEL_QUADRATIC])
def test_g2p_transfers_grid_angular_momentum_to_particles(kernel):
    """Supplement Thm 2.2, G2P part: with node masses from the same particles,
    sum x^{n+1} x m v' + sum m eps:B' equals (1/|K|) sum x_i x m_i v~_i."""
    prm = _prm(res=16, kernel=kernel, dt=2e-3)
    st = _rand_state(300, 16, seed=7)
    grids = O.p2g(st, prm)
    torch.manual_seed(0)
    vg = {k: torch.randn(prm.n_nodes ** 3, 3, dtype=F64) for k in grids}
    v, B, C = O.g2p(st, vg, prm)
    new = O.State(st.x + prm.dt * v, v, B, st.F, st.mat)
    Lp = O.particle_angular_momentum(new, prm)
    Lg = sum(torch.cross(O.grid_nodes(prm, k), grids[k][0][:, None] * vg[k], dim=-1).sum(0) for k in grids) / len(grids)
    assert torch.allclose(Lp, Lg, atol=1e-12 * float(Lg.abs().max()), rtol=0)
    Pp = O.particle_momentum(new, prm)
    Pg = sum((grids[k][0][:, None] * vg[k]).sum(0) for k in grids) / len(grids)
    assert torch.allclose(Pp, Pg, atol=1e-12 * float(Pg.abs().max()), rtol=0)


@pytest.mark.parametrize("kernel", [O.KERNEL_CK, O.KERNEL_QUADRATIC])
@pytest.mark.parametrize("model", [O.FIXED_COROTATED, O.DRUCKER_PRAGER])
def test_full_step_conserves_momentum_without_gravity_or_walls(kernel, model):
    mats = [O.Mat(model, 1e5, 0.3, 1000.0, 30.0)]
    prm = _prm(res=16, kernel=kernel, dt=1e-4, mats=mats)
    st = _rand_state(400, 16, seed=11, f_scale=0.1)
    P0, L0 = O.particle_momentum(st, prm), O.particle_angular_momentum(st, prm)
    new = O.step(st, prm, gravity=(0.0, 0.0, 0.0), bc=False)
    assert torch.allclose(O.particle_momentum(new, prm), P0, atol=1e-12 * float(P0.abs().max()), rtol=0)
    assert torch.allclose(O.particle_angular_momentum(new, prm), L0, atol=1e-11 * float(L0.abs().max()), rtol=0)


@pytest.mark.parametrize("kernel", [O.KERNEL_CK, O.KERNEL_QUADRATIC])
def test_free_fall_closed_form(kernel):
    """Symplectic Euler under gravity: v_n = v0 + n dt g,
    x_n = x0 + n dt v0 + dt^2 g n(n+1)/2; F stays I and B stays 0."""
    prm = _prm(res=32, kernel=kernel, dt=1e-3)
    x0 = torch.tensor([[0.43, 0.61, 0.52]], dtype=F64)
    v0 = torch.tensor([[0.2, 0.1, -0.3]], dtype=F64)
    st = O.make_state(x0, v0)
    g = torch.tensor(prm.gravity, dtype=F64)
    n = 25
    for _ in range(n):
        st = O.step(st, prm)
    assert torch.allclose(st.v, v0 + n * prm.dt * g, atol=1e-12, rtol=0)
    assert torch.allclose(st.x, x0 + n * prm.dt * v0 + prm.dt ** 2 * g * n * (n + 1) / 2, atol=1e-13, rtol=0)
    assert torch.allclose(st.F, torch.eye(3, dtype=F64)[None], atol=1e-11)
    assert float(st.B.abs().max()) < 1e-12


def test_particle_inside_sticky_wall_stops():
    prm = _prm(res=32, kernel=O.KERNEL_CK, dt=1e-3)
    st = O.make_state(torch.tensor([[1.6 / 32, 0.5, 0.5]], dtype=F64), torch.tensor([[-1.0, 0.5, 0.2]], dtype=F64))
    new = O.step(st, prm)
    assert float(new.v.abs().max()) == 0.0


def test_grid_force_is_minus_twice_energy_gradient():
    """Variational consistency: with F^(xh) = (I + grad v(xh - x)) F built by the
    oracle's own G2P from grid displacements, the P2G force on grid k equals
    -2 dE/dxh_ik, E = sum_p V0 psi(F^_p); the factor 2 is because each grid
    carries the full mass while grid totals are averaged (Supplement eq. 1)."""
    prm = _prm(res=12, dt=1e-3)
    st = _rand_state(60, 12, seed=13, f_scale=0.15)
    st.v.zero_()
    st.B.zero_()
    g_s = O.p2g(st, prm)
    g_0 = O.p2g(st, prm, stress=False)
    mu, lam = O.particle_lame(st, prm)
    disp = {k: torch.zeros(prm.n_nodes ** 3, 3, dtype=F64, requires_grad=True) for k in O.grid_ids(prm.kernel)}
    _, _, C = O.g2p(st, disp, prm)
    Fh = (torch.eye(3, dtype=F64) + C) @ st.F
    V = prm.dx ** 3 / 8  # physical volume per particle at 8 particles per cell
    E = (V * O.fc_energy(Fh, mu, lam, newton=True)).sum()
    grads = torch.autograd.grad(E, [disp[k] for k in O.grid_ids(prm.kernel)])
    for k, gk in zip(O.grid_ids(prm.kernel), grads):
        f = (g_s[k][1] - g_0[k][1]) / prm.dt
        assert torch.allclose(f, -2.0 * gk, atol=1e-9 * float(gk.abs().max()), rtol=0)


def test_p2g_matches_brute_force_node_loops():
    """Dense per-node summation with scalar math (no tensors) on a tiny case."""
    prm = _prm(res=8, dt=1e-3)
    st = _rand_state(6, 8, seed=17, margin_cells=2.5)
    grids = O.p2g(st, prm)
    mp = O.particle_mass(st, prm)
    tau = O.kirchhoff_stress(st, prm)
    dx = prm.dx
    n = prm.n_nodes

    def k1(t):
        t = abs(t)
        return 1 - t + math.sin(2 * math.pi * t) / (2 * math.pi) if t < 1 else 0.0

    for kk in (-1, 1):
        m_bf = np.zeros((n, n, n))
        p_bf = np.zeros((n, n, n, 3))
        for p in range(st.x.shape[0]):
            xp = st.x[p].tolist()
            D = np.zeros((3, 3))
            for k2 in (-1, 1):
                for i in range(n):
                    for j in range(n):
                        for l in range(n):
                            xi = [(i - k2 / 4) * dx, (j - k2 / 4) * dx, (l - k2 / 4) * dx]
                            w = k1((xi[0] - xp[0]) / dx) * k1((xi[1] - xp[1]) / dx) * k1((xi[2] - xp[2]) / dx)
                            if w:
                                dd = np.array(xi) - np.array(xp)
                                D += 0.5 * w * np.outer(dd, dd)
            A = (float(mp[p]) * st.B[p].numpy() - prm.dt * prm.V0 * tau[p].numpy()) @ np.linalg.inv(D)
            for i in range(n):
                for j in range(n):
                    for l in range(n):
                        xi = [(i - kk / 4) * dx, (j - kk / 4) * dx, (l - kk / 4) * dx]
                        w = k1((xi[0] - xp[0]) / dx) * k1((xi[1] - xp[1]) / dx) * k1((xi[2] - xp[2]) / dx)
                        if w:
                            dd = np.array(xi) - np.array(xp)
                            m_bf[l, j, i] += w * float(mp[p])
                            p_bf[l, j, i] += w * (float(mp[p]) * st.v[p].numpy() + A @ dd)
        m, pp = grids[kk]
        assert np.allclose(m.numpy().reshape(n, n, n), m_bf, atol=1e-15, rtol=1e-12)
        assert np.allclose(pp.numpy().reshape(n, n, n, 3), p_bf, atol=1e-13, rtol=1e-10)


# ----------------------------------------------------------------------------- constitutive

def _rotations(n, seed=0):
    g = torch.Generator().manual_seed(seed)
    q = torch.randn(n, 4, generator=g, dtype=F64)
    q = q / q.norm(dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    R = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
        2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
        2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], 1).reshape(n, 3, 3)
    return R


def test_svd_rotation_variant():
    g = torch.Generator().manual_seed(1)
    F = torch.randn(500, 3, 3, generator=g, dtype=F64)
    U, s, V = O.svd_rv(F)
    assert torch.allclose(U @ torch.diag_embed(s) @ V.transpose(-1, -2), F, atol=1e-13)
    assert torch.allclose(torch.det(U), torch.ones(500, dtype=F64), atol=1e-13)
    assert torch.allclose(torch.det(V), torch.ones(500, dtype=F64), atol=1e-13)
    ref = np.linalg.svd(F.numpy(), compute_uv=False)
    assert np.allclose(np.abs(s.numpy()), ref, atol=1e-13)
    assert bool((torch.sign(s[:, 2]) == torch.sign(torch.det(F))).all())


def test_fixed_corotated_stress_properties():
    n = 64
    R = _rotations(n)
    mu = torch.full((n,), 3e4, dtype=F64)
    lam = torch.full((n,), 5e4, dtype=F64)
    assert float(O.fc_piola(R, mu, lam).abs().max()) < 1e-9
    g = torch.Generator().manual_seed(2)
    F = torch.eye(3, dtype=F64) + 0.3 * torch.randn(n, 3, 3, generator=g, dtype=F64)
    F = F[torch.det(F) > 0.2][:16]
    m = F.shape[0]
    tau = O.fc_kirchhoff(F, mu[:m], lam[:m])
    assert torch.allclose(tau, tau.transpose(-1, -2), atol=1e-9)
    # P = d psi / dF by central differences
    P = O.fc_piola(F, mu[:m], lam[:m])
    h = 1e-6
    Pfd = torch.zeros_like(F)
    for a in range(3):
        for b in range(3):
            E = torch.zeros(3, 3, dtype=F64)
            E[a, b] = h
            Pfd[:, a, b] = (O.fc_energy(F + E, mu[:m], lam[:m]) - O.fc_energy(F - E, mu[:m], lam[:m])) / (2 * h)
    assert torch.allclose(P, Pfd, rtol=1e-6, atol=1e-4)


def test_small_strain_uniaxial_stress_gives_young_modulus():
    """Linearised fixed-corotated: under uniaxial stress the axial stress over
    axial strain is E and lateral over axial strain is -nu."""
    E, nu = 2.5e5, 0.3
    mu, lam = O.lame(E, nu)
    mu_t = torch.tensor([mu], dtype=F64)
    lam_t = torch.tensor([lam], dtype=F64)
    e = 1e-7
    F = torch.diag(torch.tensor([1 + e, 1 - nu * e, 1 - nu * e], dtype=F64))[None]
    P = O.fc_piola(F, mu_t, lam_t)[0]
    assert abs(P[0, 0].item() / e - E) < 1e-3 * E
    assert abs(P[1, 1].item()) < 1e-3 * E * e
    assert abs(P[2, 2].item()) < 1e-3 * E * e
    # Hencky model has the same linearisation
    tau = O.hencky_kirchhoff(F, mu_t, lam_t)[0]
    assert abs(tau[0, 0].item() / e - E) < 1e-3 * E
    assert abs(tau[1, 1].item()) < 1e-3 * E * e


def _dp_case(eps):
    """F = U diag(exp eps) V^T for random rotations."""
    n = eps.shape[0]
    U, V = _rotations(n, 3), _rotations(n, 4)
    return U @ torch.diag_embed(torch.exp(eps)) @ V.transpose(-1, -2), U, V


def _principal_tau(F, mu, lam):
    tau = O.hencky_kirchhoff(F, mu, lam)
    return torch.linalg.eigvalsh(tau)


def test_drucker_prager_return_map_properties():
    n = 300
    mu_v, lam_v = O.lame(3.5e5, 0.3)
    mu = torch.full((n,), mu_v, dtype=F64)
    lam = torch.full((n,), lam_v, dtype=F64)
    alpha = O.dp_alpha(30.0)
    g = torch.Generator().manual_seed(5)
    eps = 0.02 * torch.randn(n, 3, generator=g, dtype=F64)
    F, U, V = _dp_case(eps)
    Fr = O.dp_return_map(F, mu, lam, alpha)
    tau = O.hencky_kirchhoff(Fr, mu, lam)
    tr = tau.diagonal(dim1=-2, dim2=-1).sum(-1)
    dev = tau - tr[:, None, None] / 3 * torch.eye(3, dtype=F64)
    ndev = dev.norm(dim=(-1, -2))
    # inside or on the cone |dev tau| <= -alpha tr tau, tension maps to zero stress
    assert bool((ndev <= -alpha * tr + 1e-6 * mu_v).all())
    tension = eps.sum(1) >= 0
    assert float(tau[tension].abs().max()) < 1e-8 * mu_v
    # idempotent
    Fr2 = O.dp_return_map(Fr, mu, lam, alpha)
    assert torch.allclose(Fr2, Fr, atol=1e-12)
    # projected states sit on the surface; states already inside are untouched
    tr_e = eps.sum(1)
    eh = eps - tr_e[:, None] / 3
    dg = eh.norm(dim=1) + (3 * lam_v + 2 * mu_v) / (2 * mu_v) * tr_e * alpha
    inside = (tr_e < 0) & (dg <= 0)
    projected = (tr_e < 0) & (dg > 0)
    assert torch.allclose(Fr[inside], F[inside], atol=1e-14)
    assert bool(projected.any()) and bool(inside.any())
    assert torch.allclose(ndev[projected], -alpha * tr[projected], rtol=1e-9, atol=1e-6)
    # the trace of the log strain (volume) is kept by the projection
    s_new = torch.linalg.svdvals(Fr[projected])
    assert torch.allclose(torch.log(s_new).sum(1), tr_e[projected], atol=1e-12)


@pytest.mark.parametrize("c", [0.5, 0.9, 0.99, 0.995, 0.99999])
def test_drucker_prager_keeps_isotropic_compression(c):
    """Pure isotropic compression F = c R (c < 1, R a rotation): the log strain
    is ln(c) (1, 1, 1), its deviator is exactly zero and tr eps < 0, so the
    klar2016 plastic multiplier dgamma = 0 + (3 lam + 2 mu)/(2 mu) 3 ln(c) alpha
    is negative: the state lies strictly inside the cone and the return map
    leaves it unchanged (it is not the cone's tip, which is reserved for
    tr eps >= 0).  The Hencky stress is then the pressure (3 lam + 2 mu) ln(c) I."""
    mu_v, lam_v = O.lame(3.5e5, 0.3)
    alpha = O.dp_alpha(30.0)
    R = _rotations(4, 11)
    F = torch.cat([c * torch.eye(3, dtype=F64)[None], c * R])
    n = F.shape[0]
    mu = torch.full((n,), mu_v, dtype=F64)
    lam = torch.full((n,), lam_v, dtype=F64)
    Fr = O.dp_return_map(F, mu, lam, alpha)
    assert torch.allclose(Fr, F, rtol=0, atol=1e-15)
    tau = O.hencky_kirchhoff(Fr, mu, lam)
    p = (3.0 * lam_v + 2.0 * mu_v) * math.log(c)
    assert torch.allclose(tau, p * torch.eye(3, dtype=F64).expand(n, 3, 3), rtol=1e-12, atol=1e-9 * mu_v)
    # a deviatoric perturbation far below the cone's opening stays inside too
    eps = math.log(c) * torch.ones(1, 3, dtype=F64) + torch.tensor([[1e-9, -0.5e-9, -0.5e-9]], dtype=F64)
    Fp, _, _ = _dp_case(eps)
    assert torch.allclose(O.dp_return_map(Fp, mu[:1], lam[:1], alpha), Fp, rtol=0, atol=1e-15)


@pytest.mark.parametrize("c", [1.0, 1.001, 1.1])
def test_drucker_prager_sends_isotropic_tension_to_the_tip(c):
    """F = c R with c >= 1 has tr eps >= 0: the cone's tip, Sigma = I, so F
    becomes the rotation U V^T = R and carries no stress."""
    mu_v, lam_v = O.lame(3.5e5, 0.3)
    alpha = O.dp_alpha(30.0)
    R = torch.cat([torch.eye(3, dtype=F64)[None], _rotations(3, 12)])
    n = R.shape[0]
    mu = torch.full((n,), mu_v, dtype=F64)
    lam = torch.full((n,), lam_v, dtype=F64)
    Fr = O.dp_return_map(c * R, mu, lam, alpha)
    assert torch.allclose(Fr, R, rtol=0, atol=1e-14)
    assert float(O.hencky_kirchhoff(Fr, mu, lam).abs().max()) < 1e-9 * mu_v


def test_drucker_prager_matches_mohr_coulomb_in_triaxial_compression():
    """With alpha = sqrt(2/3) 2 sin(phi)/(3 - sin(phi)) the cone passes through
    the Mohr-Coulomb surface (cohesion 0) on the compression meridian:
    sigma_max - sigma_min = -(sigma_max + sigma_min) sin(phi)."""
    phi = 30.0
    mu_v, lam_v = O.lame(3.5e5, 0.3)
    mu = torch.tensor([mu_v], dtype=F64)
    lam = torch.tensor([lam_v], dtype=F64)
    alpha = O.dp_alpha(phi)
    sphi = math.sin(math.radians(phi))
    # principal log strains of a triaxial compression state eps = (-a-2b, -a+b, -a+b)
    for a, b_scale in ((0.01, 0.5), (0.01, 2.0), (0.003, 1.3)):
        eps = torch.tensor([[-a - 2 * b_scale * a, -a + b_scale * a, -a + b_scale * a]], dtype=F64)
        F, _, _ = _dp_case(eps)
        Fr = O.dp_return_map(F, mu, lam, alpha)
        s = _principal_tau(Fr, mu, lam)[0]
        smin, smax = float(s.min()), float(s.max())
        lhs = smax - smin
        rhs = -(smax + smin) * sphi
        if torch.allclose(Fr, F, atol=1e-14):
            assert lhs <= rhs * (1 + 1e-9)
        else:
            assert abs(lhs - rhs) < 1e-8 * abs(rhs)


# ----------------------------------------------------------------------------- kinematics and scale

@pytest.mark.parametrize("kernel", [O.KERNEL_CK, O.KERNEL_QUADRATIC])
def test_homogeneous_shear_flow_deforms_F_from_the_left(kernel):
    """Steady homogeneous flow v = L x with nilpotent L: dF/dt = L F has the
    exact solution F(t) = (I + t L) F0, and forward Euler reproduces it,
    F_n = (I + n dt L) F0, for any F0 (here one that does not commute with L).
    APIC carries the affine field exactly, so every particle sees grad v = L
    (over one step for CK, where D changes with position and B is stored per
    reading R6; over several steps for the quadratic path, where D is constant)."""
    mats = [O.Mat(O.FIXED_COROTATED, 0.0, 0.3, 1000.0)]
    prm = _prm(res=16, kernel=kernel, dt=1e-3, mats=mats)
    L = torch.tensor([[0.0, 0.8, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]], dtype=F64)
    x, _, _, _ = S.random_state(300, 16, seed=19, margin_cells=5.0)
    x = torch.from_numpy(x)
    F0 = torch.tensor([[1.1, 0.0, 0.2], [0.3, 0.9, 0.0], [0.0, -0.1, 1.05]], dtype=F64)
    B = L @ O.apic_D(x, prm)
    st = O.make_state(x, x @ L.T, B, F0.expand(300, 3, 3))
    n = 1 if kernel == O.KERNEL_CK else 4
    for _ in range(n):
        st = O.step(st, prm, gravity=(0.0, 0.0, 0.0), bc=False)
    want = (torch.eye(3, dtype=F64) + n * prm.dt * L) @ F0
    assert torch.allclose(st.F, want.expand_as(st.F), atol=1e-12, rtol=0)


def test_particle_masses_add_up_to_density_times_volume():
    """8 particles per filled cell: the masses of the 0.25^3 elastic cube sum to
    rho * 0.25^3 = 15.625 kg (fixes V0 = dx^3 / ppc and m = rho V0)."""
    sc = S.elastic_cube()
    prm = O.params_from_scene(sc)
    st = O.state_from_scene(sc)
    assert abs(float(O.particle_mass(st, prm).sum()) - 15.625) < 1e-9
    assert abs(prm.V0 * sc.n - 0.25 ** 3) < 1e-15
