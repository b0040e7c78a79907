"""Pins of the three-dimensional FP64 oracle (D3Q19 on P1 tetrahedra, the
paper's own setting) against what the paper and the mathematics fix.

Each test would fail under a plausible slip in the oracle (a dropped term, a
wrong sign, weight or factor, a transposed operand, a wrong lumping):
* dense brute force: M, C_e, D_e assembled by 4-point Gauss quadrature from
  shape functions obtained by solving the nodal interpolation system
  (Sec. 2.2.1, Eqs. galerkin_lbm, fem_matrices) on small tetrahedral meshes;
* streaming invariants: constants, lumped-mass conservation;
* recovery (Sec. 2.3): exact for linear fields, second-order convergence;
* D3Q19 moments of the equilibria and sources (Eqs. f_eq, g_eq, F, G and
  the exact-difference force);
* the tanh profile of width xi is the equilibrium fixed by beta and kappa;
* whole step: mass and momentum conservation, stationary uniform states,
  gravity-driven acceleration, shear-wave decay at nu = c_s^2 tau dt, and
  Poiseuille flow between walls.
"""
import numpy as np
import pytest

from oracle.oracle3d import E3, Oracle3, Params3
from paper_1608_01906_gb300 import inputs

CS2 = 1.0 / 3.0


def open_tet_grid(n, h=1.0, jitter=0.0, seed=0):
    """Kuhn-split cube lattice of n^3 nodes without wrap-around; optional
    jitter of interior nodes."""
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    i, j, k = i.ravel(order="F"), j.ravel(order="F"), k.ravel(order="F")
    xyz = np.stack([i, j, k], 1).astype(float) * h
    if jitter:
        inner = (i > 0) & (i < n - 1) & (j > 0) & (j < n - 1) & (k > 0) & (k < n - 1)
        xyz[inner] += np.random.default_rng(seed).uniform(-jitter * h, jitter * h, (inner.sum(), 3))
    nid = lambda a, b, c: a + n * (b + n * c)  # noqa: E731
    tets = []
    for a in range(n - 1):
        for b in range(n - 1):
            for c in range(n - 1):
                for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
                    cur = [a, b, c]
                    v = [nid(*cur)]
                    for ax in perm:
                        cur[ax] += 1
                        v.append(nid(*cur))
                    d = np.linalg.det(xyz[v[1:]] - xyz[v[0]])
                    tets.append(v if d > 0 else [v[0], v[2], v[1], v[3]])
    return xyz, np.array(tets, dtype=np.int32), np.zeros(3)


def oracle3(xyz, tet, box, tag=None, **kw):
    return Oracle3(xyz, tet, box, tag, Params3(**kw))


def wrapped(d, L):
    return d - L * np.round(d / L) if L > 0 else d


# ------------------------------------------------------------ brute force
def dense_operators(xyz, tet, box, e):
    """M, C_e, D_e by 4-point Gauss quadrature of P1 shape functions; each
    element's shape functions from the 4x4 interpolation system."""
    N = len(xyz)
    M = np.zeros((N, N))
    Ce = np.zeros((N, N))
    De = np.zeros((N, N))
    a, b = 0.5854101966249685, 0.1381966011250105
    bary = np.array([[a, b, b, b], [b, a, b, b], [b, b, a, b], [b, b, b, a]])
    for t in tet:
        x0 = xyz[t[0]]
        X = np.array([x0 + np.array([wrapped(xyz[v][c] - x0[c], box[c]) for c in range(3)])
                      for v in t])
        vol = abs(np.linalg.det(X[1:] - X[0])) / 6.0
        A = np.hstack([np.ones((4, 1)), X])   # rows [1 x y z] of the vertices
        coef = np.linalg.solve(A, np.eye(4))  # column a: N_a = c0 + c.x
        grad = coef[1:, :].T                  # (4, 3)
        eg = grad @ e
        for q in range(4):
            xq = bary[q] @ X
            Nq = np.array([1.0, *xq]) @ coef
            w = vol / 4.0
            for ia, va in enumerate(t):
                for ib, vb in enumerate(t):
                    M[va, vb] += w * Nq[ia] * Nq[ib]
                    Ce[va, vb] += w * Nq[ia] * eg[ib]
                    De[va, vb] += w * 0.5 * eg[ia] * eg[ib]
    return M, Ce, De


@pytest.mark.parametrize("mesh", ["periodic", "open_jittered"])
def test_stream_matches_dense_quadrature(mesh):
    if mesh == "periodic":
        xyz, tet, box, _ = inputs.structured_tet_mesh(3, 3, 3)
    else:
        xyz, tet, box = open_tet_grid(4, jitter=0.2, seed=3)
    dt = 0.5
    o = oracle3(xyz, tet, box, dt=dt)
    rng = np.random.default_rng(11)
    psi = rng.uniform(0.5, 1.5, len(xyz))
    for a in (1, 4, 6, 7, 12, 17):
        e = E3[a]
        M, Ce, De = dense_operators(xyz, tet, box, e)
        ml = M.sum(1)
        want = psi + (-dt * Ce @ psi - dt * dt * De @ psi) / ml
        assert np.allclose(o.stream(e, psi), want, rtol=0, atol=1e-12)
    assert np.allclose(o.mass, M.sum(1), atol=1e-14)


def test_stream_invariants():
    xyz, tet, box, _ = inputs.structured_tet_mesh(4, 5, 3)
    o = oracle3(xyz, tet, box, dt=0.5)
    psi = np.random.default_rng(2).uniform(0.1, 1.0, len(xyz))
    for a in range(19):
        assert np.allclose(o.stream(E3[a], np.full(len(xyz), 0.7)), 0.7, atol=1e-15)
        out = o.stream(E3[a], psi)
        assert o.mass @ out == pytest.approx(o.mass @ psi, rel=1e-14)


# ---------------------------------------------------------------- recovery
def test_recovery_exact_for_linear_fields():
    xyz, tet, box = open_tet_grid(5, jitter=0.25, seed=5)
    o = oracle3(xyz, tet, box)
    c = np.array([0.3, -1.2, 0.7])
    g = o.recover(xyz @ c + 2.0)
    assert np.allclose(g, c, atol=1e-12)


def test_recovery_and_laplacian_second_order():
    errs_g, errs_l = [], []
    for n in (8, 16, 32):
        h = 8.0 / n
        xyz, tet, box, _ = inputs.structured_tet_mesh(n, n, n, h=h)
        o = oracle3(xyz, tet, box)
        k = 2 * np.pi / 8.0
        f = np.sin(k * xyz[:, 0]) * np.cos(k * xyz[:, 2])
        g = o.recover(f)
        gx = k * np.cos(k * xyz[:, 0]) * np.cos(k * xyz[:, 2])
        errs_g.append(np.abs(g[:, 0] - gx).max())
        lap = o.fields_of(1.0 + 0.01 * f)["lap"]
        errs_l.append(np.abs(lap + 0.01 * 2 * k * k * f).max())
    for e in (errs_g, errs_l):
        assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.0, e


# ------------------------------------------------- equilibria and sources
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibria_and_source_moments(seed):
    rng = np.random.default_rng(seed)
    xyz, tet, box, _ = inputs.structured_tet_mesh(3, 3, 3)
    dt = rng.uniform(0.2, 1.0)
    g = rng.normal(size=3) * 1e-2
    o = oracle3(xyz, tet, box, dt=dt, gravity=tuple(g))
    rho, p = rng.uniform(0.1, 1.0), rng.normal() * 1e-2
    u = rng.normal(size=3) * 0.05
    dr, dm, K = rng.normal(size=3), rng.normal(size=3) * 1e-2, rng.normal(size=3) * 1e-3
    t = o.local_terms(rho, p, u, dr, dm, K)
    E = E3.T
    # D3Q19 lattice identities through the equilibria (Eqs. f_eq, g_eq)
    assert t["heq"].sum() == pytest.approx(rho, rel=1e-14)
    assert np.allclose(E @ t["heq"], rho * u, atol=1e-15)
    assert np.allclose((E * t["heq"]) @ E.T / rho, CS2 * np.eye(3) + np.outer(u, u), atol=1e-15)
    assert t["geq"].sum() == pytest.approx(p / CS2, abs=1e-15)
    assert np.allclose(E @ t["geq"], rho * u, atol=1e-15)
    # F: zero mass, first moment dt/2 (c_s^2 grad rho - rho grad mu)
    assert abs(t["F"].sum()) <= 1e-15
    assert np.allclose(E @ t["F"], 0.5 * dt * (CS2 * dr - rho * dm), atol=1e-14)
    # G: zeroth moment dt/2 u.grad rho, first moment dt/2 K
    assert t["G"].sum() == pytest.approx(0.5 * dt * u @ dr, abs=1e-14)
    assert np.allclose(E @ t["G"], 0.5 * dt * K, atol=1e-15)
    # exact-difference force: no mass, first moment rho g dt / 2
    assert abs(t["B"].sum()) <= 1e-15
    assert np.allclose(E @ t["B"], 0.5 * rho * g * dt, atol=1e-15)


def test_d3q19_fourth_moment_is_isotropic():
    # sum_a w_a e_i e_j e_k e_l = c_s^4 (d_ij d_kl + d_ik d_jl + d_il d_jk):
    # checked through the second moment of the equilibria at two velocities
    # (the u u term of Gamma needs it)
    xyz, tet, box, _ = inputs.structured_tet_mesh(3, 3, 3)
    o = oracle3(xyz, tet, box)
    for u in ([0.05, 0.0, 0.0], [0.02, -0.03, 0.04]):
        u = np.array(u)
        t = o.local_terms(1.0, 0.0, u, np.zeros(3), np.zeros(3), np.zeros(3))
        third = np.einsum("a,ai,aj,ak->ijk", t["heq"], E3, E3, E3)
        want = CS2 * (np.einsum("i,jk->ijk", u, np.eye(3)) + np.einsum("j,ik->ijk", u, np.eye(3))
                      + np.einsum("k,ij->ijk", u, np.eye(3)))
        assert np.allclose(third, want, atol=1e-15)


def test_tanh_profile_is_the_equilibrium():
    # mu = mu_phi - kappa lap rho vanishes on the tanh profile of width xi
    # only if kappa/beta = xi^2 (rho_l - rho_v)^2 / 8; refinement drives it
    # to zero at second order (flat interfaces normal to z)
    mus = []
    for n in (32, 64, 128):
        h = 32.0 / n
        xyz, tet, box, _ = inputs.structured_tet_mesh(3, 3, n, h=h)
        o = oracle3(xyz, tet, box, rho_l=1.0, rho_v=0.1, sigma=0.01, xi=4.0)
        rho = inputs.slab_fields3(xyz, 8.0, 24.0, 1.0, 0.1, 4.0)[0]
        mus.append(np.abs(o.fields_of(rho)["mu"]).max())
    scale = 12 * 0.01 / (4.0 * 0.9 ** 4) * 0.9 ** 3
    assert mus[-1] < 0.02 * scale
    assert mus[0] / mus[1] > 3.0 and mus[1] / mus[2] > 3.0, mus


# -------------------------------------------------------------- whole step
def test_step_conserves_mass_and_momentum():
    xyz, tet, box, _ = inputs.structured_tet_mesh(10, 10, 10)
    o = oracle3(xyz, tet, box, rho_l=1.0, rho_v=0.1, xi=3.0)
    rho0, u0, p0 = inputs.droplet_fields3(xyz, box, (5, 5, 5), 3.0, 1.0, 0.1, 3.0,
                                          u0=(0.01, -0.02, 0.005))
    o.init(rho0, u0, p0)
    o.step(1)
    t0 = o.totals()
    o.step(30)
    t1 = o.totals()
    assert t1[0] == pytest.approx(t0[0], rel=1e-13)
    for c in (1, 2, 3):
        assert abs(t1[c] - t0[c]) <= 1e-13 * t0[0]


def test_uniform_states_are_stationary():
    xyz, tet, box, _ = inputs.structured_tet_mesh(4, 4, 4)
    o = oracle3(xyz, tet, box)
    N = len(xyz)
    o.init(np.full(N, 0.6), np.tile([0.01, 0.02, -0.01], (N, 1)), np.full(N, 1e-3))
    h0 = o.h.copy()
    o.step(5)
    assert np.allclose(o.h, h0, atol=1e-15)
    assert np.allclose(o.u, [0.01, 0.02, -0.01], atol=1e-15)


def test_gravity_accelerates_uniform_fluid():
    xyz, tet, box, _ = inputs.structured_tet_mesh(4, 4, 4)
    g = (2e-5, -1e-5, 3e-5)
    o = oracle3(xyz, tet, box, rho_l=1.0, rho_v=0.1, dt=0.5, gravity=g)
    N = len(xyz)
    o.init(np.ones(N), np.zeros((N, 3)), np.zeros(N))
    o.step(40)
    assert np.allclose(o.u, np.array(g) * 40 * 0.5, rtol=1e-10, atol=1e-16)


@pytest.mark.parametrize("tau", [0.5, 0.2])
def test_shear_wave_decays_at_model_viscosity(tau):
    # single phase: u_x = U sin(2 pi z / L) decays as exp(-nu k^2 t), nu =
    # c_s^2 tau dt (Sec. 2.1).  The streaming adds a viscosity of second
    # order in k h: at tau = 0.2 +1.4% for L = 32, +0.36% for L = 64
    L, dt = 64, 0.5
    xyz, tet, box, _ = inputs.structured_tet_mesh(3, 3, L)
    o = oracle3(xyz, tet, box, rho_l=1.0, rho_v=0.5, sigma=0.0, tau_l=tau, tau_v=tau, dt=dt)
    rho0, u0, p0 = inputs.shear_wave_fields3(xyz, box, 1.0, 1e-4)
    o.init(rho0, u0, p0)
    s = np.sin(2 * np.pi * xyz[:, 2] / L)
    a0 = (o.u[:, 0] @ s) / (s @ s)
    steps = 800
    o.step(steps)
    a1 = (o.u[:, 0] @ s) / (s @ s)
    rate = -np.log(a1 / a0) / (steps * dt)
    assert rate == pytest.approx(CS2 * tau * dt * (2 * np.pi / L) ** 2, rel=0.01)


def test_channel_flow_between_walls_is_poiseuille():
    # walls at the bottom and top node layers (bounce-back, Sec. 3.3),
    # periodic in x and y, body force along x: the steady profile is the
    # parabola of curvature -g / nu (tau = 0.5: to round-off, as in 2-D),
    # vanishing just outside the wall layers
    nz, g, tau, dt = 17, 1e-5, 0.5, 0.5
    xyz, tet, box, tag = inputs.structured_tet_mesh(3, 3, nz, periodic_z=False)
    o = oracle3(xyz, tet, box, tag, rho_l=1.0, rho_v=0.1, tau_l=tau, tau_v=tau, dt=dt,
                gravity=(g, 0.0, 0.0))
    N = len(xyz)
    o.init(np.ones(N), np.zeros((N, 3)), np.zeros(N))
    o.step(12000)
    z = xyz[:, 2]
    u = np.array([o.u[z == k, 0].mean() for k in range(nz)])
    assert np.abs(o.u[:, 1:]).max() < 1e-14
    y = np.arange(nz, dtype=float)
    sel = slice(2, nz - 2)
    c = np.polyfit(y[sel], u[sel], 2)
    assert 2 * c[0] == pytest.approx(-g / (CS2 * tau * dt), rel=1e-5)
    assert np.abs(u[sel] - np.polyval(c, y[sel])).max() < 1e-6 * u.max()
    lo, hi = sorted(np.roots(c).real)
    assert abs(lo) < 0.05 and abs(hi - (nz - 1)) < 0.05
