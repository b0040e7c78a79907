"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test would fail under a plausible slip in the oracle: a dropped term,
a wrong sign or factor, a transposed operand, a wrong lumping or weight.
* dense brute force: M, C_e, D_e assembled by Gauss quadrature from
  shape functions obtained by solving the nodal interpolation system
  (Sec. 2.2.1, Eqs. galerkin_lbm, fem_matrices) on tiny meshes;
* streaming invariants: constants, lumped-mass conservation, exact
  translation of linear fields at interior nodes;
* recovery (Sec. 2.3): exact for linear fields, second-order convergence;
* the tanh profile of width xi is the equilibrium fixed by beta and kappa
  (Sec. 2.1): mu on it vanishes as h -> 0;
* D2Q9 moment identities of the equilibria and sources (Eqs. f_eq, g_eq, F,
  G and the exact-difference force);
* whole step: mass and momentum conservation, stationarity of uniform
  states, gravity-driven uniform acceleration, shear-wave decay at
  nu = c_s^2 tau dt (Sec. 2.1);
* walls (bounce-back, Sec. 3.3): steady channel flow is the Poiseuille
  parabola of curvature -g / nu with no slip at the wall rows; co-current
  two-phase channel flow (Sec. 3.3, planar) solves the steady momentum
  balance with the model's viscosity mixing.
"""
import numpy as np
import pytest

from oracle.oracle import EX, EY, W, Oracle, Params
from paper_1608_01906_gb300 import inputs

CS2 = 1.0 / 3.0
DIRS = list(zip(EX, EY))


def nonperiodic_grid(nx, ny, h=1.0, jitter=0.0, seed=0):
    """Unit lattice without wrap-around; optional interior jitter."""
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    xy = np.stack([i.ravel() * h, j.ravel() * h], 1).astype(float)
    if jitter:
        rng = np.random.default_rng(seed)
        inner = (i.ravel() > 0) & (i.ravel() < nx - 1) & (j.ravel() > 0) & (j.ravel() < ny - 1)
        xy[inner] += rng.uniform(-jitter * h, jitter * h, size=(inner.sum(), 2))
    tris = []
    for b in range(ny - 1):
        for a in range(nx - 1):
            p, q, r, s = a + nx * b, a + 1 + nx * b, a + 1 + nx * (b + 1), a + nx * (b + 1)
            tris += [(p, q, r), (p, r, s)]
    boundary = (xy[:, 0] < 0.5 * h) | (xy[:, 0] > (nx - 1.5) * h) | (xy[:, 1] < 0.5 * h) | (
        xy[:, 1] > (ny - 1.5) * h)
    return xy, np.array(tris, dtype=np.int32), np.zeros(2), boundary


def oracle_for(xy, tri, box, **kw):
    return Oracle(xy, tri, box, None, Params(**kw))


# ---------------------------------------------------------------- geometry
def test_geometry_areas_and_lumped_mass():
    xy, tri, box, tag = inputs.structured_mesh(8, 6)
    o = oracle_for(xy, tri, box)
    assert np.allclose(o.area, 0.5) and np.allclose(o.mass, 1.0)
    xy, tri, box, tag = inputs.jittered_delaunay_mesh(12, 10, 0.25, seed=3)
    o = oracle_for(xy, tri, box)
    assert (o.area > 0).all()
    assert o.area.sum() == pytest.approx(box[0] * box[1], rel=1e-13)
    assert o.mass.sum() == pytest.approx(box[0] * box[1], rel=1e-13)


# ------------------------------------------------- dense quadrature brute force
def dense_operators(xy, tri, box, e):
    """Consistent M, C_e, D_e by 3-point Gauss quadrature of explicit P1
    shape functions (coefficients from solving [1 x y] c = delta)."""
    N = len(xy)
    M = np.zeros((N, N))
    Cm = np.zeros((N, N))
    D = np.zeros((N, N))
    e = np.asarray(e, float)
    bary = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])
    for t in tri:
        p = xy[t].copy()
        for k in (1, 2):  # minimum image relative to the first vertex
            for d in (0, 1):
                if box[d] > 0:
                    p[k, d] = p[0, d] + (p[k, d] - p[0, d]) - box[d] * np.round(
                        (p[k, d] - p[0, d]) / box[d])
        V = np.column_stack([np.ones(3), p])
        coef = np.linalg.solve(V, np.eye(3))  # column a: N_a = c0 + c1 x + c2 y
        area = 0.5 * abs(np.linalg.det(V))
        grads = coef[1:, :].T  # (3, 2)
        for q in range(3):
            x = bary[q] @ p
            Nv = coef[0] + coef[1] * x[0] + coef[2] * x[1]
            wq = area / 3
            for a in range(3):
                for b in range(3):
                    M[t[a], t[b]] += wq * Nv[a] * Nv[b]
                    Cm[t[a], t[b]] += wq * Nv[a] * (e @ grads[b])
                    D[t[a], t[b]] += wq * 0.5 * (e @ grads[a]) * (e @ grads[b])
    return M, Cm, D


@pytest.mark.parametrize("mesh", ["structured", "delaunay", "open"])
def test_stream_matches_dense_quadrature(mesh):
    if mesh == "structured":
        xy, tri, box, _ = inputs.structured_mesh(5, 4)
    elif mesh == "delaunay":
        xy, tri, box, _ = inputs.jittered_delaunay_mesh(6, 5, 0.25, seed=11)
    else:
        xy, tri, box, _ = nonperiodic_grid(5, 5, jitter=0.2, seed=5)
    dt = 0.37
    o = oracle_for(xy, tri, box, dt=dt)
    rng = np.random.default_rng(1)
    psi = rng.normal(size=len(xy))
    for e in DIRS:
        M, Cm, D = dense_operators(xy, tri, box, e)
        ML = M.sum(axis=1)  # lumped mass: row sums of the consistent mass
        ref = psi + (-dt * Cm @ psi - dt * dt * D @ psi) / ML
        got = o.stream(e, psi)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.abs(ref).max()), e


def test_stream_invariants():
    xy, tri, box, _ = inputs.jittered_delaunay_mesh(10, 9, 0.25, seed=4)
    o = oracle_for(xy, tri, box, dt=0.3)
    rng = np.random.default_rng(2)
    psi = rng.uniform(size=len(xy))
    for e in DIRS:
        out = o.stream(e, np.full(len(xy), 0.7))
        assert np.max(np.abs(out - 0.7)) <= 1e-14
        out = o.stream(e, psi)
        assert abs(o.mass @ out - o.mass @ psi) <= 1e-13 * (o.mass @ psi)


def test_stream_translates_linear_fields_at_interior_nodes():
    xy, tri, box, boundary = nonperiodic_grid(7, 6, jitter=0.2, seed=9)
    dt = 0.45
    o = oracle_for(xy, tri, box, dt=dt)
    b = np.array([0.3, -1.1])
    psi = 2.0 + xy @ b
    for e in DIRS:
        out = o.stream(e, psi)
        want = psi - dt * (np.asarray(e) @ b)
        assert np.max(np.abs(out[~boundary] - want[~boundary])) <= 1e-13


# -------------------------------------------------------------- recovery
def test_recovery_exact_for_linear_fields():
    xy, tri, box, _ = nonperiodic_grid(6, 7, jitter=0.25, seed=8)
    o = oracle_for(xy, tri, box)
    gx, gy = o.recover(1.5 - 0.25 * xy[:, 0] + 0.75 * xy[:, 1])
    assert np.max(np.abs(gx + 0.25)) <= 1e-13 and np.max(np.abs(gy - 0.75)) <= 1e-13


def test_recovery_and_laplacian_second_order():
    errs_g, errs_l = [], []
    for n in (32, 64, 128):
        h = 64.0 / n
        xy, tri, box, _ = inputs.structured_mesh(n, n, h=h)
        o = oracle_for(xy, tri, box)
        k = 2 * np.pi / 64
        f = np.sin(k * xy[:, 0]) * np.cos(2 * k * xy[:, 1])
        gx, gy = o.recover(f)
        lap = o.recover(gx)[0] + o.recover(gy)[1]
        errs_g.append(np.abs(gx - k * np.cos(k * xy[:, 0]) * np.cos(2 * k * xy[:, 1])).max())
        errs_l.append(np.abs(lap + 5 * k * k * f).max())
    for e in (errs_g, errs_l):
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, e


def test_tanh_profile_is_the_equilibrium():
    # mu = mu_phi - kappa lap rho vanishes on the tanh profile of width xi
    # only if kappa/beta = xi^2 (rho_l - rho_v)^2 / 8 (Sec. 2.1); refinement
    # drives it to zero at second order.
    mus = []
    for n in (64, 128, 256):
        h = 64.0 / n
        xy, tri, box, _ = inputs.structured_mesh(n, 8, h=h)
        o = oracle_for(xy, tri, box, rho_l=1.0, rho_v=0.1, sigma=0.01, xi=4.0)
        # flat interfaces normal to x
        x = xy[:, 0]
        rho = 0.1 + 0.45 * (np.tanh(2 * (x - 16) / 4.0) - np.tanh(2 * (x - 48) / 4.0))
        mus.append(np.abs(o.fields_of(rho)["mu"]).max())
    beta = 12 * 0.01 / (4.0 * 0.9 ** 4)
    scale = beta * 0.9 ** 3  # magnitude of mu_phi across the interface
    assert mus[-1] < 0.02 * scale
    assert mus[0] / mus[1] > 3.0 and mus[1] / mus[2] > 3.0, mus


def test_stress_force_integrates_to_laplace_jump():
    # kappa [d_i |grad rho|^2 - d_j (d_i rho d_j rho)] of a circular tanh drop
    # integrates radially to -sigma/R in 2-D (Laplace's law, Sec. 3.1).
    n, R = 128, 32.0
    xy, tri, box, _ = inputs.structured_mesh(n, n)
    o = oracle_for(xy, tri, box, rho_l=1.0, rho_v=0.1, sigma=0.01, xi=8.0)
    rho0, _, _ = inputs.droplet_fields(xy, box, (64, 64), R, 1.0, 0.1, 8.0)
    f = o.fields_of(rho0)
    row = (xy[:, 1] == 64) & (xy[:, 0] >= 64)
    integral = np.trapezoid(f["Kx"][row]) if hasattr(np, "trapezoid") else np.trapz(f["Kx"][row])
    assert integral == pytest.approx(-0.01 / R, rel=0.03)


def test_stress_force_y_mirrors_x_and_integrates_to_laplace_jump():
    # The split of every square along its (i,j)-(i+1,j+1) diagonal is
    # symmetric under the reflection x <-> y, and so is a drop centred on a
    # node: K_y at (i, j) must equal K_x at (j, i) to rounding, and K_y
    # integrates up a column to -sigma/R like K_x along a row.  A slip in a
    # product, a sign or an index of the K_y terms breaks both.
    n, R = 128, 32.0
    xy, tri, box, _ = inputs.structured_mesh(n, n)
    o = oracle_for(xy, tri, box, rho_l=1.0, rho_v=0.1, sigma=0.01, xi=8.0)
    rho0, _, _ = inputs.droplet_fields(xy, box, (64, 64), R, 1.0, 0.1, 8.0)
    f = o.fields_of(rho0)
    kx = f["Kx"].reshape(n, n)  # [y, x]
    ky = f["Ky"].reshape(n, n)
    assert np.abs(ky - kx.T).max() <= 1e-12 * np.abs(kx).max()
    col = (xy[:, 0] == 64) & (xy[:, 1] >= 64)
    integral = np.trapezoid(f["Ky"][col]) if hasattr(np, "trapezoid") else np.trapz(f["Ky"][col])
    assert integral == pytest.approx(-0.01 / R, rel=0.03)


def test_weak_laplacian_option_exact_for_quadratics_and_second_order():
    # The alternative reading of the Laplacian (laplacian = 1): the lumped
    # weak form -(1/m_i) sum_T |T| grad N_i . grad rho_T.  On the structured
    # split it is the five-point Laplacian, exact for quadratic fields at
    # interior nodes; on smooth periodic fields it converges at second order.
    xy, tri, box, boundary = nonperiodic_grid(7, 6)
    o = oracle_for(xy, tri, box, laplacian=1)
    q = 0.5 * xy[:, 0] ** 2 + 1.5 * xy[:, 1] ** 2 - 0.25 * xy[:, 0] * xy[:, 1] + xy[:, 0]
    lap = o.fields_of(q)["lap"]
    assert np.abs(lap[~boundary] - 4.0).max() <= 1e-12
    errs = []
    k = 2 * np.pi / 64
    for n in (32, 64, 128):
        xy, tri, box, _ = inputs.structured_mesh(n, n, h=64.0 / n)
        o = oracle_for(xy, tri, box, laplacian=1)
        f = np.sin(k * xy[:, 0]) * np.cos(2 * k * xy[:, 1])
        errs.append(np.abs(o.fields_of(f)["lap"] + 5 * k * k * f).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, errs


# ------------------------------------------------------ local identities
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibria_and_source_moments(seed):
    rng = np.random.default_rng(seed)
    xy, tri, box, _ = inputs.structured_mesh(4, 4)
    dt = rng.uniform(0.2, 1.0)
    g = rng.normal(size=2) * 1e-2
    o = Oracle(xy, tri, box, None, Params(dt=dt, gravity=tuple(g)))
    rho = rng.uniform(0.1, 1.0)
    p = rng.normal() * 1e-2
    u = rng.normal(size=2) * 0.05
    dr = rng.normal(size=2)
    dm = rng.normal(size=2) * 1e-2
    K = rng.normal(size=2) * 1e-3
    t = o.local_terms(rho, p, u, dr, dm, K)
    E = np.stack([EX, EY])
    # equilibria (Eqs. f_eq, g_eq)
    assert t["heq"].sum() == pytest.approx(rho, rel=1e-14)
    assert np.allclose(E @ t["heq"], rho * u, atol=1e-15)
    P2 = (E * t["heq"]) @ E.T / rho
    assert np.allclose(P2, CS2 * np.eye(2) + np.outer(u, u), atol=1e-15)
    assert t["geq"].sum() == pytest.approx(p / CS2, abs=1e-15)
    assert np.allclose(E @ t["geq"], rho * u, atol=1e-15)
    # F (Eq. F): zero mass, first moment dt/2 (c_s^2 grad rho - rho grad mu)
    assert abs(t["F"].sum()) <= 1e-15
    assert np.allclose(E @ t["F"], 0.5 * dt * (CS2 * dr - rho * dm), atol=1e-14)
    # G (Eq. G): zeroth moment dt/2 u.grad rho, first moment dt/2 K
    assert t["G"].sum() == pytest.approx(0.5 * dt * u @ dr, abs=1e-14)
    assert np.allclose(E @ t["G"], 0.5 * dt * K, atol=1e-15)
    # exact-difference force: no mass, first moment rho g dt / 2
    assert abs(t["B"].sum()) <= 1e-15
    assert np.allclose(E @ t["B"], 0.5 * rho * g * dt, atol=1e-15)


# -------------------------------------------------------------- whole step
def droplet_oracle(mesh, ratio=10.0, **kw):
    xy, tri, box, tag = mesh
    n = np.sqrt(box[0] * box[1])
    o = Oracle(xy, tri, box, tag, Params(rho_l=1.0, rho_v=1.0 / ratio, **kw))
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (box[0] / 2, box[1] / 2), n / 4, 1.0,
                                         1.0 / ratio, 4.0)
    o.init(rho0, u0, p0)
    return o


@pytest.mark.parametrize("kind", ["structured", "delaunay"])
def test_step_conserves_mass_and_momentum(kind):
    mesh = (inputs.structured_mesh(40, 40) if kind == "structured"
            else inputs.jittered_delaunay_mesh(40, 40, 0.25, seed=1608))
    o = droplet_oracle(mesh, ratio=10.0)
    m0, _, _ = o.totals()
    o.step(300)
    m1, px, py = o.totals()
    assert abs(m1 - m0) <= 1e-13 * m0
    assert abs(px) <= 1e-13 * m0 and abs(py) <= 1e-13 * m0


def test_uniform_states_are_stationary():
    xy, tri, box, tag = inputs.jittered_delaunay_mesh(12, 12, 0.25, seed=2)
    o = Oracle(xy, tri, box, tag, Params(rho_l=1.0, rho_v=0.1))
    N = len(xy)
    u0 = np.tile([0.05, -0.02], (N, 1))
    o.init(np.full(N, 1.0), u0, np.full(N, 0.01))
    o.step(50)
    assert np.max(np.abs(o.rho - 1.0)) <= 1e-13
    assert np.max(np.abs(o.ux - 0.05)) <= 1e-13 and np.max(np.abs(o.uy + 0.02)) <= 1e-13
    assert np.max(np.abs(o.p - 0.01)) <= 1e-13


def test_gravity_accelerates_uniform_fluid():
    # periodic, uniform rho: only the body force acts; rho u grows by rho g dt
    # per step (exact-difference force + dt/2 rho g term of Eq. velocity).
    xy, tri, box, tag = inputs.structured_mesh(8, 8)
    g = (2e-5, -1e-5)
    o = Oracle(xy, tri, box, tag, Params(rho_l=1.0, rho_v=0.1, dt=0.5, gravity=g))
    N = len(xy)
    o.init(np.full(N, 1.0), np.zeros((N, 2)), np.zeros(N))
    n = 40
    o.step(n)
    assert np.allclose(o.ux, g[0] * n * 0.5, rtol=1e-10, atol=1e-16)
    assert np.allclose(o.uy, g[1] * n * 0.5, rtol=1e-10, atol=1e-16)


@pytest.mark.parametrize("tau", [0.5, 0.2])
def test_shear_wave_decays_at_model_viscosity(tau):
    # single phase (sigma = 0, uniform rho): u_x = U sin(2 pi y / L) decays
    # as exp(-nu k^2 t), nu = c_s^2 tau dt (Sec. 2.1).
    L, dt = 64, 0.5
    xy, tri, box, tag = inputs.structured_mesh(L, L)
    o = Oracle(xy, tri, box, tag,
               Params(rho_l=1.0, rho_v=0.5, sigma=0.0, tau_l=tau, tau_v=tau, dt=dt))
    rho0, u0, p0 = inputs.shear_wave_fields(xy, box, 1.0, 1e-4)
    o.init(rho0, u0, p0)
    s = np.sin(2 * np.pi * xy[:, 1] / L)
    a0 = (o.ux @ s) / (s @ s)
    steps = 400
    o.step(steps)
    a1 = (o.ux @ s) / (s @ s)
    rate = -np.log(a1 / a0) / (steps * dt)
    nu = CS2 * tau * dt
    assert rate == pytest.approx(nu * (2 * np.pi / L) ** 2, rel=0.01)


def test_flat_interface_holds_no_pressure_jump():
    # a flat slab carries no Laplace pressure: p is equal in both bulk phases
    xy, tri, box, tag = inputs.structured_mesh(32, 64)
    o = Oracle(xy, tri, box, tag, Params(rho_l=1.0, rho_v=0.1))
    rho0, u0, p0 = inputs.slab_fields(xy, box, 16, 48, 1.0, 0.1, 4.0)
    o.init(rho0, u0, p0)
    o.step(1500)
    y = xy[:, 1]
    p_liq = o.p[(y > 28) & (y < 36)].mean()
    p_vap = o.p[(y < 4) | (y > 60)].mean()
    assert abs(p_liq - p_vap) < 0.02 * 0.01 / 16  # < 2% of the droplet-case jump


def _channel_profile(tau, ny=17, g=1e-5, steps=12000):
    # walls at rows 0 and ny - 1 (bounce-back at the wall nodes, Sec. 3.3),
    # periodic in x, uniform rho, driven by a body force along x
    nx = 4
    xy, tri, box, tag = inputs.structured_mesh(nx, ny, periodic_y=False)
    dt = 0.5
    o = Oracle(xy, tri, box, tag, Params(rho_l=1.0, rho_v=0.1, tau_l=tau, tau_v=tau, dt=dt,
                                         gravity=(g, 0.0)))
    N = nx * ny
    o.init(np.ones(N), np.zeros((N, 2)), np.zeros(N))
    o.step(steps)
    ux = o.ux.reshape(ny, nx)
    assert np.abs(ux - ux[:, :1]).max() < 1e-15 and np.abs(o.uy).max() < 1e-15
    return ux[:, 0], g / (CS2 * tau * dt)


@pytest.mark.parametrize("tau", [0.5, 1.0])
def test_channel_flow_is_poiseuille(tau):
    # steady single-phase channel flow: nu u'' = -g, a parabola whose
    # curvature is -g / nu with nu = c_s^2 tau dt, vanishing at the walls.
    # At tau = 0.5 the discrete profile is that parabola to round-off, with
    # its zeros 0.013 outside the wall rows; at tau = 1 to 1e-3 away from the
    # wall rows.  A bounce-back of the wrong directions, at the wrong rows or
    # with a sign slip gives slip, a wrong curvature or no steady state.
    ny = 17
    u, g_over_nu = _channel_profile(tau, ny)
    y = np.arange(ny, dtype=float)
    sel = slice(2, ny - 2)
    c = np.polyfit(y[sel], u[sel], 2)
    resid = np.abs(u[sel] - np.polyval(c, y[sel])).max() / u.max()
    lo, hi = sorted(np.roots(c).real)
    if tau == 0.5:
        assert 2 * c[0] == pytest.approx(-g_over_nu, rel=1e-6)
        assert resid < 1e-8
        assert abs(lo) < 0.02 and abs(hi - (ny - 1)) < 0.02
    else:
        assert 2 * c[0] == pytest.approx(-g_over_nu, rel=5e-3)
        assert resid < 1e-3
        assert abs(lo) < 0.1 and abs(hi - (ny - 1)) < 0.1


def _layered_reference(rho, P, g, wall_offset):
    # steady x-momentum balance of a flow layered in y, d/dy(mu du/dy) =
    # -rho g, with mu = rho c_s^2 tau(C) dt (tau mixing rule of Sec. 2.1,
    # C clamped) from the given rho(y); the stress vanishes at the centre
    # (symmetry) and u at the walls, wall_offset outside the wall rows.
    # Integrated by the trapezoid rule on a fine grid over linear profiles.
    ny = len(rho)
    C = np.clip((rho - P.rho_v) / (P.rho_l - P.rho_v), 0.0, 1.0)
    mu = rho * CS2 * P.dt / (C / P.tau_l + (1.0 - C) / P.tau_v)
    y = np.arange(ny, dtype=float)
    yf = np.linspace(-wall_offset, ny - 1 + wall_offset, 40 * ny + 1)
    rf, mf = np.interp(yf, y, rho), np.interp(yf, y, mu)
    mass = np.concatenate([[0.0], np.cumsum(0.5 * (rf[1:] + rf[:-1]) * np.diff(yf))])
    stress = -g * (mass - np.interp((ny - 1) / 2.0, yf, mass))
    dudy = stress / mf
    u = np.concatenate([[0.0], np.cumsum(0.5 * (dudy[1:] + dudy[:-1]) * np.diff(yf))])
    return np.interp(y, yf, u)


def test_layered_channel_flow_matches_momentum_balance():
    # co-current flow (Sec. 3.3, planar): the heavier, more viscous phase in
    # the core |s| <= a, the lighter one along the walls, driven along x by
    # gravity; viscosity contrast M = mu_core / mu_wall = 4, rho 1 and 0.5.
    # The flat interfaces carry no x force, so the steady profile solves the
    # 1-D balance above with the run's own rho(y) (the diffuse interface and
    # the bulk densities the run settles to).  Outside the interface bands it
    # holds to 0.15% (a wrong tau mixing, force density or wall rule moves
    # the core by several %); inside them to the O(h^2) resolution of a
    # 4-node interface.  The sharp-interface form of the paper's closed
    # profile (rho-weighted force, continuous u and shear stress at |s| = a)
    # is approached as xi / a -> 0: 6.8% low in the core here (xi / a = 0.4),
    # 1.9% at xi / a = 0.2.
    nx, ny, xi, g = 4, 41, 4.0, 1e-6
    rho_c, rho_w, tau_w, M = 1.0, 0.5, 0.5, 4.0
    tau_c = M * rho_w * tau_w / rho_c
    yc, a = (ny - 1) / 2.0, (ny - 1) / 4.0
    xy, tri, box, tag = inputs.structured_mesh(nx, ny, periodic_y=False)
    P = Params(rho_l=rho_c, rho_v=rho_w, sigma=0.01, xi=xi, tau_l=tau_c, tau_v=tau_w, dt=0.5,
               gravity=(g, 0.0))
    rho0, _, p0 = inputs.slab_fields(xy, box, yc - a, yc + a, rho_c, rho_w, xi)
    # start from the balance of the initial profile: only a small correction
    # has to decay
    u_start = _layered_reference(rho0[::nx], P, g, 0.013)
    o = Oracle(xy, tri, box, tag, P)
    o.init(rho0, np.stack([np.repeat(u_start, nx), np.zeros(nx * ny)], 1), p0)
    o.step(20000)
    u = o.ux.reshape(ny, nx)
    assert np.abs(u - u[:, :1]).max() < 1e-15 and np.abs(o.uy).max() < 1e-12
    u = u[:, 0]
    ref = _layered_reference(o.rho[::nx], P, g, 0.013)
    s = np.abs(np.arange(ny) - yc)
    outside = np.abs(s - a) > xi
    assert np.abs(u - ref)[outside].max() < 1.5e-3 * ref.max()
    assert np.abs(u - ref).max() < 2e-2 * ref.max()
    # sharp-interface closed form
    mu_c, mu_w = rho_c * CS2 * tau_c * 0.5, rho_w * CS2 * tau_w * 0.5
    B = (rho_w - rho_c) * g * a / mu_w
    D = rho_w * g * yc ** 2 / (2 * mu_w) - B * yc
    u_a = -rho_w * g * a ** 2 / (2 * mu_w) + B * a + D + rho_c * g * a ** 2 / (2 * mu_c)
    assert 0.90 < u[int(yc)] / u_a < 0.96


def _laplace_ratio(h, L=32.0, R=8.0, xi=4.0, T=1000.0, nu=1.0 / 3.0, sigma=0.01, ratio=10.0):
    # static drop of fixed physical size on a mesh of spacing h: dt = h/2
    # (the stable Courant number of the structured split), tau = nu / (c_s^2
    # dt) so that the kinematic viscosity is the same at every h; Delta p
    # from unweighted node means of p inside R - xi and outside R + xi
    n = int(round(L / h))
    xy, tri, box, tag = inputs.structured_mesh(n, n, h=h)
    dt = 0.5 * h
    tau = nu / (CS2 * dt)
    o = Oracle(xy, tri, box, None, Params(rho_l=1.0, rho_v=1.0 / ratio, sigma=sigma, xi=xi,
                                          tau_l=tau, tau_v=tau, dt=dt))
    c = (L / 2, L / 2)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, c, R, 1.0, 1.0 / ratio, xi)
    o.init(rho0, u0, p0)
    o.step(int(round(T / dt)))
    r = np.hypot(xy[:, 0] - c[0], xy[:, 1] - c[1])
    dp = o.p[r < R - xi].mean() - o.p[r > R + xi].mean()
    return dp / (sigma / R)


def test_laplace_law_converges_with_resolution():
    # Laplace's law for a static 2-D drop, Delta p = sigma / R (Sec. 3.1,
    # restated in 2-D), approached under grid refinement as the paper's
    # Table 1 shows for its meshes M1-M5: the same drop (L = 32, R = 8,
    # xi = 4) at xi/h = 4 and 8.  The error |Delta p / (sigma/R) - 1| must
    # fall at least 3x per halving of h and the fine run must be within 10%.
    # Measured: 0.736 and 0.956 of sigma/R (error ratio 6).  Halving the
    # kappa lap rho term of mu, dropping the stress force from the velocity
    # moment, or a wrong factor in kappa or beta breaks one of the bounds
    # (u.grad rho in the pressure moment vanishes at rest; the translated
    # drop below pins it).
    coarse, fine = _laplace_ratio(1.0), _laplace_ratio(0.5)
    e1, e2 = abs(coarse - 1.0), abs(fine - 1.0)
    assert e2 < 0.10, (coarse, fine)
    assert e1 >= 3.0 * e2, (coarse, fine)


def test_translated_drop_matches_drop_at_rest():
    # Galilean invariance (Sec. 3.2, 2-D): a drop carried by u = (0.02, 0)
    # through a 32 x 32 periodic box for exactly one period coincides with
    # the same drop relaxed at rest for the same time.  The oracle reaches
    # 1.7% of rho_l - rho_v (max over nodes); dropping the second-order
    # velocity terms of the equilibrium gives 17%, dropping u.grad rho from
    # the pressure moment makes the run diverge.
    L, U, ratio, xi = 32, 0.02, 10.0, 4.0
    xy, tri, box, tag = inputs.structured_mesh(L, L)
    P = Params(rho_l=1.0, rho_v=1.0 / ratio, sigma=0.01, xi=xi, tau_l=0.5, tau_v=0.5, dt=0.5)
    steps = int(round(L / U / 0.5))
    rho = {}
    for u in (U, 0.0):
        rho0, u0, p0 = inputs.droplet_fields(xy, box, (L / 2, L / 2), L / 4, 1.0, 1.0 / ratio, xi,
                                             u0=(u, 0.0))
        o = Oracle(xy, tri, box, tag, P)
        o.init(rho0, u0, p0)
        o.step(steps)
        rho[u] = o.rho
    err = np.abs(rho[U] - rho[0.0]).max() / (1.0 - 1.0 / ratio)
    assert err < 0.03
