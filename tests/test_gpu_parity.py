"""GPU path vs FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 over all nodes, per field):
* FP64 GPU run: <= 1e-12 (reordered sums only).
* FP32 GPU run after 1000 steps: <= 1e-5 in velocity and C.  Measured: C
  1.3e-7 (ratio 10) and 9.4e-8 (ratio 1000), u 1.2e-6 to 1.5e-6 (ratio 10)
  and 5.5e-6 (ratio 1000).  The collision keeps each node's mass to one
  rounding, and its 3 w_a constants satisfy the equilibrium moment
  identities exactly in FP32 (p by a division by 3): with the nearest
  rounded weights and c_s^2 the pressure and momentum of g gain about 1e-8
  per step, 1.3e-5 and 6.3e-5 in u after 1000 steps.
"""
import numpy as np
import pytest

from conftest import rel_l2
from oracle.oracle import Oracle, Params
from paper_1608_01906_gb300 import configs, felbm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1608_01906_gb300 import build

    build.build()
    felbm.load()


def run_gpu(prob, precision, steps, general=False, lap_fp64=False):
    mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag, general=general)
    st = felbm.State(mesh, felbm.make_params(precision=precision, lap_fp64=lap_fp64, **prob.params),
                     prob.rho0, prob.u0, prob.p0)
    st.step(steps)
    m = st.moments()
    kind = mesh.info()["kind"]
    st.close()
    mesh.close()
    return m, kind


def run_oracle(prob, steps):
    o = Oracle(prob.xy, prob.tri, prob.box, prob.tag, Params(**prob.params))
    o.init(prob.rho0, prob.u0, prob.p0)
    o.step(steps)
    return o


def errors(m, o):
    return {
        "rho": rel_l2(m["rho"], o.rho),
        "C": rel_l2(m["C"], o.C),
        "u": rel_l2(m["u"], np.stack([o.ux, o.uy], 1)),
        "p": rel_l2(m["p"], o.p),
    }


def _droplet(nx, ny, R, ratio=10.0):
    xy, tri, box, tag = inputs.structured_mesh(nx, ny)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (nx / 2, ny / 2), R, 1.0, 1.0 / ratio, 4.0)
    return configs.Problem("d", xy, tri, box, tag, rho0, u0, p0,
                           configs.params(1.0, 1.0 / ratio), 0, "fp64")


@pytest.mark.parametrize("general", [False, True])
def test_fp64_structured_ragged(general):
    # 44 x 36 = 1584 nodes: several 256-node blocks and a ragged tail
    prob = _droplet(44, 36, 11.0)
    m, kind = run_gpu(prob, "fp64", 60, general=general)
    assert kind == (0 if general else 1)
    o = run_oracle(prob, 60)
    e = errors(m, o)
    assert max(e.values()) <= 1e-12, e


def test_fp64_structured_odd_width():
    # 37 x 29: rows not 16-byte aligned (element-wise halo fills), ragged
    # tiles in x and y, periodic wrap through both
    prob = _droplet(37, 29, 9.0)
    m, kind = run_gpu(prob, "fp64", 60)
    assert kind == 1
    o = run_oracle(prob, 60)
    e = errors(m, o)
    assert max(e.values()) <= 1e-12, e


def test_fp64_unstructured_delaunay():
    xy, tri, box, tag = inputs.jittered_delaunay_mesh(40, 36, 0.25, seed=7)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (20, 18), 10.0, 1.0, 0.1, 4.0)
    prob = configs.Problem("u", xy, tri, box, tag, rho0, u0, p0, configs.params(), 0, "fp64")
    m, kind = run_gpu(prob, "fp64", 60)
    assert kind == 0
    o = run_oracle(prob, 60)
    e = errors(m, o)
    assert max(e.values()) <= 1e-12, e


@pytest.mark.parametrize("nx,ny", [(32, 64), (30, 45)])
def test_fp64_walls_rayleigh_taylor_small(nx, ny):
    # 32 x 64: wall tiles and interior tiles; 30 x 45: odd width and a ragged
    # top tile row next to the wall
    prob = configs.c3_rayleigh_taylor(nx=nx, ny=ny, steps=0)
    prob.params["gravity"] = (0.0, -1e-4)
    m, kind = run_gpu(prob, "fp64", 80)
    assert kind == 1
    o = run_oracle(prob, 80)
    e = errors(m, o)
    assert max(e.values()) <= 1e-12, e


def test_fp64_walls_many_tiles():
    # 512 x 384 with walls: 768 tiles; interior tiles load their halo by TMA
    # and mix with x-wrap tiles (cp.async fills) and wall tiles
    prob = configs.c3_rayleigh_taylor(nx=512, ny=384, steps=0)
    prob.params["gravity"] = (0.0, -1e-4)
    m, kind = run_gpu(prob, "fp64", 6)
    assert kind == 1
    o = run_oracle(prob, 6)
    e = errors(m, o)
    assert max(e.values()) <= 1e-12, e


def _layered_channel():
    # co-current two-phase channel flow between wall rows (Sec. 3.3, planar):
    # core rho 1 (tau 1), wall layers rho 0.5 (tau 0.5), gravity along x
    nx, ny, xi = 4, 41, 4.0
    xy, tri, box, tag = inputs.structured_mesh(nx, ny, periodic_y=False)
    yc, a = (ny - 1) / 2.0, (ny - 1) / 4.0
    rho0, u0, p0 = inputs.slab_fields(xy, box, yc - a, yc + a, 1.0, 0.5, xi)
    params = configs.params(1.0, 0.5, 0.01, xi, 1.0, 0.5, 0.5, (1e-6, 0.0))
    return configs.Problem("channel", xy, tri, box, tag, rho0, u0, p0, params, 0, "fp64")


def test_fp64_layered_channel_walls():
    # p stays at rounding level here (flat interfaces along the flow carry no
    # jump): it is compared on the scale c_s^2 rho_l, not relative to itself
    prob = _layered_channel()
    m, kind = run_gpu(prob, "fp64", 2000)
    assert kind == 1
    o = run_oracle(prob, 2000)
    e = errors(m, o)
    dp = np.abs(m["p"] - o.p).max() / (1.0 / 3.0)
    assert max(e["rho"], e["C"], e["u"]) <= 1e-12 and dp <= 1e-13, (e, dp)


def test_fp32_layered_channel_steady_profile():
    # 20,000 FP32 steps to the steady profile against the FP64 oracle.  The
    # bulk densities drift slowly towards the discrete equilibrium over the
    # run, and FP32 rounding of that drift leaves rho 7.2e-6, C 1.7e-5 and u
    # 5.5e-6 relative L2 (measured); held as regression bounds
    prob = _layered_channel()
    m, kind = run_gpu(prob, "fp32", 20000)
    o = run_oracle(prob, 20000)
    e = errors(m, o)
    dp = np.abs(m["p"] - o.p).max() / (1.0 / 3.0)
    print("channel fp32 errors", e, "max|dp| / c_s^2", dp)
    assert e["rho"] <= 2e-5 and e["C"] <= 5e-5 and e["u"] <= 2e-5 and dp <= 1e-6, (e, dp)


def test_fp64_mass_momentum_conserved_gpu():
    prob = _droplet(48, 48, 12.0)
    mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag)
    st = felbm.State(mesh, felbm.make_params(precision="fp64", **prob.params), prob.rho0)
    t0 = st.moments()["totals"]
    st.step(300)
    t1 = st.moments()["totals"]
    assert abs(t1[0] - t0[0]) / t0[0] <= 1e-13
    assert abs(t1[1]) / t0[0] <= 1e-13 and abs(t1[2]) / t0[0] <= 1e-13


def test_fp64_totals_match_oracle_on_delaunay_mesh():
    # FP64 mass and momentum totals sum_i m_i rho_i, sum_i m_i rho_i u_i with
    # the lumped mass m_i = sum_{T contains i} |T|/3 (Sec. 2.2.1): on a
    # jittered Delaunay mesh the masses differ from node to node (0.6-1.4),
    # so unit weights or any other wrong weighting fails.  A drop carried by
    # a uniform velocity gives non-zero momentum totals.
    xy, tri, box, tag = inputs.jittered_delaunay_mesh(40, 36, 0.25, seed=21)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (20, 18), 10.0, 1.0, 0.1, 4.0,
                                         u0=(0.012, -0.007))
    prob = configs.Problem("u", xy, tri, box, tag, rho0, u0, p0, configs.params(dt=0.4), 0,
                           "fp64")
    o = Oracle(prob.xy, prob.tri, prob.box, prob.tag, Params(**prob.params))
    assert o.mass.min() < 0.8 and o.mass.max() > 1.2
    mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag)
    st = felbm.State(mesh, felbm.make_params(precision="fp64", **prob.params), prob.rho0,
                     prob.u0, prob.p0)
    o.init(prob.rho0, prob.u0, prob.p0)
    for steps in (1, 49):
        st.step(steps)
        o.step(steps)
        got = np.asarray(st.moments()["totals"])
        want = np.asarray(o.totals())
        assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want)), (steps, got, want)
        # the same sums from the returned fields (caller order) and the
        # oracle's lumped mass
        m = st.moments()
        mr = o.mass * m["rho"]
        direct = np.array([mr.sum(), (mr * m["u"][:, 0]).sum(), (mr * m["u"][:, 1]).sum()])
        assert np.all(np.abs(got - direct) <= 1e-12 * np.abs(direct)), (got, direct)
    st.close()
    mesh.close()


def test_fp32_walled_rayleigh_taylor_1000_steps():
    # Rayleigh-Taylor physics of the 512 x 2048 workload (walls, gravity,
    # At 0.5, Re 3000 at the reference width) on a 128 x 512 mesh, 1000 FP32
    # steps against the FP64 oracle.  Measured: rho 1.2e-7, C 1.9e-7, p
    # 1.9e-6 relative L2; u 5.6e-5 relative L2 and 1.1e-6 of the flow scale
    # U = sqrt(lambda g).  u starts from rest and is still small (max 1.7e-3
    # against U = 0.08) while the stored g carries the hydrostatic pressure:
    # the FP32 rounding of g, the same every step of a near-steady field,
    # adds up to ~9e-8 in u, which is 5.6e-5 of the young flow's norm.  The
    # bounds: rho, C <= 1e-5 relative L2, u <= 1e-5 of U and <= 1e-4 relative.
    prob = configs.c3_rayleigh_taylor(nx=128, ny=512, steps=0, ref_width=512)
    m, kind = run_gpu(prob, "fp32", 1000)
    assert kind == 1
    o = run_oracle(prob, 1000)
    e = errors(m, o)
    U = np.sqrt(512 * prob.meta["g"])  # sqrt(lambda g) of the 512-wide workload
    du = np.abs(m["u"] - np.stack([o.ux, o.uy], 1)).max() / U
    print("RT 128x512 fp32 1000 steps", e, "max|du|/U", du)
    assert e["C"] <= 1e-5 and e["rho"] <= 1e-5 and du <= 1e-5 and e["u"] <= 1e-4, (e, du)


def test_fp32_layered_channel_1000_steps():
    # the walled two-phase channel of the 20,000-step test at the 1000-step
    # horizon of the FP32 tolerance: <= 1e-5 in u and C
    prob = _layered_channel()
    m, _ = run_gpu(prob, "fp32", 1000)
    o = run_oracle(prob, 1000)
    e = errors(m, o)
    print("channel fp32 1000 steps", e)
    assert e["C"] <= 1e-5 and e["u"] <= 1e-5, e


@pytest.mark.parametrize("general", [False, True])
def test_fp32_droplet_1000_steps(general):
    prob = configs.droplet_structured(64, 16.0, 10.0, steps=1000, precision="fp32")
    m, _ = run_gpu(prob, "fp32", 1000, general=general)
    o = run_oracle(prob, 1000)
    e = errors(m, o)
    print("fp32 1000-step errors", e)
    assert e["C"] <= 1e-6 and e["u"] <= 1e-5, e


@pytest.mark.parametrize("nx,ny", [(40, 40), (38, 30)])
def test_checkpoint_restart_bitwise(nx, ny):
    # 38 x 30: population rows padded to a pitch of 40 slots
    prob = _droplet(nx, ny, 10.0)
    mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag)
    pr = felbm.make_params(precision="fp64", **prob.params)
    a = felbm.State(mesh, pr, prob.rho0)
    a.step(40)
    ma = a.moments()
    b = felbm.State(mesh, pr, prob.rho0)
    b.step(20)
    h, g = b.export()
    o = run_oracle(prob, 20)  # exported populations in caller order
    assert rel_l2(h.ravel(), o.h.ravel()) <= 1e-12 and rel_l2(g.ravel(), o.g.ravel()) <= 1e-12
    c = felbm.State(mesh, pr, np.ones(prob.n_nodes))
    c.import_(h, g)
    c.step(20)
    mc = c.moments()
    for k in ("rho", "u", "p"):
        assert np.array_equal(ma[k], mc[k]), k


@pytest.mark.parametrize("split", [False, True])
def test_checkpoint_restart_bitwise_on_delaunay_mesh(split):
    """Checkpoints of a general mesh go through its internal order (Hilbert
    patches, RCM inside): exported populations in caller order equal the
    oracle's, and a restart from them continues bitwise."""
    xy, tri, box, tag = inputs.jittered_delaunay_mesh(30, 26, 0.25, seed=12)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (15, 13), 7.0, 1.0, 0.1, 4.0, u0=(0.01, 0.004))
    prob = configs.Problem("d", xy, tri, box, tag, rho0, u0, p0, configs.params(dt=0.4), 0, "fp64")
    mesh = felbm.Mesh(xy, tri, box, tag, split_step=split)
    assert mesh.info()["kind"] == 0
    pr = felbm.make_params(precision="fp64", **prob.params)
    a = felbm.State(mesh, pr, rho0, u0, p0)
    a.step(30)
    ma = a.moments()
    b = felbm.State(mesh, pr, rho0, u0, p0)
    b.step(15)
    h, g = b.export()
    o = run_oracle(prob, 15)
    assert rel_l2(h.ravel(), o.h.ravel()) <= 1e-12 and rel_l2(g.ravel(), o.g.ravel()) <= 1e-12
    c = felbm.State(mesh, pr, np.ones(prob.n_nodes))
    c.import_(h, g)
    c.step(15)
    mc = c.moments()
    for k in ("rho", "u", "p"):
        assert np.array_equal(ma[k], mc[k]), k
    for s in (a, b, c):
        s.close()
    mesh.close()


def test_invalid_inputs_rejected():
    xy, tri, box, tag = inputs.structured_mesh(8, 8)
    bad = tri.copy()
    bad[0] = bad[0][::-1]  # clockwise -> negative area
    st, _ = felbm.felbm_mesh_create(xy, bad, box, felbm.flags_for(box))
    assert st == felbm.FELBM_ERR_INVALID_MESH
    mesh = felbm.Mesh(xy, tri, box)
    rho = np.ones(64)
    rho[3] = np.nan
    st, _ = felbm.felbm_state_init(mesh.handle, felbm.make_params(1.0, 0.1, 0.01, 4, 0.5, 0.5, 0.5),
                                   rho)
    assert st == felbm.FELBM_ERR_INVALID_ARG


def test_nonfinite_detected():
    # an unstable time step (Courant 3) blows up to inf/nan without any fault
    prob = _droplet(16, 16, 4.0)
    prob.params["dt"] = 3.0
    mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag)
    st = felbm.State(mesh, felbm.make_params(precision="fp32", **prob.params), prob.rho0)
    st.step(2000)
    assert felbm.felbm_state_sync(st.handle) == felbm.FELBM_ERR_NONFINITE


def test_fullsize_rayleigh_taylor_fp32_steps():
    # Early in the run u is only the gravity increment (~1e-6) and FP32
    # rounding of the hydrostatic pressure (~5e-10 per node) is a sizeable
    # fraction of it, so velocity is held to the flow's own scale
    # U = sqrt(lambda g) rather than to its (tiny) current norm.
    prob = configs.c3_rayleigh_taylor()
    m, kind = run_gpu(prob, "fp32", 4)
    assert kind == 1
    o = run_oracle(prob, 4)
    e = errors(m, o)
    U = np.sqrt(prob.meta["nx"] * prob.meta["g"])
    du = np.abs(m["u"] - np.stack([o.ux, o.uy], 1)).max() / U
    print("c3 4-step fp32 errors", e, "max|du|/U", du)
    assert e["rho"] <= 1e-6 and e["C"] <= 1e-6 and e["p"] <= 1e-5 and du <= 1e-5, (e, du)


@pytest.mark.parametrize("lap_fp64", [False, True])
def test_fullsize_unstructured_fp32_1000_steps(lap_fp64):
    # 256x256 jittered Delaunay droplet, density ratio 1000, 1000 steps; with
    # lap_fp64 the kappa lap rho term of mu is formed in FP64
    prob = configs.c2_unstructured_droplet()
    m, kind = run_gpu(prob, "fp32", 1000, lap_fp64=lap_fp64)
    assert kind == 0
    o = run_oracle(prob, 1000)
    e = errors(m, o)
    print("c2 1000-step fp32 errors (lap_fp64=%s)" % lap_fp64, e)
    assert e["C"] <= 1e-6 and e["u"] <= 1e-5, e


def test_fp64_laplacian_term_on_the_structured_lattice_ratio_1000():
    """FELBM_PARAM_LAP_FP64 on the lattice kernel (interior, TMA and wrap
    tiles) with the C2 physics (ratio 1000, xi 12) on a 96 x 80 split, 1000
    FP32 steps against the FP64 oracle, beside the plain FP32 run; the FP64
    term changes the arithmetic (the runs differ) and both hold the bounds."""
    xy, tri, box, tag = inputs.structured_mesh(96, 80)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (48, 40), 20.0, 1.0, 1e-3, 12.0)
    prob = configs.Problem("s", xy, tri, box, tag, rho0, u0, p0,
                           configs.params(1.0, 1e-3, 0.01, 12.0, 0.0025, 0.1, 0.4), 0, "fp32")
    o = run_oracle(prob, 1000)
    res = {}
    for flag in (False, True):
        m, kind = run_gpu(prob, "fp32", 1000, lap_fp64=flag)
        assert kind == 1
        res[flag] = (m, errors(m, o))
    print("structured ratio-1000 fp32 errors: plain", res[False][1], "lap_fp64", res[True][1])
    assert not np.array_equal(res[False][0]["u"], res[True][0]["u"])
    for flag in (False, True):
        e = res[flag][1]
        assert e["C"] <= 1e-6 and e["u"] <= 1e-5, (flag, e)


def test_fp64_laplacian_term_on_wall_and_ragged_tiles():
    """FELBM_PARAM_LAP_FP64 on the lattice kernel's table path: a droplet
    between bounce-back walls on a 72 x 48 split (wall rows, a ragged x tile,
    cp.async fills), 500 FP32 steps against the FP64 oracle beside the plain
    FP32 run, at the FP32 bounds; and the same on the general kernels."""
    xy, tri, box, tag = inputs.structured_mesh(72, 48, periodic_y=False)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (36, 24), 10.0, 1.0, 0.1, 4.0)
    prob = configs.Problem("w", xy, tri, box, tag, rho0, u0, p0, configs.params(), 0, "fp32")
    o = run_oracle(prob, 500)
    for general in (False, True):
        res = {}
        for flag in (False, True):
            m, kind = run_gpu(prob, "fp32", 500, general=general, lap_fp64=flag)
            assert kind == (0 if general else 1)
            res[flag] = (m, errors(m, o))
        print("walled droplet fp32 errors (general=%s): plain" % general, res[False][1], "lap_fp64", res[True][1])
        assert not np.array_equal(res[False][0]["p"], res[True][0]["p"])
        for flag in (False, True):
            e = res[flag][1]
            assert e["C"] <= 1e-6 and e["u"] <= 1e-5, (general, flag, e)


def test_fp64_laplacian_flag_is_refused_where_not_built():
    prob = _droplet(32, 32, 8.0)
    mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag)
    st = felbm.State(mesh, felbm.make_params(precision="fp32", lap_fp64=True, **prob.params), prob.rho0)
    with pytest.raises(felbm.FelbmError) as e:
        felbm.Batch([st])
    assert e.value.status == felbm.FELBM_ERR_UNSUPPORTED
    st.close()
    mesh.close()
    xyz, tet, box, _ = inputs.structured_tet_mesh(4, 4, 4)
    tm = felbm.Mesh(xyz, tet, box)
    with pytest.raises(felbm.FelbmError) as e:
        felbm.State(tm, felbm.make_params(precision="fp32", lap_fp64=True, **prob.params), np.ones(len(xyz)))
    assert e.value.status == felbm.FELBM_ERR_UNSUPPORTED
    tm.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mesh", ["delaunay", "walled_split"])
def test_patch_step_equals_four_launch_step_bitwise(precision, mesh):
    """The one-launch patch step of general meshes (regions of rings <= 4
    staged in shared memory) against the four-launch step over global
    fields (FELBM_MESH_SPLIT_STEP): the same per-node arithmetic in the same
    order, so the same bits, on a jittered Delaunay mesh with a moving drop
    and on a walled split forced onto the general kernels (bounce-back)."""
    if mesh == "delaunay":
        xy, tri, box, tag = inputs.jittered_delaunay_mesh(70, 52, 0.25, seed=8)
        rho0, u0, p0 = inputs.droplet_fields(xy, box, (35, 26), 12.0, 1.0, 0.1, 4.0, u0=(0.01, 0.005))
        prm = configs.params(dt=0.4)
    else:
        xy, tri, box, tag = inputs.structured_mesh(40, 70, periodic_y=False)
        rho0, u0, p0 = inputs.droplet_fields(xy, box, (20, 35), 10.0, 1.0, 0.1, 4.0)
        prm = configs.params(gravity=(0.0, -1e-5))
    out = []
    for split in (False, True):
        m_ = felbm.Mesh(xy, tri, box, tag, general=True, split_step=split)
        st = felbm.State(m_, felbm.make_params(precision=precision, **prm), rho0, u0, p0)
        st.profile_enable(True)
        st.step(30)
        prof = st.profile_read()
        out.append((st.moments(), st.export(), prof))
        st.close()
        m_.close()
    (ma, (ha, ga), pa), (mb, (hb, gb), pb) = out
    assert pa["k_patch_step"][2] == 30 and pb["k_patch_step"][2] == 0 and pb["k_collide"][2] == 30
    for k in ("rho", "C", "u", "p", "totals"):
        assert np.array_equal(ma[k], mb[k]), k
    assert np.array_equal(ha, hb) and np.array_equal(ga, gb)


def test_patch_step_with_fp64_laplacian_equals_four_launch_step_bitwise():
    """FELBM_PARAM_LAP_FP64 on both general steps: the patch kernel's FP64
    kappa lap rho term is k_mu_lap64's arithmetic, so the bits agree."""
    xy, tri, box, tag = inputs.jittered_delaunay_mesh(48, 40, 0.25, seed=9)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (24, 20), 10.0, 1.0, 1e-3, 12.0)
    prm = configs.params(1.0, 1e-3, 0.01, 12.0, 0.0025, 0.1, 0.4)
    out = []
    for split in (False, True):
        m_ = felbm.Mesh(xy, tri, box, tag, general=True, split_step=split)
        st = felbm.State(m_, felbm.make_params(precision="fp32", lap_fp64=True, **prm), rho0, u0, p0)
        st.step(25)
        out.append((st.moments(), st.export()))
        st.close()
        m_.close()
    (ma, (ha, ga)), (mb, (hb, gb)) = out
    for k in ("rho", "C", "u", "p"):
        assert np.array_equal(ma[k], mb[k]), k
    assert np.array_equal(ha, hb) and np.array_equal(ga, gb)


def test_profile_stride_times_every_kth_launch():
    prob = _droplet(32, 32, 8.0)
    mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag)
    st = felbm.State(mesh, felbm.make_params(precision="fp32", **prob.params), prob.rho0)
    st.profile_enable(3)
    st.step(10)
    ms, timed, issued = st.profile_read()["k_lattice_step"]
    assert issued == 10 and timed == 4 and ms > 0.0  # launches 0, 3, 6 and 9
    with pytest.raises(felbm.FelbmError):
        st.profile_enable(-1)
    st.close()
    mesh.close()


@pytest.mark.parametrize("path", ["lattice", "patch", "split", "tet"])
def test_uniform_state_is_stationary_on_every_path(path):
    """The degenerate case of no interface: a uniform density moving at a
    uniform velocity on a periodic mesh stays exactly that (no gradients, no
    force; the collision returns the equilibria).  FP64, 50 steps, every
    kernel path: the structured lattice step, the general patch and
    four-launch steps, and the tetrahedral lattice."""
    prm = configs.params(rho_l=1.0, rho_v=0.1, dt=0.4)
    if path == "tet":
        xy, tri, box, tag = inputs.structured_tet_mesh(8, 6, 5)
        prm = dict(prm, gravity=(0.0, 0.0, 0.0))
        u = np.tile([0.02, -0.01, 0.015], (len(xy), 1))
    elif path == "lattice":
        xy, tri, box, tag = inputs.structured_mesh(40, 24)
        u = np.tile([0.02, -0.01], (len(xy), 1))
    else:
        xy, tri, box, tag = inputs.jittered_delaunay_mesh(24, 20, 0.25, seed=6)
        u = np.tile([0.02, -0.01], (len(xy), 1))
    rho0 = np.full(len(xy), 0.55)
    mesh = felbm.Mesh(xy, tri, box, tag, general=path in ("patch", "split"), split_step=path == "split",
                      patch_step=path == "patch")
    st = felbm.State(mesh, felbm.make_params(precision="fp64", **prm), rho0, u, np.zeros(len(xy)))
    st.step(50)
    m = st.moments()
    st.close()
    mesh.close()
    assert np.abs(m["rho"] - 0.55).max() <= 1e-13
    assert np.abs(m["u"] - u).max() <= 1e-13
    assert np.abs(m["p"] - m["p"].mean()).max() <= 1e-13
