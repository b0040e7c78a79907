"""Halo-sharded structured lattices on one GPU: a lattice cut into slabs of
whole rows, each slab stepping its own rows and receiving 4 halo rows from
its neighbours after every step, reproduces the whole lattice's run
bitwise when the cuts are multiples of the tile height (8 rows), in FP64
and FP32, periodic and walled, with TMA and cp.async tiles; the FP64 run
matches the oracle at 1e-12; the slabs' FP64 totals add up to the whole
lattice's."""
import numpy as np
import pytest

from conftest import rel_l2
from oracle.oracle import Oracle, Params
from paper_1608_01906_gb300 import configs, felbm, inputs, sharding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1608_01906_gb300 import build

    build.build()
    felbm.load()


def droplet(nx, ny, precision):
    xy, tri, box, tag = inputs.structured_mesh(nx, ny)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (nx / 2 + 0.3, ny / 2 - 0.7), min(nx, ny) / 4, 1.0, 0.1, 4.0,
                                         u0=(0.01, -0.006))
    prm = dict(rho_l=1.0, rho_v=0.1, sigma=0.01, xi=4.0, tau_l=0.5, tau_v=0.5, dt=0.5, gravity=(0.0, 0.0))
    return xy, tri, box, tag, rho0, u0, p0, prm


def rayleigh_taylor(nx, ny):
    p = configs.c3_rayleigh_taylor(nx=nx, ny=ny, steps=0, ref_width=512)
    return p.xy, p.tri, p.box, p.tag, p.rho0, p.u0, p.p0, dict(p.params)


def whole_run(case, precision, steps):
    xy, tri, box, tag, rho0, u0, p0, prm = case
    mesh = felbm.Mesh(xy, tri, box, tag)
    st = felbm.State(mesh, felbm.make_params(precision=precision, **prm), rho0, u0, p0)
    st.step(steps)
    m, hg = st.moments(), st.export()
    st.close()
    mesh.close()
    return m, hg


def sharded_run(case, nx, ny, precision, steps, rows):
    xy, tri, box, tag, rho0, u0, p0, prm = case
    run = sharding.SlabRun(xy, tri, box, tag, nx, ny, felbm.make_params(precision=precision, **prm), rho0, u0,
                           p0, rows=rows)
    try:
        run.step(steps)
        run.sync()
        return run.moments(), run.export()
    finally:
        run.close()


def assert_bitwise(a, b):
    (ma, (ha, ga)), (mb, (hb, gb)) = a, b
    for k in ("rho", "C", "u", "p"):
        assert np.array_equal(ma[k], mb[k]), k
    assert np.array_equal(ha, hb) and np.array_equal(ga, gb)
    assert np.allclose(ma["totals"], mb["totals"], rtol=1e-12, atol=1e-12 * abs(mb["totals"][0]))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n_slabs", [1, 2, 3])
def test_periodic_slabs_equal_whole_lattice_bitwise(precision, n_slabs):
    nx, ny = 96, 96  # x tiles with and without TMA, 12 tile rows
    case = droplet(nx, ny, precision)
    whole = whole_run(case, precision, 12)
    part = sharded_run(case, nx, ny, precision, 12, sharding.slab_rows(ny, n_slabs))
    assert_bitwise(part, whole)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_walled_slabs_equal_whole_lattice_bitwise(precision):
    nx, ny = 80, 128
    case = rayleigh_taylor(nx, ny)
    whole = whole_run(case, precision, 15)
    part = sharded_run(case, nx, ny, precision, 15, [(0, 40), (40, 48), (88, 40)])
    assert_bitwise(part, whole)


def test_ragged_and_unaligned_slabs_match_whole_lattice():
    """Cuts off the tile grid (and a ragged last tile) change which tiles use
    the interior operators: same values up to rounding."""
    nx, ny = 64, 100
    case = droplet(nx, ny, "fp64")
    (mw, _), (mp, _) = whole_run(case, "fp64", 10), sharded_run(case, nx, ny, "fp64", 10, [(0, 37), (37, 30),
                                                                                            (67, 33)])
    for k in ("rho", "u", "p", "C"):
        assert rel_l2(mp[k], mw[k]) <= 1e-12, k


def test_sharded_fp64_matches_oracle_and_totals():
    nx, ny = 64, 96
    case = rayleigh_taylor(nx, ny)
    xy, tri, box, tag, rho0, u0, p0, prm = case
    m, _ = sharded_run(case, nx, ny, "fp64", 20, sharding.slab_rows(ny, 3))
    o = Oracle(xy, tri, box, tag, Params(**prm))
    o.init(rho0, u0, p0)
    o.step(20)
    r = {"rho": o.rho, "C": o.C, "u": np.stack([o.ux, o.uy], 1), "p": o.p}
    for k in ("rho", "C", "u", "p"):
        assert rel_l2(m[k], r[k]) <= 1e-12, k
    t = np.array(o.totals())
    assert np.allclose(m["totals"], t, rtol=1e-12, atol=1e-12 * abs(t[0]))


def test_slab_errors():
    nx, ny = 64, 64
    xy, tri, box, tag, rho0, u0, p0, prm = droplet(nx, ny, "fp64")
    whole = felbm.Mesh(xy, tri, box, tag)
    gen = felbm.Mesh(xy, tri, box, tag, general=True)
    try:
        with pytest.raises(felbm.FelbmError) as e:
            felbm.Mesh.slab(gen, 0, 32)
        assert e.value.status == felbm.FELBM_ERR_UNSUPPORTED
        for yb, nr in ((0, 7), (-8, 16), (56, 16)):
            with pytest.raises(felbm.FelbmError) as e:
                felbm.Mesh.slab(whole, yb, nr)
            assert e.value.status == felbm.FELBM_ERR_INVALID_ARG
        a, b = felbm.Mesh.slab(whole, 0, 32), felbm.Mesh.slab(whole, 32, 32)
        assert a.slab_info() == {"y_begin": 0, "n_rows": 32, "halo_bytes_fp32": 72 * 64 * 4}
        with pytest.raises(felbm.FelbmError):
            felbm.Mesh.slab(a, 8, 8)  # a slab of a slab
        prm_ = felbm.make_params(precision="fp64", **prm)
        rows = [sharding.storage_rows(0, 32, ny, False), sharding.storage_rows(32, 32, ny, False)]
        sa = felbm.State(a, prm_, sharding.slab_fields(rho0, nx, ny, rows[0]))
        sb = felbm.State(b, prm_, sharding.slab_fields(rho0, nx, ny, rows[1]))
        with pytest.raises(felbm.FelbmError) as e:
            felbm.slab_exchange([sb, sa])  # out of order
        assert e.value.status == felbm.FELBM_ERR_INVALID_ARG
        with pytest.raises(felbm.FelbmError) as e:
            felbm.slab_exchange([sa])  # does not cover the lattice
        assert e.value.status == felbm.FELBM_ERR_INVALID_ARG
        with pytest.raises(felbm.FelbmError) as e:
            felbm.Batch([sa, sb])
        assert e.value.status == felbm.FELBM_ERR_UNSUPPORTED
        send, recv, nb = sa.halo()
        assert nb == 72 * 64 * 8 and all(int(p) % 16 == 0 for p in send + recv)
        felbm.slab_exchange([sa, sb])
        sa.sync()
        sa.close()
        sb.close()
        a.close()
        b.close()
    finally:
        whole.close()
        gen.close()


def test_slabs_with_fp64_laplacian_term_equal_whole_lattice_bitwise():
    """FP32 slabs on the lattice kernel with the FP64 kappa lap rho term
    (FELBM_PARAM_LAP_FP64) reproduce the whole lattice's run with it."""
    nx, ny = 96, 64
    xy, tri, box, tag, rho0, u0, p0, prm = droplet(nx, ny, "fp32")
    params = felbm.make_params(precision="fp32", lap_fp64=True, **prm)
    mesh = felbm.Mesh(xy, tri, box, tag)
    st = felbm.State(mesh, params, rho0, u0, p0)
    st.step(10)
    whole = (st.moments(), st.export())
    st.close()
    mesh.close()
    run = sharding.SlabRun(xy, tri, box, tag, nx, ny, params, rho0, u0, p0, rows=sharding.slab_rows(ny, 2))
    try:
        run.step(10)
        part = (run.moments(), run.export())
    finally:
        run.close()
    assert_bitwise(part, whole)
