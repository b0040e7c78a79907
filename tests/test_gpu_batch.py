"""Batched launch: every state's result equals its stand-alone run exactly,
and the FP64 batch matches the oracle."""
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


def mixed_problems():
    probs = [configs.droplet_structured(40, 10.0, 10.0, xi=4.0),
             configs.droplet_structured(64, 20.0, 300.0, xi=configs.DROPLET_XI, tau_l=0.1, tau_v=0.1),
             configs.droplet_structured(33, 9.0, 1000.0, xi=configs.DROPLET_XI, tau_l=0.1, tau_v=0.1)]
    rt = configs.c3_rayleigh_taylor(nx=48, ny=100)
    probs.append(rt)
    xy, tri, box, tag = inputs.structured_mesh(70, 45)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (30, 20), 12.0, 1.0, 0.1, 4.0, u0=(0.02, -0.01))
    probs.append(configs.Problem("moving", xy, tri, box, tag, rho0, u0, p0, configs.params(), 0,
                                 "fp32"))
    return probs


def make_state(prob, precision):
    mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag)
    st = felbm.State(mesh, felbm.make_params(precision=precision, **prob.params), prob.rho0,
                     prob.u0, prob.p0)
    return mesh, st


def periodic_problems():
    # periodic unit lattices with one dt: every mesh has the same coefficient
    # tables, which the batched kernels then take as kernel parameters
    return [configs.droplet_structured(40, 10.0, 10.0, xi=4.0),
            configs.droplet_structured(64, 20.0, 300.0, xi=configs.DROPLET_XI, tau_l=0.1, tau_v=0.1),
            configs.droplet_structured(33, 9.0, 1000.0, xi=configs.DROPLET_XI, tau_l=0.1, tau_v=0.1),
            configs.droplet_structured(97, 30.0, 50.0, xi=configs.DROPLET_XI, tau_l=0.2, tau_v=0.1)]


def walled_problems():
    # Rayleigh-Taylor layers of different sizes with one dt: shared tables
    # whose wall-row kinds are read at run time
    return [configs.c3_rayleigh_taylor(nx=48, ny=100), configs.c3_rayleigh_taylor(nx=48, ny=64),
            configs.c3_rayleigh_taylor(nx=48, ny=41)]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("which", ["mixed", "periodic", "walled"])
def test_batch_equals_standalone_bitwise(precision, which):
    probs = {"mixed": mixed_problems, "periodic": periodic_problems, "walled": walled_problems}[which]()
    alone = []
    for p in probs:
        mesh, st = make_state(p, precision)
        st.step(121)
        alone.append(st.moments())
        st.close()
        mesh.close()
    pairs = [make_state(p, precision) for p in probs]
    batch = felbm.Batch([st for _, st in pairs], autotune=True)
    batch.step(60)
    batch.step(61)
    batch.sync()
    info = batch.info()
    assert info["n_tiles"] > 0 and info["launches"] >= 121
    for (mesh, st), ref in zip(pairs, alone):
        got = st.moments()
        for k in ("rho", "u", "p"):
            assert np.array_equal(got[k], ref[k]), k
    batch.close()


def test_batch_fp64_matches_oracle():
    probs = mixed_problems()[:2]
    pairs = [make_state(p, "fp64") for p in probs]
    batch = felbm.Batch([st for _, st in pairs], autotune=False)
    batch.step(40)
    for p, (mesh, st) in zip(probs, pairs):
        o = Oracle(p.xy, p.tri, p.box, p.tag, Params(**p.params))
        o.init(p.rho0, p.u0, p.p0)
        o.step(40)
        m = st.moments()
        assert rel_l2(m["rho"], o.rho) <= 1e-12
        assert rel_l2(m["u"], np.stack([o.ux, o.uy], 1)) <= 1e-12
        assert rel_l2(m["p"], o.p) <= 1e-12
    batch.close()


def test_member_stepped_alone_between_batch_steps():
    probs = mixed_problems()[:3]
    ref = []
    for p in probs:
        mesh, st = make_state(p, "fp32")
        st.step(30)
        ref.append(st.moments())
    pairs = [make_state(p, "fp32") for p in probs]
    batch = felbm.Batch([st for _, st in pairs], autotune=False)
    batch.step(10)
    pairs[1][1].step(7)  # one member alone
    batch.step(13)
    # members 0 and 2 have 23 steps, member 1 has 30: finish 0 and 2 alone
    pairs[0][1].step(7)
    pairs[2][1].step(7)
    for (mesh, st), r in zip(pairs, ref):
        got = st.moments()
        assert np.array_equal(got["rho"], r["rho"]) and np.array_equal(got["u"], r["u"])
    batch.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_tile_walk_equals_standalone_bitwise(precision):
    # 2304 tiles, several per block at any blocks-per-SM the autotuner tries
    # (except one block per tile): blocks claim tiles from the launch's
    # counter and load the next tile's halo early when it is on the same
    # mesh; walled (interior TMA tiles) and periodic meshes, mesh changes
    # between claimed tiles
    probs = [configs.c3_rayleigh_taylor(nx=512, ny=1024),
             configs.droplet_structured(256, 80.0, 100.0, xi=configs.DROPLET_XI, tau_l=0.1,
                                        tau_v=0.1),
             configs.droplet_structured(130, 40.0, 10.0, xi=4.0)]
    alone = []
    for p in probs:
        mesh, st = make_state(p, precision)
        st.step(9)
        alone.append(st.moments())
        st.close()
        mesh.close()
    pairs = [make_state(p, precision) for p in probs]
    batch = felbm.Batch([st for _, st in pairs], autotune=False)
    batch.step(9)
    batch.sync()
    for (mesh, st), ref in zip(pairs, alone):
        got = st.moments()
        for k in ("rho", "u", "p"):
            assert np.array_equal(got[k], ref[k]), k
    batch.close()
