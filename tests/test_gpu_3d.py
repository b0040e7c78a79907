"""Three-dimensional path (D3Q19 on P1 tetrahedra, the paper's own setting)
against the 3-D FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 per field): FP64 GPU runs <= 1e-12 (sums in another
order only); FP32 after 1000 steps <= 1e-5 in u and 1e-6 in rho and C."""
import numpy as np
import pytest

from conftest import rel_l2
from oracle.oracle3d import Oracle3, Params3
from paper_1608_01906_gb300 import felbm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1608_01906_gb300 import build

    build.build()
    felbm.load()


def droplet(n=10, R=3.0, ratio=10.0, xi=3.0, u0=(0.01, -0.02, 0.005)):
    xyz, tet, box, tag = inputs.structured_tet_mesh(n, n, n)
    rho0, u, p0 = inputs.droplet_fields3(xyz, box, (n / 2, n / 2, n / 2), R, 1.0, 1.0 / ratio, xi,
                                         u0=u0)
    params = dict(rho_l=1.0, rho_v=1.0 / ratio, sigma=0.01, xi=xi, tau_l=0.5, tau_v=0.5, dt=0.5,
                  gravity=(0.0, 0.0, 0.0))
    return xyz, tet, box, None, rho0, u, p0, params


def channel(nz=17):
    xyz, tet, box, tag = inputs.structured_tet_mesh(3, 3, nz, periodic_z=False)
    a = (nz - 1) / 4.0
    rho0, u, p0 = inputs.slab_fields3(xyz, (nz - 1) / 2.0 - a, (nz - 1) / 2.0 + a, 1.0, 0.5, 3.0)
    params = dict(rho_l=1.0, rho_v=0.5, sigma=0.01, xi=3.0, tau_l=1.0, tau_v=0.5, dt=0.5,
                  gravity=(1e-5, 0.0, 0.0))
    return xyz, tet, box, tag, rho0, u, p0, params


def run_gpu(case, precision, steps, export=False, general=False):
    xyz, tet, box, tag, rho0, u0, p0, params = case
    mesh = felbm.Mesh(xyz, tet, box, tag, general=general)
    # the Kuhn lattice runs on the lattice kernels (kind 3) unless the CSR
    # path is forced (kind 2)
    assert mesh.info()["kind"] == (2 if general else 3)
    st = felbm.State(mesh, felbm.make_params(precision=precision, **params), rho0, u0, p0)
    st.step(steps)
    m = st.moments()
    hg = st.export() if export else None
    st.close()
    mesh.close()
    return m, hg


def run_oracle(case, steps):
    xyz, tet, box, tag, rho0, u0, p0, params = case
    o = Oracle3(xyz, tet, box, tag, Params3(**params))
    o.init(rho0, u0, p0)
    o.step(steps)
    return o


def errors(m, o):
    return {"rho": rel_l2(m["rho"], o.rho), "C": rel_l2(m["C"], o.C),
            "u": rel_l2(m["u"], o.u), "p": rel_l2(m["p"], o.p)}


@pytest.mark.parametrize("general", [False, True])
def test_fp64_droplet_matches_oracle(general):
    case = droplet()
    m, (h, g) = run_gpu(case, "fp64", 40, export=True, general=general)
    o = run_oracle(case, 40)
    e = errors(m, o)
    assert max(e.values()) <= 1e-12, e
    # stored populations, D3Q19 order, caller node order
    assert rel_l2(h.ravel(), o.h.ravel()) <= 1e-12 and rel_l2(g.ravel(), o.g.ravel()) <= 1e-12


@pytest.mark.parametrize("general", [False, True])
def test_fp64_walled_channel_matches_oracle(general):
    case = channel()
    m, _ = run_gpu(case, "fp64", 300, general=general)
    o = run_oracle(case, 300)
    e = errors(m, o)
    assert max(e["rho"], e["C"], e["u"]) <= 1e-12, e
    assert np.abs(m["p"] - o.p).max() <= 1e-13 * (1.0 / 3.0), np.abs(m["p"] - o.p).max()


def test_fp64_jittered_tetrahedra_match_oracle():
    """A periodic Kuhn lattice with every node jittered by up to 0.15 h:
    not a lattice any more (general CSR kernels, kind 2), element volumes
    and lumped masses differ from node to node.  Fields, stored populations
    and the FP64 totals sum m_i rho_i, sum m_i rho_i u_i (lumped mass
    sum |T|/4, Sec. 2.2.1) against the oracle."""
    xyz, tet, box, tag = inputs.jittered_tet_mesh(8, 8, 8, 0.15, seed=11)
    rho0, u, p0 = inputs.droplet_fields3(xyz, box, (4.0, 4.0, 4.0), 2.5, 1.0, 0.2, 3.0,
                                         u0=(0.01, -0.015, 0.02))
    params = dict(rho_l=1.0, rho_v=0.2, sigma=0.01, xi=3.0, tau_l=0.6, tau_v=0.5, dt=0.4,
                  gravity=(0.0, 0.0, 0.0))
    case = (xyz, tet, box, None, rho0, u, p0, params)
    mesh = felbm.Mesh(xyz, tet, box, None)
    assert mesh.info()["kind"] == 2
    st = felbm.State(mesh, felbm.make_params(precision="fp64", **params), rho0, u, p0)
    st.step(30)
    m = st.moments()
    h, g = st.export()
    st.close()
    mesh.close()
    o = run_oracle(case, 30)
    assert o.mass.min() < 0.9 and o.mass.max() > 1.1
    e = errors(m, o)
    assert max(e.values()) <= 1e-12, e
    assert rel_l2(h.ravel(), o.h.ravel()) <= 1e-12 and rel_l2(g.ravel(), o.g.ravel()) <= 1e-12
    got, want = np.asarray(m["totals"]), np.asarray(o.totals())
    assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want)), (got, want)


def test_fp64_totals_conserved():
    case = droplet(n=12, R=3.5)
    xyz, tet, box, tag, rho0, u0, p0, params = case
    mesh = felbm.Mesh(xyz, tet, box, tag)
    st = felbm.State(mesh, felbm.make_params(precision="fp64", **params), rho0, u0, p0)
    st.step(1)
    t0 = st.moments()["totals"]
    st.step(50)
    t1 = st.moments()["totals"]
    assert t1[0] == pytest.approx(t0[0], rel=1e-13)
    assert np.all(np.abs(t1[1:] - t0[1:]) <= 1e-13 * t0[0]), (t0, t1)
    st.close()
    mesh.close()


@pytest.mark.parametrize("general", [False, True])
def test_fp32_droplet_1000_steps(general):
    case = droplet(n=12, R=3.5, u0=(0.0, 0.0, 0.0))
    m, _ = run_gpu(case, "fp32", 1000, general=general)
    o = run_oracle(case, 1000)
    e = errors(m, o)
    print("3-D fp32 1000 steps", e)
    # measured: rho 2.1e-7, C 3.4e-7, u 1.2e-6, p 1.7e-6 (lattice kernels)
    assert e["rho"] <= 1e-6 and e["C"] <= 1e-6 and e["u"] <= 1e-5 and e["p"] <= 2e-5, e


def test_fp64_box_lattice_matches_oracle():
    """A lattice of unequal sides (16 x 8 x 12), off-centre drop."""
    xyz, tet, box, tag = inputs.structured_tet_mesh(16, 8, 12)
    rho0, u, p0 = inputs.droplet_fields3(xyz, box, (8.0, 4.0, 6.0), 3.0, 1.0, 0.2, 3.0,
                                         u0=(0.01, 0.02, -0.01))
    params = dict(rho_l=1.0, rho_v=0.2, sigma=0.01, xi=3.0, tau_l=0.6, tau_v=0.5, dt=0.5,
                  gravity=(0.0, 0.0, 0.0))
    m, _ = run_gpu((xyz, tet, box, None, rho0, u, p0, params), "fp64", 30)
    e = errors(m, run_oracle((xyz, tet, box, None, rho0, u, p0, params), 30))
    assert max(e.values()) <= 1e-12, e


def test_fp64_walled_slab_lattice_matches_oracle():
    """32 x 8 x 16 with z walls, a liquid slab under oblique gravity: blocks
    of the lattice kernels hold wall-layer and interior nodes together."""
    xyz, tet, box, tag = inputs.structured_tet_mesh(32, 8, 16, periodic_z=False)
    rho0, u, p0 = inputs.slab_fields3(xyz, 4.0, 11.0, 1.0, 0.1, 3.0)
    params = dict(rho_l=1.0, rho_v=0.1, sigma=0.01, xi=3.0, tau_l=0.7, tau_v=0.5, dt=0.5,
                  gravity=(2e-5, -1e-5, 0.0))
    case = (xyz, tet, box, tag, rho0, u, p0, params)
    m, _ = run_gpu(case, "fp64", 40)
    e = errors(m, run_oracle(case, 40))
    assert max(e["rho"], e["C"], e["u"]) <= 1e-12, e
    o = run_oracle(case, 40)
    assert np.abs(m["p"] - o.p).max() <= 1e-13 / 3.0


def test_lattice_detection():
    """Only the exact Kuhn lattice takes the lattice kernels; a moved node,
    a tag off the wall layers or a forced CSR path keep the general kernels."""
    xyz, tet, box, _ = inputs.structured_tet_mesh(5, 4, 6)
    assert felbm.Mesh(xyz, tet, box).info()["kind"] == 3
    assert felbm.Mesh(xyz, tet, box, general=True).info()["kind"] == 2
    moved = xyz.copy()
    moved[7] += (0.05, -0.03, 0.02)
    assert felbm.Mesh(moved, tet, box).info()["kind"] == 2
    xyz, tet, box, tag = inputs.structured_tet_mesh(4, 5, 7, periodic_z=False)
    assert felbm.Mesh(xyz, tet, box, tag).info()["kind"] == 3
    tag2 = tag.copy()
    tag2[len(tag2) // 2] = 5
    assert felbm.Mesh(xyz, tet, box, tag2).info()["kind"] == 2
    assert felbm.Mesh(xyz, tet, box, tag).info()["device_bytes"] < \
        felbm.Mesh(xyz, tet, box, tag, general=True).info()["device_bytes"]


def test_lattice_matches_csr_fp32():
    """Both topologies of the same walled lattice agree to FP32 rounding."""
    xyz, tet, box, tag = inputs.structured_tet_mesh(8, 6, 21, periodic_z=False)
    rho0, u, p0 = inputs.slab_fields3(xyz, 5.0, 15.0, 1.0, 0.1, 3.0)
    params = dict(rho_l=1.0, rho_v=0.1, sigma=0.01, xi=3.0, tau_l=0.8, tau_v=0.5, dt=0.5,
                  gravity=(1e-5, 2e-6, -1e-6))
    out = []
    for general in (False, True):
        mesh = felbm.Mesh(xyz, tet, box, tag, general=general)
        st = felbm.State(mesh, felbm.make_params(precision="fp32", **params), rho0, u, p0)
        st.step(200)
        out.append(st.moments())
        st.close()
        mesh.close()
    for k in ("rho", "C", "u"):
        assert rel_l2(out[0][k], out[1][k]) <= 2e-6, (k, rel_l2(out[0][k], out[1][k]))
    # p is O(1e-5) here: compare it on the c_s^2 scale
    assert np.abs(out[0]["p"] - out[1]["p"]).max() <= 1e-8 / 3.0


@pytest.mark.parametrize("general", [False, True])
def test_nonfinite_detected_3d(general):
    """An unstable time step blows the 3-D state up to inf/nan without a
    fault; the step's flag reports it."""
    xyz, tet, box, _ = inputs.structured_tet_mesh(8, 8, 8)
    rho0, u, p0 = inputs.droplet_fields3(xyz, box, (4.0, 4.0, 4.0), 2.5, 1.0, 0.25, 2.0)
    mesh = felbm.Mesh(xyz, tet, box, general=general)
    st = felbm.State(mesh, felbm.make_params(1.0, 0.25, 0.01, 2.0, 0.5, 0.5, 3.0, precision="fp32"),
                     rho0, u, p0)
    st.step(2000)
    assert felbm.felbm_state_sync(st.handle) == felbm.FELBM_ERR_NONFINITE
    st.close()
    mesh.close()


def test_batch_rejects_tetrahedral_states():
    xyz, tet, box, _ = inputs.structured_tet_mesh(6, 6, 6)
    rho0, u, p0 = inputs.droplet_fields3(xyz, box, (3.0, 3.0, 3.0), 2.0, 1.0, 0.5, 2.0)
    mesh = felbm.Mesh(xyz, tet, box)
    st = felbm.State(mesh, felbm.make_params(1.0, 0.5, 0.01, 2.0, 0.5, 0.5, 0.5, precision="fp32"),
                     rho0, u, p0)
    with pytest.raises(felbm.FelbmError) as exc:
        felbm.Batch([st])
    assert exc.value.status == felbm.FELBM_ERR_UNSUPPORTED
    st.close()
    mesh.close()
