"""Allocation-free totals entry point (felbm_totals_nalloc) against the
library's own totals (felbm_moments_get), through the C ABI.

Collected last on purpose: a failure here leaves every other test already
run.  The caller owns every device buffer (PyTorch allocates them); the entry
point itself allocates nothing.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1608_01906_gb300 import configs, felbm

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1608_01906_gb300 import build

    build.build()
    lib = felbm.load()
    lib.felbm_totals_nalloc.restype = C.c_int
    lib.felbm_totals_nalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]
    return lib


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nalloc_totals_match_library_totals_twice(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    lib = _lib()
    # unit structured mesh: every lumped nodal mass is exactly 1, so unit
    # weights reproduce the library's mass-weighted totals
    prob = configs.droplet_structured(48, 12.0, 10.0, precision=precision)
    prob.u0[:, 0] = 0.01
    prob.u0[:, 1] = -0.02
    mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag)
    st = felbm.State(mesh, felbm.make_params(precision=precision, **prob.params), prob.rho0,
                     prob.u0, prob.p0)
    dt = torch.float64 if precision == "fp64" else torch.float32
    code = felbm.FELBM_FP64 if precision == "fp64" else felbm.FELBM_FP32
    stream = torch.cuda.current_stream()
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):  # two calls in a row, on different inputs
        st.step(7)
        m = st.moments()
        ref = m["totals"]
        rho = torch.tensor(m["rho"], dtype=dt, device="cuda")
        ux = torch.tensor(m["u"][:, 0], dtype=dt, device="cuda")
        uy = torch.tensor(m["u"][:, 1], dtype=dt, device="cuda")
        rc = lib.felbm_totals_nalloc(rho.data_ptr(), ux.data_ptr(), uy.data_ptr(), None,
                                     prob.n_nodes, code, out.data_ptr(), stream.cuda_stream)
        assert rc == felbm.FELBM_OK, felbm.status_string(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref).max()), (call, got, ref)
    st.close()
    mesh.close()


def test_nalloc_weighted_totals_on_delaunay_mesh_twice():
    """The weighted form, with the lumped nodal mass of a jittered Delaunay
    mesh as the weight (masses 0.6-1.4): against the library's own totals
    and against a host sum of w rho, w rho ux, w rho uy, on two calls in a
    row with different fields."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from oracle.oracle import Oracle, Params
    from paper_1608_01906_gb300 import inputs

    lib = _lib()
    xy, tri, box, tag = inputs.jittered_delaunay_mesh(40, 36, 0.25, seed=21)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (20, 18), 10.0, 1.0, 0.1, 4.0,
                                         u0=(0.012, -0.007))
    prm = configs.params(dt=0.4)
    mass = Oracle(xy, tri, box, tag, Params(**prm)).mass  # caller order
    assert mass.min() < 0.8 and mass.max() > 1.2
    mesh = felbm.Mesh(xy, tri, box, tag)
    st = felbm.State(mesh, felbm.make_params(precision="fp64", **prm), rho0, u0, p0)
    w = torch.tensor(mass, dtype=torch.float64, device="cuda")
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        st.step(5)
        m = st.moments()
        rho = torch.tensor(m["rho"], dtype=torch.float64, device="cuda")
        ux = torch.tensor(m["u"][:, 0], dtype=torch.float64, device="cuda")
        uy = torch.tensor(m["u"][:, 1], dtype=torch.float64, device="cuda")
        rc = lib.felbm_totals_nalloc(rho.data_ptr(), ux.data_ptr(), uy.data_ptr(), w.data_ptr(),
                                     len(mass), felbm.FELBM_FP64, out.data_ptr(),
                                     stream.cuda_stream)
        assert rc == felbm.FELBM_OK, felbm.status_string(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        mr = mass * m["rho"]
        host = np.array([mr.sum(), (mr * m["u"][:, 0]).sum(), (mr * m["u"][:, 1]).sum()])
        ref = np.asarray(m["totals"])
        assert np.all(np.abs(got - host) <= 1e-12 * np.abs(host)), (call, got, host)
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref)), (call, got, ref)
    st.close()
    mesh.close()


def test_nalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    lib = _lib()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for n in (0, -5, (1 << 30) + 1):
        rc = lib.felbm_totals_nalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), None, n,
                                     felbm.FELBM_FP64, out.data_ptr(), None)
        assert rc == felbm.FELBM_ERR_INVALID_ARG
