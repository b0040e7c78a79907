"""Failure detection of the bounded device waits, in the form that faults no
GPU: a block waits on an mbarrier that nothing arrives on, with a short time
limit; the wait gives up, records it in the state's flag and returns; the
host learns of it at the next synchronising call (FELBM_ERR_TIMEOUT), and the
context stays usable for other states and for the same state once new
distributions are imported."""
import time

import numpy as np
import pytest

from paper_1608_01906_gb300 import configs, felbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1608_01906_gb300 import build

    build.build()
    felbm.load()


def _state(prob, mesh):
    return felbm.State(mesh, felbm.make_params(precision="fp64", **prob.params), prob.rho0, prob.u0, prob.p0)


def test_bounded_wait_gives_up_and_is_reported():
    prob = configs.droplet_structured(n=64, R=16.0, steps=0, name="timeout_case")
    mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag)
    st, ok = _state(prob, mesh), _state(prob, mesh)
    try:
        st.step(3)
        st.sync()
        with pytest.raises(felbm.FelbmError) as bad:
            st.wait_selftest(0)
        assert bad.value.status == felbm.FELBM_ERR_INVALID_ARG
        t = time.perf_counter()
        st.wait_selftest(2_000_000)  # 2 ms
        with pytest.raises(felbm.FelbmError) as e:
            st.sync()
        assert e.value.status == felbm.FELBM_ERR_TIMEOUT
        assert time.perf_counter() - t < 1.0  # the limit, not the step's 2 s
        # the report stays until new distributions are loaded
        with pytest.raises(felbm.FelbmError) as e:
            st.moments()
        assert e.value.status == felbm.FELBM_ERR_TIMEOUT
        # the context is usable: another state steps as usual ...
        ok.step(3)
        m = ok.moments()
        assert np.all(np.isfinite(m["rho"])) and np.all(np.isfinite(m["u"]))
        # ... and the timed-out state runs again from imported distributions,
        # bitwise like the state it took them from
        h, g = ok.export()
        st.import_(h, g)
        st.step(2)
        ok.step(2)
        a, b = st.moments(), ok.moments()
        for k in ("rho", "u", "p"):
            assert np.array_equal(a[k], b[k]), k
    finally:
        st.close()
        ok.close()
        mesh.close()
