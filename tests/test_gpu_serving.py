"""Serving loop on the GPU: runs served together in the continuous batch give
exactly the results of the same runs stepped alone."""
import numpy as np
import pytest

from paper_1608_01906_gb300 import felbm, serving

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1608_01906_gb300 import build

    build.build()
    felbm.load()


def test_served_runs_equal_standalone_runs():
    reqs = serving.poisson_stream(7, rate=40.0, seed=5, side=(32, 96), steps=(40, 260))
    # room for about three of the runs at a time: later arrivals queue
    budget = 3 * (serving.run_bytes(96) + serving.mesh_bytes(96)) + serving.BATCH_FIXED_BYTES
    results, stats = serving.serve(reqs, budget, chunk=37)
    assert stats["completed"] == len(reqs)
    assert stats["p50_s"] is not None and stats["p99_s"] >= stats["p50_s"]
    by_id = {r.rid: r for r in results}
    for req in reqs:
        prob = serving.problem_for(req)
        mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag)
        st = felbm.State(mesh, felbm.make_params(precision="fp32", **prob.params), prob.rho0,
                         prob.u0, prob.p0)
        st.step(req.steps)
        alone = st.moments()
        mixed = by_id[req.rid].moments
        for k in ("rho", "u", "p"):
            assert np.array_equal(alone[k], mixed[k]), (req.rid, k)
        st.close()
        mesh.close()
