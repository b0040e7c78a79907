"""The five workloads' JSON descriptions (paper_1608_01906_gb300/workloads)
build the same problems as the builders they name, and the physical
parameters and sizes they record for the reader are the ones built."""
import json
import os

import numpy as np
import pytest

from paper_1608_01906_gb300 import configs, serving


def _doc(name):
    with open(os.path.join(configs.WORKLOAD_DIR, name + ".json")) as f:
        return json.load(f)


def _params_agree(recorded, built):
    for k, v in recorded.items():
        b = built[k]
        assert np.allclose(np.asarray(v, dtype=float), np.asarray(b, dtype=float), rtol=1e-12), (k, v, b)


@pytest.mark.parametrize("name", ["c1_static_droplet", "c2_unstructured_droplet", "c3_rayleigh_taylor"])
def test_single_problem_workloads(name):
    w = _doc(name)
    p = configs.load_workload(name)
    q = getattr(configs, w["builder"])(**w["args"])
    assert p.n_nodes == w["nodes"] == q.n_nodes
    assert p.steps == w["steps"] and p.precision == w["precision"]
    assert np.array_equal(p.xy, q.xy) and np.array_equal(p.tri, q.tri) and np.array_equal(p.rho0, q.rho0)
    _params_agree(w["params"], p.params)


def test_batched_workload():
    w = _doc("c4_batched")
    probs = configs.load_workload("c4_batched")
    assert len(probs) == w["meshes"] == 64
    for p in probs:
        assert p.precision == w["precision"]
        _params_agree(w["params"], p.params)
        assert 1.0 / 1000.0 - 1e-12 <= p.params["rho_v"] <= 0.1 + 1e-12


def test_serving_workload():
    w = _doc("c5_serving")
    with pytest.raises(ValueError):
        configs.load_workload("c5_serving")
    reqs = configs.load_workload("c5_serving", capacity_mnups=17000.0)
    assert len(reqs) == w["requests"]
    a = w["args"]
    assert all(a["side"][0] <= r.side <= a["side"][1] and a["steps"][0] <= r.steps <= a["steps"][1] for r in reqs)
    # the same stream as the serving module draws for that rate and seed
    again = configs.load_workload(os.path.join(configs.WORKLOAD_DIR, "c5_serving.json"), capacity_mnups=17000.0)
    assert [(r.arrival, r.side, r.steps) for r in reqs] == [(r.arrival, r.side, r.steps) for r in again]
    assert isinstance(reqs[0], serving.Request)
