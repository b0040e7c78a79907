"""Droplet translation (Sec. 3.2, 2-D): a drop carried by a uniform velocity
through a periodic box, GPU path.

* parity: the translating drop against the FP64 oracle, element by element;
* Galilean invariance (a property of the model, no stored values): after
  exactly one period the carried drop coincides with the same drop relaxed
  at rest for the same time, up to the scheme's error.
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


def drop(L, U, ratio, xi, tau_l=0.5, tau_v=0.5):
    xy, tri, box, tag = inputs.structured_mesh(L, L)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (L / 2, L / 2), L / 4, 1.0, 1.0 / ratio, xi,
                                         u0=(U, 0.0))
    return configs.Problem("drop", xy, tri, box, tag, rho0, u0, p0,
                           configs.params(1.0, 1.0 / ratio, 0.01, xi, tau_l, tau_v, 0.5), 0, "fp64")


def run(prob, precision, steps):
    mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag)
    st = felbm.State(mesh, felbm.make_params(precision=precision, **prob.params), prob.rho0,
                     prob.u0, prob.p0)
    st.step(steps)
    m = st.moments()
    st.close()
    mesh.close()
    return m


def test_translation_parity_fp64():
    prob = drop(32, 0.02, 10.0, 4.0)
    m = run(prob, "fp64", 400)
    o = Oracle(prob.xy, prob.tri, prob.box, prob.tag, Params(**prob.params))
    o.init(prob.rho0, prob.u0, prob.p0)
    o.step(400)
    assert rel_l2(m["rho"], o.rho) <= 1e-12
    assert rel_l2(m["u"], np.stack([o.ux, o.uy], 1)) <= 1e-12
    assert rel_l2(m["p"], o.p) <= 1e-12


def invariance_error(L, U, ratio, xi, precision, **kw):
    """max |rho_carried - rho_at_rest| / (rho_l - rho_v) after one period."""
    steps = int(round(L / U / 0.5))
    moving = run(drop(L, U, ratio, xi, **kw), precision, steps)
    rest = run(drop(L, 0.0, ratio, xi, **kw), precision, steps)
    return np.abs(moving["rho"] - rest["rho"]).max() / (1.0 - 1.0 / ratio)


def test_galilean_invariance():
    # after one period the carried drop matches the drop at rest (the FP64
    # oracle reaches 1.7% on the 32 x 32 box, 17% with the equilibrium's
    # second-order velocity terms dropped); 64 x 64 with the interface
    # resolved by twice the nodes
    e32 = invariance_error(32, 0.02, 10.0, 4.0, "fp64")
    e64 = invariance_error(64, 0.02, 10.0, 8.0, "fp64")
    print("invariance error ratio 10: L32 %.4g L64 %.4g" % (e32, e64))
    assert e32 < 0.03 and e64 < 0.03


def test_galilean_invariance_ratio_1000():
    # the paper's contrasts: density 1000, kinematic viscosity 60 (vapour
    # tau 60x the liquid's), FP32, 128 x 128 (xi 24): 0.33% measured
    e = invariance_error(128, 0.02, 1000.0, configs.DROPLET_XI, "fp32", tau_l=0.005,
                         tau_v=0.3)
    print("invariance error ratio 1000: L128 %.4g" % e)
    assert e < 0.01
