"""Von Neumann amplification of the oracle's streaming operator.

The lumped Taylor-Galerkin streaming (Sec. 2.2.1, Eq. galerkin_lbm) on the
structured split of a unit lattice is assembled column by column from the
oracle and its spectrum checked: at dt = 1 (Courant 1) the velocities that
cross the element diagonals are amplified 7x per step; dt = 0.5 is the
largest stable step (spectral radius 1); dt = 0.55 is already unstable.
This fixes the time-step reading of the unit-grid workloads.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, Params
from paper_1608_01906_gb300 import inputs


def spectral_radius(dt, e, n=12):
    xy, tri, box, tag = inputs.structured_mesh(n, n)
    o = Oracle(xy, tri, box, tag, Params(dt=dt))
    N = len(xy)
    A = np.empty((N, N))
    for j in range(N):
        v = np.zeros(N)
        v[j] = 1.0
        A[:, j] = o.stream(e, v)
    return np.abs(np.linalg.eigvals(A)).max()


@pytest.mark.parametrize("e", [(1, 0), (0, 1), (1, 1), (-1, 1), (1, -1)])
def test_half_courant_is_stable(e):
    assert spectral_radius(0.5, e) <= 1.0 + 1e-10


def test_unit_courant_diverges_across_element_diagonals():
    assert spectral_radius(1.0, (-1, 1)) == pytest.approx(7.0, rel=1e-9)
    assert spectral_radius(1.0, (1, 0)) > 1.2
    assert spectral_radius(0.55, (-1, 1)) > 1.3
