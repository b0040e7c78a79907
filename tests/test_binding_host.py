"""Host-side checks of the ctypes binding, against a fake library (no GPU):
the owning wrappers' arrays pass the binding's shape checks, and raw calls
whose arrays would be read or written past their end never reach the C
side."""
import ctypes as C
import types

import numpy as np
import pytest

from paper_1608_01906_gb300 import felbm


class FakeLib:
    """Records the C calls; a state's mesh reports n nodes of the given kind."""

    def __init__(self, n, kind):
        self.n, self.kind = n, kind
        self.calls = []

    def felbm_mesh_info(self, mesh, n, t, k, b):
        n._obj.value = self.n
        k._obj.value = self.kind
        return felbm.FELBM_OK

    def felbm_state_init(self, mesh, params, rho0, u0, p0, out):
        self.calls.append("init")
        out._obj.value = 0x1000
        return felbm.FELBM_OK

    def felbm_moments_get(self, *a):
        self.calls.append("moments")
        return felbm.FELBM_OK

    def felbm_state_export(self, *a):
        self.calls.append("export")
        return felbm.FELBM_OK

    def felbm_state_import(self, *a):
        self.calls.append("import")
        return felbm.FELBM_OK

    def felbm_state_destroy(self, s):
        self.calls.append("destroy")

    def felbm_status_string(self, st):
        return b"status"


@pytest.mark.parametrize("kind,dim,q", [(0, 2, 9), (1, 2, 9), (2, 3, 19), (3, 3, 19)])
def test_raw_calls_checked_against_the_state(monkeypatch, kind, dim, q):
    n = 12
    fake = FakeLib(n, kind)
    monkeypatch.setattr(felbm, "_lib", fake)
    mesh = types.SimpleNamespace(handle=C.c_void_p(0x2000), n_nodes=n, dim=dim, q=q)
    params = felbm.make_params(1.0, 0.1, 0.01, 4.0, 0.5, 0.5, 0.5)
    bad = felbm.FELBM_ERR_INVALID_ARG
    # mis-shaped initial fields never reach felbm_state_init
    for rho0, u0 in ((np.ones(n - 1), None), (np.ones(n), np.zeros((n, 5 - dim))), (np.ones((n, 2)), None)):
        st, _ = felbm.felbm_state_init(mesh.handle, params, rho0, u0)
        assert st == bad
    assert fake.calls == []
    s = felbm.State(mesh, params, np.ones(n), np.zeros((n, dim)), np.zeros(n))
    try:
        m = s.moments()
        assert m["u"].shape == (n, dim) and m["totals"].shape == (1 + dim,)
        h, g = s.export()
        assert h.shape == (q, n)
        s.import_(h, g)
        s.import_(h.ravel(), g.ravel())  # flat, q x n values: accepted
        assert fake.calls == ["init", "moments", "export", "import", "import"]
        raw = [
            felbm.felbm_moments_get(s.handle, rho=np.empty(n - 1)),
            felbm.felbm_moments_get(s.handle, rho=np.empty(n, dtype=np.float32)),
            felbm.felbm_moments_get(s.handle, u=np.empty((n, 5 - dim))),
            felbm.felbm_moments_get(s.handle, u=np.empty((dim, n))[:, :].T),  # not C-contiguous
            felbm.felbm_moments_get(s.handle, totals=np.empty(2 + dim)),
            felbm.felbm_state_export(s.handle, np.empty((q, n - 1)), np.empty((q, n))),
            felbm.felbm_state_export(s.handle, np.empty((q, n)), np.empty((28 - q, n))),
            felbm.felbm_state_import(s.handle, np.empty((q, n), dtype=np.float32), np.empty((q, n))),
        ]
        assert raw == [bad] * len(raw)
        with pytest.raises(felbm.FelbmError) as e:
            s.import_(np.empty((q, n + 1)), np.empty((q, n)))
        assert e.value.status == bad
        assert fake.calls == ["init", "moments", "export", "import", "import"]
    finally:
        s.close()
    assert fake.calls[-1] == "destroy" and 0x1000 not in felbm._STATE_SHAPES
