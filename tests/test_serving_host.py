"""Host-side logic of the serving loop (no GPU): the request stream and the
scheduler's admission, chunking and retirement, with the device calls faked."""
import numpy as np
import pytest

from paper_1608_01906_gb300 import serving


def test_poisson_stream_is_seeded_and_in_range():
    a = serving.poisson_stream(2000, rate=5.0, seed=1610)
    b = serving.poisson_stream(2000, rate=5.0, seed=1610)
    assert [(r.arrival, r.side, r.steps) for r in a] == [(r.arrival, r.side, r.steps) for r in b]
    sides = np.array([r.side for r in a])
    assert sides.min() >= 64 and sides.max() <= 1024
    steps = np.array([r.steps for r in a])
    assert steps.min() >= 1000 and steps.max() <= 20000
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert abs(gaps.mean() - 0.2) < 0.02  # mean inter-arrival 1 / rate


class FakeState:
    def __init__(self, *a, **k):
        self.closed = False

    def moments(self):
        return {"rho": np.zeros(1), "totals": np.array([1.0, 0.0, 0.0])}

    def close(self):
        self.closed = True


class FakeMesh(FakeState):
    def info(self):
        return {"device_bytes": serving.mesh_bytes(64)}


class FakeBatch:
    log = []

    def __init__(self, states, autotune=True):
        self.n = len(states)

    def step(self, n):
        FakeBatch.log.append((self.n, n))

    def sync(self):
        pass

    def close(self):
        pass


def test_scheduler_budget_chunks_and_retirement(monkeypatch):
    monkeypatch.setattr(serving.felbm, "Mesh", FakeMesh)
    monkeypatch.setattr(serving.felbm, "State", FakeState)
    monkeypatch.setattr(serving.felbm, "Batch", FakeBatch)
    monkeypatch.setattr(serving, "problem_for", lambda req: type(
        "P", (), {"xy": None, "tri": None, "box": None, "tag": None, "rho0": None, "u0": None,
                  "p0": None, "params": {"rho_l": 1.0, "rho_v": 0.1, "sigma": 0.01, "xi": 4.0,
                                         "tau_l": 0.1, "tau_v": 0.1, "dt": 0.5,
                                         "gravity": (0.0, 0.0)}})())
    FakeBatch.log = []
    reqs = [serving.Request(k, 0.0, 64, 10.0, 0.3, s) for k, s in enumerate([100, 250, 60, 300])]
    # two runs at a time: their states and batch shares, the shared mesh and
    # the batch's fixed part
    budget = 2 * serving.run_bytes(64) + serving.mesh_bytes(64) + serving.BATCH_FIXED_BYTES
    results, stats = serving.serve(reqs, budget, chunk=80, autotune=False)
    assert stats["completed"] == 4
    # never more than two runs in a launch, chunk never above 80 nor past a finish
    assert max(n for n, _ in FakeBatch.log) == 2
    assert all(c <= 80 for _, c in FakeBatch.log)
    done = {r.rid: r.steps for r in results}
    assert done == {0: 100, 1: 250, 2: 60, 3: 300}
    # total node-steps equal the requested work
    assert sum(n * c for n, c in FakeBatch.log) == 100 + 250 + 60 + 300


def test_diverged_run_is_retired_and_the_rest_finish(monkeypatch):
    """A run whose fields go non-finite is retired as diverged at the chunk
    where the batch reports it; the other runs carry on to their step count."""
    class DState(FakeState):
        count = 0

        def __init__(self, *a, **k):
            super().__init__()
            self.handle = DState.count
            DState.count += 1

    class DBatch(FakeBatch):
        def __init__(self, states, autotune=True):
            super().__init__(states, autotune)
            self.handles = [s.handle for s in states]
            self.steps = 0

        def step(self, n):
            super().step(n)
            self.steps += n

        def sync(self):
            if 1 in self.handles and DBatch.total + self.steps >= 120:
                raise serving.felbm.FelbmError(serving.felbm.FELBM_ERR_NONFINITE, "sync")

        def close(self):
            DBatch.total += self.steps

    DBatch.total = 0
    monkeypatch.setattr(serving.felbm, "Mesh", FakeMesh)
    monkeypatch.setattr(serving.felbm, "State", DState)
    monkeypatch.setattr(serving.felbm, "Batch", DBatch)
    monkeypatch.setattr(serving.felbm, "felbm_state_sync",
                        lambda h: serving.felbm.FELBM_ERR_NONFINITE if h == 1 else 0)
    monkeypatch.setattr(serving, "problem_for", lambda req: type(
        "P", (), {"xy": None, "tri": None, "box": None, "tag": None, "rho0": None, "u0": None,
                  "p0": None, "params": {"rho_l": 1.0, "rho_v": 0.1, "sigma": 0.01, "xi": 4.0,
                                         "tau_l": 0.1, "tau_v": 0.1, "dt": 0.5,
                                         "gravity": (0.0, 0.0)}})())
    FakeBatch.log = []
    reqs = [serving.Request(k, 0.0, 64, 10.0, 0.3, s) for k, s in enumerate([300, 400, 200])]
    budget = 3 * serving.run_bytes(64) + serving.mesh_bytes(64) + serving.BATCH_FIXED_BYTES
    results, stats = serving.serve(reqs, budget, chunk=40, autotune=False)
    by = {r.rid: r for r in results}
    assert stats["completed"] == 2 and stats["diverged"] == 1
    assert by[1].status == "diverged" and by[1].steps == 120 and by[1].moments == {}
    assert by[0].status == "ok" and by[0].steps == 300
    assert by[2].status == "ok" and by[2].steps == 200


def test_budget_counts_meshes_and_batch_memory(monkeypatch):
    """Admission counts each mesh once per side (while a run uses it) and the
    batch's own memory; the count returns to zero when every run retired."""
    monkeypatch.setattr(serving.felbm, "Mesh", FakeMesh)
    monkeypatch.setattr(serving.felbm, "State", FakeState)
    monkeypatch.setattr(serving, "problem_for", lambda req: type(
        "P", (), {"xy": None, "tri": None, "box": None, "tag": None, "rho0": None, "u0": None,
                  "p0": None, "params": {"rho_l": 1.0, "rho_v": 0.1, "sigma": 0.01, "xi": 4.0,
                                         "tau_l": 0.1, "tau_v": 0.1, "dt": 0.5,
                                         "gravity": (0.0, 0.0)}})())
    one = serving.run_bytes(64) + serving.mesh_bytes(64) + serving.BATCH_FIXED_BYTES
    srv = serving.Server(one + serving.run_bytes(64) - 1, autotune=False)
    a, b = (serving.Request(k, 0.0, 64, 10.0, 0.3, 100) for k in range(2))
    assert srv.need(a) == one and srv.fits(a)
    srv.admit(a, 0.0)
    assert srv.used == one
    # a second run on the same side shares the mesh and the batch: one byte short
    assert srv.need(b) == serving.run_bytes(64) and not srv.fits(b)
    srv.active[0]["done"] = 100
    srv.retire_finished(1.0)
    assert srv.used == 0 and not srv.meshes


def test_mass_drift_is_measured_and_flagged(monkeypatch):
    """Each completed run reports the relative change of its FP64 mass total
    from admission to completion; runs beyond MASS_DRIFT_TOL are counted."""
    class MState(FakeState):
        count = 0

        def __init__(self, *a, **k):
            super().__init__()
            self.rid = MState.count
            MState.count += 1
            self.calls = 0

        def moments(self):
            self.calls += 1
            drift = 3e-5 if (self.rid == 1 and self.calls > 1) else 0.0
            return {"rho": np.zeros(1), "totals": np.array([2.0 * (1.0 + drift), 0.0, 0.0])}

    monkeypatch.setattr(serving.felbm, "Mesh", FakeMesh)
    monkeypatch.setattr(serving.felbm, "State", MState)
    monkeypatch.setattr(serving.felbm, "Batch", FakeBatch)
    monkeypatch.setattr(serving, "problem_for", lambda req: type(
        "P", (), {"xy": None, "tri": None, "box": None, "tag": None, "rho0": None, "u0": None,
                  "p0": None, "params": {"rho_l": 1.0, "rho_v": 0.1, "sigma": 0.01, "xi": 4.0,
                                         "tau_l": 0.1, "tau_v": 0.1, "dt": 0.5,
                                         "gravity": (0.0, 0.0)}})())
    reqs = [serving.Request(k, 0.0, 64, 10.0, 0.3, 50) for k in range(3)]
    budget = 3 * serving.run_bytes(64) + serving.mesh_bytes(64) + serving.BATCH_FIXED_BYTES
    results, stats = serving.serve(reqs, budget, chunk=50, autotune=False)
    by = {r.rid: r for r in results}
    assert stats["completed"] == 3
    assert by[1].mass_drift == pytest.approx(3e-5) and by[0].mass_drift == 0.0
    assert stats["mass_drift_flagged"] == 1 and stats["max_mass_drift"] == pytest.approx(3e-5)
