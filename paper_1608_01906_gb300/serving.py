"""Continuous-batching server for binary-fluid runs.

Requests (a droplet run: mesh side, density ratio, radius, step count)
arrive as a Poisson stream.  The server keeps every admitted run's state
resident in HBM and advances all of them together with one batched launch
per time step (``felbm_batch_*``).  Between chunks of steps it

* retires runs that reached their step count (their moments are read back
  and the state is freed),
* admits arrived requests while the HBM budget allows (the mesh of a side is
  shared by every run on it),
* rebuilds the batch when its membership changed,
* retires a run whose fields went non-finite as ``diverged`` (its state's
  own flag says which run it was) while the others carry on.

A run's result does not depend on which other runs shared its launches (the
batched kernel runs the same per-node arithmetic as a stand-alone step), so
a run served in the mix equals the same run stepped alone.

All numerical work happens in ``libfelbm.so``; this module only schedules.
"""
from __future__ import annotations

import heapq
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import configs, felbm


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the stream starts
    side: int
    ratio: float
    radius_frac: float
    steps: int

    @property
    def nodes(self):
        return self.side * self.side


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    nodes: int
    moments: dict
    status: str = "ok"      # "ok" or "diverged"
    mass_drift: float = 0.0  # |M_end - M_0| / M_0 of the FP64 mass total (completed runs)

    @property
    def latency(self):
        return self.finished - self.arrival


def poisson_stream(n, rate, seed=1610, side=(64, 1024), ratio=(10.0, 1000.0),
                   steps=(1000, 20000), radius=(0.2, 0.35)):
    """n requests, exponential inter-arrival times of mean 1/rate, sides
    log-uniform, ratio and radius uniform, steps uniform (integers)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n):
        t += rng.exponential(1.0 / rate)
        s = int(round(math.exp(rng.uniform(math.log(side[0]), math.log(side[1])))))
        out.append(Request(k, t, s, float(rng.uniform(*ratio)), float(rng.uniform(*radius)),
                           int(rng.integers(steps[0], steps[1] + 1))))
    return out


def state_bytes(side, precision="fp32"):
    """Device bytes of one run: 2 x 18 populations, 6 scalar fields, 4
    moments, 5 FP64 output fields (felbm_state_init)."""
    es = 4 if precision == "fp32" else 8
    n = side * side
    return n * (36 * es + 6 * es + 4 * es + 5 * 8)


def mesh_bytes(side):
    """Device bytes of a structured side x side mesh before it exists: the
    FP64 lumped mass (structured meshes hold no assembled arrays).  Once the
    mesh is created its own count (felbm_mesh_info) replaces this."""
    return side * side * 8


# Batch memory outside the states and meshes: per run a share of the tile
# list (one 16-byte record per 32 x 8 tile), its descriptor and its 768
# bytes of tensor maps; per batch the launch counters and the autotuner's
# buffers.
BATCH_RUN_BYTES = 4096
BATCH_FIXED_BYTES = 1 << 20


def run_bytes(side, precision="fp32"):
    """Device bytes a run adds to a batch besides its mesh."""
    return state_bytes(side, precision) + (side * side // 256 + 1) * 16 + BATCH_RUN_BYTES


def problem_for(req: Request):
    return configs.droplet_structured(req.side, req.radius_frac * req.side, req.ratio,
                                      configs.DROPLET_XI, 0.01,
                                      0.1, 0.1, 0.5, req.steps, "fp32", "req%d" % req.rid)


class Server:
    """Admission by HBM budget, slot-based continuous batching."""

    def __init__(self, budget_bytes, precision="fp32", chunk=200, stream=None, autotune=True):
        self.budget = int(budget_bytes)
        self.precision = precision
        self.chunk = int(chunk)
        self.stream = stream
        self.autotune = autotune
        self.meshes = {}   # side -> (Mesh, users)
        self.active = []   # dicts: req, state, done, admitted
        self.used = 0
        self.fixed_held = False
        self.batch = None
        self.dirty = True
        self.results = []
        self.node_steps = 0
        self.t0 = time.perf_counter()

    # ---- resources ----------------------------------------------------
    def _mesh(self, req):
        ent = self.meshes.get(req.side)
        if ent is None:
            prob = problem_for(req)
            m = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag, stream=self.stream)
            ent = [m, 0, int(m.info()["device_bytes"])]
            self.meshes[req.side] = ent
            self.used += ent[2]
        ent[1] += 1
        return ent[0]

    def _release_mesh(self, side):
        ent = self.meshes[side]
        ent[1] -= 1
        if ent[1] == 0:
            ent[0].close()
            self.used -= ent[2]
            del self.meshes[side]

    def need(self, req):
        """Device bytes admitting req would add: the run, its mesh when no
        active run shares that side, and the batch's fixed part when the
        batch is empty."""
        b = run_bytes(req.side, self.precision)
        if req.side not in self.meshes:
            b += mesh_bytes(req.side)
        if not self.fixed_held:
            b += BATCH_FIXED_BYTES
        return b

    def _release_fixed(self):
        # the batch's fixed part goes with its last run
        if self.fixed_held and not self.active:
            self.used -= BATCH_FIXED_BYTES
            self.fixed_held = False

    def fits(self, req):
        return self.used + self.need(req) <= self.budget

    def admit(self, req, now):
        prob = problem_for(req)
        if not self.fixed_held:
            self.used += BATCH_FIXED_BYTES
            self.fixed_held = True
        mesh = self._mesh(req)
        st = felbm.State(mesh, felbm.make_params(precision=self.precision, **prob.params),
                         prob.rho0, prob.u0, prob.p0)
        self.used += run_bytes(req.side, self.precision)
        # the FP64 mass total at admission, for the mass-drift check at the end
        mass0 = float(st.moments()["totals"][0])
        self.active.append({"req": req, "state": st, "done": 0, "admitted": now, "mass0": mass0})
        self.dirty = True

    def _retire(self, slot, now, status="ok"):
        req = slot["req"]
        m = slot["state"].moments() if status == "ok" else {}
        drift = abs(float(m["totals"][0]) - slot["mass0"]) / abs(slot["mass0"]) if m else 0.0
        self.results.append(Result(req.rid, req.arrival, slot["admitted"], now, slot["done"],
                                   req.nodes, m, status, drift))
        slot["state"].close()
        self._release_mesh(req.side)
        self.used -= run_bytes(req.side, self.precision)
        self.dirty = True

    # ---- stepping -----------------------------------------------------
    def advance(self):
        """One chunk: every active run advances min(chunk, least remaining)."""
        if not self.active:
            return 0
        if self.dirty:
            if self.batch is not None:
                self.batch.close()
            self.batch = felbm.Batch([s["state"] for s in self.active], autotune=self.autotune)
            self.dirty = False
        n = min(self.chunk, min(s["req"].steps - s["done"] for s in self.active))
        self.batch.step(n)
        diverged = []
        try:
            self.batch.sync()
        except felbm.FelbmError as e:
            if e.status != felbm.FELBM_ERR_NONFINITE:
                raise
            diverged = [s for s in self.active
                        if felbm.felbm_state_sync(s["state"].handle) == felbm.FELBM_ERR_NONFINITE]
            if not diverged:
                raise
        for s in self.active:
            s["done"] += n
            self.node_steps += n * s["req"].nodes
        if diverged:
            now = time.perf_counter() - self.t0
            for s in diverged:
                self._retire(s, now, "diverged")
            self.active = [s for s in self.active if all(s is not d for d in diverged)]
            self._release_fixed()
        return n

    def retire_finished(self, now):
        keep = []
        for s in self.active:
            if s["done"] >= s["req"].steps:
                self._retire(s, now)
            else:
                keep.append(s)
        self.active = keep
        self._release_fixed()

    def close(self):
        if self.batch is not None:
            self.batch.close()
        for s in self.active:
            s["state"].close()
        for ent in self.meshes.values():
            ent[0].close()
        self.meshes.clear()


MASS_DRIFT_TOL = 1e-5  # relative FP64 mass-total change over a served run


def serve(requests, budget_bytes, chunk=200, stream=None, time_scale=1.0, autotune=True,
          max_wall=None):
    """Serve a request stream in real time.  time_scale stretches arrival
    times (1 = as generated).  Returns (results, stats)."""
    srv = Server(budget_bytes, chunk=chunk, stream=stream, autotune=autotune)
    pending = sorted(requests, key=lambda r: r.arrival)
    queue = []  # arrived, not yet admitted (FIFO by arrival)
    t0 = srv.t0 = time.perf_counter()
    i = 0
    try:
        while i < len(pending) or queue or srv.active:
            now = time.perf_counter() - t0
            if max_wall is not None and now > max_wall:
                break
            while i < len(pending) and pending[i].arrival * time_scale <= now:
                queue.append(pending[i])
                i += 1
            while queue and srv.fits(queue[0]):
                r = queue.pop(0)
                srv.admit(r, now)
            if not srv.active:
                if queue:  # cannot fit even alone: reject the head request
                    raise RuntimeError("request %d does not fit the HBM budget" % queue[0].rid)
                if i < len(pending):
                    time.sleep(max(0.0, pending[i].arrival * time_scale - now))
                continue
            srv.advance()
            srv.retire_finished(time.perf_counter() - t0)
    finally:
        wall = time.perf_counter() - t0
        results = list(srv.results)
        node_steps = srv.node_steps
        srv.close()
    # latencies measured from the (scaled) arrival time, over completed runs
    done = [r for r in results if r.status == "ok"]
    lat = np.array([r.finished - r.arrival * time_scale for r in done]) if done else np.zeros(0)
    stats = {
        "completed": len(done),
        "diverged": len(results) - len(done),
        "wall_s": wall,
        "aggregate_mnups": node_steps / wall / 1e6 if wall > 0 else 0.0,
        "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
        # mass-drift check: the collision keeps each node's mass to one
        # rounding, so a completed run whose total drifted beyond
        # MASS_DRIFT_TOL points at a fault
        "max_mass_drift": max((r.mass_drift for r in done), default=0.0),
        "mass_drift_flagged": sum(r.mass_drift > MASS_DRIFT_TOL for r in done),
    }
    return results, stats
