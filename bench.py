#!/usr/bin/env python
"""Throughput of the FE-LBM binary-fluid time step on GB300.

One "step" is one full time step of the method (streaming of 18 D2Q9
populations, density-gradient / Laplacian / chemical-potential recovery,
moments and the split collision) over the Rayleigh-Taylor workload:
512 x 2048 structured P1 triangulation (1,048,576 nodes), walls top and
bottom, periodic in x, Atwood 0.5, amplitude 0.1 W, Re 3000, gravity, FP32.

Metric: MNUPS (million node updates per second), whole job over all ranks.
Multi-GPU runs are independent replicas (the method's runs do not exchange
data), so scaling is weak.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl felbm|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MNUPS"
UNIT = "MNUPS"
ALGO_BYTES_PER_NODE = {"fp32": 144, "fp64": 288}  # 18 populations read + 18 written
FALLBACK_HBM_GBS = 6800.0
# FP64 runs are bound by the FP64 pipe (about 86% busy), not by HBM.  Peak:
# the FP64 FMA rate measured on the device (felbm_alu_peak), else the nominal
# dense FP64 rate of the part.  Algorithmic flops per node update in FP64:
# the 1,000 flops ncu counts per node on the current step (DADD + DMUL +
# 2 DFMA) less the halo recompute of the tile step (h streaming on the
# depth-3 density region, 1.08x extra: about 136; grad rho 0.69x and mu
# 0.33x: about 16), which agrees with an operator-by-operator count of the
# streaming, recovery, mu, force, moment and collision arithmetic (854)
FP64_PEAK_TFLOPS = 1.25
FP64_ALGO_FLOPS_PER_NODE = 850


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="felbm", choices=["felbm", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-all-cores", action="store_true",
                    help="time the oracle on one thread only")
    ap.add_argument("--no-fp64", action="store_true",
                    help="leave out the FP64 rate of the same workload")
    ap.add_argument("--fp64-steps", type=int, default=500)
    ap.add_argument("--lap-fp64", default="auto", choices=["auto", "on", "off"],
                    help="FP64 kappa lap rho term of mu in FP32 runs (auto: at density ratio >= 1000)")
    ap.add_argument("--shards", type=int, default=2,
                    help="slabs of the halo-sharded run of the same lattice on this GPU (<= 1: none)")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--split-step", action="store_true",
                    help="general triangle meshes: always the four-launch step")
    ap.add_argument("--patch-step", action="store_true",
                    help="general triangle meshes: always the one-launch patch step")
    ap.add_argument("--general", action="store_true",
                    help="force the general CSR kernels on a structured mesh")
    ap.add_argument("--serve-requests", type=int, default=40)
    ap.add_argument("--workload", default="rayleigh_taylor_512x2048",
                    choices=["rayleigh_taylor_512x2048", "droplet_2048x2048",
                             "delaunay_droplet_256x256", "delaunay_droplet_512x512", "delaunay_droplet_1024x1024", "droplet3d_64x64x64",
                             "droplet3d_128x128x128"],
                    help="droplet_2048x2048: supplementary single-mesh case (periodic, 4.2 M "
                         "nodes); delaunay_droplet_256x256: the unstructured case (general "
                         "meshes, L2-resident); droplet3d_NxNxN: D3Q19 on tetrahedra (64^3 "
                         "L2-resident, 128^3 larger than L2)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest per-rank value of x over all ranks (every rank gets it):
    the slowest rank sets the job's time.  dist: torch.distributed with an
    initialised process group, or None for one process."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, nodes, steps, seconds):
    """Whole-job MNUPS: the node updates of all ranks (each runs its own
    replica of nodes x steps) over the slowest rank's time."""
    return world * nodes * steps / seconds / 1e6


# Sources that determine a kernel's code (its ncu counters stay valid while
# these are unchanged); kernels not listed depend on every source.
KERNEL_SOURCES = {
    "k_lattice_step": ["csrc/felbm_lattice.cuh", "csrc/felbm_kernels.cuh", "csrc/felbm_internal.h",
                       "csrc/felbm_api.cu", "csrc/felbm_tmap.cu", "../include/felbm.h"],
}


def csrc_hash(kernel=None):
    import hashlib

    pkg = os.path.join(ROOT, "paper_1608_01906_gb300")
    files = KERNEL_SOURCES.get(kernel)
    if files is None:
        files = ["csrc/" + f for f in sorted(os.listdir(os.path.join(pkg, "csrc")))]
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode())
        with open(os.path.join(pkg, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_copy_gbs", "hbm_GBps"):
            if k in d:
                return float(d[k]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.15)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(name="rayleigh_taylor_512x2048"):
    from paper_1608_01906_gb300 import configs

    if name == "droplet_2048x2048":
        return configs.droplet_structured(2048, 0.3 * 2048, 100.0, configs.DROPLET_XI, 0.01, 0.1,
                                          0.1, 0.5, 0, "fp32", name)
    if name == "delaunay_droplet_256x256":
        return configs.c2_unstructured_droplet()
    if name == "delaunay_droplet_512x512":
        return configs.c2_unstructured_droplet(n=512, R=96.0)
    if name == "delaunay_droplet_1024x1024":
        # the C2 physics on a 4x wider box (state beyond L2), radius scaled
        return configs.c2_unstructured_droplet(n=1024, R=192.0)
    if name == "droplet3d_64x64x64":
        return configs.droplet_3d(64)
    if name == "droplet3d_128x128x128":
        return configs.droplet_3d(128)
    return configs.c3_rayleigh_taylor()


def config_dict(prob, precision, name="rayleigh_taylor_512x2048"):
    dim3 = name.startswith("droplet3d_")
    state_mb = 2 * (38 if dim3 else 18) * prob.n_nodes * (4 if precision == "fp32" else 8) / 1e6
    if state_mb > 126.0:
        l2_note = "inputs > L2: double-buffered state %.0f MB vs 126 MB L2, no flush" % state_mb
    else:
        l2_note = ("L2-resident: double-buffered state %.0f MB fits the 126 MB L2, no flush "
                   "(supplementary case)" % state_mb)
    if name == "droplet_2048x2048":
        phys = {"mesh": "structured P1 split, periodic x and y", "ratio": 100.0,
                "radius": 0.3 * 2048, "xi": prob.params["xi"]}
    elif name.startswith("droplet3d_"):
        side = int(round(prob.n_nodes ** (1.0 / 3.0)))
        phys = {"mesh": "%d^3 cube, 6 Kuhn tetrahedra per cube, periodic x, y, z" % side,
                "ratio": 10.0, "radius": side / 4.0, "xi": prob.params["xi"]}
    elif name.startswith("delaunay_droplet_"):
        phys = {"mesh": "jittered Delaunay (seed 1608), periodic x and y", "ratio": 1000.0,
                "radius": {"delaunay_droplet_512x512": 96.0, "delaunay_droplet_1024x1024": 192.0}.get(name, 48.0),
                "xi": prob.params["xi"], "nu_ratio": 40.0}
    else:
        phys = {"mesh": "structured P1 split, walls y, periodic x", "Re": 3000, "atwood": 0.5}
    return {"workload": name, "nodes": prob.n_nodes, "triangles": int(len(prob.tri)),
            "lattice": "D3Q19" if dim3 else "D2Q9",
            "precision": precision, **phys,
            "dt": prob.params["dt"],
            "l2": l2_note,
            "parallelism": "replicas"}


# --------------------------------------------------------------------- oracle
def make_oracle(prob):
    """The FP64 oracle of a problem: triangles (2-D) or tetrahedra (3-D)."""
    if np.shape(prob.xy)[1] == 3:
        from oracle.oracle3d import Oracle3, Params3

        return Oracle3(prob.xy, prob.tri, prob.box, prob.tag, Params3(**prob.params))
    from oracle.oracle import Oracle, Params

    return Oracle(prob.xy, prob.tri, prob.box, prob.tag, Params(**prob.params))


def oracle_rate(prob, seconds, max_steps=None):
    """Time the FP64 oracle as it stands on this host (one thread)."""
    o = make_oracle(prob)
    o.init(prob.rho0, prob.u0, prob.p0)
    t = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t
    n = max(1, int(seconds / max(one, 1e-9)))
    if max_steps:
        n = min(n, max_steps)
    t = time.perf_counter()
    o.step(n)
    el = time.perf_counter() - t
    return prob.n_nodes * n / el / 1e6, n, el


def _oracle_replica(name, seconds, barrier, out):
    """One single-threaded oracle replica of a workload (a spawned process):
    build, initialise, wait for the others, then step for about `seconds`."""
    from oracle import oracle as orc  # noqa: F401  (built by the parent)

    prob = workload(name)
    o = make_oracle(prob)
    o.init(prob.rho0, prob.u0, prob.p0)
    barrier.wait(timeout=600)
    n, t = 0, time.perf_counter()
    while True:
        o.step(1)
        n += 1
        el = time.perf_counter() - t
        if el >= seconds:
            break
    out.put((n, el))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def oracle_rate_all_cores(name, seconds, n_nodes, procs=None):
    """Aggregate rate of one plain single-threaded oracle replica per host
    core, each a separate spawned process stepping the same workload at the
    same time (the oracle itself stays free of threading)."""
    import multiprocessing as mp

    procs = procs or host_cores()
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(procs), ctx.Queue()
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    ps = []
    try:
        ps = [ctx.Process(target=_oracle_replica, args=(name, seconds, barrier, out)) for _ in range(procs)]
        for p in ps:
            p.start()
        res, t_end = [], time.monotonic() + 600 + 4 * seconds
        while len(res) < procs:
            try:
                res.append(out.get(timeout=1.0))
            except Exception:  # noqa: BLE001  (queue.Empty)
                if any(p.exitcode not in (None, 0) for p in ps) or time.monotonic() > t_end:
                    raise RuntimeError("an oracle replica failed or did not finish")
        for p in ps:
            p.join(timeout=60)
    finally:
        for p in ps:
            if p.is_alive():
                p.terminate()
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    rate = sum(n_nodes * n / el for n, el in res) / 1e6
    return rate, procs, sum(n for n, _ in res), max(el for _, el in res)


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_1608_01906_gb300 import configs

    orc.build()
    full = workload(args.workload)
    # each step: one oracle time step of a bounded sample of the same workload
    # (same physics on a smaller mesh)
    if args.workload == "droplet_2048x2048":
        samp = configs.droplet_structured(128, 0.3 * 128, 100.0, configs.DROPLET_XI, 0.01, 0.1, 0.1,
                                          0.5, 0, "fp32", "droplet_sample")
        sample = ("oracle (FP64 C, 1 thread) time step of a 128x128 periodic droplet with the "
                  "physics of the 2048x2048 case (16,384 nodes) per step")
    elif args.workload.startswith("delaunay_droplet_"):
        samp = configs.c2_unstructured_droplet(n=64, R=12.0)
        sample = ("oracle (FP64 C, 1 thread) time step of a 64x64 jittered Delaunay droplet "
                  "with the physics of the %s case (4,096 nodes) per step" % args.workload)
    elif args.workload.startswith("droplet3d_"):
        samp = configs.droplet_3d(16)
        sample = ("3-D oracle (FP64 C, 1 thread) time step of a 16^3 tetrahedral droplet with "
                  "the physics of the %s case (4,096 nodes) per step" % args.workload)
    else:
        samp = configs.c3_rayleigh_taylor(nx=64, ny=256)
        samp.params["gravity"] = full.params["gravity"]
        sample = ("oracle (FP64 C, 1 thread) time step on a 64x256 window of the 512x2048 "
                  "Rayleigh-Taylor problem (16,384 nodes) per step")
    o = make_oracle(samp)
    o.init(samp.rho0, samp.u0, samp.p0)
    o.step(args.warmup)
    t = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t
    v = samp.n_nodes * args.steps / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(full, "fp64", args.workload),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "nproc": host_cores(), "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- batched and served
def run_batched(torch, felbm, steps=200):
    """64 uneven droplet meshes: one batched launch per step vs one
    felbm_step per mesh per step (same states, same steps)."""
    from paper_1608_01906_gb300 import configs

    probs = configs.c4_batched()
    nodes = sum(p.n_nodes for p in probs)
    stream = torch.cuda.Stream()
    meshes = [felbm.Mesh(p.xy, p.tri, p.box, p.tag, stream=stream.cuda_stream) for p in probs]
    states = [felbm.State(m, felbm.make_params(precision="fp32", **p.params), p.rho0, p.u0, p.p0)
              for m, p in zip(meshes, probs)]
    for st in states:
        st.step(3)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st in states:
        st.step(steps)
    e1.record(stream)
    e1.synchronize()
    seq_ms = e0.elapsed_time(e1)
    b = felbm.Batch(states, autotune=True)
    b.step(100)  # autotuning steps
    b.sync()
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    e1.synchronize()
    b.sync()
    bat_ms = e0.elapsed_time(e1)
    info = b.info()
    b.close()
    for st in states:
        st.close()
    for m in meshes:
        m.close()
    return {"workload": "64 periodic droplet meshes, sides log-uniform [32,512] (seed 1609), "
                        "ratio U[10,1000], FP32",
            "nodes": nodes, "steps": steps,
            "value": nodes * steps / (bat_ms * 1e-3) / 1e6, "unit": UNIT,
            "sequential": nodes * steps / (seq_ms * 1e-3) / 1e6,
            "speedup": seq_ms / bat_ms, "launches_per_step": 1,
            "blocks_per_sm": info["blocks_per_sm"], "tile_order": info["tile_order"]}


def run_serving(torch, felbm, capacity_mnups, n_requests):
    """Poisson stream at 80% of the measured batched capacity."""
    import math

    from paper_1608_01906_gb300 import serving

    lo, hi = 64, 1024
    mean_nodes = (hi * hi - lo * lo) / (2.0 * math.log(hi / lo))  # E[side^2], log-uniform
    mean_work = mean_nodes * (1000 + 20000) / 2.0
    rate = 0.8 * capacity_mnups * 1e6 / mean_work
    reqs = serving.poisson_stream(n_requests, rate, seed=1610)
    stream = torch.cuda.Stream()
    budget = 64 * 1024 ** 3
    results, stats = serving.serve(reqs, budget, chunk=500, stream=stream.cuda_stream)
    stats.update({"requests": n_requests, "rate_per_s": rate, "budget_gb": 64,
                  "load": "80%% of batched capacity %.0f MNUPS" % capacity_mnups,
                  "workload": "droplet runs, sides log-uniform [64,1024], ratio U[10,1000], "
                              "steps U[1000,20000], Poisson arrivals (seed 1610), FP32"})
    return stats


# --------------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    world, rank, local = dist_env()
    import torch

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__

    __graft_entry__.build()
    from paper_1608_01906_gb300 import felbm

    prob = workload(args.workload)
    dim0 = int(np.shape(prob.xy)[1])
    stream = torch.cuda.Stream()
    mesh = felbm.Mesh(prob.xy, prob.tri, prob.box, prob.tag, general=args.general,
                      stream=stream.cuda_stream, split_step=args.split_step, patch_step=args.patch_step)
    # FP64 kappa lap rho term of mu at density ratio >= 1000 (FP32 states)
    lap64 = args.precision == "fp32" and dim0 == 2 and (
        args.lap_fp64 == "on" or (args.lap_fp64 == "auto" and prob.params["rho_l"] >= 1000.0 * prob.params["rho_v"]))
    params = felbm.make_params(precision=args.precision, lap_fp64=lap64, **prob.params)
    st = felbm.State(mesh, params, prob.rho0, prob.u0, prob.p0)
    st.step(args.warmup)
    st.sync()
    kind = mesh.info()["kind"]

    # ---- timed region: K steps, device events on the library's stream
    # time every k-th launch of each kernel (about 1000 over the region): the
    # event records then touch few launches
    st.profile_enable(max(1, args.steps // 1000))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if rank == 0 else None
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    prof = st.profile_read()
    st.sync()
    if dist:
        ms = max_over_ranks(ms, dist, "cuda")
        dist.barrier()
    value = job_rate(world, prob.n_nodes, args.steps, ms * 1e-3)
    launches = int(sum(v[2] for v in prof.values()))

    # ---- dominant kernel roofline (event-timed launches of the region).  A
    # step of several dependent launches (general and 3-D paths) is rated as
    # a whole: the step's algorithmic bytes over the summed launch times.
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_timed, _) = dom
    dom_avg_ms = dom_ms / max(dom_timed, 1)
    per_step = {k: v for k, v in prof.items() if v[2] >= args.steps}
    multi = len(per_step) > 1
    dom_single, dom_share = dom_name, dom_ms / max(sum(v[0] for v in prof.values()), 1e-12)
    if multi:
        dom_name = "+".join(per_step)
        dom_avg_ms = sum(v[0] / max(v[1], 1) for v in per_step.values())
    # the event-sampled average of the dominant kernel's timed launches; when
    # it is the only kernel the region launched, its average launch duration
    # is also the region's event time over its launches (no event records
    # between those launches), and that figure is used
    dom_event_ms = dom_avg_ms
    issued = {k: v[2] for k, v in prof.items() if v[2]}
    only_kernel = len(issued) == 1 and not multi
    if only_kernel:
        dom_avg_ms = ms / issued[dom_name]
    peak, peak_kind = hbm_peak()
    # measured ALU ceilings (after the timed region: a few ms of FMA streams)
    alu = {}
    for key, alu_kind in (("fp32", felbm.ALU_FP32), ("fp32x2", felbm.ALU_FP32X2),
                          ("fp64", felbm.ALU_FP64)):
        try:
            alu[key] = felbm.alu_peak(alu_kind) / 1e12
        except Exception:  # noqa: BLE001
            alu[key] = None
    dim = int(np.shape(prob.xy)[1])
    # 2 x Q populations per node, read once and written once
    algo = ALGO_BYTES_PER_NODE[args.precision] * (19 if dim == 3 else 9) // 9 * prob.n_nodes
    achieved = algo / (dom_avg_ms * 1e-3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        with open(tr_path) as f:
            tr = json.load(f)
        ent = tr.get(dom_name + ":" + args.precision)
        # counters are valid only for the kernel sources they were taken on
        if ent and ent.get("csrc_sha256_16") == csrc_hash(dom_name):
            traffic = ent["bytes_per_launch"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": dom_name,
                "kernel_ms": dom_avg_ms, "kernel_ms_events": dom_event_ms,
                "kernel_ms_source": ("timed region over launches (the only kernel launched)" if only_kernel
                                     else "CUDA events around its sampled launches"),
                "peak_source": peak_kind + " copy bandwidth",
                "step_gbs": algo * args.steps / (ms * 1e-3) / 1e9,
                "kernel_share": dom_ms / max(sum(v[0] for v in prof.values()), 1e-12)}
    if kind == 0:
        # general meshes: CSR metadata, reported apart from the algorithmic
        # state bytes: per node a row offset, and per neighbour a column
        # index and 5 coefficients (a_x, a_y, b_xx, b_xy, b_yy) in the
        # state's precision; the four launches read it 2 + 2 x 3/5 times
        tri = np.asarray(prob.tri, dtype=np.int64)
        ed = np.sort(np.stack([tri[:, [0, 1, 2]].ravel(), tri[:, [1, 2, 0]].ravel()], 1), axis=1)
        nnz = 2 * len(np.unique(ed[:, 0] * prob.n_nodes + ed[:, 1]))
        es = 4 if args.precision == "fp32" else 8
        deg = nnz / prob.n_nodes
        once = 4 + deg * (4 + 5 * es)
        patch = prof.get("k_patch_step", (0, 0, 0))[2] > 0
        if patch:
            # one launch: each patch reads the CSR rows of its region (rings
            # <= 3, shared with neighbouring patches through L2) and its
            # region lists; counted once per node here
            roofline["metadata"] = {"step": "patch", "nnz_per_node": deg, "csr_bytes_per_node": once,
                                    "achieved_with_metadata_gbs": (algo + once * prob.n_nodes) /
                                    (dom_avg_ms * 1e-3) / 1e9}
        else:
            meta_step = 2 * once + 2 * (4 + deg * (4 + 2 * es))
            roofline["metadata"] = {
                "step": "split", "nnz_per_node": deg, "csr_bytes_per_node": once,
                "read_per_step_bytes_per_node": meta_step,
                "achieved_with_metadata_gbs": (algo + meta_step * prob.n_nodes) / (dom_avg_ms * 1e-3) / 1e9}
    if multi:
        roofline["note"] = ("step of %d dependent launches rated as one: algorithmic bytes of the "
                            "step over the summed launch times" % len(per_step))
        roofline["kernel_share"] = 1.0
        roofline["largest_launch"] = {"kernel": dom_single, "share": dom_share}
    if args.precision == "fp64" and not multi:
        tf = FP64_ALGO_FLOPS_PER_NODE * prob.n_nodes / (dom_avg_ms * 1e-3) / 1e12
        p64 = alu.get("fp64") or FP64_PEAK_TFLOPS
        roofline = {"bound": "alu", "achieved": tf, "peak": p64, "unit": "TFLOP/s",
                    "frac": tf / p64, "traffic": traffic, "kernel": dom_name,
                    "kernel_ms": dom_avg_ms,
                    "peak_source": ("measured FP64 FMA streams (felbm_alu_peak)" if alu.get("fp64")
                                    else "nominal dense FP64 rate"),
                    "hbm_gbs": achieved, "hbm_frac": achieved / peak,
                    "kernel_share": dom_ms / max(sum(v[0] for v in prof.values()), 1e-12)}

    # ---- the same workload in FP64 (after the FP32 timed region): its rate
    # and its roofline against the measured FP64 FMA ceiling
    fp64 = None
    if args.precision == "fp32" and not args.no_fp64 and world == 1:
        p64 = felbm.make_params(precision="fp64", **prob.params)
        s64 = felbm.State(mesh, p64, prob.rho0, prob.u0, prob.p0)
        s64.step(args.warmup)
        s64.sync()
        s64.profile_enable(True)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64.step(args.fp64_steps)
        f1.record(stream)
        f1.synchronize()
        ms64 = f0.elapsed_time(f1)
        pr64 = s64.profile_read()
        s64.close()
        per64 = {k: v for k, v in pr64.items() if v[2] >= args.fp64_steps}
        k64_ms = sum(v[0] / max(v[1], 1) for v in per64.values())
        if len([v for v in pr64.values() if v[2]]) == 1:  # the only kernel: region time per launch
            k64_ms = ms64 / args.fp64_steps
        algo64 = ALGO_BYTES_PER_NODE["fp64"] * (19 if dim == 3 else 9) // 9 * prob.n_nodes
        hbm64 = algo64 / (k64_ms * 1e-3) / 1e9
        fp64 = {"value": job_rate(1, prob.n_nodes, args.fp64_steps, ms64 * 1e-3), "unit": UNIT,
                "steps": args.fp64_steps, "ms_per_step": ms64 / args.fp64_steps, "dtype": "f64",
                "kernel": "+".join(per64), "kernel_ms": k64_ms,
                "hbm": {"achieved": hbm64, "peak": peak, "unit": "GB/s", "frac": hbm64 / peak}}
        if dim == 2 and len(per64) == 1:
            tf = FP64_ALGO_FLOPS_PER_NODE * prob.n_nodes / (k64_ms * 1e-3) / 1e12
            pk = alu.get("fp64") or FP64_PEAK_TFLOPS
            fp64["roofline"] = {"bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s",
                                "frac": tf / pk,
                                "peak_source": ("measured FP64 FMA streams (felbm_alu_peak)"
                                                if alu.get("fp64") else "nominal dense FP64 rate")}

    # ---- the same lattice cut into halo-sharded slabs on this device: each
    # step is every slab's step plus the halo exchange (pack, copies, unpack)
    sharded = None
    if kind == 1 and dim == 2 and args.shards > 1 and world == 1:
        from paper_1608_01906_gb300 import sharding

        try:
            nx = int(round(prob.box[0])) if prob.box[0] > 0 else int(np.max(prob.xy[:, 0])) + 1
            ny = prob.n_nodes // nx
            run = sharding.SlabRun(prob.xy, prob.tri, prob.box, prob.tag, nx, ny, params, prob.rho0, prob.u0,
                                   prob.p0, n_slabs=args.shards, stream=stream.cuda_stream)
            run.step(args.warmup)
            torch.cuda.synchronize()
            k_sh = min(args.steps, 1000)
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            run.step(k_sh)
            g1.record(stream)
            g1.synchronize()
            ms_sh = g0.elapsed_time(g1)
            msg = run.states[0].halo()[2]
            sharded = {"slabs": [list(r) for r in run.rows], "value": job_rate(1, prob.n_nodes, k_sh, ms_sh * 1e-3),
                       "unit": UNIT, "steps": k_sh, "ms_per_step": ms_sh / k_sh,
                       "halo_bytes_per_step": 2 * len(run.rows) * msg,
                       "note": ("slabs of the same lattice on one GPU, stepped one after another, halo exchange "
                                "after every step; bitwise equal to the whole-lattice run")}
            run.close()
        except Exception as e:  # noqa: BLE001
            sharded = {"error": "%s: %s" % (type(e).__name__, e)}

    # ---- end to end through the C ABI with host buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st2 = felbm.State(mesh, params, prob.rho0, prob.u0, prob.p0)
    st2.step(args.steps)
    mom = st2.moments()
    t1 = time.perf_counter()
    st2.close()
    e2e_val = job_rate(world, prob.n_nodes, args.steps,
                       max_over_ranks(t1 - t0, dist, "cuda") if dist else t1 - t0)
    n = prob.n_nodes
    h2d = (n * 8 + dim * n * 8 + n * 8) / args.steps          # rho0, u0, p0
    d2h = ((3 + dim) * n * 8 + (1 + dim) * 8) / args.steps  # rho, C, u, p, totals

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if dim == 3 and prob.n_nodes > 300000:
            # the 3-D oracle holds about 2 KB per node: time it on the 64^3 case
            from paper_1608_01906_gb300 import configs

            v, nsteps, el = oracle_rate(configs.droplet_3d(64), args.cpu_seconds)
            what = "the 64^3 case of the same physics"
        else:
            v, nsteps, el = oracle_rate(prob, args.cpu_seconds)
            what = "full %s mesh" % args.workload
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "nproc": host_cores(),
               "sample": "FP64 C oracle (1 thread), %s, %d time steps, %.1f s" % (what, nsteps, el)}
        if dim == 2 and not args.no_all_cores:
            try:
                va, procs, nall, elall = oracle_rate_all_cores(args.workload, args.cpu_seconds, prob.n_nodes)
                cpu["all_cores"] = {
                    "value": va, "unit": UNIT, "cores": procs, "kind": "oracle",
                    "sample": ("one single-threaded FP64 C oracle replica per host core (%d spawned "
                               "processes) on the full %s mesh, stepping together: %d time steps "
                               "in all, %.1f s" % (procs, args.workload, nall, elall))}
            except Exception as e:  # noqa: BLE001
                cpu["all_cores"] = {"error": "%s: %s" % (type(e).__name__, e)}
    batched = serving = None
    if rank == 0 and world == 1 and not args.skip_batched:
        # the headline line prints even if a secondary measurement fails
        try:
            batched = run_batched(torch, felbm)
        except Exception as e:  # noqa: BLE001
            batched = {"error": "%s: %s" % (type(e).__name__, e)}
        if not args.skip_serving and "value" in batched:
            try:
                serving = run_serving(torch, felbm, batched["value"], args.serve_requests)
            except Exception as e:  # noqa: BLE001
                serving = {"error": "%s: %s" % (type(e).__name__, e)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
                "data": "synthetic", "config": dict(config_dict(prob, args.precision, args.workload),
                                                    mesh_kind=kind, kappa_lap_fp64=lap64),
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches * world, "clocks": clocks,
                "kernels": {k: {"ms": v[0], "timed": v[1], "launches": v[2]}
                            for k, v in prof.items() if v[2]},
                "mass": float(mom["totals"][0]), "alu_peaks_tflops": alu,
                "fp64": fp64, "sharded": sharded, "batched": batched, "serving": serving}
        print(json.dumps(line), flush=True)
    st.close()
    mesh.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
