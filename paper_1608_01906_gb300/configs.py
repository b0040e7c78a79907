"""The five synthetic workloads and their physical parameters.

Each workload is a seeded synthetic problem shaped like the paper's
benchmarks (static droplet of Sec. 3.1, Rayleigh-Taylor layer of Sec. 3.4)
restated in 2-D.  Readings fixed here (documented in the design notes):

* dt = 0.5 in mesh units wherever a workload states dt = 1 on a unit-spacing
  grid: the lumped Taylor-Galerkin streaming on the structured split is
  unstable above Courant number 0.5 for the diagonal velocities that cross
  the element diagonals (amplification 7 per step at dt = 1).  tau is the
  dimensionless relaxation parameter (nu = c_s^2 tau dt), so "tau = 0.5" and
  "dt = 10 tau" keep their meaning.  On the jittered Delaunay mesh dt = 0.4:
  with tau << 1 (over-relaxation) dt = 0.5 diverges there.
* rho_l = 1, rho_v = rho_l / ratio; sigma = 0.01.
* Interface width xi (mesh units): 4 where stated (64x64 droplet, ratio 10);
  12 for the ratio-1000 Delaunay droplet and 24 for the batched / served
  droplets (ratios up to 1000; see the last item).  The P1 scheme cancels the ideal-gas
  pressure of the order-parameter streaming only to O(h^2 d^4 rho); on
  interfaces of 4 to 8 mesh units that residual outgrows the capillary
  forces and ratios >= 30 diverge, so the width is the smallest tried
  (4, 8, 12, 16) that stays bounded over the run.
* "viscosity ratio 40" is a kinematic contrast nu_v / nu_l = 40 with the
  larger relaxation parameter tau_v = 0.1 (dt = 10 tau), tau_l = 0.0025.
* Rayleigh-Taylor: At = 0.5 -> rho_heavy = 1, rho_light = 1/3; lambda = W =
  512; velocity scale sqrt(lambda g) = 0.08 -> g = 1.25e-5; nu = lambda
  sqrt(lambda g) / Re (tau = 0.082 at Re 3000); equal kinematic viscosities;
  sigma = 1e-4 (the model needs sigma > 0).  With sqrt(lambda g) = 0.04 or
  0.06 (tau 0.041, 0.061) a mode at the bounce-back walls grows about 4.6x
  per 1000 steps and the run diverges.
* Batched / served droplets: tau_l = tau_v = 0.1, dt = 0.5, xi = 24.  At xi = 16
  ratio 1000 diverges after 10000-18000 steps on sides 128-1024 (ratios 10 and
  100 hold for 20000); xi = 24 and 32 hold ratio 1000 for 20000 steps on
  sides 64-1024 (measured).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import inputs

CS2 = 1.0 / 3.0


@dataclass
class Problem:
    name: str
    xy: np.ndarray
    tri: np.ndarray
    box: np.ndarray
    tag: np.ndarray
    rho0: np.ndarray
    u0: np.ndarray
    p0: np.ndarray
    params: dict
    steps: int
    precision: str
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self):
        return len(self.xy)


def params(rho_l=1.0, rho_v=0.1, sigma=0.01, xi=4.0, tau_l=0.5, tau_v=0.5, dt=0.5,
           gravity=(0.0, 0.0)):
    return dict(rho_l=rho_l, rho_v=rho_v, sigma=sigma, xi=xi, tau_l=tau_l, tau_v=tau_v, dt=dt,
                gravity=tuple(gravity))


def droplet_structured(n=64, R=16.0, ratio=10.0, xi=4.0, sigma=0.01, tau_l=0.5, tau_v=0.5,
                       dt=0.5, steps=500, precision="fp64", name="droplet"):
    xy, tri, box, tag = inputs.structured_mesh(n, n)
    rho_l, rho_v = 1.0, 1.0 / ratio
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (n / 2, n / 2), R, rho_l, rho_v, xi)
    return Problem(name, xy, tri, box, tag, rho0, u0, p0,
                   params(rho_l, rho_v, sigma, xi, tau_l, tau_v, dt), steps, precision,
                   {"n": n, "R": R, "ratio": ratio})


def c1_static_droplet():
    """64x64 periodic structured split, R = 16, ratio 10, tau = 0.5, FP64, 500 steps."""
    return droplet_structured(64, 16.0, 10.0, 4.0, 0.01, 0.5, 0.5, 0.5, 500, "fp64", "c1_droplet_64")


def c2_unstructured_droplet(n=256, R=48.0, steps=5000, seed=1608):
    """256x256 periodic box, jitter +-0.25, Lawson-Delaunay, ratio 1000,
    nu_v/nu_l = 40, tau_v = 0.1, R = 48, FP32 vs FP64 oracle."""
    xy, tri, box, tag = inputs.jittered_delaunay_mesh(n, n, 0.25, seed)
    rho_l, rho_v = 1.0, 1.0e-3
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (n / 2, n / 2), R, rho_l, rho_v, 12.0)
    return Problem("c2_unstructured_droplet_%d" % n, xy, tri, box, tag, rho0, u0, p0,
                   params(rho_l, rho_v, 0.01, 12.0, 0.0025, 0.1, 0.4), steps, "fp32",
                   {"n": n, "R": R, "ratio": 1000.0, "seed": seed})


def rt_params(width=512, Re=3000.0, uref=0.08, dt=0.5):
    g = uref * uref / width
    nu = width * uref / Re
    tau = nu / (CS2 * dt)
    return g, nu, tau


def c3_rayleigh_taylor(nx=512, ny=2048, steps=20000, Re=3000.0, uref=0.08, ref_width=None):
    """512x2048 structured split, walls top/bottom, periodic x, At = 0.5,
    amplitude 0.1 W, Re 3000, gravity body force, FP32.  ref_width: the
    width g, nu and tau are derived from (default nx); a smaller mesh with
    ref_width=512 runs the physics of the 512-wide workload."""
    xy, tri, box, tag = inputs.structured_mesh(nx, ny, periodic_y=False)
    rho_h, rho_lt = 1.0, 1.0 / 3.0
    g, nu, tau = rt_params(ref_width or nx, Re, uref)
    rho0, u0, p0 = inputs.rayleigh_taylor_fields(xy, nx, ny, rho_h, rho_lt, 4.0, 0.1 * nx, g)
    return Problem("c3_rayleigh_taylor_%dx%d" % (nx, ny), xy, tri, box, tag, rho0, u0, p0,
                   params(rho_h, rho_lt, 1e-4, 4.0, tau, tau, 0.5, (0.0, -g)), steps, "fp32",
                   {"nx": nx, "ny": ny, "Re": Re, "At": 0.5, "g": g, "nu": nu})


def droplet_3d(n=64, R=None, ratio=10.0, xi=4.0, sigma=0.01, tau_l=0.5, tau_v=0.5, dt=0.5,
               steps=0, precision="fp32", name=None):
    """Periodic n^3 cube of Kuhn-split tetrahedra (D3Q19, the paper's own
    setting) with a spherical drop of radius R (default n/4) at rest."""
    R = n / 4.0 if R is None else R
    xyz, tet, box, _ = inputs.structured_tet_mesh(n, n, n)
    rho0, u0, p0 = inputs.droplet_fields3(xyz, box, (n / 2, n / 2, n / 2), R, 1.0, 1.0 / ratio, xi)
    return Problem(name or "droplet3d_%d" % n, xyz, tet, box, None, rho0, u0, p0,
                   params(1.0, 1.0 / ratio, sigma, xi, tau_l, tau_v, dt, (0.0, 0.0, 0.0)), steps,
                   precision, {"n": n, "R": R, "ratio": ratio})


DROPLET_XI = 24.0


def batched_sides(count=64, lo=32, hi=512, seed=1609):
    """Mesh sides log-uniform in [lo, hi] (integers, multiples of 1)."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))
    ratios = rng.uniform(10.0, 1000.0, size=count)
    radii = rng.uniform(0.2, 0.35, size=count)
    return [(int(round(a)), float(b), float(c)) for a, b, c in zip(s, ratios, radii)]


def c4_batched(count=64, seed=1609, lo=32, hi=512):
    """64 independent periodic droplet runs, sides log-uniform in [32, 512],
    density ratio U[10, 1000], radius U[0.2, 0.35] of the side, FP32."""
    out = []
    for k, (side, ratio, rfrac) in enumerate(batched_sides(count, lo, hi, seed)):
        out.append(droplet_structured(side, rfrac * side, ratio, DROPLET_XI, 0.01, 0.1, 0.1, 0.5, 0,
                                      "fp32", "batch_%02d_%d" % (k, side)))
    return out


# ---- the workloads as JSON files (workloads/*.json) -----------------------
WORKLOAD_DIR = __import__("os").path.join(__import__("os").path.dirname(__file__), "workloads")


def load_workload(path_or_name, capacity_mnups=None):
    """Build a workload from its JSON description (a path, or a file name in
    workloads/ without .json).  The file names a builder of this module (or
    serving.poisson_stream) and its arguments; it also records the physical
    parameters the builder yields, for the reader (tests check they agree).
    Returns a Problem (c1-c3), a list of Problems (c4), or the request list
    of the serving stream (c5, whose arrival rate is rate_fraction x the
    batched capacity in MNUPS: pass capacity_mnups)."""
    import json
    import math
    import os

    path = path_or_name if os.path.exists(str(path_or_name)) else os.path.join(
        WORKLOAD_DIR, str(path_or_name) + ".json")
    with open(path) as f:
        w = json.load(f)
    args = dict(w.get("args", {}))
    if w["builder"] == "serving.poisson_stream":
        from . import serving

        if capacity_mnups is None:
            raise ValueError("the serving workload needs capacity_mnups")
        lo, hi = args["side"]
        mean_nodes = (hi * hi - lo * lo) / (2.0 * math.log(hi / lo))  # E[side^2], log-uniform
        mean_work = mean_nodes * (args["steps"][0] + args["steps"][1]) / 2.0
        rate = w["rate_fraction"] * capacity_mnups * 1e6 / mean_work
        return serving.poisson_stream(w["requests"], rate, seed=args["seed"], side=tuple(args["side"]),
                                      ratio=tuple(args["ratio"]), steps=tuple(args["steps"]),
                                      radius=tuple(args["radius"]))
    return globals()[w["builder"]](**args)
