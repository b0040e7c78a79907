"""Small FP64 cases through every kernel path of the library, each compared
with the oracle, for the checked build (run by tests/test_gpu_checked.py in
a process whose FELBM_LIB names libfelbm_checked.so).  Prints one JSON line:
the checked flag, the status bits after the cases, and each case's largest
relative L2 error against the oracle."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle.oracle import Oracle, Params  # noqa: E402
from oracle.oracle3d import Oracle3, Params3  # noqa: E402
from paper_1608_01906_gb300 import configs, felbm, inputs, sharding  # noqa: E402


def rel_l2(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def err2(m, o):
    return max(rel_l2(m["rho"], o.rho), rel_l2(m["C"], o.C), rel_l2(m["u"], np.stack([o.ux, o.uy], 1)),
               rel_l2(m["p"], o.p))


def oracle2(case, steps):
    xy, tri, box, tag, rho0, u0, p0, prm = case
    o = Oracle(xy, tri, box, tag, Params(**prm))
    o.init(rho0, u0, p0)
    o.step(steps)
    return o


def gpu2(case, steps, **mesh_kw):
    xy, tri, box, tag, rho0, u0, p0, prm = case
    mesh = felbm.Mesh(xy, tri, box, tag, **mesh_kw)
    st = felbm.State(mesh, felbm.make_params(precision="fp64", **prm), rho0, u0, p0)
    st.step(steps)
    m = st.moments()
    st.close()
    mesh.close()
    return m


def droplet(nx, ny, walls=False, u=(0.01, -0.004)):
    xy, tri, box, tag = inputs.structured_mesh(nx, ny, periodic_y=not walls)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (nx / 2, ny / 2), min(nx, ny) / 4, 1.0, 0.1, 4.0, u0=u)
    return xy, tri, box, tag, rho0, u0, p0, configs.params(gravity=(0.0, -1e-5) if walls else (0.0, 0.0))


def delaunay(n, walls=False):
    xy, tri, box, tag = inputs.jittered_delaunay_mesh(n, n, 0.25, seed=3)
    rho0, u0, p0 = inputs.droplet_fields(xy, box, (n / 2, n / 2), n / 4, 1.0, 0.1, 4.0, u0=(0.01, 0.005))
    return xy, tri, box, tag, rho0, u0, p0, configs.params(dt=0.4)


def main():
    out = {}
    # structured lattice: a tiny mesh (ragged, wrapping tiles only), a
    # ragged one, and one with walls and TMA tiles
    for name, case, steps in (("lattice_8x8", droplet(8, 8), 20), ("lattice_44x36", droplet(44, 36), 20),
                              ("lattice_96x64_walls", droplet(96, 64, walls=True), 15)):
        out[name] = err2(gpu2(case, steps), oracle2(case, steps))
    # general meshes: the patch step and the four-launch step
    case = delaunay(16)
    o = oracle2(case, 15)
    out["delaunay_16_patch"] = err2(gpu2(case, 15, patch_step=True), o)
    out["delaunay_16_split"] = err2(gpu2(case, 15, split_step=True), o)
    case = droplet(20, 24, walls=True)
    out["walled_general_patch"] = err2(gpu2(case, 10, general=True, patch_step=True), oracle2(case, 10))
    # halo-sharded lattice, 3 slabs
    case = droplet(40, 48)
    xy, tri, box, tag, rho0, u0, p0, prm = case
    run = sharding.SlabRun(xy, tri, box, tag, 40, 48, felbm.make_params(precision="fp64", **prm), rho0, u0, p0,
                           rows=sharding.slab_rows(48, 3))
    run.step(10)
    out["slabs_40x48"] = err2(run.moments(), oracle2(case, 10))
    run.close()
    # a batch of two lattices
    cases = [droplet(40, 40), droplet(56, 48)]
    meshes = [felbm.Mesh(c[0], c[1], c[2], c[3]) for c in cases]
    states = [felbm.State(m, felbm.make_params(precision="fp64", **c[7]), c[4], c[5], c[6])
              for m, c in zip(meshes, cases)]
    b = felbm.Batch(states)
    b.step(10)
    b.sync()
    out["batch"] = max(err2(s.moments(), oracle2(c, 10)) for s, c in zip(states, cases))
    b.close()
    for s in states:
        s.close()
    for m in meshes:
        m.close()
    # 3-D: the Kuhn lattice and the general tetrahedral kernels
    n = 6
    xyz, tet, box, tag = inputs.structured_tet_mesh(n, n, n)
    rho0, u0, p0 = inputs.droplet_fields3(xyz, box, (3, 3, 3), 2.0, 1.0, 0.1, 3.0, u0=(0.01, -0.02, 0.005))
    prm = dict(rho_l=1.0, rho_v=0.1, sigma=0.01, xi=3.0, tau_l=0.5, tau_v=0.5, dt=0.5, gravity=(0.0, 0.0, 0.0))
    o = Oracle3(xyz, tet, box, tag, Params3(**prm))
    o.init(rho0, u0, p0)
    o.step(8)
    for name, general in (("tet_lattice", False), ("tet_general", True)):
        mesh = felbm.Mesh(xyz, tet, box, tag, general=general)
        st = felbm.State(mesh, felbm.make_params(precision="fp64", **prm), rho0, u0, p0)
        st.step(8)
        m = st.moments()
        out[name] = max(rel_l2(m["rho"], o.rho), rel_l2(m["u"], o.u), rel_l2(m["p"], o.p))
        st.close()
        mesh.close()
    checked, bits = felbm.check_status()
    print(json.dumps({"checked": checked, "bits": bits, "errors": out}))


if __name__ == "__main__":
    main()
