"""Seeded synthetic inputs: meshes and initial fields.

This module is shared by the CUDA library's callers and by the CPU oracle's
callers.  It holds no arithmetic of the finite-element lattice Boltzmann method
itself (no shape functions, no mass matrix, no equilibria); it only produces
the raw inputs the method is run on:

* node coordinates and P1 triangles (structured split, jittered Delaunay),
* node tags for no-slip walls,
* initial density / velocity / pressure fields (tanh droplet, Rayleigh-Taylor
  layer with a single-mode perturbation).

Conventions
-----------
* Coordinates are float64 ``(N, 2)``; triangles are int32 ``(T, 3)`` in
  counter-clockwise order (positive signed area under the minimum-image rule of
  the periodic box).
* ``box = (Lx, Ly)``: a positive length marks a periodic direction, ``0`` a
  non-periodic one.
* ``node_tag`` is uint8 ``(N,)``: 0 = fluid node; ``k`` in 1..8 = wall node whose
  inward normal is the D2Q9 direction ``k`` (1=(1,0), 2=(0,1), 3=(-1,0),
  4=(0,-1), 5=(1,1), 6=(-1,1), 7=(-1,-1), 8=(1,-1)).

The droplet profile is the flat-interface equilibrium of the free-energy model
(tanh of width ``xi``, Sec. 2.1 "Lattice Boltzmann Method", constants beta and
kappa); the Rayleigh-Taylor perturbation is the single-mode cosine of Sec. 3.4,
restated in 2-D.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "structured_mesh",
    "jittered_delaunay_mesh",
    "droplet_fields",
    "slab_fields",
    "rayleigh_taylor_fields",
    "shear_wave_fields",
]


def _wrap(d, L):
    """Minimum-image difference along one axis (L <= 0: not periodic)."""
    if L > 0:
        return d - L * np.round(d / L)
    return d


def structured_mesh(nx, ny, h=1.0, periodic_x=True, periodic_y=True):
    """Unit-square lattice of ``nx * ny`` nodes split into P1 triangles.

    Node ``(i, j)`` has id ``i + nx * j`` and coordinates ``(i*h, j*h)``.  Each
    square with lower-left corner ``(i, j)`` is cut along its diagonal from
    ``(i, j)`` to ``(i+1, j+1)`` into the triangles
    ``[(i,j), (i+1,j), (i+1,j+1)]`` and ``[(i,j), (i+1,j+1), (i,j+1)]``.
    A periodic direction wraps the last column / row onto the first; a
    non-periodic y direction tags row 0 as a wall with inward normal +y
    (tag 2) and row ny-1 with inward normal -y (tag 4).

    Returns ``(xy, tri, box, node_tag)``.
    """
    nx, ny = int(nx), int(ny)
    if nx < 4 or ny < 4:
        raise ValueError("structured_mesh needs at least 4 nodes per direction")
    if not periodic_x:
        raise ValueError("only periodic x is supported by the generator")
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    xy = np.stack([i.ravel() * h, j.ravel() * h], axis=1).astype(np.float64)
    sq_j = ny if periodic_y else ny - 1
    si, sj = np.meshgrid(np.arange(nx), np.arange(sq_j), indexing="xy")
    si = si.ravel()
    sj = sj.ravel()
    i1 = (si + 1) % nx
    j1 = (sj + 1) % ny
    a = si + nx * sj
    b = i1 + nx * sj
    c = i1 + nx * j1
    d = si + nx * j1
    lower = np.stack([a, b, c], axis=1)
    upper = np.stack([a, c, d], axis=1)
    tri = np.empty((2 * len(a), 3), dtype=np.int32)
    tri[0::2] = lower
    tri[1::2] = upper
    box = np.array([nx * h, ny * h if periodic_y else 0.0])
    tag = np.zeros(nx * ny, dtype=np.uint8)
    if not periodic_y:
        tag[:nx] = 2
        tag[nx * (ny - 1):] = 4
    return xy, tri, box, tag


def _incircle(ax, ay, bx, by, cx, cy, dx, dy):
    """> 0 when d lies strictly inside the circumcircle of CCW triangle abc."""
    adx, ady = ax - dx, ay - dy
    bdx, bdy = bx - dx, by - dy
    cdx, cdy = cx - dx, cy - dy
    return ((adx * adx + ady * ady) * (bdx * cdy - cdx * bdy)
            - (bdx * bdx + bdy * bdy) * (adx * cdy - cdx * ady)
            + (cdx * cdx + cdy * cdy) * (adx * bdy - bdx * ady))


def jittered_delaunay_mesh(nx, ny, jitter=0.25, seed=1608, h=1.0):
    """Periodic ``nx * ny`` point set jittered uniformly by ``+-jitter*h``.

    The points start on the unit lattice; each is moved by independent uniform
    offsets drawn from ``numpy.random.default_rng(seed)``.  The triangulation
    starts as the structured split of :func:`structured_mesh` (valid for
    ``jitter < 0.5``) and Lawson edge flips are applied, with the in-circle
    test evaluated on minimum-image coordinates, until no interior edge is
    strictly non-Delaunay (ties keep their edge).

    Returns ``(xy, tri, box, node_tag)`` with coordinates wrapped into the box.
    """
    if not (0.0 <= jitter < 0.5):
        raise ValueError("jitter must lie in [0, 0.5)")
    xy0, tri, box, tag = structured_mesh(nx, ny, h, True, True)
    rng = np.random.default_rng(seed)
    xy = xy0 + rng.uniform(-jitter * h, jitter * h, size=xy0.shape)
    xy[:, 0] %= box[0]
    xy[:, 1] %= box[1]
    tri = tri.astype(np.int64)
    n = len(xy)
    Lx, Ly = box
    k0 = np.arange(3)
    # Lawson flips in rounds: every round tests all edges, then flips a set of
    # strictly non-Delaunay edges no two of which share a triangle.  For
    # points in general position the Delaunay triangulation is unique, so the
    # order of the flips does not change the result.
    while True:
        a_ = tri[:, k0].ravel()
        b_ = tri[:, (k0 + 1) % 3].ravel()
        key = np.minimum(a_, b_) * n + np.maximum(a_, b_)
        order = np.argsort(key, kind="stable")
        ks = key[order]
        first = np.nonzero(ks[:-1] == ks[1:])[0]  # each interior edge: two sides
        e1, e2 = order[first], order[first + 1]
        t1, j1 = e1 // 3, e1 % 3
        t2, j2 = e2 // 3, e2 % 3
        u, v = tri[t1, j1], tri[t1, (j1 + 1) % 3]
        c = tri[t1, (j1 + 2) % 3]
        d = tri[t2, (j2 + 2) % 3]

        def rel(o, q):
            return (_wrap(xy[q, 0] - xy[o, 0], Lx), _wrap(xy[q, 1] - xy[o, 1], Ly))

        vx, vy = rel(u, v)
        cx, cy = rel(u, c)
        dx, dy = rel(u, d)
        bad = np.nonzero(_incircle(0.0, 0.0, vx, vy, cx, cy, dx, dy) > 0.0)[0]
        if len(bad) == 0:
            break
        # keep a flip only where it is the first candidate of both triangles
        owner = np.full(len(tri), len(first), dtype=np.int64)
        np.minimum.at(owner, t1[bad], bad)
        np.minimum.at(owner, t2[bad], bad)
        sel = bad[(owner[t1[bad]] == bad) & (owner[t2[bad]] == bad)]
        # flip edge (u, v) -> (c, d): new CCW triangles (u, d, c) and (d, v, c)
        tri[t1[sel]] = np.stack([u[sel], d[sel], c[sel]], axis=1)
        tri[t2[sel]] = np.stack([d[sel], v[sel], c[sel]], axis=1)
    tri = np.asarray(tri, dtype=np.int32)
    return xy, tri, box, tag


def _min_image_delta(xy, center, box):
    dx = _wrap(xy[:, 0] - center[0], box[0])
    dy = _wrap(xy[:, 1] - center[1], box[1])
    return dx, dy


def droplet_fields(xy, box, center, radius, rho_l, rho_v, xi, u0=(0.0, 0.0)):
    """Circular liquid drop of radius ``radius`` in vapour.

    ``rho0(r) = (rho_l + rho_v)/2 + (rho_l - rho_v)/2 * tanh(2 (R - r) / xi)``
    with ``r`` the minimum-image distance to ``center``; uniform velocity ``u0``
    and zero pressure.  Returns ``(rho0, u0 (N,2), p0)`` as float64.
    """
    dx, dy = _min_image_delta(xy, center, box)
    r = np.sqrt(dx * dx + dy * dy)
    rho = 0.5 * (rho_l + rho_v) + 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (radius - r) / xi)
    u = np.zeros((len(xy), 2))
    u[:, 0] = u0[0]
    u[:, 1] = u0[1]
    return rho, u, np.zeros(len(xy))


def slab_fields(xy, box, y_lo, y_hi, rho_l, rho_v, xi):
    """Flat liquid slab ``y_lo < y < y_hi`` (two tanh interfaces), u = 0, p = 0."""
    y = xy[:, 1]
    rho = (rho_v + 0.5 * (rho_l - rho_v)
           * (np.tanh(2.0 * (y - y_lo) / xi) - np.tanh(2.0 * (y - y_hi) / xi)))
    return rho, np.zeros((len(xy), 2)), np.zeros(len(xy))


def rayleigh_taylor_fields(xy, width, height, rho_heavy, rho_light, xi, amplitude, g):
    """Heavy fluid on top of light fluid, interface ``H/2 + A cos(2 pi x / W)``.

    Density is the tanh profile across the perturbed interface, velocity is
    zero and the pressure is hydrostatic for gravity ``(0, -g)``: integrated
    column by column downward from the top row with the trapezoid rule, so
    that ``dp/dy = -rho g``.  Nodes must lie on the structured lattice
    (columns of equal x).  Returns ``(rho0, u0, p0)``.
    """
    x = xy[:, 0]
    y = xy[:, 1]
    yi = 0.5 * (height - 1) + amplitude * np.cos(2.0 * np.pi * x / width)
    rho = (0.5 * (rho_heavy + rho_light)
           + 0.5 * (rho_heavy - rho_light) * np.tanh(2.0 * (y - yi) / xi))
    nx = int(round(width))
    ny = len(xy) // nx
    r2 = rho.reshape(ny, nx)
    y2 = y.reshape(ny, nx)
    p2 = np.zeros_like(r2)
    for j in range(ny - 2, -1, -1):
        dy = y2[j + 1] - y2[j]
        p2[j] = p2[j + 1] + 0.5 * g * (r2[j] + r2[j + 1]) * dy
    return rho, np.zeros((len(xy), 2)), p2.ravel()


def shear_wave_fields(xy, box, rho, amplitude):
    """Uniform density, ``u_x = U sin(2 pi y / Ly)``, ``u_y = 0``, p = 0."""
    u = np.zeros((len(xy), 2))
    u[:, 0] = amplitude * np.sin(2.0 * np.pi * xy[:, 1] / box[1])
    return np.full(len(xy), float(rho)), u, np.zeros(len(xy))


# ---- three dimensions (D3Q19 on tetrahedra) -----------------------------

def structured_tet_mesh(nx, ny, nz, h=1.0, periodic_z=True):
    """Cubic lattice of ``nx * ny * nz`` nodes, each cube split into six
    tetrahedra around its diagonal from corner (0,0,0) to (1,1,1) (the Kuhn
    split: one tetrahedron per ordering of the three axes; conforming across
    cubes and across the periodic wrap).  Periodic in x and y; periodic in z
    unless ``periodic_z`` is false, in which case the bottom and top node
    layers are walls with inward normals +z (tag 5) and -z (tag 6) in the
    D3Q19 order of the oracle.  Periodic directions need at least 3 nodes
    (with 2 a neighbour sits half a period away and the minimum image is
    ambiguous).  Node id ``i + nx*(j + ny*k)``.  Returns
    ``(xyz (N,3), tet (T,4) positively oriented, box (3,), tag (N,))``.
    """
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    i, j, k = i.ravel(order="F"), j.ravel(order="F"), k.ravel(order="F")
    xyz = np.stack([i, j, k], 1).astype(np.float64) * h
    nid = lambda a, b, c: (a % nx) + nx * ((b % ny) + ny * (c % nz))  # noqa: E731
    cz = nz if periodic_z else nz - 1
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(cz), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    unit = np.eye(3, dtype=np.int64)
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        corners = [np.zeros(3, dtype=np.int64)]
        for ax in perm:
            corners.append(corners[-1] + unit[ax])
        v = [nid(ci + c[0], cj + c[1], ck + c[2]) for c in corners]
        t = np.stack(v, 1)
        # orientation: det of the edge vectors in unwrapped coordinates
        e = np.array([corners[1], corners[2], corners[3]], dtype=np.float64)
        if np.linalg.det(e) < 0:
            t = t[:, [0, 2, 1, 3]]
        tets.append(t)
    tet = np.concatenate(tets, 0).astype(np.int32)
    box = np.array([nx * h, ny * h, nz * h if periodic_z else 0.0])
    tag = np.zeros(len(xyz), dtype=np.uint8)
    if not periodic_z:
        tag[k == 0] = 5
        tag[k == nz - 1] = 6
    return xyz, tet, box, tag


def jittered_tet_mesh(nx, ny, nz, jitter=0.15, seed=1608, h=1.0):
    """The periodic Kuhn-split lattice of :func:`structured_tet_mesh` with
    every node moved by independent uniform offsets in ``+-jitter*h`` drawn
    from ``numpy.random.default_rng(seed)``, coordinates wrapped into the
    box.  Same tetrahedra (the orientation under the minimum-image rule holds
    for ``jitter <= 0.15``); element volumes and lumped masses then differ
    from node to node.  Returns ``(xyz, tet, box, tag)``."""
    if not (0.0 <= jitter <= 0.15):
        raise ValueError("jitter must lie in [0, 0.15]")
    xyz, tet, box, tag = structured_tet_mesh(nx, ny, nz, h, True)
    rng = np.random.default_rng(seed)
    xyz = xyz + rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
    for c in range(3):
        xyz[:, c] %= box[c]
    return xyz, tet, box, tag


def droplet_fields3(xyz, box, center, radius, rho_l, rho_v, xi, u0=(0.0, 0.0, 0.0)):
    """Spherical liquid drop of radius ``radius`` in vapour: the tanh
    profile of ``droplet_fields`` in the minimum-image distance to
    ``center``; uniform velocity ``u0``, zero pressure.  Returns
    ``(rho0, u0 (N,3), p0)``."""
    d = np.stack([_wrap(xyz[:, c] - center[c], box[c]) for c in range(3)], 1)
    r = np.sqrt((d * d).sum(1))
    rho = 0.5 * (rho_l + rho_v) + 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (radius - r) / xi)
    u = np.tile(np.asarray(u0, dtype=np.float64), (len(xyz), 1))
    return rho, u, np.zeros(len(xyz))


def slab_fields3(xyz, z_lo, z_hi, rho_l, rho_v, xi):
    """Flat liquid slab ``z_lo < z < z_hi`` (two tanh interfaces), u = 0,
    p = 0."""
    z = xyz[:, 2]
    t = np.tanh(2.0 * (z - z_lo) / xi) - np.tanh(2.0 * (z - z_hi) / xi)
    rho = rho_v + 0.5 * (rho_l - rho_v) * t
    return rho, np.zeros((len(xyz), 3)), np.zeros(len(xyz))


def shear_wave_fields3(xyz, box, rho, amplitude):
    """Uniform density, ``u_x = U sin(2 pi z / Lz)``, other components 0, p = 0."""
    u = np.zeros((len(xyz), 3))
    u[:, 0] = amplitude * np.sin(2.0 * np.pi * xyz[:, 2] / box[2])
    return np.full(len(xyz), float(rho)), u, np.zeros(len(xyz))
