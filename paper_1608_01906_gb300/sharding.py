"""Halo-sharded runs of one structured lattice: slabs of whole rows.

A lattice too large for one device is cut into slabs of whole rows, one
per device.  A node's next state depends on the present populations up to
4 rows away (h is streamed on the depth-3 density region, whose own values
are streamed from depth-1 neighbours; the derivative chain rho -> grad rho ->
lap rho, mu -> grad mu adds the rest, Sec. 2.2.1 and Sec. 2.3), so every
slab holds 4 halo rows on both sides, steps its own rows, and after each
step (and once after initialisation) receives its halo rows from its
neighbours' first and last 4 own rows.  The mass and momentum totals of the
lattice are the sum of the slabs' totals (an all-reduce across devices).

Cuts at multiples of the step's tile height (8 rows) make a sharded run
bitwise equal to the whole lattice's run: every node is then updated by the
same code path.

What runs where: `SlabRun` holds all slabs on one device, exchanging through
felbm_slab_exchange.  `slab_rows`, `storage_rows`, `neighbours` and
`exchange_ranks` are the host logic of a run with one slab per process
(rank): the partition, the slab's rows in the lattice, and the transport of
the halo messages between ranks over torch.distributed point-to-point calls
(tensors on the ranks' devices with NCCL, host tensors with gloo).
"""
from __future__ import annotations

import numpy as np

from . import felbm

TILE_ROWS = 8  # rows of a step tile: cuts at multiples keep runs bitwise equal
HALO = 4       # halo rows per side


def slab_rows(ny, n_slabs, align=TILE_ROWS):
    """Partition of rows [0, ny) into n_slabs contiguous slabs [(y_begin,
    n_rows), ...], cuts at multiples of `align`, sizes as even as the
    alignment allows, every slab at least 2 * HALO rows."""
    if n_slabs < 1:
        raise ValueError("n_slabs must be positive")
    units = ny // align  # whole aligned blocks; the remainder joins the last slab
    if units < n_slabs:
        raise ValueError("%d rows hold fewer than %d aligned slabs" % (ny, n_slabs))
    cuts = [align * ((k * units) // n_slabs) for k in range(n_slabs)] + [ny]
    out = [(cuts[k], cuts[k + 1] - cuts[k]) for k in range(n_slabs)]
    if any(r < 2 * HALO for _, r in out):
        raise ValueError("a slab would hold fewer than %d rows" % (2 * HALO))
    return out


def storage_rows(y_begin, n_rows, ny, walls):
    """Lattice row of each of a slab's n_rows + 2 * HALO storage rows:
    periodic y wraps around; with walls, rows outside the lattice take the
    nearest lattice row as a stand-in (the step never reads them)."""
    r = np.arange(y_begin - HALO, y_begin + n_rows + HALO)
    return np.clip(r, 0, ny - 1) if walls else np.mod(r, ny)


def slab_fields(field, nx, ny, rows):
    """A node field in lattice order (node x + nx y; trailing component axes
    kept) restricted to the given lattice rows, in the slab's node order."""
    a = np.asarray(field)
    return a.reshape((ny, nx) + a.shape[1:])[rows].reshape((len(rows) * nx,) + a.shape[1:])


def neighbours(rank, world, walls):
    """Ranks of the slabs below and above `rank` (None across a wall)."""
    lo = rank - 1 if rank > 0 else (None if walls else world - 1)
    hi = rank + 1 if rank < world - 1 else (None if walls else 0)
    return lo, hi


def exchange_ranks(send, recv, rank, world, walls, dist, group=None):
    """Carry one rank's halo messages to its neighbours over
    torch.distributed: send[1] (its last own rows) goes up to recv[0] of the
    slab above, send[0] down to recv[1] of the slab below.  send and recv
    are pairs of tensors of equal size ([lo, hi]); a missing neighbour (a
    wall) sends and receives nothing.  One rank alone with periodic y is its
    own neighbour both ways."""
    lo, hi = neighbours(rank, world, walls)
    if world == 1:
        if lo is not None:
            recv[0].copy_(send[1])
            recv[1].copy_(send[0])
        return
    reqs = []
    # tag 0: messages going up (recv lo <- lower's send hi); tag 1: going down
    if lo is not None:
        reqs.append(dist.irecv(recv[0], src=lo, group=group, tag=0))
    if hi is not None:
        reqs.append(dist.irecv(recv[1], src=hi, group=group, tag=1))
    if hi is not None:
        reqs.append(dist.isend(send[1], dst=hi, group=group, tag=0))
    if lo is not None:
        reqs.append(dist.isend(send[0], dst=lo, group=group, tag=1))
    for r in reqs:
        r.wait()


def allreduce_totals(totals, dist, group=None):
    """The lattice's FP64 totals from each rank's slab totals."""
    import torch

    t = torch.as_tensor(np.asarray(totals, dtype=np.float64))
    dist.all_reduce(t, group=group)
    return t.numpy()


class SlabRun:
    """All slabs of one structured lattice on one device, stepped one after
    another and exchanged after every step through felbm_slab_exchange.

    xy, tri, box, tag: the whole lattice (structured split, nx x ny nodes in
    lattice order); params: felbm_params; rho0, u0, p0: initial fields in
    lattice order; rows: the slabs as [(y_begin, n_rows), ...] (slab_rows).
    """

    def __init__(self, xy, tri, box, tag, nx, ny, params, rho0, u0=None, p0=None, rows=None,
                 n_slabs=2, stream=None):
        self.nx, self.ny = int(nx), int(ny)
        self.walls = not (box[1] > 0)
        self.rows = list(rows) if rows is not None else slab_rows(self.ny, n_slabs)
        whole = felbm.Mesh(xy, tri, box, tag, stream=stream)
        try:
            if whole.info()["kind"] != 1:
                raise felbm.FelbmError(felbm.FELBM_ERR_UNSUPPORTED, "SlabRun needs a structured lattice")
            self.meshes = [felbm.Mesh.slab(whole, yb, nr, stream) for yb, nr in self.rows]
        finally:
            whole.close()
        self.states = []
        for (yb, nr), m in zip(self.rows, self.meshes):
            r = storage_rows(yb, nr, self.ny, self.walls)
            sf = lambda f: None if f is None else slab_fields(f, self.nx, self.ny, r)  # noqa: E731
            self.states.append(felbm.State(m, params, sf(rho0), sf(u0), sf(p0)))
        felbm.slab_exchange(self.states)  # halo rows of the initial populations

    def step(self, n=1):
        for _ in range(int(n)):
            for s in self.states:
                s.step(1)
            felbm.slab_exchange(self.states)

    def sync(self):
        for s in self.states:
            s.sync()

    def _own(self, a, k):
        nr = self.rows[k][1]
        return a[HALO * self.nx:(HALO + nr) * self.nx]

    def moments(self):
        """Moments of the whole lattice (lattice order) and its totals, the
        sum of the slabs' FP64 totals."""
        parts = [s.moments() for s in self.states]
        out = {key: np.concatenate([self._own(p[key], k) for k, p in enumerate(parts)])
               for key in ("rho", "C", "u", "p")}
        out["totals"] = np.sum([p["totals"] for p in parts], axis=0)
        return out

    def export(self):
        """Stored pre-collided distributions of the whole lattice (9 x N each)."""
        hs, gs = zip(*[s.export() for s in self.states])
        h = np.concatenate([self._own(a.T, k).T for k, a in enumerate(hs)], axis=1)
        g = np.concatenate([self._own(a.T, k).T for k, a in enumerate(gs)], axis=1)
        return h, g

    def close(self):
        for s in self.states:
            s.close()
        for m in self.meshes:
            m.close()
        self.states, self.meshes = [], []
