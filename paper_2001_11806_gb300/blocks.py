"""x-slab block partition (Sec. IV-D "Framework Integration": a
block-structured domain whose blocks exchange the populations that cross
their faces through generated pack and unpack kernels).

Each block is an ordinary context over its slab x in [x0, x1) plus one ghost
layer per x face (local x = 0 and nx_b + 1): flagged LBM_GHOST where the
neighbouring block's cell is fluid, with that cell's own flag otherwise, and
NOSLIP outside a non-periodic global domain.  The block's own x axis is not
periodic; y and z are the global domain's.  After the initialisation and
after every step each block packs what crosses each face (lbm_halo_pack) and
the neighbour across that face unpacks it (lbm_halo_unpack); the pattern and
step parity decide which slots travel, inside the library.

``SlabBlocks`` runs all blocks on one device and exchanges through device
buffers.  ``exchange_plan`` and ``exchange_ranks`` give the same schedule
for blocks held by different processes (one block per rank), over
torch.distributed point-to-point calls.
"""
import ctypes

import numpy as np
import torch

from ._lib import LbmError, check, lib
from .sim import Sim

XLOW, XHIGH = 0, 1
GHOST = 8


def block_flags(flags, x0, x1, periodic_x):
    """Flags [nz][ny][x1 - x0 + 2] of the block holding global x in [x0, x1)
    of the global flag field [nz][ny][nx] (None = all fluid)."""
    nz, ny, nx = flags.shape
    out = np.zeros((nz, ny, x1 - x0 + 2), np.uint8)
    for i, gx in enumerate(range(x0 - 1, x1 + 1)):
        inside = 0 <= gx < nx
        g = gx % nx
        if 1 <= i <= x1 - x0:
            out[..., i] = flags[..., g]
        elif not inside and not periodic_x:
            out[..., i] = 1  # NOSLIP: outside a non-periodic axis
        else:
            out[..., i] = np.where(flags[..., g] == 0, GHOST, flags[..., g])
    return out


def exchange_plan(nblocks, periodic_x):
    """(sender, face, receiver, receiver_face) for every face that carries
    populations: block b's XHIGH feeds block b + 1's XLOW and back; with a
    periodic x axis the last block and the first are neighbours too (a single
    block is then its own neighbour)."""
    plan = []
    for b in range(nblocks):
        right = b + 1 if b + 1 < nblocks else (0 if periodic_x else None)
        if right is None:
            continue
        plan.append((b, XHIGH, right, XLOW))
        plan.append((right, XLOW, b, XHIGH))
    return plan


def exchange_ranks(pack, unpack, rank, world, periodic_x, dist):
    """The exchange of the block held by this rank (blocks ordered by rank
    along x): pack(face) returns the tensor to send across that face,
    unpack(face, tensor) stores what arrives there.  Sends and receives are
    posted together (isend / irecv) so that no ordering of the ranks
    deadlocks, tagged with the sender's face, so that two ranks that are
    neighbours across both faces (two periodic ranks) match each message to
    its face; a single periodic rank exchanges with itself locally."""
    left = rank - 1 if rank > 0 else (world - 1 if periodic_x else None)
    right = rank + 1 if rank + 1 < world else (0 if periodic_x else None)
    out = {f: pack(f) for f, nb in ((XLOW, left), (XHIGH, right)) if nb is not None}
    if world == 1:
        for f in out:
            unpack(XHIGH if f == XLOW else XLOW, out[f])
        return
    inbox, reqs = {}, []
    for f, nb in ((XLOW, left), (XHIGH, right)):
        if nb is None:
            continue
        inbox[f] = torch.empty_like(out[f])
        reqs.append(dist.isend(out[f], nb, tag=f))
        # what arrives across face f was sent across the neighbour's other face
        reqs.append(dist.irecv(inbox[f], nb, tag=XHIGH if f == XLOW else XLOW))
    for r in reqs:
        r.wait()
    for f, t in inbox.items():
        unpack(f, t)


class SlabBlocks:
    """The global domain `shape` = (nx, ny, nz) split at the x positions
    `cuts` (0 = cuts[0] < ... < cuts[-1] = nx), every block a Sim on one
    device; the remaining arguments are Sim's."""

    def __init__(self, stencil, collision, storage, pattern, shape, cuts, periodic=(True, True, True), flags=None,
                 device="cuda:0", **kw):
        if pattern not in ("pull", "aa"):
            raise LbmError("block halos are built for the pull and AA patterns")
        nx, ny, nz = shape
        if cuts[0] != 0 or cuts[-1] != nx or any(b - a < 1 for a, b in zip(cuts, cuts[1:])):
            raise LbmError("cuts must rise from 0 to nx")
        self.shape, self.cuts, self.periodic = tuple(shape), list(cuts), tuple(periodic)
        gflags = np.zeros((nz, ny, nx), np.uint8) if flags is None else np.asarray(flags, np.uint8).reshape(nz, ny, nx)
        self.blocks = []
        for x0, x1 in zip(cuts, cuts[1:]):
            fl = block_flags(gflags, x0, x1, periodic[0])
            self.blocks.append(Sim(stencil, collision, storage, pattern, (x1 - x0 + 2, ny, nz),
                                   periodic=(False, periodic[1], periodic[2]), flags=fl, device=device, **kw))
        p = self.blocks[0].params
        b = ctypes.c_size_t()
        check(lib().lbm_halo_bytes(ctypes.byref(p), ctypes.byref(b)), what="halo_bytes")
        self.plan = exchange_plan(len(self.blocks), periodic[0])
        self.bufs = {(s, f): torch.empty(b.value, dtype=torch.uint8, device=self.blocks[0].device)
                     for s, f, _, _ in self.plan}

    def _slab(self, arr, b, comps):
        """Rows of a global [comps][nz][ny][nx] array for block b, ghost
        columns included (wrapped; their values are replaced by the halo)."""
        x0, x1 = self.cuts[b], self.cuts[b + 1]
        idx = [x % self.shape[0] for x in range(x0 - 1, x1 + 1)]
        return np.ascontiguousarray(arr.reshape((comps,) + self.shape[::-1])[..., idx])

    def exchange(self):
        L = lib()
        for s, f, _, _ in self.plan:
            sim = self.blocks[s]
            check(L.lbm_halo_pack(sim.ctx, f, self.bufs[(s, f)].data_ptr()), sim.ctx, "halo_pack")
        for s, f, r, rf in self.plan:
            sim = self.blocks[r]
            check(L.lbm_halo_unpack(sim.ctx, rf, self.bufs[(s, f)].data_ptr()), sim.ctx, "halo_unpack")

    def init_equilibrium(self, rho, u):
        d = self.blocks[0].d
        rho, u = np.asarray(rho, np.float64), np.asarray(u, np.float64)
        for b, sim in enumerate(self.blocks):
            sim.init_equilibrium(self._slab(rho, b, 1).reshape(-1), self._slab(u, b, d).reshape(d, -1))
        self.exchange()

    def set_state(self, P):
        q = self.blocks[0].q
        for b, sim in enumerate(self.blocks):
            sim.set_state(self._slab(np.asarray(P, np.float64), b, q).reshape(q, -1))
        self.exchange()

    def step(self, n=1):
        for _ in range(int(n)):
            for sim in self.blocks:
                sim.step(1)
            self.exchange()

    def populations(self):
        """Global f [q][N] (FP64, device) assembled from the blocks' interiors."""
        q = self.blocks[0].q
        nx, ny, nz = self.shape
        out = torch.empty((q, nz, ny, nx), dtype=torch.float64, device=self.blocks[0].device)
        for b, sim in enumerate(self.blocks):
            x0, x1 = self.cuts[b], self.cuts[b + 1]
            f = sim.populations().reshape(q, nz, ny, x1 - x0 + 2)
            out[..., x0:x1] = f[..., 1:x1 - x0 + 1]
        return out.reshape(q, -1)

    def close(self):
        for sim in self.blocks:
            sim.close()
