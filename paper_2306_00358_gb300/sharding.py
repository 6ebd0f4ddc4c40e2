"""One HOTRG solve split over ranks (one GPU each): the host-side partition
and the exchange, around trg_shard_begin / trg_shard_finish.

The contraction of a half-step (Sec. 2, Tx[i,j,k,l] = sum U[a,b,i]
t[b,j,d,c] t[a,c,e,l] U[e,d,k]) is split over its free index j: rank r
computes the output rows j in j_ranges(nj, world)[r], every rank runs the
environment and the isometry itself (same inputs, same kernels, so the same
isometry everywhere), and one all-gather of the slabs per half-step gives
every rank the whole coarse tensor.  The paper reports multi-GPU speed-ups
(Sec. 3.1, Sec. 4) without saying how it partitions; this is the partition
of this library.

Layouts (the same as the C ABI's):
  slab of rank r:   S[jj][i][k][l] = O[i, j0 + jj, k, l], rows jj < slab_rows
                    (rows past the rank's range are padding);
  gathered:         G[j][i][k][l], the ranks' slabs in rank order, so row j
                    of G is O[:, j, :, :] for j < nj.
O is the output of the x formulas (Dn, nj, Dn, nj); for a y half-step the
library rotates it into place itself.

Argument marshalling and torch.distributed plumbing only: every step of the
path runs in the library's kernels.
"""
from __future__ import annotations

import math


def slab_rows(nj: int, world: int) -> int:
    """Rows of j per rank: ceil(nj / world), the same for every rank so that
    the slabs can be all-gathered."""
    if nj < 0 or world < 1:
        raise ValueError("nj >= 0 and world >= 1 required")
    return max(1, math.ceil(nj / world)) if nj else 0


def j_ranges(nj: int, world: int) -> list[tuple[int, int]]:
    """[j0, j1) of every rank: consecutive blocks of slab_rows(nj, world);
    trailing ranks may get fewer rows (or none)."""
    rows = slab_rows(nj, world)
    return [(min(nj, r * rows), min(nj, (r + 1) * rows)) for r in range(world)]


def slab_elems(rows: int, dn: int, nj: int) -> int:
    """Doubles in one slab of `rows` rows."""
    return rows * dn * dn * nj


def unpack_gathered(g, dn: int, nj: int):
    """Host statement of what trg_shard_finish reads: the gathered buffer
    (flat, rows of dn*dn*nj) as O[i, j, k, l] of shape (dn, nj, dn, nj)."""
    rows = g.reshape(-1, dn, dn, nj)
    return rows[:nj].transpose(1, 0, 2, 3)


class ShardedSolver:
    """Runs half-steps of `solver` split over the ranks of a torch.distributed
    process group.  `solver` is a Solver (or any object with state(),
    shard_extent(), shard_begin(), shard_finish()), and every rank holds one
    initialised the same way."""

    def __init__(self, solver, group=None, device=None):
        import torch
        import torch.distributed as dist

        self.s = solver
        self.group = group
        self.dist = dist
        self.torch = torch
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())

    def half_step(self, dcut: int) -> int:
        torch, dist = self.torch, self.dist
        steps, dx, dy, _ = self.s.state()
        xdir = (steps + 1) % 2 == 1
        nj = self.s.shard_extent()
        rx = dx if xdir else dy                # the blocked legs' extent
        dn_max = min(rx * rx, int(dcut))
        rows = slab_rows(nj, self.world)
        j0, j1 = j_ranges(nj, self.world)[self.rank]
        slab = torch.empty(max(1, slab_elems(rows, dn_max, nj)), dtype=torch.float64, device=self.device)
        dn = self.s.shard_begin(dcut, j0, j1, slab)
        # every rank must have kept the same dimension
        dns = [torch.zeros(1, dtype=torch.int64, device=self.device) for _ in range(self.world)]
        dist.all_gather(dns, torch.tensor([dn], dtype=torch.int64, device=self.device), group=self.group)
        if any(int(x.item()) != dn for x in dns):
            raise RuntimeError(f"ranks kept different dimensions {[int(x.item()) for x in dns]}")
        per = slab_elems(rows, dn, nj)
        gathered = torch.empty(self.world * per, dtype=torch.float64, device=self.device)
        dist.all_gather_into_tensor(gathered, slab[:per], group=self.group)
        self.s.shard_finish(gathered, self.world * rows)
        return dn

    def coarse_grain(self, dcut: int, nsteps: int):
        for _ in range(int(nsteps)):
            self.half_step(dcut)
