"""One solve split over two ranks (gloo on CPU): the partition, the exchange
and the layouts that the GPU path uses, with the oracle doing the arithmetic.

The half-step is cut where trg_shard_begin / trg_shard_finish cut it: the
environment and the isometry on every rank, the output rows j of the
contraction (Sec. 2) split by sharding.j_ranges, one all-gather of the slabs,
then the placement of the gathered rows.  ShardedSolver runs unchanged on
an oracle back end, so its partition, padding and exchange are the ones the
GPU ranks run; the result must equal the unsplit oracle solve.
"""
import math
import os
import socket

import numpy as np
import pytest

from oracle import hotrg, models
from paper_2306_00358_gb300 import sharding


class OracleShardBackend:
    """The oracle's half-step behind the same calls as the library's split
    half-step (state, shard_extent, shard_begin, shard_finish)."""

    def __init__(self, t0, beta, trunc="paper"):
        t = np.array(t0, dtype=np.float64)
        n0 = float(np.max(np.abs(t)))
        self.t = t / n0
        self.lnz = math.log(n0)
        self.beta = beta
        self.steps = 0
        self.trunc = trunc
        self.pending = None

    def state(self):
        return self.steps, self.t.shape[0], self.t.shape[1], self.lnz

    def shard_extent(self):
        k = self.steps + 1
        return self.t.shape[1] if k % 2 == 1 else self.t.shape[0]

    def shard_begin(self, dcut, j0, j1, slab):
        k = self.steps + 1
        r = self.t if k % 2 == 1 else hotrg.rotate_in(self.t)
        u, lam = hotrg.isometry(hotrg.environment_x(r), dcut, self.trunc)
        dn, nj = u.shape[2], r.shape[1]
        if j1 > j0:
            o = hotrg.contract_x_slice(r, u, j0, j1)          # (dn, j1 - j0, dn, nj)
            part = np.ascontiguousarray(o.transpose(1, 0, 2, 3)).ravel()
            slab.numpy()[:part.size] = part
        self.pending = (k, dn, nj)
        return dn

    def shard_finish(self, gathered, j_rows):
        k, dn, nj = self.pending
        self.pending = None
        assert j_rows >= nj
        o = np.ascontiguousarray(sharding.unpack_gathered(gathered.numpy(), dn, nj))
        t = o if k % 2 == 1 else hotrg.rotate_out(o)
        nk = float(np.max(np.abs(t)))
        self.t = t / nk
        self.lnz += math.ldexp(math.log(nk), -k)
        self.steps = k

    def free_energy(self):
        lnz = self.lnz + math.ldexp(math.log(hotrg.trace_pbc(self.t)), -self.steps)
        return -lnz / self.beta, lnz


def test_ranges_cover_every_row_once():
    for nj in range(0, 70):
        for world in (1, 2, 3, 4, 8):
            rg = sharding.j_ranges(nj, world)
            assert len(rg) == world
            rows = sharding.slab_rows(nj, world)
            seen = []
            for j0, j1 in rg:
                assert 0 <= j0 <= j1 <= nj and j1 - j0 <= rows
                seen.extend(range(j0, j1))
            assert seen == list(range(nj))
            assert world * rows >= nj


def test_unpack_is_the_transpose_of_the_slabs():
    rng = np.random.default_rng(0)
    dn, nj, world = 3, 5, 2
    o = rng.standard_normal((dn, nj, dn, nj))
    rows = sharding.slab_rows(nj, world)
    g = np.full((world * rows, dn, dn, nj), np.nan)
    for r, (j0, j1) in enumerate(sharding.j_ranges(nj, world)):
        g[r * rows:r * rows + (j1 - j0)] = o[:, j0:j1].transpose(1, 0, 2, 3)
    np.testing.assert_array_equal(sharding.unpack_gathered(g.ravel(), dn, nj), o)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASES = [("ising", 0.44, 1e-3, 5, 8, "paper"), ("xy", 1.0, 0.0, 7, 5, "multiplet")]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for (model, beta, h, dcut, nsteps, trunc) in CASES:
            be = OracleShardBackend(models.initial_tensor(model, beta, h), beta, trunc)
            sharding.ShardedSolver(be, device=torch.device("cpu")).coarse_grain(dcut, nsteps)
            f, lnz = be.free_energy()
            out.put((rank, model, f, lnz, be.t.shape))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_split_solve_equals_the_unsplit_oracle():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2 * len(CASES))]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for (model, beta, h, dcut, nsteps, trunc) in CASES:
        ref = hotrg.solve(models.initial_tensor(model, beta, h), beta, dcut, nsteps, trunc=trunc)
        got = [r for r in res if r[1] == model]
        assert len(got) == 2
        for _, _, f, lnz, shape in got:
            assert shape == ref.tensor.shape
            assert abs(lnz - ref.lnz_per_site) <= 1e-13 * abs(ref.lnz_per_site)
            assert abs(f - ref.f) <= 1e-13 * abs(ref.f)
        # both ranks hold the same coarse tensor, so the same free energy
        assert got[0][2] == got[1][2]
