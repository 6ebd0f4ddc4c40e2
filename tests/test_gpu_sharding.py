"""The split half-step (trg_shard_begin / trg_shard_finish) on one GPU.

Two contexts play two ranks: each runs the environment and the isometry,
contracts its rows of j (sharding.j_ranges), the slabs are concatenated as
the all-gather would lay them out, and both contexts place the result.  No
kernel waits on another context's work, so this runs safely on one GPU; the
exchange itself (torch.distributed) is covered on CPU ranks in
test_sharding.py.  The contraction's rows are independent and every product
is deterministic, so the split solve must equal the unsplit one bit for bit.
"""
import ctypes

import numpy as np
import pytest

from paper_2306_00358_gb300 import Solver, _lib, sharding
from paper_2306_00358_gb300.solver import TRGError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _split_solve(torch, world, model, beta, h, dcut, nsteps, **cfg):
    ranks = [Solver(0, **cfg) for _ in range(world)]
    try:
        for s in ranks:
            s.init_tensor(model, beta, h)
        for _ in range(nsteps):
            steps, dx, dy, _ = ranks[0].state()
            nj = ranks[0].shard_extent()
            rx = dx if (steps + 1) % 2 == 1 else dy
            dn_max = min(rx * rx, dcut)
            rows = sharding.slab_rows(nj, world)
            slabs, dns = [], []
            for r, s in enumerate(ranks):
                j0, j1 = sharding.j_ranges(nj, world)[r]
                slab = torch.full((sharding.slab_elems(rows, dn_max, nj),), float("nan"), dtype=torch.float64,
                                  device="cuda")
                dns.append(s.shard_begin(dcut, j0, j1, slab))
                slabs.append(slab)
            assert len(set(dns)) == 1
            per = sharding.slab_elems(rows, dns[0], nj)
            gathered = torch.cat([sl[:per] for sl in slabs])
            for s in ranks:
                s.shard_finish(gathered, world * rows)
        out = [s.free_energy() for s in ranks]
        tensors = [s.tensor() for s in ranks]
    finally:
        for s in ranks:
            s.close()
    return out, tensors


def _plain_solve(model, beta, h, dcut, nsteps, **cfg):
    with Solver(0, **cfg) as s:
        s.init_tensor(model, beta, h)
        s.coarse_grain(dcut, nsteps)
        return s.free_energy(), s.tensor()


@pytest.mark.parametrize("world,model,beta,h,dcut,nsteps,cfg", [
    (2, "ising", 0.44, 1e-3, 16, 14, {"precision": "fp64"}),
    (2, "ising", 0.44, 1e-3, 32, 10, {"precision": "split"}),
    (3, "ising", 0.4406868, 0.0, 24, 11, {"precision": "split"}),
    (4, "xy", 1.0, 0.0, 20, 8, {"precision": "split", "trunc": "multiplet"}),
])
def test_split_half_steps_equal_the_unsplit_solve(torch, world, model, beta, h, dcut, nsteps, cfg):
    got, tens = _split_solve(torch, world, model, beta, h, dcut, nsteps, **cfg)
    ref, ref_t = _plain_solve(model, beta, h, dcut, nsteps, **cfg)
    for (f, lnz), t in zip(got, tens):
        assert f == ref[0] and lnz == ref[1]
        np.testing.assert_array_equal(t, ref_t)


def test_split_half_step_states(torch):
    with Solver(0, precision="split") as s:
        buf = torch.empty(1 << 16, dtype=torch.float64, device="cuda")
        with pytest.raises(TRGError) as e:
            s.shard_extent()
        assert e.value.status == _lib.TRG_ESTATE
        s.init_tensor("ising", 0.44, 0.0)
        with pytest.raises(TRGError) as e:
            s.shard_finish(buf, 4)
        assert e.value.status == _lib.TRG_ESTATE
        with pytest.raises(TRGError) as e:
            s.shard_begin(8, 0, 3, buf)                 # the extent of the first step is 2
        assert e.value.status == _lib.TRG_EINVAL
        assert s.shard_begin(8, 0, 1, buf) == 4
        with pytest.raises(TRGError) as e:
            s.shard_begin(8, 1, 2, buf)                 # the first split half-step is still open
        assert e.value.status == _lib.TRG_ESTATE
        with pytest.raises(TRGError) as e:
            s.coarse_grain(8, 1)
        assert e.value.status == _lib.TRG_ESTATE
        with pytest.raises(TRGError) as e:
            s.shard_finish(buf, 1)                      # fewer rows than the extent
        assert e.value.status == _lib.TRG_EINVAL
    with Solver(0, precision="split") as s:
        s.init_tensor("ising", 0.44, 0.0)
        small = torch.empty(4, dtype=torch.float64, device="cuda")
        with pytest.raises(TRGError) as e:
            s.shard_begin(8, 0, 2, small)
        assert e.value.status == _lib.TRG_EINVAL
        s.init_tensor("ising", 0.44, 0.0)
        s.init_impure()
        with pytest.raises(TRGError) as e:
            s.shard_begin(8, 0, 2, torch.empty(1 << 10, dtype=torch.float64, device="cuda"))
        assert e.value.status == _lib.TRG_ENOTSUP
