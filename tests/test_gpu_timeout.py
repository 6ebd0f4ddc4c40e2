"""A bounded device wait that runs out, and the context afterwards.

Every mbarrier wait of the split-product kernel is bounded; on expiry the
kernel records a timeout, stops issuing, waits (bounded) for its own bulk
copies and tensor-core work in flight, frees its tensor memory and returns,
and the host reports TRG_ETIMEOUT.  The epilogue's wait for a finished
accumulator chunk gets a 1 ns limit here, far below the microseconds one
512-deep chunk of products takes, so it runs out; the products it waited
for complete on their own and every other wait keeps its 2 s limit.  Nothing
faults or hangs: the same context then computes the same product as before.
"""
import numpy as np
import pytest

from paper_2306_00358_gb300 import Solver, _lib
from paper_2306_00358_gb300.solver import TRGError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.mark.parametrize("slices", [4, 5])
def test_accumulator_wait_runs_out_then_the_context_recovers(torch, slices):
    rng = np.random.default_rng(7)
    a = torch.from_numpy(rng.standard_normal((1024, 4096))).cuda()
    b = torch.from_numpy(rng.standard_normal((4096, 512))).cuda()
    with Solver(0, precision="split", split_slices=slices) as s:
        ref = s.gemm(a, b)
        s.set_wait_limit(1)
        with pytest.raises(TRGError) as e:
            s.gemm(a, b)
        assert e.value.status == _lib.TRG_ETIMEOUT
        s.set_wait_limit(0)
        again = s.gemm(a, b)
        torch.cuda.synchronize()
        assert torch.equal(again, ref)
    # and a solve on a fresh context is unaffected
    with Solver(0, precision="split") as s:
        s.init_tensor("ising", 0.44, 0.0)
        s.coarse_grain(8, 6)
        f, _ = s.free_energy()
    assert np.isfinite(f)
