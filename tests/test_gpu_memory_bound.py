"""The admission estimate of a solve bounds what the solve allocates.

The server admits a request when its estimate (trg_solve_bytes) fits in what
the HBM budget has left, so the estimate must be an upper bound of the
device memory one solve's context holds.  A tracking allocator hook
(trg_set_allocator) records the live bytes of one context through whole
solves, with the serving slots' 1 GiB contraction workspace, and the peak is
checked against the estimate.
"""
import pytest

from paper_2306_00358_gb300 import Solver, _lib
from paper_2306_00358_gb300 import serving as sv

pytestmark = pytest.mark.gpu
WORKSPACE = 1 << 30


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


class _Tracker:
    def __init__(self, torch, device):
        self.live = 0
        self.peak = 0
        self.sizes = {}

        def alloc(nbytes, stream, user):
            try:
                p = int(torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0))
            except Exception:
                return None
            self.sizes[p] = int(nbytes)
            self.live += int(nbytes)
            self.peak = max(self.peak, self.live)
            return p

        def free(ptr, nbytes, stream, user):
            self.live -= self.sizes.pop(ptr, 0)
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc = _lib.ALLOC_FN(alloc)
        self.free = _lib.FREE_FN(free)


@pytest.mark.parametrize("model,beta,dcut,nsteps,precision,trunc", [
    ("ising", 0.4406868, 64, 12, "split", "paper"),
    ("ising", 0.4406868, 32, 12, "fp64", "paper"),
    ("xy", 1.1, 48, 8, "split", "multiplet"),
    ("potts", 1.0, 24, 10, "split", "multiplet"),
])
def test_solve_stays_within_its_admission_estimate(torch, model, beta, dcut, nsteps, precision, trunc):
    spec = sv.Spec(model=model, beta=beta, dcut=dcut, nsteps=nsteps, precision=precision, trunc=trunc)
    bound = sv.solve_bytes(spec, WORKSPACE)
    tr = _Tracker(torch, 0)
    with Solver(0, torch_alloc=False, precision=precision, trunc=trunc, workspace_bytes=WORKSPACE) as s:
        s._check(s._lib.trg_set_allocator(s._h, tr.alloc, tr.free, None), "trg_set_allocator")
        s.init_tensor(model, beta, 0.0)
        s.coarse_grain(dcut, nsteps)
        s.free_energy()
        torch.cuda.synchronize()
    assert tr.peak > 0
    assert tr.peak <= bound, (tr.peak, bound)
