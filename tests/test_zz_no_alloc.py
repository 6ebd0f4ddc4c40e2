"""The allocation-free split GEMM (trg_gemm_noalloc) against trg_gemm.

trg_gemm_noalloc serves callers that must not allocate device memory while
they run (for instance a server whose memory pool owns the whole device): it
keeps its scratch in a fixed device array inside the library.  This file is
collected last, so a run that stops at its first failure has already run
every other test; it must also pass on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2306_00358_gb300 import Solver, _lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _noalloc(lib, torch, a, b, slices, stream):
    m, k = a.shape
    n = b.shape[1]
    c = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.trg_gemm_noalloc(m, n, k, a.data_ptr(), k, b.data_ptr(), n, c.data_ptr(), n, slices,
                              ctypes.c_void_p(stream.cuda_stream))
    assert st == _lib.TRG_OK, lib.trg_status_string(st)
    torch.cuda.synchronize()
    return c.cpu().numpy()


@pytest.mark.parametrize("m,n,k,slices", [(300, 257, 1100, 4), (128, 64, 4096, 5), (7, 3, 5, 2)])
def test_noalloc_matches_trg_gemm_twice(torch, m, n, k, slices):
    lib = _lib.load()
    rng = np.random.default_rng(m + n + k)
    stream = torch.cuda.current_stream()
    results = []
    for call in range(2):
        # different operands on the two calls: the shared scratch keeps the
        # previous call's contents, which must not leak into this one
        a_h = rng.standard_normal((m, k)) * (1.0 + 10 * call)
        b_h = rng.standard_normal((k, n))
        a = torch.from_numpy(a_h).cuda()
        b = torch.from_numpy(b_h).cuda()
        got = _noalloc(lib, torch, a, b, slices, stream)
        with Solver(0, precision="split", split_slices=slices) as sv:
            ref = sv.gemm(a, b).cpu().numpy()
        # same kernels and the same arithmetic: agreement is exact
        assert np.array_equal(got, ref)
        # and within the splitting's error bound of the FP64 product
        bound = k * np.abs(a_h).max(axis=1)[:, None] * np.abs(b_h).max(axis=0)[None, :] * (slices + 2) \
            * 2.0 ** (3 - 8 * slices)
        assert np.all(np.abs(got - a_h @ b_h) <= bound)
        results.append(got)
    assert not np.array_equal(results[0], results[1])


def test_noalloc_rejects_oversized_and_bad_arguments(torch):
    lib = _lib.load()
    a = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    # 8192 x 8192 x 8192 needs far more than the 64 MiB scratch
    st = lib.trg_gemm_noalloc(8192, 8192, 8192, a.data_ptr(), 8192, a.data_ptr(), 8192, a.data_ptr(), 8192, 4,
                              None)
    assert st == _lib.TRG_EINVAL
    assert lib.trg_gemm_noalloc(8, 8, 8, a.data_ptr(), 8, a.data_ptr(), 8, a.data_ptr(), 8, 6, None) == \
        _lib.TRG_EINVAL
    assert lib.trg_gemm_noalloc(8, 8, 8, None, 8, a.data_ptr(), 8, a.data_ptr(), 8, 4, None) == _lib.TRG_EINVAL
