"""Split-precision path (BF16 slices on tcgen05, exact FP32 partial sums).

* Integer-valued operands are represented exactly by the slices and their
  products sum exactly, so the split GEMM must agree bit for bit with the
  FP64 product (this checks slicing, TMA layouts, MMA descriptors, the
  exact chunk drains and the integer-built FP64 epilogue).
* Random operands must stay inside the error bound of the splitting:
  |C - AB| <= K rowmax|A| colmax|B| (S + 2) 2^(3 - 8 S).
* Components and full solves against the oracle within the split tolerance
  (|f_split - f_oracle| <= 1e-9).
"""
import json
import os

import numpy as np
import pytest

from oracle import hotrg
from paper_2306_00358_gb300 import Solver, workloads

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "oracle_solves.json")))
F_TOL_SPLIT = 1e-9


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _bound(a, b, s):
    k = a.shape[1]
    return k * np.abs(a).max(axis=1)[:, None] * np.abs(b).max(axis=0)[None, :] * (s + 2) * 2.0 ** (3 - 8 * s)


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (128, 128, 32), (130, 257, 100), (300, 70, 2100), (64, 200, 1025)])
@pytest.mark.parametrize("s", [2, 4])
def test_split_gemm_exact_on_integers(torch, m, n, k, s):
    rng = np.random.default_rng(m * 7 + n * 3 + k + s)
    a = rng.integers(-100, 101, size=(m, k)).astype(np.float64)
    b = rng.integers(-100, 101, size=(k, n)).astype(np.float64)
    ref = a @ b
    with Solver(0, precision="split", split_slices=s) as sv:
        c = sv.gemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    assert np.array_equal(c, ref)


@pytest.mark.parametrize("m,n", [(2_200_000, 3), (3, 2_200_000)])
def test_split_gemm_exact_with_many_rows(torch, m, n):
    # more than 65535 x 32 rows in one operand: the exponent and slicing
    # kernels stride over their row blocks instead of one block per row group
    k = 40
    rng = np.random.default_rng(m + n)
    a = rng.integers(-100, 101, size=(m, k)).astype(np.float64)
    b = rng.integers(-100, 101, size=(k, n)).astype(np.float64)
    ref = a @ b
    with Solver(0, precision="split", split_slices=4) as sv:
        c = sv.gemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    assert np.array_equal(c, ref)


@pytest.mark.parametrize("m,n,k", [(200, 300, 4096), (129, 64, 777), (512, 80, 4096)])
@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_split_gemm_error_bound(torch, m, n, k, s):
    rng = np.random.default_rng(1000 + s)
    a = rng.standard_normal((m, k)) * np.exp(rng.uniform(-8, 8, size=(m, 1)))
    b = rng.standard_normal((k, n)) * np.exp(rng.uniform(-8, 8, size=(1, n)))
    ref = a @ b
    with Solver(0, precision="split", split_slices=s) as sv:
        c = sv.gemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    assert np.all(np.abs(c - ref) <= _bound(a, b, s))


@pytest.mark.parametrize("m,n,k", [(130, 257, 100), (300, 70, 2100), (513, 128, 1100)])
@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_split_gemm_pairs_exact_on_integers(torch, m, n, k, s):
    # the CTA-pair kernel (256-row tiles, cta_group::2) on the same exact cases
    rng = np.random.default_rng(m * 11 + n * 5 + k + s)
    a = rng.integers(-100, 101, size=(m, k)).astype(np.float64)
    b = rng.integers(-100, 101, size=(k, n)).astype(np.float64)
    with Solver(0, precision="split", split_slices=s, mma_pairs=1, autotune=0) as sv:
        c = sv.gemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    assert np.array_equal(c, a @ b)


@pytest.mark.parametrize("m,n,k", [(257, 300, 4096), (1000, 129, 3000), (4096, 512, 2048)])
@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_split_gemm_pairs_match_single(torch, m, n, k, s):
    # the pair kernel issues the single-CTA product table at M = 256: the same
    # products into the same accumulators in the same order, identical bits
    rng = np.random.default_rng(m + n + k + s)
    an = rng.standard_normal((m, k)) * np.exp(rng.uniform(-6, 6, size=(m, 1)))
    bn = rng.standard_normal((k, n))
    a, b = torch.from_numpy(an).cuda(), torch.from_numpy(bn).cuda()
    with Solver(0, precision="split", mma_pairs=0, split_slices=s, autotune=0) as s1, \
            Solver(0, precision="split", mma_pairs=1, split_slices=s, autotune=0) as s2:
        c1 = s1.gemm(a, b)
        c2 = s2.gemm(a, b)
    assert torch.equal(c1, c2)
    ref = an @ bn
    assert np.all(np.abs(c2.cpu().numpy() - ref) <= _bound(an, bn, s))


def test_split_gemm_zero_rows_and_tiny_values(torch):
    a = np.zeros((40, 64))
    a[3] = 1e-300
    a[5, 7] = 3.0
    b = np.ones((64, 33))
    with Solver(0, precision="split", split_slices=4) as sv:
        c = sv.gemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    ref = a @ b
    assert np.array_equal(c[5], ref[5])
    assert np.all(c[[0, 1, 2, 4, 6]] == 0.0)
    assert np.allclose(c[3], ref[3], rtol=1e-9, atol=0)


@pytest.mark.parametrize("dx,dy", [(5, 3), (12, 7), (16, 16)])
def test_split_environment(torch, dx, dy):
    t = workloads.random_tensor((dx, dy, dx, dy), seed=500 + dx)
    ref = hotrg.environment_x(t)
    with Solver(0, precision="split", split_slices=4) as sv:
        m = sv.environment(torch.from_numpy(t).cuda()).cpu().numpy()
    assert np.abs(m - ref).max() <= 1e-7 * np.abs(ref).max()


@pytest.mark.parametrize("dx,dy,dn,ws,pairs", [(8, 8, 20, 0, 0), (12, 7, 33, 0, 0), (16, 16, 64, 3_000_000, 0),
                                               (16, 16, 64, 3_000_000, 1), (32, 32, 40, 0, 1)])
def test_split_contraction(torch, dx, dy, dn, ws, pairs):
    t = workloads.random_tensor((dx, dy, dx, dy), seed=600 + dx)
    u = workloads.random_isometry(dx, dn, seed=700 + dn)
    ref = hotrg.contract_x(t, u)
    with Solver(0, precision="split", split_slices=4, workspace_bytes=ws, mma_pairs=pairs, autotune=0) as sv:
        out = sv.contract(torch.from_numpy(t).cuda(), torch.from_numpy(u).cuda()).cpu().numpy()
    assert np.abs(out - ref).max() <= 1e-7 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["ising_b0.44_d16_n40", "ising_bc_d16_h1e-3_n40", "xy_b1.0_d12_n12"])
@pytest.mark.parametrize("s", [4, 5])
def test_split_solve_matches_oracle(torch, name, s):
    g = GOLDEN[name]
    with Solver(0, precision="split", split_slices=s, trunc=g["trunc"]) as sv:
        sv.init_tensor(g["model"], g["beta"], g["h"])
        sv.coarse_grain(g["dcut"], g["nsteps"])
        f, _ = sv.free_energy()
    assert abs(f - g["f"]) <= F_TOL_SPLIT, (f, g["f"], abs(f - g["f"]))


@pytest.mark.parametrize("dx,dy,dn,ws", [(32, 32, 40, 0), (64, 32, 48, 0), (32, 64, 24, 0),
                                         (64, 64, 20, 200_000_000)])
def test_fused_handover_is_bit_identical(torch, dx, dy, dn, ws):
    # the producer writing the next product's slices must give exactly what
    # slicing its FP64 output gives (several j-blocks, a ragged last one)
    t = workloads.random_tensor((dx, dy, dx, dy), seed=800 + dx + dy)
    u = workloads.random_isometry(dx, dn, seed=900 + dn)
    tt, uu = torch.from_numpy(t).cuda(), torch.from_numpy(u).cuda()
    outs = []
    for fused in (0, 1, 2):
        with Solver(0, precision="split", fused_slices=fused, workspace_bytes=ws) as sv:
            outs.append(sv.contract(tt, uu))
    assert torch.equal(outs[0], outs[1])
    assert torch.equal(outs[0], outs[2])
    ref = hotrg.contract_x(t, u)
    assert np.abs(outs[1].cpu().numpy() - ref).max() <= 1e-7 * np.abs(ref).max()


def test_fused_handover_solve_is_bit_identical(torch):
    # a solve whose bond dimension reaches 32 (x and rotated y half-steps)
    res = []
    for fused in (0, 1, 2):
        with Solver(0, precision="split", fused_slices=fused) as sv:
            sv.init_tensor("ising", 0.44, 0.0)
            sv.coarse_grain(32, 12)
            res.append(sv.free_energy())
    assert res[0] == res[1] == res[2]


@pytest.mark.parametrize("model,beta,h,dcut,nsteps", [("ising", 0.4406868, 1e-3, 32, 12), ("xy", 1.0, 0.0, 24, 8)])
def test_split_solve_pairs_match_single(torch, model, beta, h, dcut, nsteps):
    # every product of the solve on CTA pairs or on single CTAs: identical bits
    out = []
    for pairs in (0, 1):
        with Solver(0, precision="split", mma_pairs=pairs, autotune=0,
                    trunc="multiplet" if model == "xy" else "paper") as sv:
            sv.init_tensor(model, beta, h)
            sv.coarse_grain(dcut, nsteps)
            out.append((sv.free_energy(), sv.tensor()))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])


def test_autotuned_launches_give_the_model_bits(torch):
    # the tuner picks among launch choices that all give identical bits
    rng = np.random.default_rng(77)
    a = torch.from_numpy(rng.standard_normal((4096, 2048))).cuda()
    b = torch.from_numpy(rng.standard_normal((2048, 1024))).cuda()
    with Solver(0, precision="split", autotune=0) as s0, Solver(0, precision="split", autotune=1) as s1:
        c0 = s0.gemm(a, b)
        c1 = s1.gemm(a, b)
        c2 = s1.gemm(a, b)
        tuned = s1.counters()["shapes_tuned"]
    assert torch.equal(c0, c1) and torch.equal(c1, c2)
    assert tuned <= 1
