"""The components of one half-step at the timed size, against the oracle.

Input: the 2D Ising tensor at beta_c after six half-steps of the oracle
(Dx = Dy = 64, the steady state of the timed workload), its environment M (4096 x 4096, a
graded PSD matrix), the isometry of M with Dcut = 64, and the contraction with
that isometry, each run through the C ABI in the default launch configuration
(split precision: 4 slices, one CTA per tile, D^7 product handing its slices
to the last product; FP64 as well).

* Environment: the whole M against the oracle's (Sec. 2, Eq. for M).
* Isometry: the full-size Jacobi of the oracle takes too long, so the kept
  eigenvalues are compared with LAPACK's eigvalsh of the same M (an
  independent routine), and U is checked for orthonormal columns and small
  Ritz residuals.
* Contraction: three whole j-slices of Tx (D^3 entries each, the first,
  a middle and the last) against the oracle's contraction of those slices.
"""
import math

import numpy as np
import pytest

from oracle import hotrg, models

from paper_2306_00358_gb300 import Solver

pytestmark = pytest.mark.gpu
BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))
DCUT = 64
# elementwise tolerances relative to the largest entry.  Split: each slice
# product carries ~2^-31 relative error per term, accumulated over K = 4096
# and over chained products (P and Q, then M; X1, X2, then the last
# product); measured 3.6e-7 on M at this size.  A dropped slice product or a
# wrong index gives errors above 1e-3.
TOL = {"split": 2e-6, "fp64": 1e-12}
LAM_TOL = {"split": 1e-6, "fp64": 1e-9}


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def tensor64():
    res = hotrg.solve(models.ising_tensor(BETA_C, 0.0), BETA_C, DCUT, 6)
    assert res.dims[-1] == (64, 64)
    return np.ascontiguousarray(res.tensor)


@pytest.fixture(scope="module")
def env_ref(tensor64):
    return hotrg.environment_x(tensor64)


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_environment_d64(torch, tensor64, env_ref, precision):
    with Solver(0, precision=precision) as s:
        m = s.environment(torch.from_numpy(tensor64).cuda()).cpu().numpy()
    assert np.abs(m - env_ref).max() <= TOL[precision] * np.abs(env_ref).max()


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_isometry_d64(torch, env_ref, precision):
    msym = 0.5 * (env_ref + env_ref.T)
    ref = np.linalg.eigvalsh(msym)[::-1][:DCUT]
    with Solver(0, precision=precision) as s:
        u, lam, dn = s.isometry(torch.from_numpy(np.ascontiguousarray(msym)).cuda(), DCUT)
        u = u.cpu().numpy()
    assert dn == DCUT
    assert np.abs(lam - ref).max() <= LAM_TOL[precision] * ref[0]
    assert np.abs(u.T @ u - np.eye(dn)).max() <= 1e-12
    resid = np.linalg.norm(msym @ u - u * lam[None, :], axis=0).max()
    assert resid <= LAM_TOL[precision] * ref[0]


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_contraction_d64_slices(torch, tensor64, env_ref, precision):
    msym = 0.5 * (env_ref + env_ref.T)
    w, v = np.linalg.eigh(msym)
    u = np.ascontiguousarray(v[:, ::-1][:, :DCUT]).reshape(64, 64, DCUT)
    with Solver(0, precision=precision) as s:
        out = s.contract(torch.from_numpy(tensor64).cuda(), torch.from_numpy(u).cuda()).cpu().numpy()
    assert out.shape == (DCUT, 64, DCUT, 64)
    refs = {j: hotrg.contract_x_slice(tensor64, u, j, j + 1) for j in (0, 37, 63)}
    scale = max(np.abs(r).max() for r in refs.values())
    for j, ref in refs.items():
        assert np.abs(out[:, j:j + 1] - ref).max() <= TOL[precision] * scale, j
