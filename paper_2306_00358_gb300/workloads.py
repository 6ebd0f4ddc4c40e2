"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds no arithmetic of the method: only the parameters of the workloads
(couplings, cut-offs, step counts) and seeded random tensors for component
checks.  Both the CUDA path and the oracle receive what is generated here.
"""
from __future__ import annotations

import math

import numpy as np

BETA_C_ISING = 0.5 * math.log(1.0 + math.sqrt(2.0))

# 2D Ising, h = 0, beta = 0.44, Dcut = 16, 40 half-steps, FP64
ISING_SMALL = dict(model="ising", beta=0.44, h=0.0, dcut=16, nsteps=40)
# 2D Ising at beta_c, Dcut = 64, 40 half-steps (the headline workload)
ISING_DCUT64 = dict(model="ising", beta=BETA_C_ISING, h=0.0, dcut=64, nsteps=40)
# couplings of the Ising sweep
ISING_BETAS = (BETA_C_ISING, 0.40, 0.48)
ISING_FIELDS = (0.0, 1e-3)
ISING_DCUTS = (32, 48, 64)
# XY (D0 = 9, |n| <= 4)
XY_BETAS = (0.9, 1.0, 1.1, 1.2)
XY_DCUTS = (64, 96)


def random_tensor(shape, seed: int, positive: bool = False) -> np.ndarray:
    rng = np.random.default_rng(seed)
    t = rng.standard_normal(shape)
    return np.abs(t) + 0.05 if positive else t


def random_isometry(dx: int, dn: int, seed: int) -> np.ndarray:
    """Orthonormal columns (dx*dx, dn) reshaped (dx, dx, dn), seeded."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((dx * dx, dn)))
    return np.ascontiguousarray(q.reshape(dx, dx, dn))


def graded_psd(n: int, decades: float, seed: int) -> np.ndarray:
    """Symmetric PSD matrix with eigenvalues 10^-(decades * i / (n-1))."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = 10.0 ** (-decades * np.arange(n) / max(1, n - 1))
    return (q * lam) @ q.T
