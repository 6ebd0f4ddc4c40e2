"""Python face of the oracle's cyclic Jacobi eigensolver (``jacobi.c``).

ORACLE / TEST INFRASTRUCTURE ONLY.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native

_P = ctypes.POINTER(ctypes.c_double)


def eigh(a: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Eigendecomposition of a real symmetric matrix by cyclic Jacobi.

    Returns ``(w, v, sweeps)`` with the eigenvalues ``w`` sorted in descending
    order and ``v[:, k]`` the unit eigenvector of ``w[k]``.  Raises
    ``RuntimeError`` if the sweeps do not converge.
    """
    a = np.array(a, dtype=np.float64, order="C", copy=True)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("eigh: square matrix expected")
    n = a.shape[0]
    if n == 0:
        return np.zeros(0), np.zeros((0, 0)), 0
    w = np.empty(n, dtype=np.float64)
    vt = np.empty((n, n), dtype=np.float64)
    sweeps = ctypes.c_int(0)
    rc = _native.lib().oracle_jacobi_eigh(
        n, a.ctypes.data_as(_P), w.ctypes.data_as(_P), vt.ctypes.data_as(_P),
        float(tol), int(max_sweeps), ctypes.byref(sweeps))
    if rc < 0:
        raise ValueError("eigh: bad arguments")
    if rc > 0:
        raise RuntimeError(f"eigh: Jacobi did not converge in {max_sweeps} sweeps")
    # Descending order; a stable sort keeps equal eigenvalues in diagonal order.
    order = np.argsort(-w, kind="stable")
    return w[order], vt[order].T.copy(), int(sweeps.value)
