"""Plain CPU FP64 HOTRG on the cubic lattice: the oracle for the 3D path.

ORACLE / TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU
baseline leg of the benchmark import this module; the GPU product path never
does, and this module imports nothing from the GPU package.

The paper carries its method to three dimensions only as the direction of
future work (Sec. 1 and Sec. 4): it gives no 3D blocking.  This is the 2D
variant of Sec. 2 (the coarse-graining listing) with one more pair of legs,
read as follows (each reading is named in the design notes):

  * the site tensor t[x, x', y, y', z, z'] has legs (left, right, front,
    back, down, up), shape (Dx, Dx, Dy, Dy, Dz, Dz);
  * a z step stacks two copies along z, the lower one's up leg bonded to
    the upper one's down leg (bond m), and keeps the lower one's down leg
    and the upper one's up leg;
  * each transverse pair of legs is truncated by an isometry taken, as in
    the listing, from one side only: U_x (first index the lower tensor's
    leg) from the environment of the two left legs, applied to the left pair
    and to the right pair; U_y likewise from the two front legs;
  * the environment of the left legs is the Gram matrix of the stacked pair
    over all its other legs,
        M_x[(x1, x2), (a1, a2)] = sum_{m, n} P1[x1, m, a1, n] P2[x2, m, a2, n],
        P1[x1, m, a1, n] = sum t[x1, x1', y1, y1', z, m] t[a1, x1', y1, y1', z, n],
        P2[x2, m, a2, n] = sum t[x2, x2', y2, y2', m, z'] t[a2, x2', y2, y2', n, z'],
    (the sums over the lower tensor's down leg z and the upper one's up leg
    z' fall inside P1 and P2), and M_y the same with the front legs;
  * the blocked tensor is
        T'[X, X', Y, Y', z, z'] = sum U_x[x1, x2, X] U_x[x1', x2', X']
            U_y[y1, y2, Y] U_y[y1', y2', Y'] t[x1, x1', y1, y1', z, m] t[x2, x2', y2, y2', m, z'],
    shape (Nx, Nx, Ny, Ny, Dz, Dz) with Nx = min(Dx^2, Dcut), Ny = min(Dy^2, Dcut);
  * steps cycle z, x, y: after each one the tensor is rotated,
    R = permute(T', (2, 3, 4, 5, 0, 1)), so that the next axis to block sits
    in the z slot; three rotations restore the original frame;
  * normalisation by max |T| after every step and
        ln Z / V = ln n0 + sum_k 2^-k ln n_k + 2^-N ln Tr T_N,
    Tr T = sum T[x, x, y, y, z, z] (periodic boundaries), as in 2D.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import hotrg


def ising3d_tensor(beta: float, h: float = 0.0) -> np.ndarray:
    """Rank-6 Ising site tensor on the cubic lattice, shape (2,)*6:
    T[x, x', y, y', z, z'] = sum_s e^{beta h s} W_sx W_sx' W_sy W_sy' W_sz W_sz'
    with W the symmetric square root of the bond matrix (the 2D tensor's
    construction with two more legs)."""
    if not (beta >= 0.0 and math.isfinite(beta)):
        raise ValueError("beta must be finite and >= 0")
    from .models import ising_weight_sqrt
    w = ising_weight_sqrt(beta)
    t = np.zeros((2,) * 6)
    for s_idx, s in enumerate((1.0, -1.0)):
        ws = w[s_idx]
        t += math.exp(beta * h * s) * np.einsum("a,b,c,d,e,f->abcdef", ws, ws, ws, ws, ws, ws)
    return t


def environments_z(t: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(M_x, M_y) of the z step, shapes (Dx^2, Dx^2) and (Dy^2, Dy^2),
    rows and columns (lower leg, upper leg)."""
    dx, dy = t.shape[0], t.shape[2]
    p1 = np.tensordot(t, t, axes=([1, 2, 3, 4], [1, 2, 3, 4]))     # (x1, m, a1, n)
    p2 = np.tensordot(t, t, axes=([1, 2, 3, 5], [1, 2, 3, 5]))     # (x2, m, a2, n)
    mx = np.tensordot(p1, p2, axes=([1, 3], [1, 3]))               # (x1, a1, x2, a2)
    mx = mx.transpose(0, 2, 1, 3).reshape(dx * dx, dx * dx)
    q1 = np.tensordot(t, t, axes=([0, 1, 3, 4], [0, 1, 3, 4]))     # (y1, m, b1, n)
    q2 = np.tensordot(t, t, axes=([0, 1, 3, 5], [0, 1, 3, 5]))     # (y2, m, b2, n)
    my = np.tensordot(q1, q2, axes=([1, 3], [1, 3]))               # (y1, b1, y2, b2)
    my = my.transpose(0, 2, 1, 3).reshape(dy * dy, dy * dy)
    return mx, my


def contract_z(t: np.ndarray, ux: np.ndarray, uy: np.ndarray) -> np.ndarray:
    """T'[X, X', Y, Y', z, z'] of the z step, evaluated pairwise (each step a
    library tensordot): U_x into the lower tensor, the upper tensor over
    (x2, m), U_x on the right pair, U_y on the front pair, U_y on the back
    pair."""
    a = np.tensordot(ux, t, axes=([0], [0]))                 # (x2, X, x1', y1, y1', z, m)
    b = np.tensordot(a, t, axes=([0, 6], [0, 4]))            # (X, x1', y1, y1', z, x2', y2, y2', z')
    c = np.tensordot(b, ux, axes=([1, 5], [0, 1]))           # (X, y1, y1', z, y2, y2', z', X')
    d = np.tensordot(c, uy, axes=([1, 4], [0, 1]))           # (X, y1', z, y2', z', X', Y)
    e = np.tensordot(d, uy, axes=([1, 3], [0, 1]))           # (X, z, z', X', Y, Y')
    return np.ascontiguousarray(e.transpose(0, 3, 4, 5, 1, 2))


def rotate(t: np.ndarray) -> np.ndarray:
    """Put the next axis to block (the current x pair) in the z slot."""
    return np.ascontiguousarray(t.transpose(2, 3, 4, 5, 0, 1))


def trace(t: np.ndarray) -> float:
    """Tr T = sum_{x, y, z} T[x, x, y, y, z, z] (periodic boundaries)."""
    return float(np.einsum("aabbcc->", t))


@dataclass
class Step3:
    tensor: np.ndarray
    lam_x: np.ndarray
    lam_y: np.ndarray
    nx: int
    ny: int


def step_z(t: np.ndarray, dcut: int, trunc: str = "paper", gap_tol: float = 1e-6) -> Step3:
    """One z step (environments, two isometries, contraction); identity
    isometries where Dx^2 or Dy^2 fits under Dcut."""
    dx, dy = t.shape[0], t.shape[2]
    mx, my = environments_z(t)
    if dx * dx <= dcut:
        ux, lx = np.eye(dx * dx).reshape(dx, dx, dx * dx), np.zeros(0)
    else:
        ux, lx = hotrg.isometry(mx, dcut, trunc, gap_tol)
    if dy * dy <= dcut:
        uy, ly = np.eye(dy * dy).reshape(dy, dy, dy * dy), np.zeros(0)
    else:
        uy, ly = hotrg.isometry(my, dcut, trunc, gap_tol)
    return Step3(contract_z(t, ux, uy), lx, ly, ux.shape[2], uy.shape[2])


@dataclass
class Solve3:
    beta: float
    ln_n0: float
    ln_norms: list = field(default_factory=list)
    spectra: list = field(default_factory=list)    # (kept lam_x, kept lam_y) per step
    dims: list = field(default_factory=list)       # tensor shape after each step (rotated frame)
    lnz_per_site: float = float("nan")
    f: float = float("nan")
    trace: float = float("nan")
    tensor: np.ndarray | None = None


def solve3d(t0: np.ndarray, beta: float, dcut: int, nsteps: int, trunc: str = "paper",
            gap_tol: float = 1e-6) -> Solve3:
    """nsteps steps (z, x, y, z, ...) from the raw tensor t0; ln Z / V and
    f = -(ln Z / V) / beta of the periodic lattice the final trace closes."""
    t = np.array(t0, dtype=np.float64)
    n0 = float(np.max(np.abs(t)))
    if not n0 > 0:
        raise ValueError("initial tensor is zero")
    t = t / n0
    res = Solve3(beta=beta, ln_n0=math.log(n0))
    lnz = math.log(n0)
    for k in range(1, nsteps + 1):
        st = step_z(t, dcut, trunc, gap_tol)
        t = st.tensor
        res.spectra.append((st.lam_x[:st.nx].copy(), st.lam_y[:st.ny].copy()))
        nk = float(np.max(np.abs(t)))
        if not (nk > 0 and math.isfinite(nk)):
            raise FloatingPointError(f"non-positive norm at step {k}")
        t = rotate(t / nk)
        res.dims.append(t.shape)
        res.ln_norms.append(math.log(nk))
        lnz += math.ldexp(math.log(nk), -k)
    tr = trace(t)
    if not tr > 0:
        raise FloatingPointError("non-positive trace")
    res.trace = tr
    lnz += math.ldexp(math.log(tr), -nsteps)
    res.lnz_per_site = lnz
    res.f = -lnz / beta if beta > 0 else float("nan")
    res.tensor = t
    return res


def block3d(nsteps: int) -> tuple[int, int, int]:
    """(Lx, Ly, Lz) of the periodic lattice after nsteps steps z, x, y, ..."""
    lz = 2 ** ((nsteps + 2) // 3)
    lx = 2 ** ((nsteps + 1) // 3)
    ly = 2 ** (nsteps // 3)
    return lx, ly, lz
