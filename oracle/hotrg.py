"""Plain CPU FP64 HOTRG: the oracle for the coarse-graining hot path.

ORACLE / TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU
baseline leg of the benchmark import this module; the GPU product path never
does, and this module imports nothing from the GPU package.

Everything follows the coarse-graining step of Sec. 2 (the listing with the
environment, SVD and contraction einsums, and the caption of Fig. 1):

x half-step on t[l, u, r, d] (shape (Dx, Dy, Dx, Dy)):
  1. environment   M[i, j, k, l] = sum t[j,a,b,e] t[i,e,c,d] t[l,a,b,f] t[k,f,c,d]
     (two tensors stacked vertically: t[j,...] on top, t[i,...] below, bond e;
     the doubled left legs (i, j) are kept),
  2. isometry      U = leading Dn = min(Dx^2, Dcut) left singular vectors of M
     viewed as the (Dx^2, Dx^2) matrix [(i, j), (k, l)],
  3. contraction   Tx[i, j, k, l] = sum U[a,b,i] t[b,j,d,c] t[a,c,e,l] U[e,d,k]
     (shape (Dn, Dy, Dn, Dy)),
y half-step: the same three operations on the rotated tensor
  R = permute(T, (1, 2, 3, 0)), result rotated back with permute(O, (3, 0, 1, 2)).
  (Substituting R into the x formulas reproduces the y einsums of the listing
  index for index; tests check this against the literal y einsums.)
normalise: after every half-step divide by n_k = max |T| and accumulate
  ln Z / V = ln n0 + sum_{k=1..N} 2^-k ln n_k + 2^-N ln Tr T_N,
  Tr T = sum_{i,j} T[i, j, i, j] (periodic boundary conditions, Sec. 2 and the
  caption of Fig. 1), f = -(ln Z / V) / beta (Sec. 3.2).

Readings where the paper is silent or ambiguous (each is a keyword here):
  * the SVD of M is taken as the eigendecomposition of the symmetrised M
    (M is a Gram matrix, so both give the same leading vectors and values),
    computed by the oracle's own cyclic Jacobi solver;
  * normalisation by max |T| after every half-step ("halfstep", default) or by
    the signed max once per full x+y iteration as the listing does ("paper");
  * truncation "paper" keeps exactly min(Dx^2, Dcut) vectors; "multiplet"
    lowers Dn until the relative gap (lam[Dn-1] - lam[Dn]) / lam[0] is at
    least gap_tol (default 1e-6), so that a degenerate multiplet is never
    split.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import jacobi


# ----------------------------------------------------------------- x step ---
def environment_x(t: np.ndarray) -> np.ndarray:
    """Environment matrix of the x half-step, shape (Dx*Dx, Dx*Dx).

    Evaluated pairwise as M = sum_{e,f} P[j,e,l,f] Q[i,e,k,f] with
    P[j,e,l,f] = sum_{a,b} t[j,a,b,e] t[l,a,b,f] (top pair) and
    Q[i,e,k,f] = sum_{c,d} t[i,e,c,d] t[k,f,c,d] (bottom pair): a grouping of
    the same sum of products, each step a library tensordot."""
    dx = t.shape[0]
    p = np.tensordot(t, t, axes=([1, 2], [1, 2]))        # (j, e, l, f)
    q = np.tensordot(t, t, axes=([2, 3], [2, 3]))        # (i, e, k, f)
    m = np.tensordot(q, p, axes=([1, 3], [1, 3]))        # (i, k, j, l)
    m = m.transpose(0, 2, 1, 3)                          # (i, j, k, l)
    return m.reshape(dx * dx, dx * dx)


def truncation_dim(lam: np.ndarray, dcut: int, trunc: str = "paper",
                   gap_tol: float = 1e-6) -> int:
    """Number of kept vectors: min(size, Dcut) as the SVD helper of the
    listing does; with trunc="multiplet", lowered until the cut does not split
    a (near-)degenerate multiplet."""
    n = lam.shape[0]
    dn = min(n, int(dcut))
    if trunc == "paper" or dn == n:
        return dn
    if trunc != "multiplet":
        raise ValueError(f"unknown truncation rule {trunc!r}")
    scale = abs(lam[0]) if n else 1.0
    k = dn
    while k > 1 and (lam[k - 1] - lam[k]) < gap_tol * scale:
        k -= 1
    return k


def isometry(m: np.ndarray, dcut: int, trunc: str = "paper", gap_tol: float = 1e-6):
    """Leading eigenvectors of the symmetrised environment matrix.

    Returns (U, lam_all) with U of shape (Dx, Dx, Dn) (first index: the leg of
    the lower tensor, second: the leg of the upper tensor) and all
    eigenvalues in descending order."""
    n = m.shape[0]
    dx = int(round(math.sqrt(n)))
    msym = 0.5 * (m + m.T)
    lam, v, _ = jacobi.eigh(msym)
    dn = truncation_dim(lam, dcut, trunc, gap_tol)
    u = v[:, :dn].reshape(dx, dx, dn)
    return u, lam


def contract_x(t: np.ndarray, u: np.ndarray, j_chunk: int | None = None) -> np.ndarray:
    """Tx[i,j,k,l] = sum U[a,b,i] t[b,j,d,c] t[a,c,e,l] U[e,d,k].

    Pairwise order X1 = U.t (over b), X2 = X1.t (over a, c), Tx = X2.U (over
    d, e).  The free index j (the up leg of the upper tensor) is processed in
    chunks so that the D^5 intermediates stay bounded in host memory."""
    dx, dy = t.shape[0], t.shape[1]
    dn = u.shape[2]
    out = np.empty((dn, dy, dn, dy))
    if j_chunk is None:
        j_chunk = max(1, min(dy, int(2 ** 27 // max(1, dx * dx * dn * dy))))
    for j0 in range(0, dy, j_chunk):
        j1 = min(dy, j0 + j_chunk)
        out[:, j0:j1] = contract_x_slice(t, u, j0, j1)
    return out


def contract_x_slice(t: np.ndarray, u: np.ndarray, j0: int, j1: int,
                     bottom: np.ndarray | None = None) -> np.ndarray:
    """Tx[:, j0:j1, :, :] of contract_x; `bottom` (default t) is the lower
    tensor t[a,c,e,l] of the pair, t the upper one t[b,j,d,c]."""
    if bottom is None:
        bottom = t
    tj = t[:, j0:j1]                                   # (b, j, d, c)
    x1 = np.tensordot(u, tj, axes=([1], [0]))          # (a, i, j, d, c)
    x2 = np.tensordot(x1, bottom, axes=([0, 4], [0, 1]))   # (i, j, d, e, l)
    x3 = np.tensordot(x2, u, axes=([2, 3], [1, 0]))    # (i, j, l, k)
    return x3.transpose(0, 1, 3, 2)


def contract_pair_x(top: np.ndarray, bottom: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Tx[i,j,k,l] = sum U[a,b,i] top[b,j,d,c] bottom[a,c,e,l] U[e,d,k]: the
    x blocking of two different tensors (an impure one with a pure one)."""
    dn, dy = u.shape[2], top.shape[1]
    out = np.empty((dn, dy, dn, dy))
    j_chunk = max(1, min(dy, int(2 ** 27 // max(1, top.shape[0] ** 2 * dn * dy))))
    for j0 in range(0, dy, j_chunk):
        j1 = min(dy, j0 + j_chunk)
        out[:, j0:j1] = contract_x_slice(top, u, j0, j1, bottom=bottom)
    return out


def rotate_in(t: np.ndarray) -> np.ndarray:
    """R = permute(T, (1, 2, 3, 0)): the y half-step run as an x half-step."""
    return np.ascontiguousarray(t.transpose(1, 2, 3, 0))


def rotate_out(o: np.ndarray) -> np.ndarray:
    """Txy = permute(O, (3, 0, 1, 2))."""
    return np.ascontiguousarray(o.transpose(3, 0, 1, 2))


@dataclass
class HalfStep:
    tensor: np.ndarray          # coarse tensor (not normalised)
    lam: np.ndarray             # all eigenvalues of M, descending
    dn: int                     # kept dimension
    u: np.ndarray               # isometry (Dx, Dx, Dn)


def half_step(t: np.ndarray, dcut: int, direction: str, trunc: str = "paper",
              gap_tol: float = 1e-6) -> HalfStep:
    """One directional blocking (x: stack vertically; y: stack horizontally)."""
    if direction == "x":
        m = environment_x(t)
        u, lam = isometry(m, dcut, trunc, gap_tol)
        return HalfStep(contract_x(t, u), lam, u.shape[2], u)
    if direction == "y":
        r = rotate_in(t)
        m = environment_x(r)
        u, lam = isometry(m, dcut, trunc, gap_tol)
        return HalfStep(rotate_out(contract_x(r, u)), lam, u.shape[2], u)
    raise ValueError("direction must be 'x' or 'y'")


def half_step_impure(t: np.ndarray, t_imp: np.ndarray, dcut: int, direction: str, trunc: str = "paper",
                     gap_tol: float = 1e-6):
    """One half-step of the pure tensor and of an impure one blocked with it.

    The isometry comes from the pure tensor's environment (the impure tensor
    is one site in the whole lattice and leaves it unchanged); the impure
    block is the mean of the two placements of the impurity in the pair,
    (C(imp, pure) + C(pure, imp)) / 2, so after N half-steps it is the mean
    of the insertion over all 2^N sites of the block."""
    if direction == "x":
        m = environment_x(t)
        u, lam = isometry(m, dcut, trunc, gap_tol)
        pure = contract_x(t, u)
        imp = 0.5 * (contract_pair_x(t_imp, t, u) + contract_pair_x(t, t_imp, u))
        return HalfStep(pure, lam, u.shape[2], u), imp
    if direction == "y":
        r, ri = rotate_in(t), rotate_in(t_imp)
        m = environment_x(r)
        u, lam = isometry(m, dcut, trunc, gap_tol)
        pure = rotate_out(contract_x(r, u))
        imp = rotate_out(0.5 * (contract_pair_x(ri, r, u) + contract_pair_x(r, ri, u)))
        return HalfStep(pure, lam, u.shape[2], u), imp
    raise ValueError("direction must be 'x' or 'y'")


def trace_pbc(t: np.ndarray) -> float:
    """Tr T = sum_{i,j} T[i, j, i, j]: one tensor closed on itself."""
    return float(np.einsum("ijij->", t))


# ----------------------------------------------------------------- solver ---
@dataclass
class Solve:
    beta: float
    ln_n0: float
    ln_norms: list = field(default_factory=list)   # ln n_k, k = 1..N
    spectra: list = field(default_factory=list)    # kept eigenvalues per half-step
    full_spectra: list = field(default_factory=list)
    dims: list = field(default_factory=list)       # (Dx, Dy) after each half-step
    lnz_per_site: float = float("nan")
    f: float = float("nan")
    trace: float = float("nan")
    tensor: np.ndarray | None = None
    expectation: float = float("nan")              # Tr T_imp / Tr T when an impure tensor ran along


def solve(t0: np.ndarray, beta: float, dcut: int, nsteps: int, trunc: str = "paper",
          gap_tol: float = 1e-6, norm: str = "halfstep", keep_full_spectra: bool = False,
          first_direction: str = "x", impure: np.ndarray | None = None) -> Solve:
    """Run nsteps alternating half-steps (x first) from the raw tensor t0 and
    return ln Z / V and f = -(ln Z / V) / beta for the periodic lattice of
    2^nsteps sites that the final trace closes.  With an impure tensor (t0
    with an observable inserted) it is blocked alongside, divided by the same
    norms, and expectation = Tr T_imp / Tr T is the site mean of <O>."""
    t = np.array(t0, dtype=np.float64)
    n0 = float(np.max(np.abs(t)))
    if not n0 > 0:
        raise ValueError("initial tensor is zero")
    t = t / n0
    t_imp = None if impure is None else np.array(impure, dtype=np.float64) / n0
    res = Solve(beta=beta, ln_n0=math.log(n0))
    lnz = math.log(n0)
    # a tensor after half-step k stands for 2^k sites, so its norm enters
    # ln Z / V with weight 2^-k whichever schedule divides it out
    directions = ("x", "y") if first_direction == "x" else ("y", "x")
    for k in range(1, nsteps + 1):
        if t_imp is None:
            hs = half_step(t, dcut, directions[(k - 1) % 2], trunc, gap_tol)
        else:
            hs, t_imp = half_step_impure(t, t_imp, dcut, directions[(k - 1) % 2], trunc, gap_tol)
        t = hs.tensor
        res.spectra.append(hs.lam[:hs.dn].copy())
        if keep_full_spectra:
            res.full_spectra.append(hs.lam.copy())
        res.dims.append((t.shape[0], t.shape[1]))
        if norm == "halfstep":
            nk = float(np.max(np.abs(t)))
            if not (nk > 0 and math.isfinite(nk)):
                raise FloatingPointError(f"non-positive norm at half-step {k}")
            t = t / nk
            if t_imp is not None:
                t_imp = t_imp / nk
            res.ln_norms.append(math.log(nk))
            lnz += math.ldexp(math.log(nk), -k)
        elif norm == "paper":
            # the listing divides by the signed maximum after the y step only
            if k % 2 == 0 or k == nsteps:
                nk = float(np.max(t))
                if not (nk > 0 and math.isfinite(nk)):
                    raise FloatingPointError(f"non-positive norm at half-step {k}")
                t = t / nk
                if t_imp is not None:
                    t_imp = t_imp / nk
                res.ln_norms.append(math.log(nk))
                lnz += math.ldexp(math.log(nk), -k)
            else:
                res.ln_norms.append(0.0)
        else:
            raise ValueError(f"unknown normalisation schedule {norm!r}")
    tr = trace_pbc(t)
    if not (tr > 0 and math.isfinite(tr)):
        raise FloatingPointError("non-positive trace")
    res.trace = tr
    lnz += math.ldexp(math.log(tr), -nsteps)
    res.lnz_per_site = lnz
    res.f = -lnz / beta if beta > 0 else float("nan")
    res.tensor = t
    if t_imp is not None:
        res.expectation = trace_pbc(t_imp) / tr
    return res
