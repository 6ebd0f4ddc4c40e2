"""Initial site tensors of the oracle (the first step of the method, FP64).

ORACLE / TEST INFRASTRUCTURE ONLY.

Leg order of every rank-4 site tensor is t[l, u, r, d]: left, up, right,
down.  Legs 0 and 2 are the horizontal pair, legs 1 and 3 the vertical pair
(the bond pattern the coarse-graining listing of Sec. 2 implies).  The paper
does not print the Ising or XY tensors (Sec. 2 names the models, Sec. 3.1
gives the XY Hamiltonian, Sec. 3.2 the Ising closed form); the forms below are
the standard ones for the Hamiltonians the paper states:

* Ising, H = -sum_<ij> s_i s_j - h sum_i s_i (Sec. 3.2; field sign chosen to
  match the -h cos(theta) term of the XY Hamiltonian, Eq. 1):
  B[s, s'] = exp(beta s s'), W = B^(1/2) (symmetric square root),
  T[i, j, k, l] = sum_s exp(beta h s) W[s, i] W[s, j] W[s, k] W[s, l].
  Contracting W W^T on every bond gives back B, so the network of T is Z.

* XY (Eq. 1 with Delta = 1) in the character expansion
  exp(x cos phi) = sum_n I_n(x) exp(i n phi), with measure d theta / (2 pi):
  T[n_l, n_u, n_r, n_d] = prod_legs sqrt(I_n(beta)) * I_{n_l+n_u-n_r-n_d}(beta h),
  charges truncated to |n| <= nmax, leg index = n + nmax (D0 = 2 nmax + 1).
  At h = 0 the last factor is the charge-conservation delta.
"""
from __future__ import annotations

import math

import numpy as np


def bessel_i(n: int, x: float, terms: int = 200) -> float:
    """Modified Bessel function of the first kind, integer order, by its
    power series I_n(x) = sum_k (x/2)^(2k+n) / (k! (k+n)!)  (|n| used, since
    I_{-n} = I_n for integer n)."""
    n = abs(int(n))
    x = float(x)
    if x == 0.0:
        return 1.0 if n == 0 else 0.0
    half = 0.5 * x
    term = half ** n / math.factorial(n)  # k = 0
    total = term
    for k in range(1, terms):
        term *= half * half / (k * (k + n))
        total += term
        if term < 1e-18 * total:
            break
    return total


def ising_weight_sqrt(beta: float) -> np.ndarray:
    """Symmetric square root W of B = [[e^b, e^-b], [e^-b, e^b]] (rows and
    columns ordered s = +1, -1), from B's eigenpairs: 2 cosh(beta) on
    (1, 1)/sqrt(2) and 2 sinh(beta) on (1, -1)/sqrt(2)."""
    a = math.sqrt(2.0 * math.cosh(beta))
    b = math.sqrt(2.0 * math.sinh(beta)) if beta > 0 else 0.0
    # W = V diag(a, b) V^T with V = [[1, 1], [1, -1]] / sqrt(2)
    return 0.5 * np.array([[a + b, a - b], [a - b, a + b]], dtype=np.float64)


def ising_tensor(beta: float, h: float = 0.0) -> np.ndarray:
    """Rank-4 Ising site tensor, shape (2, 2, 2, 2), legs (l, u, r, d)."""
    if not (beta >= 0.0 and math.isfinite(beta)):
        raise ValueError("beta must be finite and >= 0")
    w = ising_weight_sqrt(beta)
    spins = (1.0, -1.0)
    t = np.zeros((2, 2, 2, 2))
    for s_idx, s in enumerate(spins):
        ws = w[s_idx]
        t += math.exp(beta * h * s) * np.einsum("i,j,k,l->ijkl", ws, ws, ws, ws)
    return t


def xy_tensor(beta: float, h: float = 0.0, d0: int = 9) -> np.ndarray:
    """Rank-4 XY site tensor in the character expansion, shape (d0,)*4."""
    if d0 < 1 or d0 % 2 == 0:
        raise ValueError("XY: D0 must be odd (2*nmax+1)")
    if not (beta >= 0.0 and math.isfinite(beta)):
        raise ValueError("beta must be finite and >= 0")
    nmax = d0 // 2
    charges = np.arange(-nmax, nmax + 1)
    leg = np.array([math.sqrt(bessel_i(n, beta)) for n in charges])
    t = np.zeros((d0, d0, d0, d0))
    for a, nl in enumerate(charges):
        for b, nu in enumerate(charges):
            for c, nr in enumerate(charges):
                for d, nd in enumerate(charges):
                    div = nl + nu - nr - nd
                    site = bessel_i(div, beta * h)
                    t[a, b, c, d] = leg[a] * leg[b] * leg[c] * leg[d] * site
    return t


def potts_weight_factor(beta: float, q: int = 3) -> np.ndarray:
    """Lower Cholesky factor L of the q-state Potts bond weight
    W[s, s'] = e^beta if s == s' else 1 (Sec. 3.3), W = L L^T."""
    w = np.ones((q, q)) + (math.exp(beta) - 1.0) * np.eye(q)
    return np.linalg.cholesky(w)


def potts_tensor(beta: float, h: float = 0.0, q: int = 3) -> np.ndarray:
    """q-state Potts site tensor T[i,j,k,l] = sum_s e^{beta h [s=0]} L[s,i] L[s,j] L[s,k] L[s,l].

    Sec. 3.3 prints T_ijkl = L_ia L_ib L_ic L_id, which drops the sum over the
    spin index; contracting two such legs gives sum_i L[s,i] L[s',i] = W[s,s'],
    so the network of T is Z.  The field h favours state 0 (the paper says a
    field can be added to this tensor but does not give the form)."""
    if not (beta >= 0.0 and math.isfinite(beta)):
        raise ValueError("beta must be finite and >= 0")
    L = potts_weight_factor(beta, q)
    t = np.zeros((q, q, q, q))
    for s in range(q):
        ls = L[s]
        t += math.exp(beta * h * (1.0 if s == 0 else 0.0)) * np.einsum("i,j,k,l->ijkl", ls, ls, ls, ls)
    return t


# ------------------------------------------------------- impure tensors ---
# The site tensor with an observable O(s) inserted at its site: the same sum
# over the site's spin with O as an extra factor.  Ising: O = s; XY: O =
# cos(theta), which in the character expansion turns the site factor
# I_div(beta h) into (I_{div-1}(beta h) + I_{div+1}(beta h)) / 2 (from
# cos(theta) = (e^{i theta} + e^{-i theta}) / 2); Potts: O = [s = 0].

def ising_impure_tensor(beta: float, h: float = 0.0) -> np.ndarray:
    """Ising site tensor with the spin s inserted, shape (2, 2, 2, 2)."""
    w = ising_weight_sqrt(beta)
    t = np.zeros((2, 2, 2, 2))
    for s_idx, s in enumerate((1.0, -1.0)):
        ws = w[s_idx]
        t += s * math.exp(beta * h * s) * np.einsum("i,j,k,l->ijkl", ws, ws, ws, ws)
    return t


def xy_impure_tensor(beta: float, h: float = 0.0, d0: int = 9) -> np.ndarray:
    """XY site tensor with cos(theta) inserted, shape (d0,)*4."""
    nmax = d0 // 2
    charges = np.arange(-nmax, nmax + 1)
    leg = np.array([math.sqrt(bessel_i(n, beta)) for n in charges])
    t = np.zeros((d0, d0, d0, d0))
    for a, nl in enumerate(charges):
        for b, nu in enumerate(charges):
            for c, nr in enumerate(charges):
                for d, nd in enumerate(charges):
                    div = nl + nu - nr - nd
                    site = 0.5 * (bessel_i(div - 1, beta * h) + bessel_i(div + 1, beta * h))
                    t[a, b, c, d] = leg[a] * leg[b] * leg[c] * leg[d] * site
    return t


def potts_impure_tensor(beta: float, h: float = 0.0, q: int = 3) -> np.ndarray:
    """q-state Potts site tensor with [s = 0] inserted: only the s = 0 term."""
    L = potts_weight_factor(beta, q)
    l0 = L[0]
    return math.exp(beta * h) * np.einsum("i,j,k,l->ijkl", l0, l0, l0, l0)


def impure_tensor(model: str, beta: float, h: float = 0.0, d0: int | None = None) -> np.ndarray:
    model = model.lower()
    if model == "ising":
        return ising_impure_tensor(beta, h)
    if model == "xy":
        return xy_impure_tensor(beta, h, 9 if d0 is None else d0)
    if model == "potts":
        return potts_impure_tensor(beta, h, 3 if d0 is None else d0)
    raise ValueError(f"unknown model {model!r}")


def initial_tensor(model: str, beta: float, h: float = 0.0, d0: int | None = None) -> np.ndarray:
    model = model.lower()
    if model == "ising":
        if d0 not in (None, 2):
            raise ValueError("Ising: D0 must be 2")
        return ising_tensor(beta, h)
    if model == "xy":
        return xy_tensor(beta, h, 9 if d0 is None else d0)
    if model == "potts":
        return potts_tensor(beta, h, 3 if d0 is None else d0)
    raise ValueError(f"unknown model {model!r}")
