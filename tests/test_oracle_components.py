"""Pins for the oracle's building blocks (CPU only).

Each check compares the oracle with something other than itself: closed
forms, a library routine for a special case, or brute force.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import exact, hotrg, jacobi, models


# ------------------------------------------------------------------ Jacobi ---
def test_jacobi_two_by_two_closed_form():
    a, b, c = 2.0, 0.75, -1.25
    w, v, _ = jacobi.eigh(np.array([[a, b], [b, c]]))
    mid, rad = 0.5 * (a + c), math.hypot(0.5 * (a - c), b)
    assert w[0] == pytest.approx(mid + rad, abs=1e-15)
    assert w[1] == pytest.approx(mid - rad, abs=1e-15)
    # eigenvector of the larger eigenvalue: (b, lam - a) up to sign and norm
    ref = np.array([b, w[0] - a])
    ref /= np.linalg.norm(ref)
    assert abs(abs(ref @ v[:, 0]) - 1.0) < 1e-15


def test_jacobi_diagonal_is_fixed_point():
    d = np.array([3.0, -1.0, 7.5, 0.0, 2.0])
    w, v, sweeps = jacobi.eigh(np.diag(d))
    assert np.array_equal(w, np.sort(d)[::-1])
    assert sweeps == 0
    assert np.array_equal(np.abs(v), np.abs(v).round())


@pytest.mark.parametrize("n", [3, 17, 64, 130])
def test_jacobi_random_symmetric(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n))
    a = a + a.T
    w, v, _ = jacobi.eigh(a)
    scale = np.abs(w).max()
    assert np.abs(a @ v - v * w).max() <= 1e-12 * scale * n ** 0.5
    assert np.abs(v.T @ v - np.eye(n)).max() <= 1e-13 * n
    assert np.all(np.diff(w) <= 0)
    # eigenvalues against LAPACK's symmetric solver
    assert np.abs(w - np.linalg.eigvalsh(a)[::-1]).max() <= 1e-12 * scale


def test_jacobi_graded_psd():
    # a Gram matrix whose spectrum spans 24 decades, like the environments
    rng = np.random.default_rng(7)
    n = 40
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = 10.0 ** (-np.linspace(0, 24, n))
    a = (q * lam) @ q.T
    w, v, _ = jacobi.eigh(a)
    assert np.abs(a @ v - v * w).max() <= 1e-14
    assert np.abs(w[:10] - lam[:10]).max() <= 1e-14
    # leading eigenvectors agree with the construction up to sign
    for k in range(6):
        assert abs(abs(v[:, k] @ q[:, k]) - 1.0) < 1e-10


# ------------------------------------------------------------------ Bessel ---
@pytest.mark.parametrize("x", [0.0, 1e-3, 0.05, 0.9, 1.0, 1.3, 3.0])
def test_bessel_series_vs_library(x):
    scipy_special = pytest.importorskip("scipy.special")
    for n in range(-6, 7):
        ref = float(scipy_special.iv(n, x))
        got = models.bessel_i(n, x)
        if ref == 0.0:
            assert got == 0.0
        else:
            assert abs(got - ref) <= 1e-14 * abs(ref)


# ---------------------------------------------------------------- tensors ---
@pytest.mark.parametrize("beta,h", [(0.44, 0.0), (0.3, 0.05), (0.6, -0.2)])
def test_ising_tensor_leg_permutation_symmetry(beta, h):
    t = models.ising_tensor(beta, h)
    for perm in itertools.permutations(range(4)):
        # exact in arithmetic; the products may round in a different order
        assert np.abs(t - t.transpose(perm)).max() <= 1e-15 * np.abs(t).max()


def test_ising_bond_weight_reconstructed():
    # W W^T = B: contracting two half-bonds gives the Boltzmann weight
    for beta in (0.0, 0.2, 0.44, 1.5):
        w = models.ising_weight_sqrt(beta)
        b = np.array([[math.exp(beta), math.exp(-beta)], [math.exp(-beta), math.exp(beta)]])
        assert np.abs(w @ w.T - b).max() <= 1e-14 * b.max()


def test_ising_single_site_trace():
    # one site closed on itself (1x1 torus): Z = sum_s e^{2 beta} e^{beta h s}
    beta, h = 0.37, 0.21
    t = models.ising_tensor(beta, h)
    z = hotrg.trace_pbc(t)
    ref = sum(math.exp(2 * beta + beta * h * s) for s in (1, -1))
    assert z == pytest.approx(ref, rel=1e-14)


def test_xy_tensor_charge_conservation():
    t = models.xy_tensor(1.1, 0.0, 9)
    n = np.arange(-4, 5)
    div = n[:, None, None, None] + n[None, :, None, None] - n[None, None, :, None] - n[None, None, None, :]
    assert np.all(t[div != 0] == 0.0)
    assert np.all(t[div == 0] > 0.0)
    # charge conjugation n -> -n on every leg is a symmetry
    assert np.array_equal(t, t[::-1, ::-1, ::-1, ::-1])


# ---------------------------------------------------------------- Onsager ---
@pytest.mark.parametrize("beta", [0.2, 0.3, 0.40, 0.48, 0.6, 1.0])
def test_onsager_forms_agree(beta):
    series = exact.onsager_series(beta)
    single = exact.onsager_integral(beta)
    assert abs(series - single) <= 1e-13
    if abs(beta - exact.BETA_C) > 0.1:
        assert abs(exact.onsager_double_integral(beta) - single) <= 1e-12


def test_onsager_limits():
    # beta -> 0: ln Z / V -> ln 2; large beta: -beta f -> 2 beta (ground state)
    assert exact.onsager_integral(1e-8) == pytest.approx(math.log(2.0), abs=1e-12)
    b = 5.0
    assert exact.onsager_integral(b) == pytest.approx(2 * b, abs=1e-8)


def test_onsager_continuous_at_beta_c():
    # the 4F3 series does not converge at beta_c; the integral form there is
    # pinned by its agreement with the series on both sides of beta_c
    bc = exact.BETA_C
    for d in (2e-2, 1e-2):
        lo = exact.onsager_integral(bc - d)
        hi = exact.onsager_integral(bc + d)
        assert abs(lo - exact.onsager_series(bc - d)) <= 1e-13
        assert abs(hi - exact.onsager_series(bc + d)) <= 1e-13
    mid = exact.onsager_integral(bc)
    assert min(exact.onsager_integral(bc - 1e-6), exact.onsager_integral(bc + 1e-6)) - 1e-5 < mid
    assert mid < max(exact.onsager_integral(bc - 1e-6), exact.onsager_integral(bc + 1e-6)) + 1e-5


# ------------------------------------------------------------- enumeration ---
def test_ising_enumeration_known_cases():
    # 1x1 torus: two self-bonds, Z = sum_s e^{2 beta + beta h s}
    beta, h = 0.31, 0.2
    ref = math.log(sum(math.exp(2 * beta + beta * h * s) for s in (1, -1)))
    assert exact.ising_lnz_exact(1, 1, beta, h) == pytest.approx(ref, abs=1e-14)
    # beta = 0: Z = 2^V
    assert exact.ising_lnz_exact(4, 4, 0.0, 0.0) == pytest.approx(16 * math.log(2), abs=1e-12)


def test_xy_enumeration_known_cases():
    # 1x1 torus: two self-bonds, div = 0 always; Z = (sum_n I_n(b))^2 * I_0(b h)
    beta, h = 0.9, 0.3
    s = sum(models.bessel_i(n, beta) for n in range(-4, 5))
    ref = math.log(s * s * models.bessel_i(0, beta * h))
    assert exact.xy_lnz_exact(1, 1, beta, h) == pytest.approx(ref, abs=1e-13)


# ------------------------------------------------------------------ Potts ---
def test_potts_cholesky_reconstructs_bond_weight():
    for beta in (0.3, math.log(1 + math.sqrt(3)), 2.0):
        L = models.potts_weight_factor(beta, 3)
        w = np.ones((3, 3)) + (math.exp(beta) - 1.0) * np.eye(3)
        assert np.abs(L @ L.T - w).max() <= 1e-14 * w.max()
        assert np.allclose(np.triu(L, 1), 0.0)


def test_potts_single_site_trace():
    # one site closed on itself: two self-bonds, each W_ss = e^beta
    beta, h = 0.7, 0.3
    t = models.potts_tensor(beta, h, 3)
    ref = sum(math.exp(2 * beta + beta * h * (s == 0)) for s in range(3))
    assert hotrg.trace_pbc(t) == pytest.approx(ref, rel=1e-14)


def test_potts_enumeration_known_cases():
    # beta = 0: Z = q^V
    assert exact.potts_lnz_exact(2, 2, 0.0) == pytest.approx(4 * math.log(3), abs=1e-13)
    # q = 2 Potts with W = e^{beta delta} is Ising at K = beta/2 (+ beta per bond pair)
    beta = 0.9
    ref = exact.ising_lnz_exact(2, 2, beta / 2) + 8 * beta / 2
    assert exact.potts_lnz_exact(2, 2, beta, q=2) == pytest.approx(ref, abs=1e-12)


def test_potts_critical_closed_form_special_cases():
    # q = 1: every configuration weighs e^{2 K_c} per site, K_c = ln 2
    assert exact.potts_critical_lnz(1.0) == pytest.approx(2 * math.log(2), abs=1e-13)
    # q = 2: Ising at K = K_c / 2 (Onsager's integral form) plus K_c per site
    kc = math.log(1 + math.sqrt(2))
    assert exact.potts_critical_lnz(2.0) == pytest.approx(exact.onsager_integral(kc / 2) + kc, abs=1e-13)
    # weights >= 1 bound ln Z / V from below by ln q, and the Peierls-type
    # bound ln Z / V <= ln q + 2 K_c from above
    for q in (1.5, 2.5, 3.0, 3.5):
        kc = math.log(1 + math.sqrt(q))
        assert math.log(q) < exact.potts_critical_lnz(q) < math.log(q) + 2 * kc


def test_impure_tensors_reduce_to_pure_ones():
    # inserting O = 1 gives the pure tensor: Ising s = +-1 splits it in two
    # signed halves, Potts [s = 0] is one of the q terms, and the XY site
    # factor (I_{n-1} + I_{n+1}) / 2 equals I_n'(x) (the recurrence of I_n)
    from oracle import models
    beta, h = 0.7, 0.3
    t = models.ising_tensor(beta, h)
    ti = models.ising_impure_tensor(beta, h)
    w = models.ising_weight_sqrt(beta)
    plus = math.exp(beta * h) * np.einsum("i,j,k,l->ijkl", w[0], w[0], w[0], w[0])
    assert np.abs(t + ti - 2 * plus).max() <= 1e-14 * np.abs(t).max()
    tp = models.potts_tensor(beta, 0.0, 3)
    total = sum(np.einsum("i,j,k,l->ijkl", *(models.potts_weight_factor(beta, 3)[s],) * 4) for s in range(3))
    assert np.allclose(tp, total, rtol=1e-14)
    x = beta * h
    for n in range(-3, 4):
        deriv = (models.bessel_i(n, x + 1e-6) - models.bessel_i(n, x - 1e-6)) / 2e-6
        assert abs(0.5 * (models.bessel_i(n - 1, x) + models.bessel_i(n + 1, x)) - deriv) <= 1e-8
