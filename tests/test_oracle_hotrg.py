"""Pins for the oracle's HOTRG step and solver (CPU only).

The partition function of small periodic lattices with no truncation must
equal brute-force enumeration (1e-12 relative in Z); truncated runs must
approach Onsager's free energy at the rate the paper reports; the literal
einsums of the coarse-graining listing (Sec. 2) must equal the oracle's
pairwise evaluation; lattice rotation and the normalisation schedule must not
change f.
"""
import math

import numpy as np
import pytest

from oracle import exact, hotrg, models

NO_TRUNC = 10 ** 6


# ----------------------------------------------- the listing, index by index ---
def _rand_tensor(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_environment_x_equals_listing_einsum():
    t = _rand_tensor((3, 4, 3, 4), 1)
    lit = np.einsum("jabe,iecd,labf,kfcd->ijkl", t, t, t, t, optimize=True)
    got = hotrg.environment_x(t)
    assert np.abs(got - lit.reshape(9, 9)).max() <= 1e-12 * np.abs(lit).max()


def test_contract_x_equals_listing_einsum():
    t = _rand_tensor((3, 4, 3, 4), 2)
    u = _rand_tensor((3, 3, 5), 3)
    lit = np.einsum("abi,bjdc,acel,edk->ijkl", u, t, t, u, optimize=True)
    got = hotrg.contract_x(t, u, j_chunk=1)
    assert got.shape == (5, 4, 5, 4)
    assert np.abs(got - lit).max() <= 1e-12 * np.abs(lit).max()


def test_y_half_step_is_rotated_x_half_step():
    # the y einsums of the listing equal the x formulas applied to
    # R = permute(T, (1,2,3,0)), with the result rotated back by (3,0,1,2)
    t = _rand_tensor((5, 3, 5, 3), 4)
    env_lit = np.einsum("aibc,bjde,akfc,flde->ijkl", t, t, t, t, optimize=True)
    env_rot = hotrg.environment_x(hotrg.rotate_in(t))
    assert np.abs(env_rot - env_lit.reshape(9, 9)).max() <= 1e-12 * np.abs(env_lit).max()
    u = _rand_tensor((3, 3, 7), 5)
    con_lit = np.einsum("abj,iacd,cbke,del->ijkl", u, t, t, u, optimize=True)
    con_rot = hotrg.rotate_out(hotrg.contract_x(hotrg.rotate_in(t), u))
    assert con_rot.shape == con_lit.shape == (5, 7, 5, 7)
    assert np.abs(con_rot - con_lit).max() <= 1e-12 * np.abs(con_lit).max()


def test_isometry_keeps_leading_eigenvectors():
    t = np.abs(_rand_tensor((4, 3, 4, 3), 6))
    m = hotrg.environment_x(t)
    u, lam = hotrg.isometry(m, 5)
    v = u.reshape(16, 5)
    ref = np.linalg.eigvalsh(0.5 * (m + m.T))[::-1]
    assert np.abs(lam - ref).max() <= 1e-12 * ref[0]
    assert np.abs(v.T @ v - np.eye(5)).max() <= 1e-13
    assert np.abs(m @ v - v * lam[:5]).max() <= 1e-11 * ref[0]


def test_truncation_rules():
    lam = np.array([4.0, 2.0, 2.0, 1.0, 0.5])
    assert hotrg.truncation_dim(lam, 2, "paper") == 2
    assert hotrg.truncation_dim(lam, 2, "multiplet") == 1
    assert hotrg.truncation_dim(lam, 3, "multiplet") == 3
    assert hotrg.truncation_dim(lam, 9, "multiplet") == 5


# ------------------------------------------------------ exact enumeration ---
@pytest.mark.parametrize("nsteps", [2, 3, 4])
@pytest.mark.parametrize("beta,h", [(0.44, 0.0), (0.44, 0.01), (0.3, -0.25)])
def test_ising_untruncated_matches_enumeration(nsteps, beta, h):
    width, height = exact.hotrg_block(nsteps)
    sol = hotrg.solve(models.ising_tensor(beta, h), beta, NO_TRUNC, nsteps)
    lnz = sol.lnz_per_site * width * height
    ref = exact.ising_lnz_exact(width, height, beta, h)
    # 1e-12 relative in Z is 1e-12 absolute in ln Z
    assert abs(lnz - ref) <= 1e-12 * max(1.0, abs(ref)) + 1e-12


@pytest.mark.parametrize("nsteps", [1, 2])
@pytest.mark.parametrize("beta,h", [(1.0, 0.0), (0.9, 0.1)])
def test_xy_untruncated_matches_enumeration(nsteps, beta, h):
    width, height = exact.hotrg_block(nsteps)
    sol = hotrg.solve(models.xy_tensor(beta, h, 9), beta, NO_TRUNC, nsteps)
    lnz = sol.lnz_per_site * width * height
    ref = exact.xy_lnz_exact(width, height, beta, h, 9)
    assert abs(lnz - ref) <= 1e-12 * max(1.0, abs(ref))


def test_beta_zero_limits():
    s = hotrg.solve(models.ising_tensor(0.0), 1.0, 8, 12)
    assert s.lnz_per_site == pytest.approx(math.log(2.0), abs=1e-13)
    s = hotrg.solve(models.xy_tensor(0.0, 0.0, 5), 1.0, 8, 8)
    assert s.lnz_per_site == pytest.approx(0.0, abs=1e-13)


# ------------------------------------------------------------ truncation ---
@pytest.mark.slow
def test_ising_onsager_convergence_in_dcut():
    beta = 0.44
    fe = exact.onsager_free_energy(beta)
    err = {}
    for dcut in (8, 16):
        sol = hotrg.solve(models.ising_tensor(beta), beta, dcut, 40)
        err[dcut] = abs(sol.f - fe) / abs(fe)
    # the paper's fit |df/f| ~ D^-4.12 (Sec. 3.2) puts Dcut=16 near 5.7e-7
    assert err[16] <= 2e-6
    assert err[16] < err[8] / 10


def test_rotation_invariance_untruncated():
    # a 4x4 torus of T and a 4x4 torus of the rotated tensor are the same lattice
    t = np.abs(_rand_tensor((2, 3, 2, 3), 8)) + 0.1
    a = hotrg.solve(t, 1.0, NO_TRUNC, 4)
    r = hotrg.solve(t.transpose(1, 2, 3, 0), 1.0, NO_TRUNC, 4)
    assert abs(a.lnz_per_site - r.lnz_per_site) <= 1e-13


def test_xy_rotation_is_gauge_transform():
    # rotating the XY tensor conjugates the charge on one pair of legs, a
    # relabelling of the basis; with multiplet-aware truncation f is unchanged
    beta = 1.0
    t = models.xy_tensor(beta, 0.0, 5)
    a = hotrg.solve(t, beta, 12, 10, trunc="multiplet")
    r = hotrg.solve(t.transpose(1, 2, 3, 0), beta, 12, 10, trunc="multiplet")
    assert abs(a.f - r.f) <= 1e-12


def test_normalisation_schedule_does_not_change_f():
    beta = 0.44
    t0 = models.ising_tensor(beta)
    a = hotrg.solve(t0, beta, 8, 20, norm="halfstep")
    b = hotrg.solve(t0, beta, 8, 20, norm="paper")
    assert abs(a.f - b.f) <= 1e-13


def test_identity_isometry_when_untruncated(monkeypatch):
    # when Dn = Dx^2 the isometry is a basis change, so U = I gives the same f
    beta, h = 0.44, 0.02
    t0 = models.ising_tensor(beta, h)
    ref = hotrg.solve(t0, beta, 16, 6)
    real = hotrg.isometry

    def identity_when_full(m, dcut, trunc="paper", gap_tol=1e-6):
        n = m.shape[0]
        if min(n, dcut) == n:
            dx = int(round(math.sqrt(n)))
            lam = np.sort(np.linalg.eigvalsh(0.5 * (m + m.T)))[::-1]
            return np.eye(n).reshape(dx, dx, n), lam
        return real(m, dcut, trunc, gap_tol)

    monkeypatch.setattr(hotrg, "isometry", identity_when_full)
    ident = hotrg.solve(t0, beta, 16, 6)
    assert abs(ident.f - ref.f) <= 1e-13


@pytest.mark.parametrize("nsteps", [2, 3])
@pytest.mark.parametrize("beta,h", [(1.0, 0.0), (0.8, 0.05)])
def test_potts_untruncated_matches_enumeration(nsteps, beta, h):
    width, height = exact.hotrg_block(nsteps)
    sol = hotrg.solve(models.potts_tensor(beta, h, 3), beta, NO_TRUNC, nsteps)
    lnz = sol.lnz_per_site * width * height
    ref = exact.potts_lnz_exact(width, height, beta, h, 3)
    assert abs(lnz - ref) <= 1e-12 * max(1.0, abs(ref))


def test_potts_q2_is_ising_onsager():
    # q = 2 Potts with W = e^{beta delta} equals Ising at K = beta/2, plus beta per site
    beta = 0.6
    sol = hotrg.solve(models.potts_tensor(beta, 0.0, 2), beta, 16, 40)
    ref = exact.onsager_integral(beta / 2) + beta
    assert abs(sol.lnz_per_site - ref) <= 1e-9


def test_potts_q3_at_tc_approaches_baxter():
    # Sec. 3.3: q = 3 at T_c = 1 / ln(1 + sqrt 3) on a 2^20 x 2^20 lattice;
    # truncated HOTRG at Dcut = 16 lies within 1e-4 of Baxter's
    # infinite-lattice value (the finite-size shift is of order L^-2)
    beta = math.log(1 + math.sqrt(3))
    sol = hotrg.solve(models.potts_tensor(beta, 0.0, 3), beta, 16, 40)
    assert abs(sol.lnz_per_site - exact.potts_critical_lnz(3)) <= 1e-4


# ------------------------------------------------ impure tensors (observables) ---
@pytest.mark.parametrize("nsteps", [2, 3, 4])
@pytest.mark.parametrize("beta,h", [(0.44, 0.01), (0.3, -0.25), (0.6, 0.0)])
def test_ising_magnetization_matches_enumeration(nsteps, beta, h):
    width, height = exact.hotrg_block(nsteps)
    sol = hotrg.solve(models.ising_tensor(beta, h), beta, NO_TRUNC, nsteps,
                      impure=models.ising_impure_tensor(beta, h))
    ref = exact.ising_magnetization_exact(width, height, beta, h)
    assert abs(sol.expectation - ref) <= 1e-12


@pytest.mark.parametrize("nsteps", [1, 2])
def test_xy_cos_matches_enumeration(nsteps):
    width, height = exact.hotrg_block(nsteps)
    beta, h = 0.9, 0.1
    sol = hotrg.solve(models.xy_tensor(beta, h, 5), beta, NO_TRUNC, nsteps,
                      impure=models.xy_impure_tensor(beta, h, 5))
    assert abs(sol.expectation - exact.xy_cos_exact(width, height, beta, h, 5)) <= 1e-12


@pytest.mark.parametrize("nsteps", [2, 3])
def test_potts_fraction_matches_enumeration(nsteps):
    width, height = exact.hotrg_block(nsteps)
    beta, h = 0.8, 0.05
    sol = hotrg.solve(models.potts_tensor(beta, h, 3), beta, NO_TRUNC, nsteps,
                      impure=models.potts_impure_tensor(beta, h, 3))
    assert abs(sol.expectation - exact.potts_fraction0_exact(width, height, beta, h, 3)) <= 1e-12


def test_magnetization_vanishes_in_the_symmetric_phase():
    # h = 0: the impure tensor is odd under the global spin flip, the
    # isometries keep the two sectors apart, so the trace is zero
    sol = hotrg.solve(models.ising_tensor(0.3), 0.3, 8, 20, impure=models.ising_impure_tensor(0.3))
    assert abs(sol.expectation) <= 1e-14


def test_spontaneous_magnetization_approaches_yang():
    # beta > beta_c with a field that only picks the + state on 2^20 x 2^20
    # sites: M -> (1 - sinh(2 beta)^-4)^(1/8), the error shrinking with Dcut
    beta, h = 0.6, 1e-10
    ref = exact.onsager_yang_magnetization(beta)
    err = {}
    for dcut in (8, 16):
        sol = hotrg.solve(models.ising_tensor(beta, h), beta, dcut, 40, impure=models.ising_impure_tensor(beta, h))
        err[dcut] = abs(sol.expectation - ref)
    assert err[16] <= 5e-6
    assert err[16] < err[8] / 4
