"""Pins of the 3D oracle (oracle/hotrg3d.py), CPU only.

* Untruncated blocking equals enumeration of Z on the 1x1x2, 2x1x2 and
  2x2x2 tori (field included) to 1e-12 in ln Z.
* The environment's pairwise grouping equals the Gram matrix of the fully
  formed stacked pair, and the pairwise contraction equals the defining
  sum evaluated in one einsum, on small random tensors.
* At beta = 0 every spin is free: ln Z / V = ln 2 at any Dcut.
* Truncation converges: ln Z / V at Dcut 4 and 6 differ by less than at
  Dcut 2 and 4 (nearer the bulk value).
"""
import math

import numpy as np
import pytest

from oracle import exact, hotrg3d


@pytest.mark.parametrize("nsteps", [1, 2, 3])
@pytest.mark.parametrize("beta,h", [(0.22, 0.0), (0.3, 0.1), (0.15, -0.4)])
def test_untruncated_matches_enumeration(nsteps, beta, h):
    lx, ly, lz = hotrg3d.block3d(nsteps)
    sol = hotrg3d.solve3d(hotrg3d.ising3d_tensor(beta, h), beta, 10 ** 6, nsteps)
    lnz = sol.lnz_per_site * lx * ly * lz
    ref = exact.ising3d_lnz_exact(lx, ly, lz, beta, h)
    assert abs(lnz - ref) <= 1e-12 * max(1.0, abs(ref))


def test_single_site_trace():
    # a 1x1x1 torus: each site bonds to itself three times, Z = sum_s e^{3 beta + beta h s}
    beta, h = 0.4, 0.25
    t = hotrg3d.ising3d_tensor(beta, h)
    ref = sum(math.exp(3 * beta + beta * h * s) for s in (1, -1))
    assert hotrg3d.trace(t) == pytest.approx(ref, rel=1e-14)
    assert exact.ising3d_lnz_exact(1, 1, 1, beta, h) == pytest.approx(math.log(ref), abs=1e-13)


def test_enumeration_known_cases():
    # beta = 0: Z = 2^V
    assert exact.ising3d_lnz_exact(2, 1, 2, 0.0) == pytest.approx(4 * math.log(2), abs=1e-13)
    # a 2x1x1 ring with bonds in x (two between the sites) and self-bonds in y, z:
    # Z = sum_{s1,s2} e^{2 beta s1 s2 + 4 beta} = 2 e^{4b} (e^{2b} + e^{-2b})
    b = 0.37
    ref = math.log(2 * math.exp(4 * b) * (math.exp(2 * b) + math.exp(-2 * b)))
    assert exact.ising3d_lnz_exact(2, 1, 1, b) == pytest.approx(ref, abs=1e-13)


def test_site_tensor_leg_symmetry():
    # every leg carries the same W row of the site spin, so the tensor is
    # invariant under all 720 leg permutations (field included), up to the
    # rounding of the six-factor products taken in different orders
    import itertools
    t = hotrg3d.ising3d_tensor(0.31, 0.2)
    for perm in itertools.permutations(range(6)):
        assert np.abs(t - t.transpose(perm)).max() <= 4e-16 * np.abs(t).max()


def _stack(t):
    # S[x1, x2, x1', x2', y1, y2, y1', y2', z, z'] = sum_m t[x1,x1',y1,y1',z,m] t[x2,x2',y2,y2',m,z']
    return np.einsum("abcdem,fghimj->afbgchdiej", t, t)


def test_environment_is_gram_of_stacked_pair():
    rng = np.random.default_rng(5)
    t = rng.standard_normal((2, 2, 3, 3, 2, 2))
    mx, my = hotrg3d.environments_z(t)
    s = _stack(t)
    sx = s.reshape(4, -1)
    assert np.abs(mx - sx @ sx.T).max() <= 1e-12 * np.abs(mx).max()
    sy = s.transpose(4, 5, 0, 1, 2, 3, 6, 7, 8, 9).reshape(9, -1)
    assert np.abs(my - sy @ sy.T).max() <= 1e-12 * np.abs(my).max()


def test_contraction_matches_defining_sum():
    rng = np.random.default_rng(6)
    t = rng.standard_normal((2, 2, 2, 2, 3, 3))
    ux = np.linalg.qr(rng.standard_normal((4, 3)))[0].reshape(2, 2, 3)
    uy = np.linalg.qr(rng.standard_normal((4, 4)))[0].reshape(2, 2, 4)
    ref = np.einsum("aeX,bfW,cgY,dhV,abcdzm,efghmw->XWYVzw", ux, ux, uy, uy, t, t)
    out = hotrg3d.contract_z(t, ux, uy)
    assert out.shape == (3, 3, 4, 4, 3, 3)
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("dcut", [2, 4])
def test_free_spins_at_beta_zero(dcut):
    sol = hotrg3d.solve3d(hotrg3d.ising3d_tensor(0.0, 0.0), 0.0, dcut, 7)
    assert abs(sol.lnz_per_site - math.log(2)) <= 1e-14


def test_truncation_converges():
    beta = 0.2
    t0 = hotrg3d.ising3d_tensor(beta, 0.0)
    v = [hotrg3d.solve3d(t0, beta, d, 9).lnz_per_site for d in (2, 4, 6)]
    assert abs(v[2] - v[1]) < abs(v[1] - v[0])
