"""Exact results that pin the oracle (closed forms and brute-force sums).

ORACLE / TEST INFRASTRUCTURE ONLY.

* Onsager's free energy of the square-lattice Ising model at h = 0, in three
  independent forms:
    - the generalised-hypergeometric form the paper prints (Sec. 3.2, Eq. 3),
      -beta f = ln(2 cosh 2b) - kappa^2 4F3(1,1,3/2,3/2; 2,2,2; 16 kappa^2),
      kappa = sinh(2b) / (2 cosh^2(2b));
    - the single-integral form (Onsager 1944; e.g. Huang, Statistical
      Mechanics, sec. 17.5):
      -beta f = ln(2 cosh 2b) + (1/2pi) int_0^pi ln[(1 + sqrt(1 - k^2 sin^2 p))/2] dp,
      k = 2 sinh(2b) / cosh^2(2b)  (= 4 kappa);
    - the double-integral form
      -beta f = ln 2 + (1/8pi^2) int int ln[cosh^2(2b) - sinh(2b)(cos t1 + cos t2)].
* Baxter's free energy of the q-state Potts model (weights e^{K [s = s']})
  at its self-dual critical point e^{K_c} = 1 + sqrt(q), 0 < q < 4
  (Baxter 1973; Baxter, Exactly Solved Models, sec. 12.5):
      ln Z / V = (1/2) ln q + 2 int_0^inf sinh((pi - mu) x) tanh(mu x) / (x sinh(pi x)) dx,
      sqrt(q) = 2 cos(mu).
  It reduces to 2 ln 2 at q = 1 and to Onsager's value plus K_c at q = 2.
* Brute-force partition function of the Ising model on small periodic
  cubic lattices (every site bonds to its +x, +y and +z neighbours, a
  lattice one site wide bonding a site to itself), for the 3D blocking.
* Brute-force partition functions of small periodic lattices: Ising by
  enumerating spins, XY by enumerating bond charges of the character
  expansion.  Bonds: every site couples to its right and its upper
  neighbour (periodic), so a W x H torus has 2 W H bonds, and a torus of
  width 2 has two distinct bonds between horizontal neighbours -- the same
  bonds the traced tensor network has.

Geometry of the HOTRG lattice: the x half-step stacks two tensors vertically
and the y half-step horizontally, so after N half-steps (x first) one tensor
covers a block of width 2^floor(N/2) and height 2^ceil(N/2).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from .models import bessel_i

BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))


# --------------------------------------------------------------- Onsager ---
def onsager_series(beta: float, max_terms: int = 20_000_000, tol: float = 1e-17) -> float:
    """-beta f from the 4F3 form.  The series converges for 16 kappa^2 < 1
    (every beta except beta_c); close to beta_c it needs many terms."""
    c2 = math.cosh(2 * beta)
    kappa = math.sinh(2 * beta) / (2 * c2 * c2)
    z = 16 * kappa * kappa
    if z >= 1.0:
        raise ValueError("4F3 series does not converge at beta_c")
    total = 0.0
    term = 1.0
    n = 0
    # term_{n+1}/term_n = (n+1)^2 (n+3/2)^2 / ((n+2)^3 (n+1)) z
    chunk = 4096
    while n < max_terms:
        idx = np.arange(n, n + chunk, dtype=np.float64)
        ratios = (idx + 1.0) * (idx + 1.5) ** 2 / (idx + 2.0) ** 3 * z
        terms = term * np.concatenate(([1.0], np.cumprod(ratios[:-1])))
        total += float(np.sum(terms))
        term = float(terms[-1] * ratios[-1])
        n += chunk
        if term < tol * total:
            break
    return math.log(2 * c2) - kappa * kappa * total


def _gauss_legendre(f, a: float, b: float, npts: int) -> float:
    x, w = np.polynomial.legendre.leggauss(npts)
    xm, xr = 0.5 * (b + a), 0.5 * (b - a)
    return float(xr * np.sum(w * f(xm + xr * x)))


def onsager_integral(beta: float) -> float:
    """-beta f from the single-integral form, by composite Gauss-Legendre on
    [0, pi] split at pi/2 and graded geometrically towards pi/2, where the
    integrand is (nearly) non-smooth at and near beta_c."""
    c2 = math.cosh(2 * beta)
    k = 2 * math.sinh(2 * beta) / (c2 * c2)
    k2 = k * k

    def g(p):
        s = np.sin(p)
        return np.log(0.5 * (1.0 + np.sqrt(np.maximum(0.0, 1.0 - k2 * s * s))))

    half = 0.5 * math.pi
    total = 0.0
    # [0, pi/2] and [pi/2, pi] are mirror images (sin is symmetric about pi/2)
    edges = [0.0]
    width = half
    for _ in range(60):
        width *= 0.5
        edges.append(half - width)
    edges.append(half)
    for a, b in zip(edges[:-1], edges[1:]):
        total += _gauss_legendre(g, a, b, 40)
    total *= 2.0
    return math.log(2 * c2) + total / (2 * math.pi)


def onsager_double_integral(beta: float, npts: int = 400) -> float:
    """-beta f from the double-integral form (tensor-product Gauss-Legendre
    over [0, pi]^2, using the symmetry of cos).  Accurate away from beta_c."""
    c2 = math.cosh(2 * beta)
    s2 = math.sinh(2 * beta)
    x, w = np.polynomial.legendre.leggauss(npts)
    th = 0.5 * math.pi * (x + 1.0)
    wt = 0.5 * math.pi * w
    ct = np.cos(th)
    arg = c2 * c2 - s2 * (ct[:, None] + ct[None, :])
    val = float(np.sum(wt[:, None] * wt[None, :] * np.log(arg)))
    # integral over [0, 2pi]^2 = 4 x integral over [0, pi]^2
    return math.log(2.0) + 4.0 * val / (8 * math.pi ** 2)


def onsager_free_energy(beta: float) -> float:
    """Exact f = -(1/beta) ln Z / V of the 2D Ising model at h = 0."""
    return -onsager_integral(beta) / beta


# ----------------------------------------------------------- enumeration ---
def hotrg_block(nsteps: int, first_direction: str = "x") -> tuple[int, int]:
    """(width, height) of the periodic lattice that nsteps half-steps close."""
    n_x = (nsteps + 1) // 2 if first_direction == "x" else nsteps // 2
    n_y = nsteps - n_x
    # an x half-step doubles the height, a y half-step the width
    return 2 ** n_y, 2 ** n_x


def ising_lnz_exact(width: int, height: int, beta: float, h: float = 0.0) -> float:
    """ln Z of the Ising model on a width x height torus by enumeration."""
    nsite = width * height
    if nsite > 24:
        raise ValueError("lattice too large to enumerate")
    states = np.arange(2 ** nsite, dtype=np.int64)
    bits = (states[:, None] >> np.arange(nsite)) & 1
    spins = 1 - 2 * bits                             # bit 0 -> +1, bit 1 -> -1
    s = spins.reshape(-1, height, width)             # [state, y, x]
    bond = np.sum(s * np.roll(s, -1, axis=2), axis=(1, 2)) \
        + np.sum(s * np.roll(s, -1, axis=1), axis=(1, 2))
    mag = np.sum(s, axis=(1, 2))
    e = beta * bond + beta * h * mag
    emax = float(np.max(e))
    return emax + math.log(float(np.sum(np.exp(e - emax))))


def ising_magnetization_exact(width: int, height: int, beta: float, h: float = 0.0) -> float:
    """<(1/V) sum_i s_i> on a width x height torus by enumeration."""
    nsite = width * height
    if nsite > 24:
        raise ValueError("lattice too large to enumerate")
    states = np.arange(2 ** nsite, dtype=np.int64)
    s = (1 - 2 * ((states[:, None] >> np.arange(nsite)) & 1)).reshape(-1, height, width)
    bond = np.sum(s * np.roll(s, -1, axis=2), axis=(1, 2)) + np.sum(s * np.roll(s, -1, axis=1), axis=(1, 2))
    mag = np.sum(s, axis=(1, 2))
    e = beta * bond + beta * h * mag
    w = np.exp(e - np.max(e))
    return float(np.sum(w * mag) / np.sum(w)) / nsite


def potts_fraction0_exact(width: int, height: int, beta: float, h: float = 0.0, q: int = 3) -> float:
    """<(1/V) sum_i [s_i = 0]> on a torus by enumeration."""
    nsite = width * height
    if q ** nsite > 5e7:
        raise ValueError("lattice too large to enumerate")
    states = np.arange(q ** nsite, dtype=np.int64)
    s = ((states[:, None] // (q ** np.arange(nsite))) % q).reshape(-1, height, width)
    same = np.sum(s == np.roll(s, -1, axis=2), axis=(1, 2)) + np.sum(s == np.roll(s, -1, axis=1), axis=(1, 2))
    zeros = np.sum(s == 0, axis=(1, 2))
    e = beta * same + beta * h * zeros
    w = np.exp(e - np.max(e))
    return float(np.sum(w * zeros) / np.sum(w)) / nsite


def onsager_yang_magnetization(beta: float) -> float:
    """Spontaneous magnetization of the square-lattice Ising model (Yang 1952):
    M = (1 - sinh(2 beta)^-4)^(1/8) for beta > beta_c, else 0."""
    if beta <= BETA_C:
        return 0.0
    return (1.0 - math.sinh(2.0 * beta) ** -4) ** 0.125


def ising3d_lnz_exact(lx: int, ly: int, lz: int, beta: float, h: float = 0.0) -> float:
    """ln Z of the Ising model on an lx x ly x lz torus by enumeration:
    Z = sum_s exp(beta sum_<ij> s_i s_j + beta h sum_i s_i) over the 3 V bonds
    (i, i + e) for e = x, y, z (periodic)."""
    nsite = lx * ly * lz
    if nsite > 20:
        raise ValueError("lattice too large to enumerate")
    states = np.arange(2 ** nsite, dtype=np.int64)
    s = (1 - 2 * ((states[:, None] >> np.arange(nsite)) & 1)).reshape(-1, lz, ly, lx)
    bond = (np.sum(s * np.roll(s, -1, axis=3), axis=(1, 2, 3)) + np.sum(s * np.roll(s, -1, axis=2), axis=(1, 2, 3))
            + np.sum(s * np.roll(s, -1, axis=1), axis=(1, 2, 3)))
    e = beta * bond + beta * h * np.sum(s, axis=(1, 2, 3))
    emax = float(np.max(e))
    return emax + math.log(float(np.sum(np.exp(e - emax))))


def potts_critical_lnz(q: float) -> float:
    """ln Z / V of the q-state Potts model at its critical point
    T_c = 1 / ln(1 + sqrt(q)) (Sec. 3.3), infinite lattice, 0 < q < 4:
    Baxter's closed form, the integral evaluated by adaptive quadrature with
    sinh((pi - mu) x) / sinh(pi x) written as decaying exponentials."""
    from scipy.integrate import quad

    if not 0.0 < q < 4.0:
        raise ValueError("the closed form holds for 0 < q < 4")
    mu = math.acos(math.sqrt(q) / 2.0)

    def integrand(x: float) -> float:
        if x == 0.0:
            return mu * (math.pi - mu) / math.pi   # limit x -> 0
        ratio = math.exp(-mu * x) * (-math.expm1(-2.0 * (math.pi - mu) * x)) / (-math.expm1(-2.0 * math.pi * x))
        return ratio * math.tanh(mu * x) / x

    # the integrand decays like exp(-mu x) / x: nothing beyond x = 80 / mu counts
    val, _ = quad(integrand, 0.0, 80.0 / mu, limit=2000, epsabs=1e-15, epsrel=1e-13)
    return 0.5 * math.log(q) + 2.0 * val


def potts_lnz_exact(width: int, height: int, beta: float, h: float = 0.0, q: int = 3) -> float:
    """ln Z of the q-state Potts model on a torus by enumeration:
    Z = sum_s exp(beta * #(equal neighbour pairs) + beta h * #(sites in state 0))."""
    nsite = width * height
    if q ** nsite > 5e7:
        raise ValueError("lattice too large to enumerate")
    states = np.arange(q ** nsite, dtype=np.int64)
    digits = (states[:, None] // (q ** np.arange(nsite))) % q
    s = digits.reshape(-1, height, width)
    same = np.sum(s == np.roll(s, -1, axis=2), axis=(1, 2)) + np.sum(s == np.roll(s, -1, axis=1), axis=(1, 2))
    zeros = np.sum(s == 0, axis=(1, 2))
    e = beta * same + beta * h * zeros
    emax = float(np.max(e))
    return emax + math.log(float(np.sum(np.exp(e - emax))))


def xy_cos_exact(width: int, height: int, beta: float, h: float = 0.0, d0: int = 9) -> float:
    """<cos theta> of the charge-truncated XY model on a torus: the charge
    sum with the site factor of site (0, 0) replaced by
    (I_{div-1}(beta h) + I_{div+1}(beta h)) / 2, divided by Z (all sites
    are equivalent on the torus)."""
    return math.exp(_xy_log_charge_sum(width, height, beta, h, d0, impure_site=True) -
                    _xy_log_charge_sum(width, height, beta, h, d0, impure_site=False))


def xy_lnz_exact(width: int, height: int, beta: float, h: float = 0.0, d0: int = 9) -> float:
    """ln Z of the charge-truncated XY model (|n| <= (d0-1)/2) on a torus, by
    summing over all bond charges of the character expansion:
    Z = sum_n prod_bonds I_n(beta) prod_sites I_div(beta h),
    div = n_left + n_up - n_right - n_down at each site."""
    return _xy_log_charge_sum(width, height, beta, h, d0, impure_site=False)


def _xy_log_charge_sum(width: int, height: int, beta: float, h: float, d0: int, impure_site: bool) -> float:
    nmax = d0 // 2
    charges = np.arange(-nmax, nmax + 1)
    ib = np.array([bessel_i(int(n), beta) for n in charges])
    ndiv = 4 * nmax
    isite = {int(m): bessel_i(int(m), beta * h) for m in range(-ndiv, ndiv + 1)}
    site_tab = np.array([isite[m] for m in range(-ndiv, ndiv + 1)])
    # site (0, 0) with cos(theta) inserted (the charge sum may be negative then)
    imp_tab = np.array([0.5 * (bessel_i(m - 1, beta * h) + bessel_i(m + 1, beta * h))
                        for m in range(-ndiv, ndiv + 1)])
    nsite = width * height
    nbond = 2 * nsite
    if d0 ** nbond > 2e8:
        raise ValueError("lattice too large to enumerate")
    # bond numbering: horizontal bond from (x, y) to (x+1, y): y*W + x;
    # vertical bond from (x, y) to (x, y+1): nsite + y*W + x
    total = 0.0
    # enumerate the last bonds vectorised, the first ones in a Python loop
    nvec = min(nbond, 6)
    grids = np.array(list(itertools.product(range(d0), repeat=nvec)), dtype=np.int64).T
    for head in itertools.product(range(d0), repeat=nbond - nvec):
        idx = list(head) + [grids[i] for i in range(nvec)]
        n = [charges[i] if np.ndim(i) == 0 else charges[i] for i in idx]
        w = np.ones(grids.shape[1])
        for b in range(nbond):
            w = w * ib[idx[b]]
        for y in range(height):
            for x in range(width):
                n_r = n[y * width + x]
                n_l = n[y * width + (x - 1) % width]
                n_u = n[nsite + y * width + x]
                n_d = n[nsite + ((y - 1) % height) * width + x]
                div = n_l + n_u - n_r - n_d
                tab = imp_tab if (impure_site and x == 0 and y == 0) else site_tab
                w = w * tab[np.asarray(div) + ndiv]
        total += float(np.sum(w))
    return math.log(total)
