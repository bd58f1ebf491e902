"""Exact results for the 2D Ising model (J = 1, h = 0, periodic L x L).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

- ``enumerate_lattice``: brute force over all 2**(L*L) states of a small torus.
- ``kaufman_logZ`` / ``kaufman_energy``: Kaufman's exact partition function of
  the finite periodic lattice (B. Kaufman, Phys. Rev. 76, 1232 (1949)), in the
  form of A. E. Ferdinand and M. E. Fisher, Phys. Rev. 185, 832 (1969), Eq. 2.
- ``onsager_energy``: Onsager's bulk internal energy per site (L. Onsager,
  Phys. Rev. 65, 117 (1944)).
- ``onsager_magnetisation``: the spontaneous magnetisation
  (1 - sinh(2 beta)^-4)^(1/8) below T_c (paper, Sec. 5.3, Eq. 7, with J = 1
  and beta = 1/T).
- ``BETA_C``: the critical point sinh(2 beta_c) = 1, i.e.
  T_c = 2 / ln(1 + sqrt 2) = 2.269185... (paper, Sec. 5.3; the printed
  condition there is garbled, the value is not).
"""
from __future__ import annotations

import math

import mpmath
import numpy as np

BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))


# --------------------------------------------------------------------------
# Brute-force enumeration
# --------------------------------------------------------------------------
def _all_states(L: int) -> np.ndarray:
    n = L * L
    if n > 20:
        raise ValueError("enumeration is limited to L*L <= 20")
    idx = np.arange(1 << n, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(n, dtype=np.int64)[None, :]) & 1
    return (2 * bits - 1).astype(np.int8).reshape(-1, L, L)


def state_sums(L: int):
    """(sum s, sum over bonds s_i s_j) of every state of the L x L torus,
    state k having spin +1 at flat position p iff bit p of k is set."""
    s = _all_states(L).astype(np.int32)
    m = s.sum(axis=(1, 2))
    bonds = (s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) + (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    return m.astype(np.int64), bonds.astype(np.int64)


def enumerate_lattice(L: int, beta: float) -> dict:
    """Exact Boltzmann averages on the L x L torus by summing over all states.

    Returns Z and the averages of e = E/N, |m|, m^2, m^4 (N = L*L,
    E = -sum bonds, m = sum s / N), plus the exact distribution of the bond
    sum (``levels`` -> ``probs``)."""
    m, b = state_sums(L)
    N = L * L
    w = np.exp(beta * (b - b.max()).astype(np.float64))  # exp(-beta E) rescaled
    Z = w.sum()
    mm = m / N
    e = -b / N
    levels, inv = np.unique(b, return_inverse=True)
    probs = np.bincount(inv, weights=w) / Z
    return {
        "logZ": float(np.log(Z) + beta * b.max()),
        "e": float((w * e).sum() / Z),
        "absm": float((w * np.abs(mm)).sum() / Z),
        "m2": float((w * mm**2).sum() / Z),
        "m4": float((w * mm**4).sum() / Z),
        "bond_levels": levels,
        "bond_probs": probs,
    }


# --------------------------------------------------------------------------
# Kaufman's finite-lattice partition function
# --------------------------------------------------------------------------
def kaufman_logZ(L: int, beta, dps: int = 40):
    """ln Z of the periodic L x L lattice at coupling K = beta (J = 1).

    Z = 1/2 (2 sinh 2K)^(L^2/2) (Z1 + Z2 + Z3 + Z4), with
      Z1 = prod_{r=0}^{L-1} 2 cosh(L g_{2r+1} / 2),  Z2 = same with sinh,
      Z3 = prod_{r=0}^{L-1} 2 cosh(L g_{2r} / 2),    Z4 = same with sinh,
      cosh g_l = cosh 2K coth 2K - cos(pi l / L)  (g_l > 0, l >= 1),
      g_0 = 2K + ln tanh K  (negative above T_c, which flips the sign of Z4).
    """
    with mpmath.workdps(dps):
        return _logZ(L, mpmath.mpf(beta))


def _logZ(L: int, K):
    """kaufman_logZ at the current mpmath precision (no precision change, so
    that numerical differentiation can raise it)."""
    c = mpmath.cosh(2 * K) * mpmath.coth(2 * K)

    def gamma(l: int):
        if l == 0:
            return 2 * K + mpmath.log(mpmath.tanh(K))
        return mpmath.acosh(c - mpmath.cos(mpmath.pi * l / L))

    z = [mpmath.mpf(1)] * 4
    for r in range(L):
        go, ge = gamma(2 * r + 1), gamma(2 * r)
        z[0] *= 2 * mpmath.cosh(L * go / 2)
        z[1] *= 2 * mpmath.sinh(L * go / 2)
        z[2] *= 2 * mpmath.cosh(L * ge / 2)
        z[3] *= 2 * mpmath.sinh(L * ge / 2)
    pref = (L * L / mpmath.mpf(2)) * mpmath.log(2 * mpmath.sinh(2 * K))
    return pref + mpmath.log(sum(z) / 2)


def kaufman_energy(L: int, beta: float, dps: int = 40) -> float:
    """Exact <E>/N = -(1/N) d lnZ / d beta on the periodic L x L lattice."""
    with mpmath.workdps(dps):
        d = mpmath.diff(lambda k: _logZ(L, k), mpmath.mpf(beta))
        return float(-d / (L * L))


# --------------------------------------------------------------------------
# Onsager's bulk results
# --------------------------------------------------------------------------
def onsager_energy(beta: float) -> float:
    """Bulk energy per site: u = -coth(2b) [1 + (2/pi)(2 tanh^2(2b) - 1) K(k)],
    k = 2 sinh(2b) / cosh^2(2b), K the complete elliptic integral of the first
    kind with modulus k."""
    with mpmath.workdps(30):
        b = mpmath.mpf(beta)
        kappa = 2 * mpmath.sinh(2 * b) / mpmath.cosh(2 * b) ** 2
        pre = -mpmath.coth(2 * b)
        fac = 2 * mpmath.tanh(2 * b) ** 2 - 1
        if abs(kappa - 1) < mpmath.mpf(10) ** -25:  # at beta_c the product tends to 0
            return float(pre)
        return float(pre * (1 + 2 / mpmath.pi * fac * mpmath.ellipk(kappa**2)))


def onsager_magnetisation(beta: float) -> float:
    """Spontaneous magnetisation per site; 0 at and above T_c."""
    if beta <= BETA_C:
        return 0.0
    return (1.0 - math.sinh(2.0 * beta) ** -4) ** 0.125
