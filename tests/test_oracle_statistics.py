"""Pins for the oracle's stationary law against exact results.

The checkerboard Metropolis chain must sample the Boltzmann distribution of
Eq. 1: each half-sweep is a product of commuting single-site Metropolis
kernels, each of which satisfies detailed balance.  The oracle's long-run
averages are compared with
  - brute-force enumeration of the 4 x 4 torus (2^16 states),
  - Kaufman's exact finite-lattice energy at beta_c (L = 16),
  - Onsager's bulk energy and spontaneous magnetisation (Sec. 5.3, Eq. 7)
off criticality, where finite-size corrections are exponentially small.
Error bars use the integrated autocorrelation time (oracle.stats).  All
seeds are fixed, so each check is deterministic; the bounds are 4 sigma.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import exact, stats

NSIG = 4.0


def _chains(L, beta, n_chains, n_sweeps, burn, mode=oracle.MODE_RANDOM, seed0=1000):
    es, ms = [], []
    N = L * L
    for k in range(n_chains):
        s = oracle.init(L, mode, seed0 + k)
        oracle.run(s, beta, burn, seed0 + k, trace=False, nthreads=1)
        tr = oracle.run(s, beta, n_sweeps, seed0 + k, off=burn, nthreads=1)
        es.append(-tr[:, 1] / N)
        ms.append(tr[:, 0] / N)
    return es, ms


def _check(name, chains, target):
    m, err = stats.pooled_mean_and_error(chains)
    assert err > 0
    assert abs(m - target) < NSIG * err, f"{name}: {m} +- {err} vs exact {target}"


def test_stats_estimator_on_ar1():
    """tau_int of an AR(1) series with coefficient phi is (1+phi)/(2(1-phi))."""
    rng = np.random.default_rng(0)
    phi, n = 0.8, 400_000
    x = np.empty(n)
    x[0] = 0.0
    eps = rng.standard_normal(n)
    for i in range(1, n):
        x[i] = phi * x[i - 1] + eps[i]
    tau = stats.tau_int(x)
    assert abs(tau - (1 + phi) / (2 * (1 - phi))) < 0.3


@pytest.mark.parametrize("beta", [0.30, exact.BETA_C, 0.60])
def test_4x4_enumeration(beta):
    L = 4
    ex = exact.enumerate_lattice(L, beta)
    es, ms = _chains(L, beta, n_chains=16, n_sweeps=40_000, burn=500)
    _check("e", es, ex["e"])
    _check("|m|", [np.abs(m) for m in ms], ex["absm"])
    _check("m^2", [m**2 for m in ms], ex["m2"])
    _check("m^4", [m**4 for m in ms], ex["m4"])
    # full distribution of the bond sum, level by level
    bonds = np.concatenate([-e * L * L for e in es]).round().astype(np.int64)
    for lev, p in zip(ex["bond_levels"], ex["bond_probs"]):
        ind = [(-e * L * L).round() == lev for e in es]
        m, err = stats.pooled_mean_and_error([i.astype(float) for i in ind])
        tol = NSIG * max(err, math.sqrt(p * (1 - p) / bonds.size))
        assert abs(m - p) < tol + 1e-4, (lev, m, p, err)


def test_kaufman_matches_enumeration_at_l4():
    for beta in (0.2, exact.BETA_C, 0.7):
        ex = exact.enumerate_lattice(4, beta)
        assert abs(float(exact.kaufman_logZ(4, beta)) - ex["logZ"]) < 1e-10
        assert abs(exact.kaufman_energy(4, beta) - ex["e"]) < 1e-10


def test_kaufman_tends_to_onsager_off_critical():
    for beta in (0.30, 0.60):
        assert abs(exact.kaufman_energy(96, beta) - exact.onsager_energy(beta)) < 1e-9


def test_onsager_closed_form_values():
    assert abs(exact.onsager_energy(exact.BETA_C) + math.sqrt(2.0)) < 1e-12
    assert abs(exact.onsager_energy(0.30) - (-0.7044990708)) < 1e-9
    assert abs(exact.onsager_energy(0.60) - (-1.9090861777)) < 1e-9
    assert exact.onsager_magnetisation(exact.BETA_C) == 0.0
    # low-temperature series m = 1 - 2x^4 - 8x^6 - 34x^8 - ..., x = exp(-2 beta)
    b = 2.0
    x = math.exp(-2 * b)
    assert abs(exact.onsager_magnetisation(b) - (1 - 2 * x**4 - 8 * x**6 - 34 * x**8)) < 1e-12
    assert abs(exact.onsager_magnetisation(0.60) - 0.9736086674) < 1e-9
    # beta_c: sinh(2 beta_c) = 1 and T_c = 2.269185 (Sec. 5.3)
    assert abs(math.sinh(2 * exact.BETA_C) - 1.0) < 1e-15
    assert abs(1 / exact.BETA_C - 2.269185) < 1e-6


def test_finite_lattice_energy_at_beta_c():
    L = 16
    target = exact.kaufman_energy(L, exact.BETA_C)
    es, _ = _chains(L, exact.BETA_C, n_chains=4, n_sweeps=25_000, burn=2_000)
    _check("e(L=16, beta_c)", es, target)


def test_onsager_energy_hot_phase():
    es, _ = _chains(64, 0.30, n_chains=2, n_sweeps=3_000, burn=500)
    _check("e(0.30)", es, exact.onsager_energy(0.30))


def test_onsager_energy_and_magnetisation_ordered_phase():
    es, ms = _chains(64, 0.60, n_chains=2, n_sweeps=3_000, burn=500, mode=oracle.MODE_UP)
    _check("e(0.60)", es, exact.onsager_energy(0.60))
    _check("|m|(0.60)", [np.abs(m) for m in ms], exact.onsager_magnetisation(0.60))
