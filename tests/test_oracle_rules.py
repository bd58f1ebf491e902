"""Pins for the oracle's acceptance table and its deterministic dynamics.

Every expected value here comes from the definitions (Metropolis rule,
Hamiltonian, checkerboard order) or from closed forms, never from the oracle
itself.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle
from oracle import exact

TWO32 = 1 << 32


def _exact_threshold(p) -> int:
    """floor(p * 2^32) from a 50-digit p."""
    with mpmath.workdps(50):
        return int(mpmath.floor(p * TWO32))


# ----------------------------------------------------------------------------
# threshold table: T[a] = 2^32 min(1, exp(-beta (4a - 8)))
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("beta", [1e-6, 0.1, 0.3, exact.BETA_C, 0.4406868, 0.6, 1.0, 3.0])
def test_thresholds_match_closed_form(beta):
    T = oracle.thresholds(beta)
    assert T[0] == T[1] == T[2] == TWO32  # dE <= 0 is always accepted
    with mpmath.workdps(50):
        p3 = mpmath.exp(-4 * mpmath.mpf(beta))
        p4 = mpmath.exp(-8 * mpmath.mpf(beta))
    # the oracle builds p in double precision: allow one unit of 2^-32
    assert abs(int(T[3]) - _exact_threshold(p3)) <= 1
    assert abs(int(T[4]) - _exact_threshold(p4)) <= 1
    assert T[4] < T[3] < TWO32


def test_thresholds_at_beta_c_are_silver_ratio_powers():
    # exp(-4 beta_c) = (1 + sqrt 2)^-2 = 3 - 2 sqrt 2; exp(-8 beta_c) = 17 - 12 sqrt 2
    T = oracle.thresholds(exact.BETA_C)
    with mpmath.workdps(50):
        s2 = mpmath.sqrt(2)
        assert abs(int(T[3]) - _exact_threshold(3 - 2 * s2)) <= 1
        assert abs(int(T[4]) - _exact_threshold(17 - 12 * s2)) <= 1


def test_thresholds_printed_values():
    # p3 = e^{-4b}, p4 = e^{-8b} to 6 significant digits
    for beta, p3, p4 in [(0.30, 0.301194, 0.0907180), (0.60, 0.0907180, 0.00822975),
                         (0.4406868, 0.171572871, 0.0294372515)]:
        T = oracle.thresholds(beta)
        assert math.isclose(int(T[3]) / TWO32, p3, rel_tol=2e-6)
        assert math.isclose(int(T[4]) / TWO32, p4, rel_tol=2e-6)


def test_thresholds_special_betas():
    assert list(oracle.thresholds(0.0)) == [TWO32] * 5  # infinite temperature: always flip
    T = oracle.thresholds(50.0)
    assert T[3] == 0 and T[4] == 0  # zero temperature: never climb
    for bad in (-0.1, float("nan"), float("inf")):
        with pytest.raises(ValueError):
            oracle.thresholds(bad)


# ----------------------------------------------------------------------------
# deterministic special cases
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("L", [2, 4, 6, 10, 16])
def test_beta_zero_negates_the_lattice_each_sweep(L):
    s0 = oracle.init(L, oracle.MODE_RANDOM, 99)
    s = s0.copy()
    oracle.run(s, 0.0, 1, 99)
    np.testing.assert_array_equal(s, -s0)
    tr = oracle.run(s, 0.0, 2, 99, off=1)
    np.testing.assert_array_equal(s, -s0)
    o0 = exact_bond_sum(s0)
    assert tr[0, 0] == s0.sum() and tr[1, 0] == -s0.sum()
    assert tr[0, 1] == tr[1, 1] == o0


def exact_bond_sum(s):
    s = s.astype(np.int64)
    return int((s * np.roll(s, -1, axis=1)).sum() + (s * np.roll(s, -1, axis=0)).sum())


def neel(L):
    i, c = np.indices((L, L))
    return np.where((i + c) % 2 == 0, 1, -1).astype(np.int8)  # black +1, white -1


@pytest.mark.parametrize("L", [4, 8, 12])
def test_zero_temperature_neel_start_black_first(L):
    s = neel(L)
    oracle.half_sweep(s, 50.0, 0, seed=5, t=0)
    # every black spin had 4 opposite neighbours (dE = -8): all flipped
    np.testing.assert_array_equal(s, -np.ones((L, L), np.int8))
    s = neel(L)
    oracle.run(s, 50.0, 3, seed=5)
    # black first -> uniform -1, then nothing can climb at beta = 50
    np.testing.assert_array_equal(s, -np.ones((L, L), np.int8))


@pytest.mark.parametrize("mode", [oracle.MODE_UP, oracle.MODE_DOWN])
def test_zero_temperature_cold_start_is_frozen(mode):
    s = oracle.init(16, mode)
    s0 = s.copy()
    oracle.run(s, 50.0, 5, seed=1)
    np.testing.assert_array_equal(s, s0)


def test_half_sweep_touches_one_colour_only():
    L = 12
    i, c = np.indices((L, L))
    for colour in (0, 1):
        s0 = oracle.init(L, oracle.MODE_RANDOM, 3)
        s = s0.copy()
        oracle.half_sweep(s, 0.0, colour, seed=3, t=0)
        mine = (i + c) % 2 == colour
        np.testing.assert_array_equal(s[~mine], s0[~mine])
        np.testing.assert_array_equal(s[mine], -s0[mine])


def test_resume_equals_one_run():
    a, b = 7, 11
    s1 = oracle.init(20, oracle.MODE_RANDOM, 42)
    s2 = s1.copy()
    t1 = oracle.run(s1, 0.4, a + b, 42)
    ta = oracle.run(s2, 0.4, a, 42)
    tb = oracle.run(s2, 0.4, b, 42, off=a)
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(t1, np.vstack([ta, tb]))


def test_thread_count_does_not_change_the_result():
    s1 = oracle.init(64, oracle.MODE_RANDOM, 8)
    s2 = s1.copy()
    t1 = oracle.run(s1, exact.BETA_C, 10, 8, nthreads=1)
    t2 = oracle.run(s2, exact.BETA_C, 10, 8, nthreads=4)
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(t1, t2)


def test_trace_is_the_observables_after_each_sweep():
    s = oracle.init(10, oracle.MODE_RANDOM, 2)
    ref = s.copy()
    tr = oracle.run(s, 0.35, 4, 2)
    for k in range(4):
        oracle.run(ref, 0.35, 1, 2, off=k, trace=False)
        assert tr[k, 0] == int(ref.sum())
        assert tr[k, 1] == exact_bond_sum(ref)


def test_random_init_uses_top_bit_of_the_init_draw():
    L = 6
    s = oracle.init(L, oracle.MODE_RANDOM, 77)
    for i in range(L):
        for c in range(L):
            site = i * (L // 2) + c // 2
            u = oracle.draw(77, site, 0, (i + c) % 2, oracle.PURPOSE_INIT)
            assert s[i, c] == (1 if u < 2**31 else -1)


# ----------------------------------------------------------------------------
# the Metropolis rule, site by site, against the Hamiltonian
# ----------------------------------------------------------------------------
def hamiltonian(s):
    return -exact_bond_sum(s)  # Eq. 1 with J = 1


def test_metropolis_flip_probability_per_site():
    """Flip frequency of every site over many independent half-sweeps equals
    min(1, exp(-beta dE)), dE taken from the full Hamiltonian."""
    L, beta, n = 6, 0.3, 6000
    rng = np.random.default_rng(11)
    start = rng.choice(np.array([-1, 1], np.int8), size=(L, L))
    for colour in (0, 1):
        flips = np.zeros((L, L))
        for t in range(n):
            s = start.copy()
            oracle.half_sweep(s, beta, colour, seed=2024, t=t)
            flips += s != start
        for i in range(L):
            for c in range(L):
                if (i + c) % 2 != colour:
                    assert flips[i, c] == 0
                    continue
                f = start.copy()
                f[i, c] = -f[i, c]
                dE = hamiltonian(f) - hamiltonian(start)
                p = min(1.0, math.exp(-beta * dE))
                sd = math.sqrt(max(p * (1 - p), 1e-12) / n)
                assert abs(flips[i, c] / n - p) < 5 * sd + 1e-12, (i, c, dE, flips[i, c] / n, p)


def test_metropolis_uses_the_sites_own_draw():
    """At beta = ln 2 / 4, a site with 3 aligned neighbours flips with p = 1/2;
    it must flip exactly when its own draw is below 2^31."""
    beta = math.log(2.0) / 4
    T = oracle.thresholds(beta)
    assert abs(int(T[3]) - 2**31) <= 1
    L = 8
    s0 = np.ones((L, L), np.int8)
    i, c = 3, 5  # black? (3 + 5) even -> black
    s0[i, (c + 1) % L] = -1  # one opposite neighbour -> a = 3
    site = i * (L // 2) + c // 2
    for seed in range(200):
        s = s0.copy()
        oracle.half_sweep(s, beta, 0, seed=seed, t=9)
        u = oracle.draw(seed, site, 9, 0, oracle.PURPOSE_METROPOLIS)
        assert (s[i, c] == -1) == (u < int(T[3]))
