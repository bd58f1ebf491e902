"""Pins for the oracle's batched sweeps with replica exchange.

A batch is n independent lattices; ladders of S lattices exchange
temperatures every `record_every` sweeps with probability
min(1, exp((beta_hi - beta_lo)(E_b - E_a))).  The pins: the threshold against
a 50-digit exponential, the swap frequency per energy difference against that
formula, the joint stationary law of a two-replica ladder against exact
enumeration (the product of the two Boltzmann laws), and lattice 0 of a
batch against the single-lattice oracle.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle
from oracle import exact, stats


def test_swap_threshold_closed_form():
    for lo, hi in [(0.3, 0.6), (0.30, 0.30 + 0.3 / 63), (0.44, 0.45)]:
        assert oracle.swap_threshold(lo, hi, 0) == 1 << 32
        assert oracle.swap_threshold(lo, hi, 8) == 1 << 32
        for D in (-4, -8, -40, -400):
            with mpmath.workdps(50):
                p = mpmath.exp(-(mpmath.mpf(hi) - mpmath.mpf(lo)) * (-D))
                want = int(mpmath.floor(p * 2**32))
            assert abs(oracle.swap_threshold(lo, hi, D) - want) <= 1
    assert oracle.swap_threshold(0.3, 0.6, -4000) == 0


def test_batch_lattice_zero_is_the_single_lattice_oracle():
    b = oracle.Batch([8, 8, 8, 8], 4, [0.3, 0.4, 0.5, 0.6], seed=11)
    s = oracle.init(8, oracle.MODE_RANDOM, 11)
    np.testing.assert_array_equal(b.lattice(0), s)
    b.run(15, 11, swaps=False)
    oracle.run(s, 0.3, 15, 11)
    np.testing.assert_array_equal(b.lattice(0), s)
    # the other lattices use other streams: same start rule, different draws
    assert not np.array_equal(b.lattice(1), b.lattice(0))


def test_batch_without_swaps_keeps_slots_and_records_observables():
    b = oracle.Batch([6, 6, 10, 10], 2, [0.35, 0.45], seed=3)
    tr = b.run(12, 3, record_every=4, swaps=False)
    assert tr.shape == (3, 4, 2)
    np.testing.assert_array_equal(b.slot_of, [0, 1, 0, 1])
    for i in range(4):
        np.testing.assert_array_equal(tr[-1, i], oracle.observables(b.lattice(i)))


def test_swap_frequency_matches_replica_exchange_rule():
    """Over many events, the fraction of accepted exchanges at each energy
    difference D equals min(1, exp(dbeta * D))."""
    lo, hi = 0.40, 0.48
    b = oracle.Batch([4, 4], 2, [lo, hi], seed=21)
    tried, done = {}, {}
    n = 12000
    tr = b.run(2 * n, 21, record_every=1)  # exchanges on even events only (S = 2)
    # replay the slot history: rerun event by event would be slow; instead
    # recompute acceptance from consecutive traces: the lattice at slot 0 in
    # event e+1 differs from slot 0 in event e only through a sweep, so track
    # exchanges directly from a second run that records slots
    b2 = oracle.Batch([4, 4], 2, [lo, hi], seed=21)
    for e in range(0, 2 * n, 2):
        before = b2.lattice_at.copy()
        t = b2.run(1, 21, off=e, record_every=1)
        D = int(t[0, 0, 1] - t[0, 1, 1])  # bonds_a - bonds_b
        tried[D] = tried.get(D, 0) + 1
        done[D] = done.get(D, 0) + int(b2.lattice_at[0] != before[0])
        b2.run(1, 21, off=e + 1, record_every=1)  # odd event: no pair for S = 2
    np.testing.assert_array_equal(b2.spins, b.spins)  # same trajectory both ways
    assert tr.shape == (2 * n, 2, 2)
    checked = 0
    for D, m in tried.items():
        if m < 200:
            continue
        p = min(1.0, math.exp((hi - lo) * D))
        f = done[D] / m
        sd = math.sqrt(max(p * (1 - p), 1e-12) / m)
        assert abs(f - p) < 5 * sd + 1e-12, (D, f, p, m)
        checked += 1
    assert checked >= 4


def test_two_replica_ladder_samples_the_product_law():
    """Slots at beta 0.30 and 0.60 of a 4x4 two-replica ladder with an
    exchange every other sweep: each slot's bond-sum distribution equals the
    exact Boltzmann law at its own beta, and the joint law is their product."""
    lo, hi = 0.30, 0.60
    ex_lo, ex_hi = exact.enumerate_lattice(4, lo), exact.enumerate_lattice(4, hi)
    chains = 6
    series = []
    for c in range(chains):
        b = oracle.Batch([4, 4], 2, [lo, hi], seed=100 + c)
        b.run(200, 100 + c, record_every=1)
        tr = b.run(30000, 100 + c, off=200, record_every=1)
        series.append(tr[:, :, 1])  # (events, slot) bond sums
    for slot, ex in ((0, ex_lo), (1, ex_hi)):
        es = [-s[:, slot] / 16.0 for s in series]
        m, err = stats.pooled_mean_and_error(es)
        assert abs(m - ex["e"]) < 4 * err, (slot, m, err, ex["e"])
        for lev, p in zip(ex["bond_levels"], ex["bond_probs"]):
            if p < 0.02:
                continue
            ind = [(s[:, slot] == lev).astype(float) for s in series]
            f, ferr = stats.pooled_mean_and_error(ind)
            assert abs(f - p) < 4 * ferr + 1e-4, (slot, lev, f, p)
    # independence across slots: P(a, b) = P(a) P(b) for the largest cells
    pa = dict(zip(ex_lo["bond_levels"], ex_lo["bond_probs"]))
    pb = dict(zip(ex_hi["bond_levels"], ex_hi["bond_probs"]))
    for a in sorted(pa, key=pa.get)[-2:]:
        for bb in sorted(pb, key=pb.get)[-2:]:
            ind = [((s[:, 0] == a) & (s[:, 1] == bb)).astype(float) for s in series]
            f, ferr = stats.pooled_mean_and_error(ind)
            want = pa[a] * pb[bb]
            assert abs(f - want) < 4 * ferr + 1e-4, (a, bb, f, want)
