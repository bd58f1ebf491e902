"""Parity of the batched sweep with replica exchange against the oracle.

Every lattice of the batch, the slot state of every ladder and the recorded
trace must equal the oracle's batched run bit for bit, for any launch shape,
with and without the captured graph, and across split runs.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1906_06297_gb300 as ising

pytestmark = pytest.mark.gpu

MIXED_L = [32] * 4 + [64] * 4 + [96] * 2 + [128] * 2 + [256] * 2
MIXED_BETA = [0.400, 0.403]  # close enough that replicas exchange


@pytest.fixture(scope="module", autouse=True)
def built():
    ising.build()
    oracle.build()


def gpu_full(batch, i):
    b, w = batch.planes_numpy(i)
    return oracle.from_planes_msc4(int(batch.L[i]), b, w)


def run_both(L, S, beta, seed, sweeps, record_every, swaps, offset=0, configs=None, use_graph=True):
    g = ising.Batch(L, S, beta)
    g.init(ising.ISING_INIT_RANDOM, seed)
    if configs:
        g.config(*configs)
    n_ev = g.n_events(sweeps, offset, record_every)
    tr = torch.zeros((max(n_ev, 1), len(L), 2), dtype=torch.int64, device="cuda")
    if offset:
        # bring both sides to the offset first (no records)
        g.run(offset, seed, 0, 0, False, None, use_graph)
    g.run(sweeps, seed, offset, record_every, swaps, tr if n_ev else None, use_graph)
    g.check()
    o = oracle.Batch(L, S, beta, oracle.MODE_RANDOM, seed)
    if offset:
        o.run(offset, seed, 0, 0, False)
    tr_o = o.run(sweeps, seed, offset, record_every, swaps)
    return g, o, tr[:n_ev].cpu().numpy() if n_ev else None, tr_o


def assert_same(g, o, tr, tr_o):
    for i in range(g.n):
        np.testing.assert_array_equal(gpu_full(g, i), o.lattice(i), err_msg=f"lattice {i}")
    slot, at = g.state_numpy()
    np.testing.assert_array_equal(slot, o.slot_of)
    np.testing.assert_array_equal(at, o.lattice_at)
    if tr_o is not None:
        np.testing.assert_array_equal(tr, tr_o)


def test_init_matches_oracle():
    g = ising.Batch(MIXED_L, 2, MIXED_BETA)
    g.init(ising.ISING_INIT_RANDOM, 9)
    torch.cuda.synchronize()
    o = oracle.Batch(MIXED_L, 2, MIXED_BETA, oracle.MODE_RANDOM, 9)
    for i in range(g.n):
        np.testing.assert_array_equal(gpu_full(g, i), o.lattice(i))


@pytest.mark.parametrize("swaps", [False, True])
def test_mixed_sizes_with_exchanges(swaps):
    g, o, tr, tr_o = run_both(MIXED_L, 2, MIXED_BETA, 5, 37, 4, swaps)
    assert_same(g, o, tr, tr_o)
    if swaps:
        assert not np.array_equal(o.slot_of, np.arange(len(MIXED_L)) % 2)  # some exchange happened


def test_ladders_of_eight_temperatures():
    L = [32] * 16 + [64] * 8
    beta = list(np.linspace(0.30, 0.60, 8))
    g, o, tr, tr_o = run_both(L, 8, beta, 77, 60, 3, True)
    assert_same(g, o, tr, tr_o)


@pytest.mark.parametrize("threads,wpt", [(256, 1), (256, 2), (512, 4), (512, 1)])
def test_launch_shape_does_not_change_results(threads, wpt):
    g, o, tr, tr_o = run_both(MIXED_L, 2, MIXED_BETA, 13, 21, 5, True, configs=(threads, wpt))
    assert_same(g, o, tr, tr_o)


def test_direct_launch_equals_graph_and_split_runs():
    g, o, tr, tr_o = run_both(MIXED_L, 2, MIXED_BETA, 21, 30, 5, True, use_graph=False)
    assert_same(g, o, tr, tr_o)
    g2 = ising.Batch(MIXED_L, 2, MIXED_BETA)
    g2.init(ising.ISING_INIT_RANDOM, 21)
    tr2 = torch.zeros((6, len(MIXED_L), 2), dtype=torch.int64, device="cuda")
    g2.run(12, 21, 0, 5, True, tr2[:2])
    g2.run(18, 21, 12, 5, True, tr2[2:])
    g2.check()
    for i in range(g.n):
        np.testing.assert_array_equal(gpu_full(g2, i), o.lattice(i))
    np.testing.assert_array_equal(tr2.cpu().numpy(), tr_o)


def test_lattice_zero_is_the_single_lattice_sweep():
    L, seed, beta, n = 128, 31, 0.4406868, 25
    g = ising.Batch([L, L, L], 1, [beta])
    g.init(ising.ISING_INIT_RANDOM, seed)
    g.run(n, seed)
    g.check()
    single = ising.Lattice(L, "msc4")
    ising.ising_init_lattice(single, ising.ISING_INIT_RANDOM, seed)
    ising.ising_sweep(single, beta, n, seed)
    torch.cuda.synchronize()
    b, w = single.planes_numpy()
    np.testing.assert_array_equal(gpu_full(g, 0), oracle.from_planes_msc4(L, b, w))


def test_autotune_keeps_results():
    g = ising.Batch(MIXED_L, 2, MIXED_BETA)
    g.init(ising.ISING_INIT_RANDOM, 3)
    cfg = g.autotune(2)
    assert cfg[0] in (256, 512) and cfg[1] in (1, 2, 4)
    g.run(10, 3, 0, 5, True)
    g.check()
    o = oracle.Batch(MIXED_L, 2, MIXED_BETA, oracle.MODE_RANDOM, 3)
    o.run(10, 3, 0, 5, True)
    for i in range(g.n):
        np.testing.assert_array_equal(gpu_full(g, i), o.lattice(i))


def test_barrier_timeout_is_reported_and_the_context_survives():
    g = ising.Batch([32, 32], 2, MIXED_BETA)
    g.init(ising.ISING_INIT_RANDOM, 1)
    # ~2 ms at 2 GHz: every wait of the impossible barrier runs out
    assert g.barrier_selftest(4_000_000) == ising.ISING_ETIMEOUT
    g.run(5, 1, 0, 5, True)
    g.check()
    o = oracle.Batch([32, 32], 2, MIXED_BETA, oracle.MODE_RANDOM, 1)
    o.run(5, 1, 0, 5, True)
    np.testing.assert_array_equal(gpu_full(g, 1), o.lattice(1))


def test_invalid_batches_are_rejected():
    for L, S, beta in [([32, 32, 32], 2, MIXED_BETA), ([32, 48], 2, MIXED_BETA), ([32, 64], 2, MIXED_BETA),
                       ([32, 32], 2, [0.5, 0.4]), ([32, 32], 2, [0.0, 0.4])]:
        with pytest.raises(ising.IsingError) as e:
            ising.Batch(L, S, beta)
        assert e.value.status == ising.ISING_EINVAL


def test_beta_whose_threshold_reaches_two_to_the_32_is_refused():
    """At beta = 1e-18, exp(-4 beta) rounds to 1 and T3 = 2^32, which the
    batched 32-bit compare cannot hold: creation refuses it."""
    with pytest.raises(ising.IsingError) as e:
        ising.Batch([32, 32, 64, 64], 2, [1e-18, 0.4])
    assert e.value.status == ising.ISING_EINVAL


def test_smallest_betas_near_the_cutoff_match_oracle():
    """beta = 2e-16 has T3 = 2^32 - 1 and T4 < 2^32: ordinary tables, and the
    batch must follow the oracle's uint64 rule bit for bit (Sec. 2)."""
    L = [32] * 2 + [64] * 2
    g, o, tr, tr_o = run_both(L, 2, [2e-16, 0.3], 21, 12, 3, True)
    assert_same(g, o, tr, tr_o)


@pytest.mark.parametrize("L,S,beta", [
    ([512] * 2 + [1024] * 2 + [2048] * 2, 2, MIXED_BETA),           # 8, 16 and 32 lanes per row
    ([160] * 2 + [128] * 4 + [96] * 2 + [2048] * 2, 2, MIXED_BETA),  # item and march groups interleaved
])
def test_row_marching_sides_match_oracle(L, S, beta):
    """Sides 128 .. 2048 that are powers of two go through the row-marching
    path (a row held by L/64 lanes, lane groups marching down whole rows);
    other sides through the item path.  Both, side by side in one launch and
    across lattice starts within a lane group's run, equal the oracle's
    batched run bit for bit, with exchanges and traces."""
    g, o, tr, tr_o = run_both(L, S, beta, 61, 9, 3, True)
    assert_same(g, o, tr, tr_o)
