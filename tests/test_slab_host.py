"""Host logic of the slab decomposition (Sec. 4: horizontal slabs, each needing
the boundary rows of its two neighbours), on CPU with gloo ranks.

Each rank holds one slab with halo rows; the package's exchange and sweep
driver (``exchange_halos``, ``slab_sweep``) move the boundary rows between
ranks and order the half-sweeps.  The update of a slab's own rows is done
here by the oracle's row update, so the test checks the exchange pattern,
the halo placement, the colour order and the all-reduced trace against the
oracle's whole-lattice run, bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import paper_1906_06297_gb300 as ising

BETA = 0.4406868


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _decode(sl):
    """Int8 rows of plane rows 0 .. rows+1 (halo above, own rows, halo below)."""
    L = sl.L
    b = np.ascontiguousarray(sl.black.numpy()).view(np.uint64)
    w = np.ascontiguousarray(sl.white.numpy()).view(np.uint64)
    return [oracle.row_from_planes_msc4(L, (sl.row0 + pr - 1) % L, b[pr], w[pr]) for pr in range(sl.rows + 2)]


def oracle_slab_half_sweep(sl, beta, colour, seed, t, obs):
    """One colour of the slab's own rows by the oracle's row update, reading the
    neighbour rows from the halos; obs gets the slab's share of the sums, every
    bond counted at its white end."""
    L = sl.L
    full = _decode(sl)
    out = [r.copy() for r in full]
    for r in range(sl.rows):
        oracle.update_row(L, full[r], out[r + 1], full[r + 2], (sl.row0 + r) % L, colour, beta, seed, t)
        b, w = oracle.row_to_planes_msc4(L, sl.row0 + r, out[r + 1])
        sl.plane(colour)[r + 1].copy_(torch.from_numpy((b if colour == 0 else w).view(np.uint8)))
    if obs is not None:
        A = np.stack(out).astype(np.int64)
        ssum = int(A[1:sl.rows + 1].sum())
        bonds = 0
        for r in range(1, sl.rows + 1):
            i = sl.row0 + r - 1
            nb = A[r - 1] + A[r + 1] + np.roll(A[r], 1) + np.roll(A[r], -1)
            white = (np.arange(L) + i) % 2 == 1
            bonds += int((A[r] * nb)[white].sum())
        obs[0] += ssum
        obs[1] += bonds


def _worker(rank, world, port, L, n_sweeps, seed, q, overlap=True):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        row0, rows = ising.slab_partition(L, world)[rank]
        sl = ising.Slab(L, row0, rows, device="cpu")
        s = oracle.init(L, oracle.MODE_RANDOM, seed)
        b, w = oracle.to_planes_msc4(s)
        sl.load_own_numpy(b[row0:row0 + rows], w[row0:row0 + rows])
        trace = torch.zeros((n_sweeps, 2), dtype=torch.int64)
        ising.slab_sweep(sl, BETA, n_sweeps, seed, 5, trace, half_sweep=oracle_slab_half_sweep, overlap=overlap)
        want_trace = oracle.run(s, BETA, n_sweeps, seed, 5)
        wb, ww = oracle.to_planes_msc4(s)
        gb, gw = sl.own_numpy()
        ok_planes = np.array_equal(gb, wb[row0:row0 + rows]) and np.array_equal(gw, ww[row0:row0 + rows])
        # after the last exchange the black halos hold the neighbours' rows
        halo_ok = (np.array_equal(np.ascontiguousarray(sl.black[0].numpy()).view(np.uint64), wb[(row0 - 1) % L])
                   and np.array_equal(np.ascontiguousarray(sl.black[rows + 1].numpy()).view(np.uint64),
                                      wb[(row0 + rows) % L]))
        q.put((rank, ok_planes, halo_ok, np.array_equal(trace.numpy(), want_trace)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("world,L", [(2, 64), (3, 128)])
def test_gloo_slabs_match_the_whole_lattice(world, L, overlap):
    """Two ranks (the pair exchanges both rows with each other) and three
    ranks (slabs of 43/43/42 rows: a slab starting on an odd row), in the
    serial order and in the overlapped one (boundary rows first, their
    messages posted before the interior rows are updated)."""
    oracle.build()
    ising.build()
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, L, 4, 99, q, overlap)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == list(range(world))
    for rank, ok_planes, halo_ok, ok_trace in out:
        assert ok_planes, f"rank {rank}: own rows differ from the whole-lattice run"
        assert halo_ok, f"rank {rank}: halo rows are not the neighbours' boundary rows"
        assert ok_trace, f"rank {rank}: all-reduced trace differs"


def test_slab_partition_and_sizes():
    assert ising.slab_partition(10, 3) == [(0, 4), (4, 3), (7, 3)]
    assert ising.slab_partition(64, 1) == [(0, 64)]
    parts = ising.slab_partition(65536, 7)
    assert sum(r for _, r in parts) == 65536 and max(r for _, r in parts) - min(r for _, r in parts) <= 1
    with pytest.raises(ValueError):
        ising.slab_partition(4, 5)
    ising.build()
    assert ising.ising_slab_bytes(256, 10) == (64, 64 * 12)
    for L, rows, layout in [(96, 4, ising.ISING_MSC4), (256, 0, ising.ISING_MSC4), (256, 257, ising.ISING_MSC4),
                            (256, 4, ising.ISING_INT8)]:
        with pytest.raises(ising.IsingError) as e:
            ising.ising_slab_bytes(L, rows, layout)
        assert e.value.status == ising.ISING_EINVAL
