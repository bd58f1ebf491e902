"""Parity at the full benchmark sizes, in the launch configuration the
benchmark times (ising_sweep on a dense MSC4 lattice).

The oracle cannot sweep 4.3e9 or 6.9e10 spins in test time, so rows are
checked one at a time: rows r-1, r, r+1 of both planes are copied back before
a half-sweep, the oracle updates row r from them, and the GPU's row r after
the half-sweep must match bit for bit.  Whole-lattice properties (beta = 0
negation, fused trace == separate observables kernel) hold at any size.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1906_06297_gb300 as ising

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ising.build()
    oracle.build()


def row_words(plane: torch.Tensor, r: int, row_bytes: int) -> np.ndarray:
    return np.ascontiguousarray(plane[r, :row_bytes].cpu().numpy()).view(np.uint64)


def full_row(lat, r):
    r %= lat.L
    return oracle.row_from_planes_msc4(lat.L, r, row_words(lat.black, r, lat.row_bytes),
                                       row_words(lat.white, r, lat.row_bytes))


def banded_half_sweep_check(lat, beta, colour, seed, t, rows, obs=None):
    before = {r: (full_row(lat, r - 1), full_row(lat, r), full_row(lat, r + 1)) for r in rows}
    ising.ising_half_sweep(lat, beta, colour, seed, t, obs)
    torch.cuda.synchronize()
    for r in rows:
        above, row, below = before[r]
        expect = oracle.update_row(lat.L, above, row.copy(), below, r, colour, beta, seed, t)
        np.testing.assert_array_equal(full_row(lat, r), expect, err_msg=f"row {r} colour {colour}")


def test_65536_random_start_rows_match_oracle():
    L, seed, beta = 65536, 1234, 0.4406868
    lat = ising.Lattice(L, "msc4")
    ising.ising_init_lattice(lat, ising.ISING_INIT_RANDOM, seed)
    torch.cuda.synchronize()
    for r in (0, 1, 4097, 32768, L - 1):
        np.testing.assert_array_equal(full_row(lat, r), oracle.init_row(L, r, oracle.MODE_RANDOM, seed))
    trace = torch.zeros((3, 2), dtype=torch.int64, device="cuda")
    ising.ising_sweep(lat, beta, 3, seed, 0, trace)
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    ising.ising_observables(lat, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(trace[2].cpu().numpy(), out.cpu().numpy())
    rows = [0, 1, 2, 1023, 4096, 32767, 32768, 54321, L - 2, L - 1]
    for t in (3, 4):
        banded_half_sweep_check(lat, beta, 0, seed, t, rows)
        banded_half_sweep_check(lat, beta, 1, seed, t, rows)


def test_65536_beta_zero_negates():
    L, seed = 65536, 9
    lat = ising.Lattice(L, "msc4")
    ising.ising_init_lattice(lat, ising.ISING_INIT_RANDOM, seed)
    o0 = torch.zeros(2, dtype=torch.int64, device="cuda")
    ising.ising_observables(lat, o0)
    torch.cuda.synchronize()
    rows = [0, 777, L - 1]
    before = {r: full_row(lat, r) for r in rows}
    trace = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    ising.ising_sweep(lat, 0.0, 1, seed, 0, trace)
    torch.cuda.synchronize()
    m0, b0 = o0.cpu().numpy()
    np.testing.assert_array_equal(trace[0].cpu().numpy(), [-m0, b0])
    for r in rows:
        np.testing.assert_array_equal(full_row(lat, r), -before[r])


def test_262144_cold_start_rows_beyond_2_32_sites():
    """Rows past 32768 have plane-site indices above 2^32, so their Philox
    counters use the high counter word."""
    L = 262144
    need = 2 * L * L // 4 + (1 << 30)
    free, _ = torch.cuda.mem_get_info()
    if free < need:
        pytest.skip(f"needs {need / 2**30:.1f} GiB free")
    seed, beta = 5, 0.4406868
    lat = ising.Lattice(L, "msc4")
    ising.ising_init_lattice(lat, ising.ISING_INIT_UP, seed)
    trace = torch.zeros((2, 2), dtype=torch.int64, device="cuda")
    ising.ising_sweep(lat, beta, 2, seed, 0, trace)
    torch.cuda.synchronize()
    tr = trace.cpu().numpy()
    assert abs(int(tr[0, 1])) <= 2 * L * L and int(tr[1, 0]) <= L * L
    rows = [0, 32767, 32768, 40000, 200001, L - 1]
    banded_half_sweep_check(lat, beta, 0, seed, 2, rows)
    obs = torch.zeros(2, dtype=torch.int64, device="cuda")
    banded_half_sweep_check(lat, beta, 1, seed, 2, rows, obs)
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    ising.ising_observables(lat, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(obs.cpu().numpy(), out.cpu().numpy())
    del lat
    torch.cuda.empty_cache()
