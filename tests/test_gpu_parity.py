"""Parity of the CUDA path with the oracle: bit-exact lattices and traces.

Every GPU result is decoded into a full L x L lattice by the oracle's own
decoder of the documented plane layouts and compared element by element with
the oracle's lattice for the same seed, beta, sweep offset and start state.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1906_06297_gb300 as ising
from oracle import exact
from tests import inputs

pytestmark = pytest.mark.gpu

BETAS = [0.0, 0.30, 0.4406868, 0.60, 50.0]
MODES = {"random": ising.ISING_INIT_RANDOM, "up": ising.ISING_INIT_UP, "down": ising.ISING_INIT_DOWN}


@pytest.fixture(scope="module", autouse=True)
def built():
    ising.build()
    oracle.build()
    torch.cuda.init()


def full_from_gpu(lat: ising.Lattice) -> np.ndarray:
    b, w = lat.planes_numpy()
    if lat.layout == ising.ISING_MSC4:
        return oracle.from_planes_msc4(lat.L, b, w)
    return oracle.from_planes_int8(lat.L, b, w)


def load_full(lat: ising.Lattice, s: np.ndarray):
    if lat.layout == ising.ISING_MSC4:
        b, w = oracle.to_planes_msc4(s)
    else:
        b, w = oracle.to_planes_int8(s)
    lat.load_numpy(b, w)


def gpu_run(lat, beta, n, seed, off=0, trace=True):
    tr = torch.zeros((max(n, 1), 2), dtype=torch.int64, device="cuda") if trace else None
    ising.ising_sweep(lat, beta, n, seed, off, tr)
    torch.cuda.synchronize()
    return tr[:n].cpu().numpy() if trace else None


# ---------------------------------------------------------------------------
# initial state
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("layout,L", [("int8", 2), ("int8", 6), ("int8", 10), ("int8", 130), ("int8", 256),
                                      ("msc4", 64), ("msc4", 192), ("msc4", 256), ("msc4", 4224)])
@pytest.mark.parametrize("mode", ["random", "up", "down"])
def test_init_matches_oracle(layout, L, mode):
    lat = ising.Lattice(L, layout)
    ising.ising_init_lattice(lat, MODES[mode], 1234)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(full_from_gpu(lat), oracle.init(L, MODES[mode], 1234))


# ---------------------------------------------------------------------------
# sweeps from the library's own initial state
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("layout,L", [("int8", 2), ("int8", 6), ("int8", 18), ("int8", 130), ("int8", 256),
                                      ("msc4", 64), ("msc4", 128), ("msc4", 192), ("msc4", 640),
                                      ("msc4", 2112)])
@pytest.mark.parametrize("beta", BETAS)
def test_sweeps_bit_exact(layout, L, beta):
    n, seed = 12, 77
    lat = ising.Lattice(L, layout)
    ising.ising_init_lattice(lat, ising.ISING_INIT_RANDOM, seed)
    tr = gpu_run(lat, beta, n, seed)
    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    tr_o = oracle.run(s, beta, n, seed)
    np.testing.assert_array_equal(full_from_gpu(lat), s)
    np.testing.assert_array_equal(tr, tr_o)


@pytest.mark.parametrize("layout", ["int8", "msc4"])
def test_reference_workload_1000_sweeps(layout):
    """L = 256, beta = 0.4406868, random start from seed 1234, 1000 sweeps:
    final lattice and the per-sweep {M, bond sum} trace bit-exact."""
    L, beta, seed, n = 256, 0.4406868, 1234, 1000
    lat = ising.Lattice(L, layout)
    ising.ising_init_lattice(lat, ising.ISING_INIT_RANDOM, seed)
    tr = gpu_run(lat, beta, n, seed)
    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    tr_o = oracle.run(s, beta, n, seed)
    np.testing.assert_array_equal(full_from_gpu(lat), s)
    np.testing.assert_array_equal(tr, tr_o)


@pytest.mark.parametrize("beta", [exact.BETA_C, 0.6])
def test_several_tiles_with_ragged_tail(beta):
    """L = 4224: 132 words per plane row = two full 64-word chunks and a
    4-word tail; 4224 rows split over many warps."""
    L, n, seed = 4224, 3, 5
    lat = ising.Lattice(L, "msc4")
    ising.ising_init_lattice(lat, ising.ISING_INIT_RANDOM, seed)
    tr = gpu_run(lat, beta, n, seed, off=40)
    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    tr_o = oracle.run(s, beta, n, seed, off=40)
    np.testing.assert_array_equal(full_from_gpu(lat), s)
    np.testing.assert_array_equal(tr, tr_o)


# ---------------------------------------------------------------------------
# arbitrary start states, padded strides, half-sweeps
# ---------------------------------------------------------------------------
STARTS = {
    "neel": lambda L: inputs.neel(L),
    "random": lambda L: inputs.random_lattice(L, 3),
    "biased": lambda L: inputs.random_lattice(L, 4, p_up=0.9),
    "domains": lambda L: inputs.domains(L, 5),
}


@pytest.mark.parametrize("layout,L,stride", [("int8", 64, None), ("int8", 66, 40), ("msc4", 128, None),
                                             ("msc4", 192, 64), ("msc4", 256, 96)])
@pytest.mark.parametrize("start", sorted(STARTS))
@pytest.mark.parametrize("beta", [0.3, 0.4406868, 50.0])
def test_half_sweeps_from_arbitrary_states(layout, L, stride, start, beta):
    s = STARTS[start](L)
    lat = ising.Lattice(L, layout, row_stride_bytes=stride)
    load_full(lat, s)
    seed, t = 99, 7
    obs = torch.zeros(2, dtype=torch.int64, device="cuda")
    ising.ising_half_sweep(lat, beta, 0, seed, t)
    ising.ising_half_sweep(lat, beta, 1, seed, t, obs)
    torch.cuda.synchronize()
    oracle.half_sweep(s, beta, 0, seed, t)
    oracle.half_sweep(s, beta, 1, seed, t)
    np.testing.assert_array_equal(full_from_gpu(lat), s)
    np.testing.assert_array_equal(obs.cpu().numpy(), oracle.observables(s))


def test_padding_is_not_touched():
    L, stride = 128, 64  # 16 bytes of data per row, 48 of padding
    lat = ising.Lattice(L, "msc4", row_stride_bytes=stride)
    lat.black.fill_(0xAB)
    lat.white.fill_(0xCD)
    ising.ising_init_lattice(lat, ising.ISING_INIT_RANDOM, 1)
    ising.ising_sweep(lat, 0.44, 5, 1, 0, None)
    torch.cuda.synchronize()
    assert bool((lat.black[:, lat.row_bytes:] == 0xAB).all())
    assert bool((lat.white[:, lat.row_bytes:] == 0xCD).all())


# ---------------------------------------------------------------------------
# invariants of the API
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("layout", ["int8", "msc4"])
def test_resume_equals_single_call(layout):
    L, beta, seed, a, b = 128, 0.4406868, 11, 9, 14
    one = ising.Lattice(L, layout)
    two = ising.Lattice(L, layout)
    for lat in (one, two):
        ising.ising_init_lattice(lat, ising.ISING_INIT_RANDOM, seed)
    t1 = gpu_run(one, beta, a + b, seed)
    ta = gpu_run(two, beta, a, seed)
    tb = gpu_run(two, beta, b, seed, off=a)
    np.testing.assert_array_equal(full_from_gpu(one), full_from_gpu(two))
    np.testing.assert_array_equal(t1, np.vstack([ta, tb]))


def test_int8_and_msc4_give_the_same_lattice():
    L, beta, seed, n = 256, 0.35, 21, 30
    a = ising.Lattice(L, "int8")
    b = ising.Lattice(L, "msc4")
    for lat in (a, b):
        ising.ising_init_lattice(lat, ising.ISING_INIT_RANDOM, seed)
    ta = gpu_run(a, beta, n, seed)
    tb = gpu_run(b, beta, n, seed)
    np.testing.assert_array_equal(full_from_gpu(a), full_from_gpu(b))
    np.testing.assert_array_equal(ta, tb)
    # and through the library's own conversion
    c = ising.Lattice(L, "int8")
    ising.ising_unpack(b, c)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(full_from_gpu(c), full_from_gpu(a))


@pytest.mark.parametrize("layout,L", [("int8", 6), ("int8", 130), ("msc4", 64), ("msc4", 2112)])
@pytest.mark.parametrize("start", sorted(STARTS))
def test_observables_kernel(layout, L, start):
    s = STARTS[start](L)
    lat = ising.Lattice(L, layout)
    load_full(lat, s)
    out = torch.full((2,), 7, dtype=torch.int64, device="cuda")
    ising.ising_observables(lat, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.observables(s))


@pytest.mark.parametrize("L", [64, 192, 2112])
def test_pack_unpack_against_oracle_encoding(L):
    s = inputs.random_lattice(L, 8)
    src = ising.Lattice(L, "int8")
    load_full(src, s)
    dst = ising.Lattice(L, "msc4")
    ising.ising_pack(src, dst)
    back = ising.Lattice(L, "int8", row_stride_bytes=L // 2 + 3)
    ising.ising_unpack(dst, back)
    torch.cuda.synchronize()
    ob, ow = oracle.to_planes_msc4(s)
    gb, gw = dst.planes_numpy()
    np.testing.assert_array_equal(gb, ob)
    np.testing.assert_array_equal(gw, ow)
    np.testing.assert_array_equal(full_from_gpu(back), s)


@pytest.mark.parametrize("n_blocks", [5000, 5003, 7, 1, 8 * 40000 + 5])
def test_rng_probe_counts_match_oracle(n_blocks):
    """The Philox-only probe (groups of 8 blocks sharing counter words 1..3,
    a ragged last group) counts exactly the oracle's draws below T3."""
    seed, t, colour = 321, 3, 1
    T3 = int(oracle.thresholds(0.4406868)[3])
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ising.ising_rng_probe(n_blocks, seed, t, colour, T3, cnt)
    torch.cuda.synchronize()
    expect = sum(int(oracle.draw(seed, site, t, colour) < T3) for site in range(4 * n_blocks))
    assert int(cnt.item()) == expect


def test_mulwide_probe_launches_a_full_grid():
    """The wide-multiply probe runs and reports the multiplies of one launch:
    a whole number of 256-thread blocks per SM, 16 chains, `iters` each."""
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for form in (0, 1):
        n = ising.ising_mulwide_probe(form, 64, sink)
        torch.cuda.synchronize()
        assert n % (sms * 256 * 16 * 64) == 0 and n >= sms * 256 * 16 * 64
    for form, iters in ((0, 0), (2, 64)):
        with pytest.raises(ising.IsingError):
            ising.ising_mulwide_probe(form, iters, sink)


@pytest.mark.parametrize("layout,L,stride", [("msc4", 256, None), ("int8", 256, None), ("int8", 130, 80)])
def test_host_buffer_entry_point(layout, L, stride):
    """Several sweeps through host memory (whole planes copied in and out
    around ising_sweep): planes and trace equal the oracle, in both layouts
    and with padded device rows."""
    beta, seed, n = 0.4406868, 4, 7
    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    if layout == "msc4":
        b, w = oracle.to_planes_msc4(s)
    else:
        b, w = oracle.to_planes_int8(s)
    hb = torch.from_numpy(b.view(np.uint8).copy()).pin_memory()
    hw = torch.from_numpy(w.view(np.uint8).copy()).pin_memory()
    dev = ising.Lattice(L, layout, row_stride_bytes=stride)
    tr_dev = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    tr_host = torch.zeros((n, 2), dtype=torch.int64).pin_memory()
    ising.ising_sweep_host(dev, hb.data_ptr(), hw.data_ptr(), beta, n, seed, 0, tr_dev, tr_host.data_ptr())
    torch.cuda.synchronize()
    tr_o = oracle.run(s, beta, n, seed)
    if layout == "msc4":
        got = oracle.from_planes_msc4(L, hb.numpy().view(np.uint64).reshape(L, -1),
                                      hw.numpy().view(np.uint64).reshape(L, -1))
    else:
        got = oracle.from_planes_int8(L, hb.numpy().view(np.int8).reshape(L, -1),
                                      hw.numpy().view(np.int8).reshape(L, -1))
    np.testing.assert_array_equal(got, s)
    np.testing.assert_array_equal(tr_host.numpy(), tr_o)


@pytest.mark.parametrize("L,beta,stride", [(64, 0.4406868, None), (192, 0.3, None), (256, 0.0, None),
                                           (640, 50.0, None), (2112, 0.4406868, 2112 // 4 + 64),
                                           (4224, 0.6, None)])
def test_host_buffer_single_sweep_in_bands(L, beta, stride):
    """One sweep through host memory runs in row bands that overlap the copies
    (8 or 16 bands, padded device rows): each step of 3 sweeps equals
    the oracle bit for bit, planes and trace, and the host planes feed the
    next call."""
    seed, n = 9, 3
    init = ising.Lattice(L, "msc4")
    ising.ising_init_lattice(init, ising.ISING_INIT_RANDOM, seed)
    torch.cuda.synchronize()
    hb = init.black.cpu().pin_memory()
    hw = init.white.cpu().pin_memory()
    dev = ising.Lattice(L, "msc4", row_stride_bytes=stride)
    tr_dev = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    tr_host = torch.zeros((1, 2), dtype=torch.int64).pin_memory()
    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    for k in range(n):
        ising.ising_sweep_host(dev, hb.data_ptr(), hw.data_ptr(), beta, 1, seed, k, tr_dev, tr_host.data_ptr())
        torch.cuda.synchronize()
        tr_o = oracle.run(s, beta, 1, seed, off=k)
        got = oracle.from_planes_msc4(L, hb.numpy().view(np.uint64), hw.numpy().view(np.uint64))
        np.testing.assert_array_equal(got, s)
        np.testing.assert_array_equal(tr_host.numpy(), tr_o)


def test_host_buffer_sweep_in_many_ragged_bands_equals_device_sweep():
    """At 36864^2 (two 340 MB planes) the host path uses 20 bands of 1844
    rows, the last one ragged: two calls equal two sweeps of the device path
    (itself bit-exact against the oracle above), planes and trace."""
    L, beta, seed = 36864, 0.4406868, 17
    ref = ising.Lattice(L, "msc4")
    ising.ising_init_lattice(ref, ising.ISING_INIT_RANDOM, seed)
    torch.cuda.synchronize()
    hb = ref.black.cpu().pin_memory()
    hw = ref.white.cpu().pin_memory()
    dev = ising.Lattice(L, "msc4")
    tr_dev = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    tr_host = torch.zeros((1, 2), dtype=torch.int64).pin_memory()
    tr_ref = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    for k in range(2):
        ising.ising_sweep_host(dev, hb.data_ptr(), hw.data_ptr(), beta, 1, seed, k, tr_dev, tr_host.data_ptr())
        ising.ising_sweep(ref, beta, 1, seed, k, tr_ref)
        torch.cuda.synchronize()
        assert torch.equal(hb, ref.black.cpu()) and torch.equal(hw, ref.white.cpu())
        assert torch.equal(tr_host, tr_ref.cpu())
    del ref, dev
    torch.cuda.empty_cache()


def pinned_bits(b, w):
    return torch.from_numpy(b.copy()).pin_memory(), torch.from_numpy(w.copy()).pin_memory()


@pytest.mark.parametrize("L,stride", [(64, None), (192, None), (256, None), (320, 320 // 4 + 32),
                                      (1024, 1024 // 4 + 16), (2112, None)])
def test_bit_planes_convert_both_ways_like_the_oracle(L, stride):
    """MSC4 device planes -> bit planes equals the oracle's encoding of the
    same lattice, and the oracle's bit planes -> MSC4 give back the lattice
    (padded device rows included)."""
    seed = 21
    lat = ising.Lattice(L, "msc4", row_stride_bytes=stride)
    ising.ising_init_lattice(lat, ising.ISING_INIT_RANDOM, seed)
    nb = ising.ising_bits_bytes(L)
    bits = torch.zeros(2 * nb, dtype=torch.uint8, device="cuda")
    ising.ising_msc4_to_bits(lat, bits[:nb], bits[nb:])
    torch.cuda.synchronize()
    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    eb, ew = oracle.to_planes_bits(s)
    got = bits.cpu().numpy()
    np.testing.assert_array_equal(got[:nb].reshape(L, L // 16), eb)
    np.testing.assert_array_equal(got[nb:].reshape(L, L // 16), ew)
    back = ising.Lattice(L, "msc4", row_stride_bytes=stride)
    up = torch.from_numpy(np.concatenate([eb.ravel(), ew.ravel()])).cuda()
    ising.ising_bits_to_msc4(up[:nb], up[nb:], back)
    torch.cuda.synchronize()
    words = (back.row_stride_bytes // 8)
    pb = back.black.cpu().numpy().view(np.uint64).reshape(L, words)[:, :L // 32]
    pw = back.white.cpu().numpy().view(np.uint64).reshape(L, words)[:, :L // 32]
    np.testing.assert_array_equal(oracle.from_planes_msc4(L, pb, pw), s)


@pytest.mark.parametrize("L,beta,stride", [(64, 0.4406868, None), (256, 0.0, None), (640, 50.0, None),
                                           (2112, 0.4406868, 2112 // 4 + 64), (4224, 0.6, None)])
def test_host_bits_single_sweep_in_bands(L, beta, stride):
    """One sweep of a bit-packed host lattice (bands converted on the device
    after their copy in and before their copy out): each of 3 calls equals
    the oracle bit for bit, planes and trace."""
    seed, n = 9, 3
    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    hb, hw = pinned_bits(*oracle.to_planes_bits(s))
    dev = ising.Lattice(L, "msc4", row_stride_bytes=stride)
    nb = ising.ising_bits_bytes(L)
    stage = torch.empty(2 * nb, dtype=torch.uint8, device="cuda")
    tr_dev = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    tr_host = torch.zeros((1, 2), dtype=torch.int64).pin_memory()
    for k in range(n):
        ising.ising_sweep_host_bits(dev, hb, hw, stage, beta, 1, seed, k, tr_dev, tr_host.data_ptr())
        torch.cuda.synchronize()
        tr_o = oracle.run(s, beta, 1, seed, off=k)
        np.testing.assert_array_equal(oracle.from_planes_bits(L, hb.numpy(), hw.numpy()), s)
        np.testing.assert_array_equal(tr_host.numpy(), tr_o)


def test_host_bits_several_sweeps_per_call():
    """n_sweeps != 1 converts whole planes around ising_sweep: 2 calls of 4
    sweeps equal the oracle's 8, planes and trace."""
    L, beta, seed = 256, 0.4406868, 5
    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    hb, hw = pinned_bits(*oracle.to_planes_bits(s))
    dev = ising.Lattice(L, "msc4")
    nb = ising.ising_bits_bytes(L)
    stage = torch.empty(2 * nb, dtype=torch.uint8, device="cuda")
    tr_dev = torch.zeros((4, 2), dtype=torch.int64, device="cuda")
    tr_host = torch.zeros((4, 2), dtype=torch.int64).pin_memory()
    for k in range(2):
        ising.ising_sweep_host_bits(dev, hb, hw, stage, beta, 4, seed, 4 * k, tr_dev, tr_host.data_ptr())
        torch.cuda.synchronize()
        tr_o = oracle.run(s, beta, 4, seed, off=4 * k)
        np.testing.assert_array_equal(oracle.from_planes_bits(L, hb.numpy(), hw.numpy()), s)
        np.testing.assert_array_equal(tr_host.numpy(), tr_o)


def test_host_bits_sweep_in_many_ragged_bands_equals_device_sweep():
    """At 69632^2 (bit planes of 303 MB) the bit path uses 18 bands of 3869
    rows, the last one ragged: two calls equal two sweeps of the device path,
    converted to bits on the device (conversion checked above), and the trace."""
    L, beta, seed = 69632, 0.4406868, 23
    ref = ising.Lattice(L, "msc4")
    ising.ising_init_lattice(ref, ising.ISING_INIT_RANDOM, seed)
    nb = ising.ising_bits_bytes(L)
    refbits = torch.empty(2 * nb, dtype=torch.uint8, device="cuda")
    ising.ising_msc4_to_bits(ref, refbits[:nb], refbits[nb:])
    torch.cuda.synchronize()
    hb = refbits[:nb].cpu().pin_memory()
    hw = refbits[nb:].cpu().pin_memory()
    dev = ising.Lattice(L, "msc4")
    stage = torch.empty(2 * nb, dtype=torch.uint8, device="cuda")
    tr_dev = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    tr_host = torch.zeros((1, 2), dtype=torch.int64).pin_memory()
    tr_ref = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    for k in range(2):
        ising.ising_sweep_host_bits(dev, hb, hw, stage, beta, 1, seed, k, tr_dev, tr_host.data_ptr())
        ising.ising_sweep(ref, beta, 1, seed, k, tr_ref)
        ising.ising_msc4_to_bits(ref, refbits[:nb], refbits[nb:])
        torch.cuda.synchronize()
        assert torch.equal(hb, refbits[:nb].cpu()) and torch.equal(hw, refbits[nb:].cpu())
        assert torch.equal(tr_host, tr_ref.cpu())
    del ref, dev, refbits, stage
    torch.cuda.empty_cache()


def test_host_sweeps_alternating_between_lattices_of_one_size():
    """Calls that alternate between lattices of the same size (other host
    planes, stage, device lattice and seed, the same band schedule, so the
    replayed schedule of one call is updated in place for the next) must each
    act on their own buffers; switching host format changes the schedule and
    re-instantiates it.  Both formats, 3 rounds, against the oracle."""
    L, beta = 2112, 0.4406868
    runs = []
    # consecutive calls of one format (same schedule, other buffers), then the other format
    for fmt, seed in (("bits", 41), ("bits", 43), ("msc4", 42), ("msc4", 44)):
        s = oracle.init(L, oracle.MODE_RANDOM, seed)
        if fmt == "bits":
            hb, hw = pinned_bits(*oracle.to_planes_bits(s))
            nb = ising.ising_bits_bytes(L)
            extra = torch.empty(2 * nb, dtype=torch.uint8, device="cuda")
        else:
            b, w = oracle.to_planes_msc4(s)
            hb = torch.from_numpy(b.view(np.uint8).copy()).pin_memory()
            hw = torch.from_numpy(w.view(np.uint8).copy()).pin_memory()
            extra = None
        dev = ising.Lattice(L, "msc4")
        tr_dev = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
        tr_host = torch.zeros((1, 2), dtype=torch.int64).pin_memory()
        runs.append(dict(fmt=fmt, seed=seed, s=s, hb=hb, hw=hw, stage=extra, dev=dev, tr_dev=tr_dev,
                         tr_host=tr_host))
    for k in range(3):
        for r in runs:
            if r["fmt"] == "bits":
                ising.ising_sweep_host_bits(r["dev"], r["hb"], r["hw"], r["stage"], beta, 1, r["seed"], k,
                                            r["tr_dev"], r["tr_host"].data_ptr())
            else:
                ising.ising_sweep_host(r["dev"], r["hb"].data_ptr(), r["hw"].data_ptr(), beta, 1, r["seed"], k,
                                       r["tr_dev"], r["tr_host"].data_ptr())
        torch.cuda.synchronize()
        for r in runs:
            tr_o = oracle.run(r["s"], beta, 1, r["seed"], off=k)
            if r["fmt"] == "bits":
                got = oracle.from_planes_bits(L, r["hb"].numpy(), r["hw"].numpy())
            else:
                got = oracle.from_planes_msc4(L, r["hb"].numpy().view(np.uint64).reshape(L, -1),
                                              r["hw"].numpy().view(np.uint64).reshape(L, -1))
            np.testing.assert_array_equal(got, r["s"])
            np.testing.assert_array_equal(r["tr_host"].numpy(), tr_o)


@pytest.mark.parametrize("fmt", ["msc4", "bits"])
def test_host_sweeps_on_pageable_host_planes(fmt):
    """Plain numpy (pageable, not pinned) host planes through the banded
    one-sweep path, two calls in a row: the schedule's copies from and to
    pageable memory (captured and replayed, or launched directly where the
    capture is refused) give the oracle's lattice and trace bit for bit."""
    L, beta, seed = 2112, 0.4406868, 47
    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    if fmt == "bits":
        hb, hw = (np.ascontiguousarray(x) for x in oracle.to_planes_bits(s))
        nb = ising.ising_bits_bytes(L)
        stage = torch.empty(2 * nb, dtype=torch.uint8, device="cuda")
    else:
        hb, hw = (np.ascontiguousarray(x).copy() for x in oracle.to_planes_msc4(s))
    dev = ising.Lattice(L, "msc4")
    tr_dev = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    tr_host = np.zeros((1, 2), dtype=np.int64)
    for k in range(2):
        if fmt == "bits":
            ising.ising_sweep_host_bits(dev, hb, hw, stage, beta, 1, seed, k, tr_dev, tr_host)
        else:
            ising.ising_sweep_host(dev, hb, hw, beta, 1, seed, k, tr_dev, tr_host)
        torch.cuda.synchronize()
        tr_o = oracle.run(s, beta, 1, seed, off=k)
        if fmt == "bits":
            got = oracle.from_planes_bits(L, hb, hw)
        else:
            got = oracle.from_planes_msc4(L, hb.view(np.uint64).reshape(L, -1), hw.view(np.uint64).reshape(L, -1))
        np.testing.assert_array_equal(got, s)
        np.testing.assert_array_equal(tr_host, tr_o)


def test_host_entry_points_with_zero_sweeps_return_the_lattice_unchanged():
    """n_sweeps = 0: the lattice goes in and comes back out (through the MSC4
    device lattice) unchanged, in both host formats; trace buffers untouched."""
    L, seed = 192, 31
    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    b, w = oracle.to_planes_msc4(s)
    hb = torch.from_numpy(b.view(np.uint8).copy()).pin_memory()
    hw = torch.from_numpy(w.view(np.uint8).copy()).pin_memory()
    dev = ising.Lattice(L, "msc4", row_stride_bytes=L // 4 + 16)
    tr_dev = torch.full((1, 2), 7, dtype=torch.int64, device="cuda")
    tr_host = torch.full((1, 2), 7, dtype=torch.int64).pin_memory()
    ising.ising_sweep_host(dev, hb.data_ptr(), hw.data_ptr(), 0.44, 0, seed, 0, tr_dev, tr_host.data_ptr())
    bb, bw = pinned_bits(*oracle.to_planes_bits(s))
    nb = ising.ising_bits_bytes(L)
    stage = torch.empty(2 * nb, dtype=torch.uint8, device="cuda")
    ising.ising_sweep_host_bits(dev, bb, bw, stage, 0.44, 0, seed, 0, tr_dev, tr_host.data_ptr())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(oracle.from_planes_msc4(L, hb.numpy().view(np.uint64).reshape(L, -1),
                                                          hw.numpy().view(np.uint64).reshape(L, -1)), s)
    np.testing.assert_array_equal(oracle.from_planes_bits(L, bb.numpy(), bw.numpy()), s)
    assert int(tr_host[0, 0]) == 7 and int(tr_dev[0, 0].item()) == 7


def test_bit_format_arguments_are_checked_before_any_work():
    """Wrong layout, unaligned host planes, a missing stage or trace staging
    buffer and a negative beta are rejected with ISING_EINVAL, and nothing is
    written."""
    L = 128
    nb = ising.ising_bits_bytes(L)
    dev = ising.Lattice(L, "msc4")
    stage = torch.zeros(2 * nb, dtype=torch.uint8, device="cuda")
    hb = torch.zeros(nb + 4, dtype=torch.uint8).pin_memory()
    hw = torch.zeros(nb + 4, dtype=torch.uint8).pin_memory()
    i8 = ising.Lattice(L, "int8")
    bad = [
        lambda: ising.ising_sweep_host_bits(i8, hb, hw, stage, 0.4, 1, 1),
        lambda: ising.ising_sweep_host_bits(dev, hb.data_ptr() + 2, hw, stage, 0.4, 1, 1),
        lambda: ising.ising_sweep_host_bits(dev, hb, hw, None, 0.4, 1, 1),
        lambda: ising.ising_sweep_host_bits(dev, hb, hw, stage, 0.4, 1, 1, 0, None, hb.data_ptr()),
        lambda: ising.ising_sweep_host_bits(dev, hb, hw, stage, -0.1, 1, 1),
        lambda: ising.ising_msc4_to_bits(i8, stage[:nb], stage[nb:]),
    ]
    for call in bad:
        with pytest.raises(ising.IsingError) as e:
            call()
        assert e.value.status == ising.ISING_EINVAL
    torch.cuda.synchronize()
    assert int(stage.count_nonzero()) == 0


def test_undersized_buffers_are_rejected():
    """The library checks each plane against the extent of its CUDA allocation
    (the caching allocator's segment, so only overruns past the segment can be
    seen: the claims below are far larger than any segment)."""
    lat = ising.Lattice(64, "msc4")
    big = ising.ising_lattice_t(lat.black.data_ptr(), lat.white.data_ptr(), 1 << 16, ising.ISING_MSC4, 0, 1 << 14)
    with pytest.raises(ising.IsingError) as e:
        ising.ising_sweep(big, 0.4, 1, 1, 0, None)
    assert e.value.status == ising.ISING_EINVAL
    tr = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(ising.IsingError):
        ising.ising_sweep(lat, 0.4, 1 << 24, 1, 0, tr)  # trace for 2^24 sweeps
