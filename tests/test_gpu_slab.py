"""Slabs on one GPU (Sec. 4: horizontal slabs in the single-GPU layout, each
reading the boundary rows of its two neighbours): a lattice swept as K slabs
with explicit halo rows equals the same lattice swept whole, bit for bit
(planes and traces), because every random number is keyed by the global
site.  Also the slab initial state, the halo copies, the distributed driver
on one rank, a full-size spot check and argument validation."""
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
    torch.cuda.init()


def whole(L, seed, init=ising.ISING_INIT_RANDOM):
    lat = ising.Lattice(L, "msc4")
    ising.ising_init_lattice(lat, init, seed)
    return lat


def slabs_of(L, parts, seed, init=ising.ISING_INIT_RANDOM):
    out = []
    for row0, rows in parts:
        sl = ising.Slab(L, row0, rows)
        ising.ising_slab_init(sl, init, seed)
        out.append(sl)
    return out


def own_rows_equal(sl, lat):
    a, b = sl.row0, sl.row0 + sl.rows
    return torch.equal(sl.black[1:sl.rows + 1], lat.black[a:b]) and torch.equal(sl.white[1:sl.rows + 1],
                                                                                lat.white[a:b])


PARTS = {
    "one": lambda L: [(0, L)],
    "two": lambda L: ising.slab_partition(L, 2),
    "three": lambda L: ising.slab_partition(L, 3),
    "five": lambda L: ising.slab_partition(L, 5),
    "thin": lambda L: [(0, 1), (1, 2), (3, L - 5), (L - 2, 1), (L - 1, 1)],
}


@pytest.mark.parametrize("L", [64, 192, 256])
@pytest.mark.parametrize("parts", list(PARTS))
def test_slab_init_equals_lattice_init(L, parts):
    lat = whole(L, 7)
    for sl in slabs_of(L, PARTS[parts](L), 7):
        assert own_rows_equal(sl, lat)


@pytest.mark.parametrize("L", [64, 192, 256])
@pytest.mark.parametrize("parts", list(PARTS))
@pytest.mark.parametrize("beta", [0.0, 0.30, 0.4406868, 50.0])
def test_slab_sweep_equals_whole_sweep(L, parts, beta):
    n, seed = 6, 31
    lat = whole(L, seed)
    sls = slabs_of(L, PARTS[parts](L), seed)
    tr_w = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    tr_s = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    ising.ising_sweep(lat, beta, n, seed, 3, tr_w)
    ising.ising_slab_sweep(sls, beta, n, seed, 3, tr_s)
    torch.cuda.synchronize()
    assert torch.equal(tr_s, tr_w)
    for sl in sls:
        assert own_rows_equal(sl, lat)


def test_slab_sweep_equals_the_oracle():
    L, n, seed = 192, 5, 4
    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    want = oracle.run(s, 0.4406868, n, seed, 0)
    sls = slabs_of(L, ising.slab_partition(L, 3), seed)
    tr = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    ising.ising_slab_sweep(sls, 0.4406868, n, seed, 0, tr)
    torch.cuda.synchronize()
    assert np.array_equal(tr.cpu().numpy(), want)
    b, w = oracle.to_planes_msc4(s)
    for sl in sls:
        gb, gw = sl.own_numpy()
        assert np.array_equal(gb, b[sl.row0:sl.row0 + sl.rows]) and np.array_equal(gw, w[sl.row0:sl.row0 + sl.rows])


def test_exchange_fills_halos_with_neighbour_rows():
    L = 256
    parts = PARTS["thin"](L)
    lat = whole(L, 3)
    sls = slabs_of(L, parts, 3)
    for colour in (0, 1):
        ising.ising_slab_exchange(sls, colour)
    torch.cuda.synchronize()
    for sl in sls:
        for plane_s, plane_w in ((sl.black, lat.black), (sl.white, lat.white)):
            assert torch.equal(plane_s[0], plane_w[(sl.row0 - 1) % L])
            assert torch.equal(plane_s[sl.rows + 1], plane_w[(sl.row0 + sl.rows) % L])


def test_half_sweeps_by_hand_equal_slab_sweep():
    """The per-slab entry points, called in the documented order, give the
    same lattice and trace as ising_slab_sweep (and as the single-rank
    distributed driver, whose exchange is the library's copy)."""
    L, n, seed, beta = 128, 4, 8, 0.4406868
    parts = ising.slab_partition(L, 2)
    a = slabs_of(L, parts, seed)
    tr_a = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    ising.ising_slab_sweep(a, beta, n, seed, 0, tr_a)
    b = slabs_of(L, parts, seed)
    tr_b = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    for k in range(n):
        for colour in (0, 1):
            ising.ising_slab_exchange(b, 1 - colour)
            for sl in b:
                ising.ising_slab_half_sweep(sl, beta, colour, seed, k, tr_b[k] if colour == 1 else None)
    one = slabs_of(L, [(0, L)], seed)[0]
    tr_c = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    ising.slab_sweep(one, beta, n, seed, 0, tr_c)
    torch.cuda.synchronize()
    assert torch.equal(tr_a, tr_b) and torch.equal(tr_a, tr_c)
    for x, y in zip(a, b):
        assert torch.equal(x.black, y.black) and torch.equal(x.white, y.white)
    lat = whole(L, seed)
    ising.ising_sweep(lat, beta, n, seed, 0)
    torch.cuda.synchronize()
    assert own_rows_equal(one, lat)


@pytest.mark.parametrize("spare", [0, 8])
def test_overlapped_driver_order_equals_the_serial_order(spare):
    """The driver's overlapped order (first and last own rows, then their
    halo exchange beside the interior rows, views of the slab's storage) and
    its serial order give the whole-lattice sweep, planes and trace, also when
    the half-sweep kernel leaves SMs free."""
    L, n, seed, beta = 256, 5, 12, 0.4406868
    lat = whole(L, seed)
    tr_w = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    ising.ising_sweep(lat, beta, n, seed, 2, tr_w)
    for overlap in (False, True):
        one = slabs_of(L, [(0, L)], seed)[0]
        one.spare_sms = spare
        tr = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
        ising.slab_sweep(one, beta, n, seed, 2, tr, overlap=overlap)
        torch.cuda.synchronize()
        assert torch.equal(tr, tr_w), f"overlap={overlap}"
        assert own_rows_equal(one, lat), f"overlap={overlap}"


def test_slab_views_are_bounded():
    sl = slabs_of(128, [(0, 128)], 1)[0]
    for first, count in ((-1, 2), (0, 0), (120, 9)):
        with pytest.raises(ValueError):
            sl.view(first, count)
    v = sl.view(5, 7)
    assert (v.row0, v.rows) == (5, 7) and v.black.data_ptr() == sl.black[5].data_ptr()


def test_full_size_four_slabs_match_whole_lattice():
    """65536^2 as four slabs of 16384 rows, 2 sweeps, cold start and random
    start: planes compared on the device, traces exactly."""
    L, n = 65536, 2
    for init, seed in ((ising.ISING_INIT_UP, 1), (ising.ISING_INIT_RANDOM, 1234)):
        lat = whole(L, seed, init)
        tr_w = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
        ising.ising_sweep(lat, 0.4406868, n, seed, 0, tr_w)
        sls = slabs_of(L, ising.slab_partition(L, 4), seed, init)
        tr_s = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
        ising.ising_slab_sweep(sls, 0.4406868, n, seed, 0, tr_s)
        torch.cuda.synchronize()
        assert torch.equal(tr_s, tr_w)
        for sl in sls:
            assert own_rows_equal(sl, lat)
        del lat, sls
        torch.cuda.empty_cache()


def test_bad_slabs_are_rejected():
    L = 128
    good = slabs_of(L, ising.slab_partition(L, 2), 1)
    st = [x.struct() for x in good]

    def expect_einval(fn):
        with pytest.raises(ising.IsingError) as e:
            fn()
        assert e.value.status == ising.ISING_EINVAL

    bad = ising.ising_slab_t.from_buffer_copy(st[0])
    bad.layout = ising.ISING_INT8
    expect_einval(lambda: ising.ising_slab_half_sweep(bad, 0.4, 0, 1, 0))
    bad = ising.ising_slab_t.from_buffer_copy(st[0])
    bad.rows = 0
    expect_einval(lambda: ising.ising_slab_half_sweep(bad, 0.4, 0, 1, 0))
    bad = ising.ising_slab_t.from_buffer_copy(st[1])
    bad.row0 = 100  # 100 + 64 > 128
    expect_einval(lambda: ising.ising_slab_half_sweep(bad, 0.4, 0, 1, 0))
    bad = ising.ising_slab_t.from_buffer_copy(st[0])
    bad.row_stride_bytes = 1 << 30  # planes far larger than their allocations
    expect_einval(lambda: ising.ising_slab_half_sweep(bad, 0.4, 0, 1, 0))
    # a gap between slabs, a missing last slab, a wrong order, a shared plane
    expect_einval(lambda: ising.ising_slab_exchange([st[0]], 0))
    expect_einval(lambda: ising.ising_slab_exchange([st[1], st[0]], 0))
    dup = ising.ising_slab_t.from_buffer_copy(st[1])
    dup.white = st[0].white
    expect_einval(lambda: ising.ising_slab_exchange([st[0], dup], 0))
    expect_einval(lambda: ising.ising_slab_exchange(st * 33, 0))  # more than 64 slabs
    expect_einval(lambda: ising.ising_slab_half_sweep(st[0], -1.0, 0, 1, 0))
    obs = torch.zeros(2, dtype=torch.int64, device="cuda")
    expect_einval(lambda: ising.ising_slab_half_sweep(st[0], 0.4, 0, 1, 0, obs))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for spare in (-1, sms):  # no SM left, or a negative count
        bad = ising.ising_slab_t.from_buffer_copy(st[0])
        bad.spare_sms = spare
        expect_einval(lambda: ising.ising_slab_half_sweep(bad, 0.4, 0, 1, 0))
    # nothing above touched the planes
    fresh = slabs_of(L, ising.slab_partition(L, 2), 1)
    torch.cuda.synchronize()
    for x, y in zip(good, fresh):
        assert torch.equal(x.black, y.black) and torch.equal(x.white, y.white)
