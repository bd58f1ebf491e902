"""The C ABI library builds, loads, exports every symbol its header declares,
and rejects bad arguments before touching a GPU (runs without one)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1906_06297_gb300 as ising
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ising.h")


@pytest.fixture(scope="module")
def lib():
    ising.build()
    return ctypes.CDLL(ising.library_path())


def declared_functions():
    text = open(HEADER).read()
    return re.findall(r"ISING_API\s+[\w\s\*]+?\b(ising_\w+)\s*\(", text)


def test_header_declares_the_entry_points():
    names = set(declared_functions())
    for required in ("ising_init_lattice", "ising_sweep", "ising_observables", "ising_thresholds",
                     "ising_lattice_bytes", "ising_half_sweep", "ising_pack", "ising_unpack", "ising_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_lattice_bytes():
    assert ising.ising_lattice_bytes(256, ising.ISING_INT8) == (128, 128 * 256)
    assert ising.ising_lattice_bytes(65536, ising.ISING_MSC4) == (65536 // 4, 65536 * 65536 // 4)
    for L, layout in [(0, 0), (-2, 0), (3, 0), (96, 1), (256, 7)]:
        with pytest.raises(ising.IsingError) as e:
            ising.ising_lattice_bytes(L, layout)
        assert e.value.status == ising.ISING_EINVAL


@pytest.mark.parametrize("beta", [0.0, 1e-3, 0.3, 0.4406868, 0.6, 50.0])
def test_library_table_equals_oracle_table(beta):
    """Both sides build T[a] independently from exp(); same machine, same libm."""
    assert ising.ising_thresholds(beta) == [int(x) for x in oracle.thresholds(beta)]


def test_thresholds_reject_bad_beta():
    for beta in (-1e-9, float("nan"), float("inf"), -float("inf")):
        with pytest.raises(ising.IsingError) as e:
            ising.ising_thresholds(beta)
        assert e.value.status == ising.ISING_EINVAL


def test_strerror():
    assert ising.ising_strerror(0) == "ok"
    assert ising.ising_strerror(ising.ISING_EINVAL) == "invalid argument"
    assert ising.ising_strerror(12345) == "unknown status"


def _bad(**kw):
    f = dict(black=None, white=None, L=64, layout=ising.ISING_MSC4, reserved=0, row_stride_bytes=16)
    f.update(kw)
    return ising.ising_lattice_t(f["black"], f["white"], f["L"], f["layout"], f["reserved"], f["row_stride_bytes"])


@pytest.mark.parametrize("kw", [
    dict(),                                   # NULL planes
    dict(L=63),                               # odd
    dict(L=96),                               # MSC4 needs L % 64 == 0
    dict(reserved=1),
    dict(row_stride_bytes=8),                 # below the row size
    dict(black=0x1000, white=0x1000),         # aliasing planes
    dict(black=0x1008, white=0x2000),         # misaligned MSC4 plane
    dict(layout=3),
])
def test_invalid_lattices_are_rejected_without_a_launch(kw):
    lat = _bad(**kw)
    with pytest.raises(ising.IsingError) as e:
        ising.ising_sweep(lat, 0.4, 1, 1, 0, None, stream=0)
    assert e.value.status == ising.ISING_EINVAL
    with pytest.raises(ising.IsingError):
        ising.ising_init_lattice(lat, 0, 1, stream=0)


def test_host_memory_is_not_accepted_as_a_device_plane():
    buf = np.zeros((64, 16), dtype=np.uint8)
    buf2 = np.zeros((64, 16), dtype=np.uint8)
    lat = _bad(black=buf.ctypes.data, white=buf2.ctypes.data)
    with pytest.raises(ising.IsingError) as e:
        ising.ising_sweep(lat, 0.4, 1, 1, 0, None, stream=0)
    assert e.value.status == ising.ISING_EINVAL


def test_sweep_rejects_bad_counts_and_colours():
    lat = _bad()
    with pytest.raises(ising.IsingError):
        ising.ising_half_sweep(lat, 0.4, 2, 1, 0, None, stream=0)
    with pytest.raises(ising.IsingError):
        ising.ising_rng_probe(10, 1, 0, 5, 0, None, stream=0)


def test_batch_refuses_betas_whose_thresholds_reach_two_to_the_32():
    """exp(-4 beta) rounds to 1 in FP64 below beta ~ 1.4e-17; the batched
    decision keeps T3, T4 as 32-bit words, so such a beta is refused
    (Sec. 2 Metropolis rule: p = 1 would need the entry 2^32)."""
    for beta in ([1e-18, 0.4], [1e-17, 0.3], [0.2, 0.3]):
        if beta[0] < 1.4e-17:
            assert oracle.thresholds(beta[0])[3] == 2 ** 32
            with pytest.raises(ising.IsingError) as e:
                ising.ising_batch_bytes([32, 32], 2, beta)
            assert e.value.status == ising.ISING_EINVAL
        else:
            assert ising.ising_batch_bytes([32, 32], 2, beta) > 0
    # just above the cut-off the table is ordinary: T3 < 2^32
    assert oracle.thresholds(2e-16)[3] < 2 ** 32
    assert ising.ising_batch_bytes([32, 32], 2, [2e-16, 0.3]) > 0
