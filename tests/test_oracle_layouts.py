"""The oracle's storage layouts against their definitions, decoded here with
numpy alone: one int8 per spin, MSC4 (four bits per spin, Sec. 3.3) and the
bit-packed I/O format (one bit per spin, the MSC4 order)."""
import numpy as np
import pytest

import oracle
import paper_1906_06297_gb300 as ising


def random_lattice(L, seed):
    rng = np.random.default_rng(seed)
    return np.where(rng.random((L, L)) < 0.5, 1, -1).astype(np.int8)


def colour_planes(s):
    """Plane c holds the spins with (i + col) % 2 == c at column col // 2."""
    L = s.shape[0]
    i, col = np.indices((L, L))
    planes = []
    for c in (0, 1):
        m = (i + col) % 2 == c
        planes.append(s[m].reshape(L, L // 2))
    return planes


@pytest.mark.parametrize("L", [64, 128, 192])
def test_int8_planes_are_the_colour_sublattices(L):
    s = random_lattice(L, L)
    b, w = oracle.to_planes_int8(s)
    eb, ew = colour_planes(s)
    np.testing.assert_array_equal(b, eb)
    np.testing.assert_array_equal(w, ew)


@pytest.mark.parametrize("L", [64, 128, 192])
def test_msc4_words_hold_each_spin_in_a_nibble(L):
    s = random_lattice(L, L + 1)
    b, w = oracle.to_planes_msc4(s)
    for plane, expect in zip((b, w), colour_planes(s)):
        nib = (plane[:, :, None] >> (4 * np.arange(16, dtype=np.uint64))) & np.uint64(0xF)
        np.testing.assert_array_equal(nib.reshape(L, L // 2), (expect > 0).astype(np.uint64))
    np.testing.assert_array_equal(oracle.from_planes_msc4(L, b, w), s)


@pytest.mark.parametrize("L", [64, 128, 192, 320])
def test_bit_planes_are_little_endian_bits_of_the_colour_planes(L):
    s = random_lattice(L, L + 2)
    b, w = oracle.to_planes_bits(s)
    assert b.shape == (L, L // 16) and b.dtype == np.uint8
    for plane, expect in zip((b, w), colour_planes(s)):
        np.testing.assert_array_equal(plane, np.packbits(expect > 0, axis=1, bitorder="little"))
    np.testing.assert_array_equal(oracle.from_planes_bits(L, b, w), s)


def test_bit_planes_follow_the_msc4_spin_order():
    """Bits 16 k .. 16 k + 15 of a row are the low bits of MSC4 word k's nibbles."""
    L = 128
    s = random_lattice(L, 7)
    bb, bw = oracle.to_planes_bits(s)
    mb, mw = oracle.to_planes_msc4(s)
    for bits, words in ((bb, mb), (bw, mw)):
        as16 = bits.view("<u2").astype(np.uint64)
        lows = np.zeros_like(words)
        for k in range(16):
            lows |= ((words >> np.uint64(4 * k)) & np.uint64(1)) << np.uint64(k)
        np.testing.assert_array_equal(as16, lows)


def test_bits_bytes():
    assert ising.ising_bits_bytes(64) == 64 * 4
    assert ising.ising_bits_bytes(65536) == 65536 * 65536 // 16
    for L in (0, 32, 96, -64):
        with pytest.raises(ising.IsingError) as e:
            ising.ising_bits_bytes(L)
        assert e.value.status == ising.ISING_EINVAL
