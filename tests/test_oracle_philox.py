"""Pins for the oracle's Philox4x32-10 and its site keying.

The block function is checked against a second, independently written
implementation that we only *run*: PyTorch's CPU ``at::Philox4_32`` engine
(header ``ATen/core/PhiloxRNGEngine.h``), whose (seed, subsequence, offset)
map onto the key and counter words.  Statistical checks then catch a
generator that is well-formed but biased.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

_ENGINE_SRC = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>
int main() {
  unsigned c0, c1, c2, c3, k0, k1;
  while (std::scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
    uint64_t sub = (uint64_t)c2 | ((uint64_t)c3 << 32);
    uint64_t off = (uint64_t)c0 | ((uint64_t)c1 << 32);
    at::Philox4_32 e(seed, sub, off);
    for (int i = 0; i < 4; i++) std::printf("%u ", e());
    std::printf("\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def torch_engine(tmp_path_factory):
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("PhiloxRNGEngine.h not shipped with this torch")
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("philox")
    src = d / "engine.cpp"
    src.write_text(_ENGINE_SRC)
    exe = d / "engine"
    subprocess.run(["g++", "-O1", "-std=c++17", f"-I{inc}", str(src), "-o", str(exe)], check=True)

    def run(rows):
        text = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
        out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True)
        return np.array([[int(v) for v in line.split()] for line in out.stdout.strip().splitlines()],
                        dtype=np.uint64)

    return run


def test_philox_matches_torch_engine(torch_engine):
    rng = np.random.default_rng(7)
    rows = rng.integers(0, 2**32, size=(300, 6), dtype=np.uint64)
    # special words: all zero, all ones, counter words near wrap-around
    rows[0] = 0
    rows[1] = 2**32 - 1
    rows[2] = [2**32 - 1, 2**32 - 1, 0, 0, 1, 0]
    rows[3] = [0, 0, 2**32 - 1, 2**32 - 1, 0, 2**32 - 1]
    expect = torch_engine(rows)
    got = np.array([oracle.philox4x32_10(r[:4], r[4:]) for r in rows], dtype=np.uint64)
    np.testing.assert_array_equal(got, expect)


def test_draw_keying_convention():
    """The draw of a plane site is word (site & 3) of the block with counter
    (q_lo, q_hi, t_lo, colour | purpose << 1 | t_hi << 8), q = site >> 2, and
    key (seed_lo, seed_hi)."""
    cases = [
        (1234, 0, 0, 0, 0),
        (1234, 5, 17, 1, 0),
        (2**63 + 99, 2**35 + 3, 2**33 + 7, 1, 1),
        (0xFFFFFFFF_FFFFFFFF, 2**40 - 1, 2**40 + 5, 0, 3),
    ]
    for seed, site, t, colour, purpose in cases:
        q = site >> 2
        ctr = [q & 0xFFFFFFFF, q >> 32, t & 0xFFFFFFFF, colour | (purpose << 1) | ((t >> 32) << 8)]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        assert oracle.draw(seed, site, t, colour, purpose) == int(oracle.philox4x32_10(ctr, key)[site & 3])


def test_draws_differ_across_every_key_field():
    base = oracle.draw(1234, 100, 5, 0, 0)
    assert oracle.draw(1235, 100, 5, 0, 0) != base
    assert oracle.draw(1234 + (1 << 32), 100, 5, 0, 0) != base
    assert oracle.draw(1234, 101, 5, 0, 0) != base
    assert oracle.draw(1234, 104, 5, 0, 0) != base
    assert oracle.draw(1234, 100, 6, 0, 0) != base
    assert oracle.draw(1234, 100, 5 + (1 << 32), 0, 0) != base
    assert oracle.draw(1234, 100, 5, 1, 0) != base
    assert oracle.draw(1234, 100, 5, 0, 1) != base


def test_philox_uniformity_and_bit_balance():
    """chi^2 over 256 bins and per-bit balance on 2^16 blocks (2^18 words)."""
    key = [0x12345678, 0x9ABCDEF0]
    words = []
    for q in range(1 << 16):
        words.extend(oracle.philox4x32_10([q, 0, 3, 0], key))
    w = np.array(words, dtype=np.uint64)
    n = w.size
    counts = np.bincount((w >> 24).astype(np.int64), minlength=256)
    expected = n / 256
    chi2 = ((counts - expected) ** 2 / expected).sum()
    # 255 degrees of freedom: mean 255, sd ~22.6; 6 sd bound
    assert abs(chi2 - 255) < 6 * np.sqrt(2 * 255)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint64)[None, :]) & 1).sum(axis=0)
    sd = np.sqrt(n / 4)
    assert np.all(np.abs(bits - n / 2) < 6 * sd)
