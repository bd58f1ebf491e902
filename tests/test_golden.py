"""The values the paper prints, kept as text fixtures under tests/golden/ (each
line with where it is printed), against the oracle and the library's host
logic.  Nothing here needs a GPU.

- fig3_neighbour_words.txt: the worked example of the multi-spin layout
  (caption of Fig. 3, Sec. 3.3): which words of the other colour the update of
  a target word reads.  Checked twice: through the oracle's colour planes and
  the nearest-neighbour definition of Sec. 2, and by perturbing the oracle's
  own half-sweep, which must depend on exactly those spins.
- critical_point.txt: T_c = 2.269185 (Sec. 5.3, Fig. 6).
- lattice_memory.txt: lattice sides with their memory footprints (Sec. 5.1,
  Sec. 5.2, Table 2) at 4 bits per spin.
"""
import os

import numpy as np
import pytest

import oracle
import paper_1906_06297_gb300 as ising
from oracle import exact
from tests import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
COLOURS = {"black": 0, "white": 1}
# the example lattice of Fig. 3: 12 columns, so 6 spins per colour-array row
WIDTH = 12
ROW = WIDTH // 2


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def _fig3_cases():
    cases = []
    for colour, target, above, below, centre, side, where in _lines("fig3_neighbour_words.txt"):
        ints = lambda t: [int(v) for v in t.split(",")]
        cases.append((colour, ints(target), ints(above), ints(below), ints(centre), int(side), where))
    return cases


FIG3 = _fig3_cases()


def _plane_coordinates():
    """For each colour plane position (i, j) of the 12 x 12 example lattice,
    its lattice row and column, through the oracle's own plane split."""
    r, c = np.indices((WIDTH, WIDTH), dtype=np.int64)
    rb, rw = oracle.to_planes_int8(r.astype(np.int8))
    cb, cw = oracle.to_planes_int8(c.astype(np.int8))
    return {0: (rb.astype(int), cb.astype(int)), 1: (rw.astype(int), cw.astype(int))}


def test_fig3_fixture_is_the_printed_example():
    assert len(FIG3) == 4
    assert FIG3[0][:2] == ("black", [8, 9]) and FIG3[1][:2] == ("black", [38, 39])


@pytest.mark.parametrize("case", FIG3, ids=[f"{c[0]}{c[1][0]}" for c in FIG3])
def test_fig3_words_from_the_oracle_planes_and_the_neighbour_definition(case):
    colour, target, above, below, centre, side, where = case
    tc = COLOURS[colour]
    coords = _plane_coordinates()
    rows, cols = coords[tc]
    orows, ocols = coords[1 - tc]
    # lattice site -> compact index in the other colour's array
    other = {(int(orows[i, j]), int(ocols[i, j])): i * ROW + j for i in range(WIDTH) for j in range(ROW)}
    needed = set()
    for k in target:
        i, j = divmod(k, ROW)
        r, c = int(rows[i, j]), int(cols[i, j])
        # Sec. 2: the four nearest neighbours on the periodic square lattice
        for rr, cc in ((r - 1, c), (r + 1, c), (r, c - 1), (r, c + 1)):
            needed.add(other[(rr % WIDTH, cc % WIDTH)])
    assert needed == set(above) | set(below) | set(centre) | {side}
    i0, j0 = divmod(target[0], ROW)
    # the vertical words sit straight above and below the target word, the
    # centre word at its own coordinates
    assert [divmod(k, ROW) for k in above] == [(i0 - 1, j0), (i0 - 1, j0 + 1)]
    assert [divmod(k, ROW) for k in below] == [(i0 + 1, j0), (i0 + 1, j0 + 1)]
    assert centre == target
    # the side spin is the nearest spin of the neighbouring word: the first of
    # the word to the right, or the last of the word to the left.  For black
    # targets the right word goes with odd rows (Sec. 3.3); white is reversed.
    assert side == (target[-1] + 1 if where == "right" else target[0] - 1)
    right = (i0 % 2 == 1) if colour == "black" else (i0 % 2 == 0)
    assert where == ("right" if right else "left")


@pytest.mark.parametrize("case", FIG3, ids=[f"{c[0]}{c[1][0]}" for c in FIG3])
def test_fig3_oracle_half_sweep_reads_exactly_those_spins(case):
    """At beta = 50 a site flips iff its energy does not rise (the table is
    2^32, 2^32, 2^32, 0, 0), so the update is a deterministic function of
    the neighbours.  Toggling one spin of the other colour and re-running
    the oracle's half-sweep shows which target spins depend on it; over
    48 random lattices the union must be exactly the printed words."""
    colour, target, above, below, centre, side, where = case
    tc = COLOURS[colour]
    coords = _plane_coordinates()
    rows, cols = coords[tc]
    orows, ocols = coords[1 - tc]
    sites = [(int(rows[divmod(k, ROW)]), int(cols[divmod(k, ROW)])) for k in target]
    found = set()
    for n in range(48):
        s = inputs.random_lattice(WIDTH, 500 + n)
        base = oracle.half_sweep(s.copy(), 50.0, tc, 7, 0)
        for i in range(WIDTH):
            for j in range(ROW):
                t = s.copy()
                t[orows[i, j], ocols[i, j]] *= -1
                out = oracle.half_sweep(t, 50.0, tc, 7, 0)
                if any(out[r, c] != base[r, c] for r, c in sites):
                    found.add(i * ROW + j)
    assert found == set(above) | set(below) | set(centre) | {side}


def test_critical_temperature():
    (tc_line,) = list(_lines("critical_point.txt"))
    assert tc_line[0] == "T_c"
    Tc = float(tc_line[1])
    # printed to 6 decimals
    assert abs(1.0 / exact.BETA_C - Tc) <= 0.5e-6
    # the spontaneous magnetisation (Eq. 7) vanishes above T_c and not below
    assert exact.onsager_magnetisation(1.0 / (Tc + 1e-4)) == 0.0
    assert exact.onsager_magnetisation(1.0 / (Tc - 1e-4)) > 0.0


UNITS = {"MB": 2**20, "GB": 2**30}


def _significant(text: str) -> int:
    """Significant digits of a number as printed."""
    return len(text.split("e")[0].replace(".", "").lstrip("0"))


def _rounded(x: float, digits: int) -> float:
    return float(f"{x:.{digits}g}")


def test_lattice_memory_footprints():
    for side, quantity, value, *_ in _lines("lattice_memory.txt"):
        L = int(side)
        if quantity == "spins":
            assert _rounded(L * L, _significant(value)) == float(value)
            continue
        number, unit = value[:-2], value[-2:]
        # the library's two MSC4 colour planes of an L x L lattice
        row_bytes, plane_bytes = ising.ising_lattice_bytes(L, ising.ISING_MSC4)
        total = 2 * plane_bytes
        assert total * 2 == L * L  # 4 bits per spin
        assert row_bytes * L == plane_bytes
        # as printed: to the digits given, in binary units
        assert _rounded(total / UNITS[unit], _significant(number)) == float(number)
    # and the oracle's own MSC4 planes at the smallest printed side: exactly 2 MB
    b, w = oracle.to_planes_msc4(np.ones((2048, 2048), dtype=np.int8))
    assert b.nbytes + w.nbytes == 2 * UNITS["MB"]
