"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of ``oracle/ising_oracle.c`` (a
dropped term, a wrong sign, a wrong index, a transposed operand, a swapped
order), builds it on the CPU into a temporary library, and runs the pin tests
against that build in a subprocess.  The pins must fail for every mutant.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ising_oracle.c")

MUTANTS = {
    "dropped_neighbour": ("above[c] + below[c] + row[wrap(c - 1, L)]", "above[c] + row[wrap(c - 1, L)]"),
    "wrong_exponent_sign": ("double p = exp(-beta * dE);", "double p = exp(beta * dE);"),
    "wrong_neighbour_index": ("row[wrap(c + 1, L)];\n        int s", "row[wrap(c + 3, L)];\n        int s"),
    "transposed_philox_operand": ("(uint64_t)PHILOX_M0 * (uint64_t)x[0]", "(uint64_t)PHILOX_M0 * (uint64_t)x[1]"),
    "missing_key_bump": ("        k1 += PHILOX_W1;\n", ""),
    "wrong_draw_word": ("return out[site & 3];", "return out[(site + 1) & 3];"),
    "white_first": ("oracle_half_sweep(L, s, 0, T, seed, t, nthreads);\n        oracle_half_sweep(L, s, 1, T, seed, t, nthreads);",
                    "oracle_half_sweep(L, s, 1, T, seed, t, nthreads);\n        oracle_half_sweep(L, s, 0, T, seed, t, nthreads);"),
    "right_bonds_only": ("        b += v * s[wrap(i + 1, L) * L + c];\n", ""),
    "wrong_plane_site": ("return (uint64_t)i * (uint64_t)(L / 2) + (uint64_t)(c / 2);",
                         "return (uint64_t)i * (uint64_t)(L / 2) + (uint64_t)(c % (L / 2));"),
    "swap_exponent_sign": ("double p = exp(-x);", "double p = exp(x);"),
    "swap_keeps_slot": ("                    slot_of[a] = (int32_t)(k + 1);\n", ""),
    "stream_ignored": ("ctr[1] = (uint32_t)(q >> 32) + stream;", "ctr[1] = (uint32_t)(q >> 32);"),
    "black_is_odd": ("return (int)((i + c) & 1); }", "return (int)((i + c + 1) & 1); }"),
    "plane_split_shifted": ("int8_t *dst = colour_of(i, c) == 0 ? black_row : white_row;",
                            "int8_t *dst = colour_of(i, c + 1) == 0 ? black_row : white_row;"),
}

PIN_FILES = ["tests/test_oracle_philox.py", "tests/test_oracle_rules.py", "tests/test_oracle_batch.py",
             "tests/test_oracle_statistics.py", "tests/test_golden.py"]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name} not found exactly once"
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", str(lib), str(src), "-lm"],
                   check=True)
    env = dict(os.environ, ISING_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PIN_FILES],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
