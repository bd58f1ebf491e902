"""CPU oracle for the checkerboard Metropolis sweep of the 2D Ising model.

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users; the product path never imports this
package.  The arithmetic lives in ``ising_oracle.c`` (plain C, compiled here
with gcc) and, for the exact results it is checked against, in
``oracle.exact`` (enumeration, Kaufman and Onsager closed forms) and
``oracle.stats`` (autocorrelation-aware error bars).

This module only marshals numpy arrays to the C functions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ising_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# A test may point the wrapper at a deliberately broken build of the oracle
# (see tests/test_oracle_mutations.py); nothing else sets this.
_LIB_OVERRIDE = os.environ.get("ISING_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

MODE_RANDOM, MODE_UP, MODE_DOWN = 0, 1, 2
PURPOSE_METROPOLIS, PURPOSE_INIT = 0, 1


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(_LIB_OVERRIDE or build())
        i64, u64, i32, u32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
        p = ctypes.c_void_p
        lib.oracle_philox4x32_10.argtypes = [p, p, p]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_draw.argtypes = [u64, u64, u64, i32, i32]
        lib.oracle_draw.restype = u32
        lib.oracle_thresholds.argtypes = [ctypes.c_double, p]
        lib.oracle_thresholds.restype = i32
        lib.oracle_init_row.argtypes = [i64, i64, p, i32, u64]
        lib.oracle_init_row.restype = None
        lib.oracle_init.argtypes = [i64, p, i32, u64]
        lib.oracle_init.restype = i32
        lib.oracle_update_row.argtypes = [i64, p, p, p, i64, i32, p, u64, u64]
        lib.oracle_update_row.restype = None
        lib.oracle_half_sweep.argtypes = [i64, p, i32, p, u64, u64, i32]
        lib.oracle_half_sweep.restype = None
        lib.oracle_observables.argtypes = [i64, p, p]
        lib.oracle_observables.restype = None
        lib.oracle_run.argtypes = [i64, p, ctypes.c_double, i64, u64, u64, p, i32]
        lib.oracle_run.restype = i32
        for name in ("oracle_row_to_planes_int8", "oracle_row_from_planes_int8",
                     "oracle_row_to_planes_msc4", "oracle_row_from_planes_msc4"):
            getattr(lib, name).argtypes = [i64, i64, p, p, p]
            getattr(lib, name).restype = None
        for name in ("oracle_to_planes_int8", "oracle_to_planes_msc4"):
            getattr(lib, name).argtypes = [i64, p, p, p, i64]
            getattr(lib, name).restype = None
        lib.oracle_to_planes_bits.argtypes = [i64, p, p, p]
        lib.oracle_from_planes_bits.argtypes = [i64, p, p, p]
        lib.oracle_to_planes_bits.restype = None
        lib.oracle_from_planes_bits.restype = None
        for name in ("oracle_from_planes_int8", "oracle_from_planes_msc4"):
            getattr(lib, name).argtypes = [i64, p, p, i64, p]
            getattr(lib, name).restype = None
        lib.oracle_draw_stream.argtypes = [u64, u32, u64, u64, i32, i32]
        lib.oracle_draw_stream.restype = u32
        lib.oracle_init_row_stream.argtypes = [i64, i64, p, i32, u64, u32]
        lib.oracle_init_row_stream.restype = None
        lib.oracle_swap_threshold.argtypes = [ctypes.c_double, ctypes.c_double, i64]
        lib.oracle_swap_threshold.restype = u64
        lib.oracle_batch_run.argtypes = [i64, p, p, i64, p, p, p, i64, u64, u64, i64, i32, p, i32, i64]
        lib.oracle_batch_run.restype = i32
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = i32
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: 4 counter words, 2 key words -> 4 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw(seed: int, site: int, t: int, colour: int, purpose: int = PURPOSE_METROPOLIS) -> int:
    """The 32-bit random number of one colour-plane site at sweep t."""
    return int(_load().oracle_draw(seed, site, t, colour, purpose))


def thresholds(beta: float) -> np.ndarray:
    """The 5-entry acceptance table T[a] (uint64; 2**32 means always flip)."""
    T = np.zeros(5, dtype=np.uint64)
    if _load().oracle_thresholds(float(beta), _ptr(T)) != 0:
        raise ValueError(f"invalid beta {beta!r}")
    return T


def init(L: int, mode: int = MODE_RANDOM, seed: int = 0) -> np.ndarray:
    """An L x L int8 lattice in the requested initial state."""
    s = np.zeros((L, L), dtype=np.int8)
    if _load().oracle_init(L, _ptr(s), mode, seed) != 0:
        raise ValueError(f"invalid lattice size {L}")
    return s


def init_row(L: int, i: int, mode: int = MODE_RANDOM, seed: int = 0) -> np.ndarray:
    """Row i of the initial state of an L x L lattice (int8, length L)."""
    row = np.zeros(L, dtype=np.int8)
    _load().oracle_init_row(L, i, _ptr(row), mode, seed)
    return row


def half_sweep(s: np.ndarray, beta: float, colour: int, seed: int, t: int, nthreads: int = 0):
    """Update every site of one colour of ``s`` in place."""
    T = thresholds(beta)
    _load().oracle_half_sweep(s.shape[0], _ptr(s), colour, _ptr(T), seed, t, nthreads)
    return s


def update_row(L: int, above: np.ndarray, row: np.ndarray, below: np.ndarray, i: int,
               colour: int, beta: float, seed: int, t: int) -> np.ndarray:
    """Update the given colour's sites of row i (in place) from rows i-1 and i+1."""
    T = thresholds(beta)
    _load().oracle_update_row(L, _ptr(above), _ptr(row), _ptr(below), i, colour, _ptr(T), seed, t)
    return row


def observables(s: np.ndarray) -> np.ndarray:
    """[sum of spins, sum over bonds of s_i s_j] as int64."""
    out = np.zeros(2, dtype=np.int64)
    _load().oracle_observables(s.shape[0], _ptr(s), _ptr(out))
    return out


def run(s: np.ndarray, beta: float, n: int, seed: int, off: int = 0, nthreads: int = 0,
        trace: bool = True):
    """n sweeps of ``s`` in place starting at sweep index ``off``; returns the
    per-sweep trace (n x 2 int64: sum s, sum bonds) or None."""
    tr = np.zeros((max(n, 0), 2), dtype=np.int64) if trace else None
    rc = _load().oracle_run(s.shape[0], _ptr(s), float(beta), n, seed, off,
                            _ptr(tr) if trace else None, nthreads)
    if rc != 0:
        raise ValueError("invalid oracle arguments")
    return tr


def to_planes_int8(s: np.ndarray, stride: int | None = None):
    L = s.shape[0]
    stride = L // 2 if stride is None else stride
    b = np.zeros((L, stride), dtype=np.int8)
    w = np.zeros((L, stride), dtype=np.int8)
    _load().oracle_to_planes_int8(L, _ptr(s), _ptr(b), _ptr(w), stride)
    return b, w


def from_planes_int8(L: int, black: np.ndarray, white: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(black, dtype=np.int8)
    w = np.ascontiguousarray(white, dtype=np.int8)
    s = np.zeros((L, L), dtype=np.int8)
    _load().oracle_from_planes_int8(L, _ptr(b), _ptr(w), b.shape[1], _ptr(s))
    return s


def to_planes_msc4(s: np.ndarray, stride_words: int | None = None):
    L = s.shape[0]
    stride_words = L // 32 if stride_words is None else stride_words
    b = np.zeros((L, stride_words), dtype=np.uint64)
    w = np.zeros((L, stride_words), dtype=np.uint64)
    _load().oracle_to_planes_msc4(L, _ptr(s), _ptr(b), _ptr(w), stride_words)
    return b, w


def from_planes_msc4(L: int, black: np.ndarray, white: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(black, dtype=np.uint64)
    w = np.ascontiguousarray(white, dtype=np.uint64)
    s = np.zeros((L, L), dtype=np.int8)
    _load().oracle_from_planes_msc4(L, _ptr(b), _ptr(w), b.shape[1], _ptr(s))
    return s


def to_planes_bits(s: np.ndarray):
    """The two colour planes in the bit-packed format: (L, L/16) uint8 each."""
    L = s.shape[0]
    s = np.ascontiguousarray(s, dtype=np.int8)
    b = np.zeros((L, L // 16), dtype=np.uint8)
    w = np.zeros((L, L // 16), dtype=np.uint8)
    _load().oracle_to_planes_bits(L, _ptr(s), _ptr(b), _ptr(w))
    return b, w


def from_planes_bits(L: int, black: np.ndarray, white: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(black, dtype=np.uint8).reshape(L, L // 16)
    w = np.ascontiguousarray(white, dtype=np.uint8).reshape(L, L // 16)
    s = np.zeros((L, L), dtype=np.int8)
    _load().oracle_from_planes_bits(L, _ptr(b), _ptr(w), _ptr(s))
    return s


def row_from_planes_msc4(L: int, i: int, black_row: np.ndarray, white_row: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(black_row, dtype=np.uint64)
    w = np.ascontiguousarray(white_row, dtype=np.uint64)
    row = np.zeros(L, dtype=np.int8)
    _load().oracle_row_from_planes_msc4(L, i, _ptr(b), _ptr(w), _ptr(row))
    return row


def row_to_planes_msc4(L: int, i: int, row: np.ndarray):
    r = np.ascontiguousarray(row, dtype=np.int8)
    b = np.zeros(L // 32, dtype=np.uint64)
    w = np.zeros(L // 32, dtype=np.uint64)
    _load().oracle_row_to_planes_msc4(L, i, _ptr(r), _ptr(b), _ptr(w))
    return b, w


def row_from_planes_int8(L: int, i: int, black_row: np.ndarray, white_row: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(black_row, dtype=np.int8)
    w = np.ascontiguousarray(white_row, dtype=np.int8)
    row = np.zeros(L, dtype=np.int8)
    _load().oracle_row_from_planes_int8(L, i, _ptr(b), _ptr(w), _ptr(row))
    return row


def max_threads() -> int:
    return int(_load().oracle_max_threads())


# ---------------------------------------------------------------------------
# batches with replica exchange
# ---------------------------------------------------------------------------
def draw_stream(seed: int, stream: int, site: int, t: int, colour: int, purpose: int = PURPOSE_METROPOLIS) -> int:
    return int(_load().oracle_draw_stream(seed, stream, site, t, colour, purpose))


def swap_threshold(beta_lo: float, beta_hi: float, D: int) -> int:
    return int(_load().oracle_swap_threshold(float(beta_lo), float(beta_hi), int(D)))


class Batch:
    """n full int8 lattices with sides L[i]; ladders of S consecutive lattices
    over the inverse temperatures `beta` (S ascending values)."""

    def __init__(self, L, S: int, beta, mode: int = MODE_RANDOM, seed: int = 0, lattice_base: int = 0):
        self.L = np.ascontiguousarray(L, dtype=np.int64)
        self.n = int(self.L.size)
        self.S = int(S)
        self.beta = np.ascontiguousarray(beta, dtype=np.float64)
        self.lattice_base = int(lattice_base)
        assert self.beta.size == self.S and self.n % self.S == 0 and self.lattice_base % self.S == 0
        self.start = np.concatenate([[0], np.cumsum(self.L * self.L)])
        self.spins = np.zeros(int(self.start[-1]), dtype=np.int8)
        for i in range(self.n):
            Li = int(self.L[i])
            view = self.spins[self.start[i]:self.start[i + 1]].reshape(Li, Li)
            for r in range(Li):
                row = np.zeros(Li, dtype=np.int8)
                _load().oracle_init_row_stream(Li, r, _ptr(row), mode, seed, self.lattice_base + i)
                view[r] = row
        self.slot_of = (np.arange(self.n) % self.S).astype(np.int32)
        self.lattice_at = np.arange(self.n, dtype=np.int32)

    def lattice(self, i: int) -> np.ndarray:
        Li = int(self.L[i])
        return self.spins[self.start[i]:self.start[i + 1]].reshape(Li, Li)

    def run(self, n_sweeps: int, seed: int, off: int = 0, record_every: int = 0, swaps: bool = True,
            nthreads: int = 0):
        """Sweeps in place; returns the trace (events x n x 2, slot-ordered
        within each ladder) when record_every > 0."""
        n_events = 0
        if record_every > 0:
            n_events = (off + n_sweeps) // record_every - off // record_every
        tr = np.zeros((max(n_events, 0), self.n, 2), dtype=np.int64) if record_every > 0 else None
        rc = _load().oracle_batch_run(self.n, _ptr(self.L), _ptr(self.spins), self.S, _ptr(self.beta),
                                      _ptr(self.slot_of), _ptr(self.lattice_at), n_sweeps, seed, off,
                                      record_every, int(bool(swaps)), _ptr(tr) if tr is not None else None,
                                      nthreads, self.lattice_base)
        if rc != 0:
            raise ValueError("invalid batch arguments")
        return tr
