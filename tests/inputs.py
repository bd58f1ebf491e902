"""Seeded synthetic spin configurations fed to both the CUDA path and the
oracle.  This module holds none of the method's arithmetic: it only draws
+1/-1 patterns with numpy."""
import numpy as np


def random_lattice(L: int, seed: int, p_up: float = 0.5) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.where(rng.random((L, L)) < p_up, 1, -1).astype(np.int8)


def neel(L: int) -> np.ndarray:
    i, c = np.indices((L, L))
    return np.where((i + c) % 2 == 0, 1, -1).astype(np.int8)


def domains(L: int, seed: int, n: int = 6) -> np.ndarray:
    """Large random rectangles of flipped spins on an all-up background:
    mostly aligned neighbourhoods (a = 3, 4), like an ordered phase."""
    rng = np.random.default_rng(seed)
    s = np.ones((L, L), dtype=np.int8)
    for _ in range(n):
        r0, c0 = rng.integers(0, L, size=2)
        h, w = rng.integers(1, max(2, L // 2), size=2)
        rows = (np.arange(h) + r0) % L
        cols = (np.arange(w) + c0) % L
        s[np.ix_(rows, cols)] *= -1
    return s
