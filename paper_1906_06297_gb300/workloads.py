"""Shapes of the synthetic workloads (no arithmetic of the method here).

pt_batch(): the parallel-tempering batch -- 4096 periodic lattices in 64
ladders of 64 inverse temperatures evenly spaced in [0.30, 0.60]; ladder sides
drawn from {32, 64, 128, 256, 512, 1024} in proportions 8:8:4:2:1:1, rounded
to whole ladders by largest remainder: 21, 21, 11, 5, 3, 3 ladders.
"""
from __future__ import annotations

import numpy as np

PT_SIDES = (32, 64, 128, 256, 512, 1024)
PT_WEIGHTS = (8, 8, 4, 2, 1, 1)


def ladders_by_largest_remainder(n_ladders: int, weights) -> list[int]:
    w = np.asarray(weights, dtype=np.float64)
    quota = n_ladders * w / w.sum()
    base = np.floor(quota).astype(int)
    rest = n_ladders - int(base.sum())
    order = np.argsort(-(quota - base), kind="stable")
    base[order[:rest]] += 1
    return base.tolist()


def pt_batch(n_ladders: int = 64, ladder_size: int = 64, beta_lo: float = 0.30, beta_hi: float = 0.60):
    counts = ladders_by_largest_remainder(n_ladders, PT_WEIGHTS)
    L = []
    for side, c in zip(PT_SIDES, counts):
        L += [side] * (c * ladder_size)
    beta = np.linspace(beta_lo, beta_hi, ladder_size)
    return L, ladder_size, beta
