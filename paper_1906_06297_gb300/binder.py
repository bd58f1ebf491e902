"""Binder cumulant crossing (Sec. 5.3, Fig. 6): locate the critical point as
the inverse temperature where U_L(beta) of different lattice sizes cross.

U_L = 1 - <m^4> / (3 <m^2>^2), m the magnetisation per site.  The paper prints
the ratio without the factor 3; the two forms are affine images of each other
(U_printed = 3 U - 2), so they cross at the same beta, and the form with the
factor 3 is the one whose critical value (about 0.611 for the periodic square
lattice) is tabulated in the literature.

The sampler is the batched sweep with replica exchange: one batch holds, for
every size, `ladders` ladders of S inverse temperatures spanning the window
around beta_c; the per-record magnetisations of the slot-ordered trace are
pooled per (size, beta).  Everything that moves spins runs in the library's
kernels; this module only schedules the runs and reduces the recorded sums.
"""
from __future__ import annotations

import math

import numpy as np

BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))


def binder_from_moments(m2: np.ndarray, m4: np.ndarray) -> np.ndarray:
    return 1.0 - m4 / (3.0 * m2 * m2)


def crossings(beta, u_a, u_b) -> list[float]:
    """Inverse temperatures where u_a - u_b changes sign, by linear
    interpolation between neighbouring grid points."""
    beta = np.asarray(beta, dtype=np.float64)
    d = np.asarray(u_a, dtype=np.float64) - np.asarray(u_b, dtype=np.float64)
    out = []
    for k in range(len(d) - 1):
        if d[k] == 0.0:
            out.append(float(beta[k]))
        elif d[k] * d[k + 1] < 0.0:
            out.append(float(beta[k] + (beta[k + 1] - beta[k]) * d[k] / (d[k] - d[k + 1])))
    return out


def binder_study(sizes=(32, 64), ladders: int = 8, ladder_size: int = 16, beta_lo: float = 0.41,
                 beta_hi: float = 0.47, sweeps: int = 20000, thermalize: int = 2000, record_every: int = 2,
                 chunks: int = 10, seed: int = 1, device="cuda", stream=None) -> dict:
    """U_L(beta) for every size on an evenly spaced beta grid, with jackknife
    errors over `chunks` consecutive blocks of the measured sweeps, and the
    crossing points of consecutive sizes."""
    import torch

    import paper_1906_06297_gb300 as ising

    betas = np.linspace(beta_lo, beta_hi, ladder_size)
    L = []
    for side in sizes:
        L += [int(side)] * (ladders * ladder_size)
    S = ladder_size
    # the trace fills and reads in the stream order of the batched runs
    with ising._on_stream(stream):
        b = ising.Batch(L, S, betas, device=device)
        b.init(ising.ISING_INIT_RANDOM, seed, stream)
        b.run(thermalize, seed, 0, record_every, True, None, True, stream)
        b.check(stream)
        per_chunk = max(record_every, (sweeps // chunks) // record_every * record_every)
        n_lat = len(L)
        area = torch.tensor([float(x) * float(x) for x in L], dtype=torch.float64, device=device)
        # sums over events per chunk and lattice column: m^2, m^4
        m2 = np.zeros((chunks, n_lat))
        m4 = np.zeros((chunks, n_lat))
        off = thermalize
        events = 0
        for c in range(chunks):
            n_ev = b.n_events(per_chunk, off, record_every)
            tr = torch.zeros((n_ev, n_lat, 2), dtype=torch.int64, device=device)
            b.run(per_chunk, seed, off, record_every, True, tr, True, stream)
            b.check(stream)
            m = tr[:, :, 0].to(torch.float64) / area
            m2[c] = (m * m).sum(dim=0).cpu().numpy()
            m4[c] = (m * m * m * m).sum(dim=0).cpu().numpy()
            events += n_ev
            off += per_chunk
    n_per_chunk = events / chunks
    # trace column l*S + k holds the lattice at slot k of ladder l: pool the
    # ladders of each size per slot
    out = {"betas": betas.tolist(), "sizes": list(sizes), "ladders": ladders, "sweeps": off - thermalize,
           "thermalize": thermalize, "record_every": record_every, "U": {}, "U_err": {}}
    for si, side in enumerate(sizes):
        cols = np.arange(si * ladders * S, (si + 1) * ladders * S).reshape(ladders, S)
        c2 = m2[:, cols].sum(axis=1)  # chunks x S
        c4 = m4[:, cols].sum(axis=1)
        cnt = n_per_chunk * ladders
        full = binder_from_moments(c2.sum(0) / (cnt * chunks), c4.sum(0) / (cnt * chunks))
        jk = np.stack([binder_from_moments((c2.sum(0) - c2[j]) / (cnt * (chunks - 1)),
                                           (c4.sum(0) - c4[j]) / (cnt * (chunks - 1))) for j in range(chunks)])
        err = np.sqrt((chunks - 1) / chunks * ((jk - jk.mean(0)) ** 2).sum(0))
        out["U"][str(side)] = full.tolist()
        out["U_err"][str(side)] = err.tolist()
    out["crossings"] = {f"{a}/{c}": crossings(betas, out["U"][str(a)], out["U"][str(c)])
                        for a, c in zip(sizes[:-1], sizes[1:])}
    k = int(np.argmin(np.abs(betas - BETA_C)))
    out["beta_nearest_c"] = float(betas[k])
    out["U_at_beta_nearest_c"] = {str(s): out["U"][str(s)][k] for s in sizes}
    del b
    return out
