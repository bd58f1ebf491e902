"""Effective sample size of Monte Carlo time series (host-side measurement).

The integrated autocorrelation time uses the self-consistent window of
Madras and Sokal (J. Stat. Phys. 50, 109 (1988)): sum the normalised
autocorrelation up to the first lag W with W >= c * tau(W), c = 6.  A series
of n samples then carries n / (2 tau) independent samples.
"""
from __future__ import annotations

import numpy as np


def integrated_time(x, c: float = 6.0) -> float:
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 4 or np.allclose(x, x[0]):
        return 0.5
    d = x - x.mean()
    spec = np.fft.rfft(d, 2 * n)
    acov = np.fft.irfft(spec * np.conj(spec))[:n]
    rho = acov / acov[0]
    tau = 0.5
    for lag in range(1, n):
        tau += rho[lag]
        if lag >= c * tau:
            break
    return max(float(tau), 0.5)


def effective_samples(series_list) -> dict:
    """Independent-sample count of equally long series (one per chain)."""
    taus = [integrated_time(s) for s in series_list]
    n = sum(len(s) for s in series_list)
    tau = float(np.mean(taus))
    return {"tau_int": tau, "samples": n, "effective": n / (2.0 * tau)}
