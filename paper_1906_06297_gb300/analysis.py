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


def seconds_to_error(series_list, seconds: float, eps: float) -> dict:
    """Wall time a method needs for standard error `eps` on the mean of an
    observable, from a run of `seconds` that produced `series_list` (equally
    long series, one per chain, all at the temperature of interest).

    With N samples in all, integrated time tau (in samples) and per-sample
    variance var, the squared standard error of the mean is var * 2 tau / N;
    error eps needs N_eps = 2 tau var / eps^2 samples, i.e. seconds * N_eps / N
    of the same run (the cost grows linearly with the samples).  `reliable`
    says whether each series is at least 50 tau long, the length from which
    tau itself is well estimated; shorter series give lower bounds on tau and
    on the time."""
    xs = [np.asarray(s, dtype=np.float64) for s in series_list]
    es = effective_samples(xs)
    allx = np.concatenate(xs)
    var = float(allx.var(ddof=1)) if allx.size > 1 else 0.0
    n = es["samples"]
    tau = es["tau_int"]
    n_eps = 2.0 * tau * var / (eps * eps)
    return {"seconds_to_error": seconds * n_eps / n, "eps": eps, "tau_int": tau, "var": var,
            "mean": float(allx.mean()), "stderr_reached": float(np.sqrt(var * 2.0 * tau / n)),
            "series_over_tau": float(len(xs[0]) / tau) if xs else 0.0,
            "reliable": bool(xs) and len(xs[0]) >= 50.0 * tau}
