"""Error bars for Markov-chain time series.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

``tau_int`` is the integrated autocorrelation time with Sokal's automatic
window (A. D. Sokal, "Monte Carlo methods in statistical mechanics:
foundations and new algorithms", 1996 lecture notes, Sec. 3): the window W is
the smallest with W >= c * tau_int(W), c = 6.  The error of a time average of
n correlated samples is sqrt(2 tau_int var / n).
"""
from __future__ import annotations

import numpy as np


def autocorrelation(x: np.ndarray) -> np.ndarray:
    """Normalised autocorrelation function rho(t), t = 0 .. n-1 (via FFT)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    y = x - x.mean()
    f = np.fft.rfft(y, n=2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n]
    if acf[0] == 0:
        return np.zeros(n)
    return acf / acf[0]


def tau_int(x: np.ndarray, c: float = 6.0) -> float:
    """Integrated autocorrelation time, tau = 1/2 + sum_{t=1}^{W} rho(t)."""
    rho = autocorrelation(x)
    tau = 0.5
    for w in range(1, rho.size):
        tau += rho[w]
        if w >= c * tau:
            return max(tau, 0.5)
    return max(tau, 0.5)


def mean_and_error(x: np.ndarray, c: float = 6.0):
    """(mean, standard error, tau_int) of a correlated series."""
    x = np.asarray(x, dtype=np.float64)
    tau = tau_int(x, c)
    var = x.var(ddof=1) if x.size > 1 else 0.0
    return float(x.mean()), float(np.sqrt(2.0 * tau * var / x.size)), tau


def pooled_mean_and_error(chains) -> tuple[float, float]:
    """Mean and error over independent chains, each with its own tau_int."""
    means, errs = [], []
    for x in chains:
        m, e, _ = mean_and_error(x)
        means.append(m)
        errs.append(e)
    means = np.asarray(means)
    errs = np.asarray(errs)
    # equal-length chains: the plain average, with the per-chain errors combined
    m = float(means.mean())
    e = float(np.sqrt((errs**2).sum()) / len(means))
    return m, e
