"""Host-side statistics of Monte Carlo series: integrated autocorrelation time by Sokal's automatic
window and the effective sample size it implies (Madras & Sokal, J. Stat. Phys. 50, 109 (1988))."""
from __future__ import annotations

import numpy as np


def autocorrelation(x: np.ndarray) -> np.ndarray:
    """Normalised autocorrelation rho(t), t = 0..T-1, of a series x [T] or of M independent series x [T, M]
    of one process (the autocovariances are averaged over the M series)."""
    x = np.asarray(x, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    T = x.shape[0]
    x = x - x.mean(0)
    n = 1 << int(2 * T - 1).bit_length()
    f = np.fft.rfft(x, n=n, axis=0)
    c = np.fft.irfft(f * np.conj(f), n=n, axis=0)[:T].mean(1)
    return c / c[0] if c[0] > 0 else np.zeros(T)


def tau_int(x: np.ndarray, c: float = 5.0) -> float:
    """tau_int = 1/2 + sum_{t=1}^{W} rho(t) with the smallest window W >= c tau_int(W); a series of n
    measurements then carries n / (2 tau_int) independent samples."""
    rho = autocorrelation(x)
    tau = 0.5 + np.cumsum(rho[1:])
    W = np.arange(1, len(rho))
    ok = W >= c * tau
    if not ok.any():
        return float(tau[-1]) if len(tau) else 0.5
    return float(tau[np.argmax(ok)])


def ess(x: np.ndarray, c: float = 5.0) -> float:
    """Effective number of independent samples in x [T] or x [T, M]."""
    x = np.asarray(x, np.float64)
    T = x.shape[0]
    M = 1 if x.ndim == 1 else x.shape[1]
    return T * M / (2.0 * tau_int(x, c))
