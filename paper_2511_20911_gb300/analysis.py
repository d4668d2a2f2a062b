"""Host-side analysis of sampler output: energies from exact integer sums and
effective sample sizes.  Post-processing only (not on the sampling path)."""
from __future__ import annotations

import numpy as np


def energy_series(series, J, Jp, h):
    """E = J NJ + J' NJ' - h M per measurement; series[..., 3] int32, and J,
    Jp, h broadcastable to series[..., 0] (e.g. per chain)."""
    s = series.astype(np.float64)
    return J * s[..., 0] + Jp * s[..., 1] - h * s[..., 2]


def integrated_autocorr_time(x, c=5.0):
    """Sokal's automatic windowing (Sokal, "Monte Carlo methods in statistical
    mechanics", 1997): tau = 1/2 + sum_{t=1}^{W} rho(t) with the smallest
    window W >= c tau(W).  x: [chains][T]; returns tau per chain."""
    x = np.asarray(x, np.float64)
    n_ch, T = x.shape
    y = x - x.mean(1, keepdims=True)
    nfft = 1 << int(np.ceil(np.log2(2 * T)))
    f = np.fft.rfft(y, nfft, axis=1)
    acf = np.fft.irfft(f * np.conj(f), nfft, axis=1)[:, :T]
    var = acf[:, :1]
    tau = np.full(n_ch, np.nan)
    ok = var[:, 0] > 0
    rho = np.zeros_like(acf)
    rho[ok] = acf[ok] / var[ok]
    cum = 0.5 + np.cumsum(rho[:, 1:], axis=1)        # tau(W) for W = 1..T-1
    W = np.arange(1, T)
    cond = W[None, :] >= c * cum
    first = np.where(cond.any(1), cond.argmax(1), T - 2)
    tau[ok] = np.maximum(cum[ok, first[ok]], 0.5)
    return tau


def effective_samples(x, burn_frac=0.1, c=5.0):
    """Per-chain ESS = n / (2 tau) after discarding the first burn_frac; chains
    with zero variance (frozen) contribute 0."""
    x = np.asarray(x, np.float64)
    b = int(x.shape[1] * burn_frac)
    x = x[:, b:]
    tau = integrated_autocorr_time(x, c)
    ess = x.shape[1] / (2.0 * tau)
    return np.where(np.isfinite(ess), ess, 0.0)


def structure_factor(spins):
    """Static structure factor per spin of configurations [n][rows][cols] of
    +-1, S(q) = |sum_r s_r e^{i q.r}|^2 / N averaged over the n configurations,
    at q = 2 pi (nR / rows, nC / cols) (Sec. IV.B, Eq. 11; defined for open
    edges too, unlike the periodic correlation sums the sampler accumulates).
    Returns [rows][cols] doubles."""
    s = np.asarray(spins, dtype=np.float64)
    f = np.fft.fft2(s, axes=(-2, -1))
    return (np.abs(f) ** 2).mean(0) / (s.shape[-1] * s.shape[-2])
