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


def ss_counts(spins):
    """Exact (N_J, N_J', M) of periodic SS configurations [n][rows][cols] of
    +-1 (even sides): J bonds between lattice neighbours, J' dimers on the
    plaquettes (2i, 2j) ('\\') and (2i+1, 2j+1) ('/'), as the ten filters place
    them.  Returns three int64 arrays of length n."""
    s = np.asarray(spins, dtype=np.int64)
    nJ = (s * np.roll(s, -1, axis=2)).sum((1, 2)) + (s * np.roll(s, -1, axis=1)).sum((1, 2))
    a = s[:, 0::2, 0::2] * np.roll(np.roll(s, -1, 1), -1, 2)[:, 0::2, 0::2]           # (2i,2j)-(2i+1,2j+1)
    b = np.roll(s, -2, 2)[:, 1::2, 0::2] * np.roll(np.roll(s, -2, 1), -1, 2)[:, 0::2, 0::2]
    return nJ, a.sum((1, 2)) + b.sum((1, 2)), s.sum((1, 2))


def ground_state_energy(L, J, Jp, h, max_sites=16):
    """Lowest energy per lattice (1/16 units, E = qJ N_J + qJ' N_J' - qh M with
    Q.4 couplings) over all configurations of an L x L periodic lattice that
    repeat with an even a x b supercell (a, b dividing L, a b <= max_sites):
    the exact ground state whenever it has such a period, as the FM, Neel,
    dimer and 1/3-plateau states do.  Also returns the supercell and pattern."""
    qJ, qJp, qh = (int(round(16 * x)) for x in (J, Jp, h))
    best = None
    for a in range(2, L + 1, 2):
        for b in range(2, L + 1, 2):
            if L % a or L % b or a * b > max_sites:
                continue
            n = a * b
            x = np.arange(1 << n, dtype=np.int64)
            cells = (((x[:, None] >> np.arange(n)) & 1) * 2 - 1).reshape(-1, a, b)
            nJ, nP, M = ss_counts(cells)
            E = (qJ * nJ + qJp * nP - qh * M) * (L * L // n)
            i = int(np.argmin(E))
            if best is None or E[i] < best[0]:
                best = (int(E[i]), (a, b), cells[i].copy())
    return best


def phase_label(nJ, nJp, M, N):
    """A name for a ground state of N spins from its counts: FM (|M| = N),
    Neel (M = 0, every J bond antiparallel: N_J = -2N), dimer (M = 0, every
    J' dimer antiparallel: N_J' = -N/2, N_J = 0), the 1/3 and 1/2
    magnetisation plateaus, else its magnetisation per spin."""
    from fractions import Fraction
    m = abs(Fraction(int(M), int(N)))
    if m == 1:
        return "FM"
    if m == 0:
        if nJ == -2 * N:
            return "Neel"
        if nJp == -(N // 2) and nJ == 0:
            return "dimer"
        return "m=0"
    if m == Fraction(1, 3):
        return "1/3 plateau"
    if m == Fraction(1, 2):
        return "1/2 plateau"
    return f"m={m}"


def time_to_solution(first_hits, n_sweeps, level=99.0):
    """TTS_l = T log(1 - l/100) / log(1 - p_gnd) (Sec. III, "Hardware
    Acceleration"), in sweeps, from the first hitting sweeps of independent
    runs of n_sweeps sweeps (-1: no hit): p_gnd = fraction of runs that reached
    the ground state, T = their mean hitting sweep.  p_gnd = 1 gives TTS_100 =
    T; p_gnd = 0 gives None.  Returns (p_gnd, T, TTS_l)."""
    h = np.asarray(first_hits)
    ok = (h >= 0) & (h <= n_sweeps)
    p = float(ok.mean())
    if p == 0.0:
        return p, None, None
    T = float(h[ok].mean())
    if p == 1.0:
        return p, T, T
    return p, T, T * np.log(1.0 - level / 100.0) / np.log(1.0 - p)
