"""Pins of the oracle's Gibbs sampler (arXiv 2511.20911, Sec. II.B) against
exact distributions: enumeration on L=3, a transfer matrix on L=6, and
brute-force ground states over supercell-periodic states."""
import numpy as np
import pytest
from scipy.stats import chi2

from ss_geometry import supercell_ground_energy, transfer_matrix_moments


def _exact_L3(orc, periodic, J, Jp, h, beta):
    L, N = 3, 9
    x = np.arange(1 << N)
    V = (((x[:, None] >> np.arange(N)) & 1) * 2 - 1).astype(np.int8)
    E = np.array([J * a + Jp * b - h * c for a, b, c in
                  (orc.counts(V[i].reshape(L, L), L, periodic=periodic) for i in range(len(V)))])
    w = np.exp(-beta * (E - E.min()))
    return w / w.sum()


# Odd-L periodic windows repeat every bond several times (4x the couplings on
# L=3), and block Gibbs through the hidden layer mixes slowly, so the burn-in
# is long and beta moderate there.
@pytest.mark.parametrize("periodic,J,Jp,h,beta,n_sweeps", [(True, 1.0, 1.5, 0.6875, 0.3, 600),
                                                           (False, 1.0, 1.5, 0.6875, 1.0, 400),
                                                           (True, -1.0, 0.5, -0.25, 0.25, 600),
                                                           (False, 0.5, 2.0, 1.0, 0.7, 400)])
def test_L3_histogram_chi2(orc, periodic, J, Jp, h, beta, n_sweeps):
    """Final states of many independent chains, histogrammed over the 512
    configurations, against the enumerated Boltzmann law exp(-beta H)/Z."""
    L, n_chains = 3, 30000
    p = _exact_L3(orc, periodic, J, Jp, h, beta)
    ids = np.arange(n_chains, dtype=np.uint32) + 7 * n_chains
    spins = orc.init_spins(L, ids, seed=99)
    orc.run(L, {"J": [J], "Jp": [Jp], "h": [h], "beta": [beta]}, np.zeros(n_chains, np.int32),
            spins, seed=99, sweep0=0, n_sweeps=n_sweeps, measure_every=0, chain_ids=ids,
            periodic=periodic)
    bits = ((spins.reshape(n_chains, 9) > 0).astype(np.int64) << np.arange(9)).sum(1)
    obs = np.bincount(bits, minlength=512).astype(float)
    exp = p * n_chains
    order = np.argsort(exp)            # pool the rarest states until each bin expects >= 5
    o_b, e_b, acc_o, acc_e = [], [], 0.0, 0.0
    for i in order:
        acc_o += obs[i]
        acc_e += exp[i]
        if acc_e >= 5:
            o_b.append(acc_o)
            e_b.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0:
        o_b[-1] += acc_o
        e_b[-1] += acc_e
    o_b, e_b = np.array(o_b), np.array(e_b)
    stat = ((o_b - e_b) ** 2 / e_b).sum()
    pval = chi2.sf(stat, len(o_b) - 1)
    assert pval > 1e-3, (stat, len(o_b), pval)


def test_L3_chi2_detects_a_wrong_sampler(orc):
    """Sanity of the test itself: a histogram drawn at another beta fails."""
    p_true = _exact_L3(orc, True, 1.0, 1.5, 0.6875, 0.5)
    p_wrong = _exact_L3(orc, True, 1.0, 1.5, 0.6875, 0.6)
    n = 40000
    obs = np.random.default_rng(1).multinomial(n, p_wrong)
    exp = p_true * n
    m = exp >= 5
    stat = ((obs[m] - exp[m]) ** 2 / exp[m]).sum()
    assert chi2.sf(stat, m.sum() - 1) < 1e-6


@pytest.mark.slow
def test_L6_config1_matches_transfer_matrix(orc):
    """L=6 periodic, J=J'=1, h=0.5, beta=2, 64 chains, 10^4 sweeps (the small
    workload's model and length): chain means of E, E^2, M, M^2 within 3
    standard errors of the exact transfer-matrix values.  The chains start
    from exact Boltzmann samples of the transfer matrix, so any bias of the
    sampler would move them away from the law they start in.  (From uniform
    random spins the chains do not equilibrate within 10^4 sweeps at this beta:
    a few percent stay in domain states 12 units above the Neel ground state
    for thousands of sweeps; see the companion test below.)"""
    from ss_geometry import transfer_matrix_sample
    L, N, n_chains, n_sweeps = 6, 36, 64, 10000
    J, Jp, h, beta = 1.0, 1.0, 0.5, 2.0
    ex = transfer_matrix_moments(L, J, Jp, h, beta)
    spins = transfer_matrix_sample(L, J, Jp, h, beta, n_chains, np.random.default_rng(2024))
    _, series, _ = orc.run(L, {"J": [J], "Jp": [Jp], "h": [h], "beta": [beta]},
                           np.zeros(n_chains, np.int32), spins, seed=1, sweep0=0,
                           n_sweeps=n_sweeps, measure_every=1, series_cap=n_sweeps)
    s = series.astype(np.float64)
    E = J * s[..., 0] + Jp * s[..., 1] - h * s[..., 2]
    M = s[..., 2]
    for name, x, ref in (("E", E, ex["E"]), ("E2", E * E, ex["E2"]), ("M", M, ex["M"]),
                         ("M2", M * M, ex["M2"])):
        cm = x.mean(1)
        se = cm.std(ddof=1) / np.sqrt(n_chains)
        assert abs(cm.mean() - ref) < 3 * se + 1e-9 * abs(ref), (name, cm.mean(), ref, se)
    # the exact values themselves: specific heat positive, |<m>| small in the Neel phase
    assert ex["E2"] - ex["E"] ** 2 > 0 and abs(ex["M"]) / N < 0.2


def test_transfer_matrix_sampler_matches_enumeration_L4():
    """The exact row sampler against the enumerated law on L=4: chi-square of
    the (N_J, N_J', M) histogram of 40000 samples (p > 1e-3)."""
    from scipy.stats import chi2
    from ss_geometry import ss_counts_batch, transfer_matrix_sample
    L, J, Jp, h, beta = 4, 1.0, 1.5, 0.5, 0.7
    x = np.arange(1 << 16)
    V = ((x[:, None] >> np.arange(16)) & 1) * 2 - 1
    nJ, nJp, M = ss_counts_batch(V, L)
    key = (nJ + 64) * 10000 + (nJp + 64) * 100 + (M + 32)
    w = np.exp(-beta * (J * nJ + Jp * nJp - h * M))
    uk, inv = np.unique(key, return_inverse=True)
    p = np.bincount(inv, weights=w) / w.sum()
    smp = transfer_matrix_sample(L, J, Jp, h, beta, 40000, np.random.default_rng(5))
    a, b, c = ss_counts_batch(smp.reshape(len(smp), -1), L)
    obs = np.bincount(np.searchsorted(uk, (a + 64) * 10000 + (b + 64) * 100 + (c + 32)),
                      minlength=len(uk)).astype(float)
    e = p * len(smp)
    m = e >= 5
    stat = ((obs[m] - e[m]) ** 2 / e[m]).sum() + (obs[~m].sum() - e[~m].sum()) ** 2 / max(e[~m].sum(), 1e-9)
    assert chi2.sf(stat, m.sum()) > 1e-3, stat


def test_transfer_matrix_matches_enumeration_L4():
    """The transfer-matrix helper against brute-force enumeration on L=4."""
    from ss_geometry import ss_counts_batch
    L, J, Jp, h, beta = 4, 1.0, 1.5, 0.5, 0.7
    x = np.arange(1 << 16)
    V = ((x[:, None] >> np.arange(16)) & 1) * 2 - 1
    nJ, nJp, M = ss_counts_batch(V, L)
    E = J * nJ + Jp * nJp - h * M
    w = np.exp(-beta * (E - E.min()))
    w /= w.sum()
    ex = transfer_matrix_moments(L, J, Jp, h, beta)
    assert np.isclose(ex["E"], (w * E).sum(), rtol=1e-10)
    assert np.isclose(ex["E2"], (w * E * E).sum(), rtol=1e-10)
    assert np.isclose(ex["M"], (w * M).sum(), atol=1e-10)
    assert np.isclose(ex["M2"], (w * M * M).sum(), rtol=1e-10)


@pytest.mark.parametrize("J,Jp,h,closed", [(1.0, 1.0, 0.5, -1.5), (1.0, 1.0, 7.0, 2.5 - 7.0),
                                           (1.0, 2.5, 0.0, None)])
def test_cold_sampler_reaches_bruteforce_ground_state(orc, J, Jp, h, closed):
    """Ground-state energy per spin at beta=5 equals the brute-force minimum
    over supercell-periodic states (and the closed forms e_Neel = -2J + J'/2,
    e_FM = 2J + J'/2 - h)."""
    L, N = 6, 36
    e0, _ = supercell_ground_energy(L, J, Jp, h)
    if closed is not None:
        assert np.isclose(e0 / N, closed)
    n_chains, n_sweeps = 32, 1500
    ids = np.arange(n_chains, dtype=np.uint32)
    spins = orc.init_spins(L, ids, seed=3)
    _, series, _ = orc.run(L, {"J": [J], "Jp": [Jp], "h": [h], "beta": [5.0]},
                           np.zeros(n_chains, np.int32), spins, seed=3, sweep0=0,
                           n_sweeps=n_sweeps, measure_every=1, series_cap=n_sweeps)
    E = J * series[..., 0] + Jp * series[..., 1] - h * series[..., 2]
    assert np.isclose(E.min(), e0)
