"""Pins of the oracle's parallel tempering: replica exchange must leave every
rung's marginal equal to the Boltzmann law at that rung's beta (detailed
balance of the swap move), and the swap thresholds must match the closed form."""
import math

import numpy as np
import pytest
from scipy.stats import chi2

from test_oracle_sampler import _exact_L3


def ladder_params(betas, J=1.0, Jp=1.5, h=0.6875):
    n = len(betas)
    return dict(J=[J] * n, Jp=[Jp] * n, h=[h] * n, beta=list(betas))


def chi2_pvalue(obs, p):
    n = obs.sum()
    exp = p * n
    order = np.argsort(exp)
    o_b, e_b, ao, ae = [], [], 0.0, 0.0
    for i in order:
        ao += obs[i]
        ae += exp[i]
        if ae >= 5:
            o_b.append(ao)
            e_b.append(ae)
            ao = ae = 0.0
    if ae > 0:
        o_b[-1] += ao
        e_b[-1] += ae
    o_b, e_b = np.array(o_b), np.array(e_b)
    return chi2.sf(((o_b - e_b) ** 2 / e_b).sum(), len(o_b) - 1)


@pytest.mark.slow
def test_tempering_preserves_each_rung_marginal(orc):
    L, n_lad = 3, 1500
    betas = 0.1 * (20.0 ** (np.arange(32) / 31.0))          # geometric in [0.1, 2]
    params = ladder_params(betas)
    cp = np.tile(np.arange(32, dtype=np.int32), n_lad)
    ids = np.arange(32 * n_lad, dtype=np.uint32)
    spins = orc.init_spins(L, ids, 17)
    sob = np.tile(np.arange(32, dtype=np.int32), (n_lad, 1))
    orc.run_pt(L, params, cp, spins, sob, 17, 0, 300, measure_every=0, swap_every=2,
               periodic=False)
    assert (sob != np.arange(32)).any(1).mean() > 0.9              # the ladders do exchange
    for k in (0, 8, 16, 24, 31):
        conf = spins[np.arange(n_lad) * 32 + sob[:, k]]            # rung k of every ladder
        bits = ((conf.reshape(n_lad, 9) > 0).astype(np.int64) << np.arange(9)).sum(1)
        p = _exact_L3(orc, False, 1.0, 1.5, 0.6875, betas[k])
        assert chi2_pvalue(np.bincount(bits, minlength=512).astype(float), p) > 1e-3, k


def test_tempering_with_wrong_swap_sign_would_fail(orc):
    """Sanity of the test: a ladder whose rungs held the configurations of the
    neighbouring beta fails the chi-square at a cold rung."""
    p_true = _exact_L3(orc, False, 1.0, 1.5, 0.6875, 2.0)
    p_wrong = _exact_L3(orc, False, 1.0, 1.5, 0.6875, 1.6)
    obs = np.random.default_rng(3).multinomial(1500, p_wrong).astype(float)
    assert chi2_pvalue(obs, p_true) < 1e-4


def test_swap_threshold_closed_form(orc):
    for x in (-1e-9, -0.5, -3.0, -20.0, -25.0, -700.0):
        t = orc.swap_threshold(x)
        assert abs(t - min(2.0**32 - 1, 2.0**32 * math.exp(x))) <= 0.5 + 1e-9
    assert orc.swap_threshold(-30.0) == 0


def test_tempering_measures_per_rung(orc):
    """Sums rows follow the rungs: row 32 l + k always holds rung k's
    configuration, whichever slot carries it."""
    L, n_lad = 6, 2
    betas = 0.2 * (50.0 ** (np.arange(32) / 31.0))
    params = ladder_params(betas, 1.0, 1.5, 1.0)
    cp = np.tile(np.arange(32, dtype=np.int32), n_lad)
    spins = orc.init_spins(L, np.arange(64, dtype=np.uint32), 4)
    sob = np.tile(np.arange(32, dtype=np.int32), (n_lad, 1))
    # swaps after sweeps 10, 20, 30; the measurement (after sweep 35) sees the final rungs
    sums, ser = orc.run_pt(L, params, cp, spins, sob, 4, 0, 35, measure_every=35, swap_every=10,
                           series_cap=1)
    assert (sob != np.arange(32)).any()
    for l in range(n_lad):
        for k in range(32):
            nJ, nP, M = orc.counts(spins[32 * l + sob[l, k]], L)
            assert tuple(ser[32 * l + k, 0]) == (nJ, nP, M)
            assert sums[32 * l + k, 0] == 1 and sums[32 * l + k, 3] == M
