"""Pins of the oracle's paper-precision mode (Sec. III, "Dimension and
Precision"): 10-bit weights and visible bias with 4 fraction bits, a 12-bit
accumulator, a 16-bit sigmoid table and 16-bit uniforms, two per Philox word.

What fixes it, independently of the oracle's own formulas: the sigmoid's
symmetry and monotonicity, the size of a quantisation step, and the law the
chain must sample -- block Gibbs with weights A/16 is exact for the Ising model
whose couplings are 1/2 ln cosh(2 A / 16) (the identity of Eqs. 5-7 read
backwards), so the chain's histogram on L=3 must follow that quantised model
and must not follow the unquantised one."""
import math

import numpy as np
import pytest
from scipy.stats import chi2

PAPER = 1


def test_lut16_is_a_16_bit_sigmoid(orc):
    acc = np.arange(-2100, 2101)
    t = np.array([orc.lut16(int(a)) for a in acc], np.uint64)
    assert (t & 0xFFFF).max() == 0                         # 16-bit values in the upper half
    t16 = t >> 16
    assert (np.diff(t16.astype(np.int64)) >= 0).all()      # monotone in the accumulator
    assert t16[acc == 0][0] == 32768                       # sigmoid(0) = 1/2
    mirror = t16 + t16[::-1]                               # sigma(y) + sigma(-y) = 1
    assert set(np.unique(mirror)) <= {65535, 65536}
    assert t16[acc == 2047][0] == t16[-1] == 65535         # 12-bit accumulator saturates
    assert t16[acc == -2047][0] == t16[0] == 0
    # one step of 1/16 in the accumulator moves the probability by at most
    # the sigmoid's largest slope (1/2 per unit of 2y) times 2/16, plus rounding
    assert np.abs(np.diff(t16.astype(np.int64))).max() <= 65536 * 2 / 16 / 4 + 1


def test_q54_steps_and_saturation(orc):
    for x in np.linspace(-31.9, 31.9, 997):
        q = orc.q54(x)
        assert abs(q / 16.0 - x) <= 1.0 / 32 + 1e-12
    assert orc.q54(40.0) == 511 and orc.q54(-40.0) == -511
    assert orc.q54(0.03125 + 1e-9) == 1 and orc.q54(-0.03125 - 1e-9) == -1


@pytest.mark.parametrize("J,Jp,h,beta", [(1.0, 1.0, 3.0, 2.0), (1.0, 1.5, 0.6875, 0.8),
                                         (-0.5, 2.0, -1.25, 1.3), (2.0, 0.25, 0.0, 0.4)])
def test_paper_tables_stay_within_the_quantisation_error(orc, J, Jp, h, beta):
    """Each entry is the exact conditional probability up to one quantisation
    step of its weights (slope of sigma(2y) <= 1/2 per unit of y) and the
    16-bit rounding."""
    L = 18
    th_e, tv_e = orc.tables(L, J, Jp, h, beta)
    th_p, tv_p = orc.tables(L, J, Jp, h, beta, precision=PAPER)
    dj, djp = orc.degrees(L)
    for cls in range(2):
        for m in range(-2, 3):
            dp = abs(int(th_p[cls, m + 2]) - int(th_e[cls, m + 2])) / 2.0**32
            assert dp <= 0.5 * abs(m) / 32 + 2.0**-16, (cls, m, dp)
    for nJ in range(-dj, dj + 1):
        for nJp in range(-djp, djp + 1):
            dp = abs(int(tv_p[nJ + dj, nJp + djp]) - int(tv_e[nJ + dj, nJp + djp])) / 2.0**32
            assert dp <= 0.5 * (1 + abs(nJ) + abs(nJp)) / 32 + 2.0**-16, (nJ, nJp, dp)


def _L3_law(orc, KJ, KP, B):
    L, N = 3, 9
    x = np.arange(1 << N)
    V = (((x[:, None] >> np.arange(N)) & 1) * 2 - 1).astype(np.int8)
    c = np.array([orc.counts(V[i].reshape(L, L), L, periodic=False) for i in range(len(V))], float)
    lw = KJ * c[:, 0] + KP * c[:, 1] + B * c[:, 2]
    w = np.exp(lw - lw.max())
    return w / w.sum()


def _chi2_p(obs, p):
    exp = p * obs.sum()
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
def test_paper_chain_samples_the_quantised_model(orc):
    """L=3 open, beta=0.8, J=1, J'=1.5, h=0.6875: a_J = 1.141 and a_J' = 1.546
    become 18/16 and 25/16, beta h = 0.55 becomes 9/16.  The paper-precision
    chain must sample exp(K_J N_J + K_J' N_J' + B M) with
    K = -1/2 ln cosh(2 A / 16) and B = 9/16, not the exact model."""
    L, n_chains, beta, J, Jp, h = 3, 30000, 0.8, 1.0, 1.5, 0.6875
    aJ, sJ = orc.weight(beta, J)
    aP, sP = orc.weight(beta, Jp)
    AJ, AP, B = orc.q54(aJ), orc.q54(aP), orc.q54(beta * h)
    assert (AJ, AP, B) == (18, 25, 9)
    q_model = _L3_law(orc, sJ * 0.5 * math.log(math.cosh(2 * AJ / 16)),
                      sP * 0.5 * math.log(math.cosh(2 * AP / 16)), B / 16)
    exact = _L3_law(orc, -beta * J, -beta * Jp, beta * h)
    ids = np.arange(n_chains, dtype=np.uint32) + 3 * n_chains
    spins = orc.init_spins(L, ids, seed=21)
    orc.run(L, {"J": [J], "Jp": [Jp], "h": [h], "beta": [beta]}, np.zeros(n_chains, np.int32),
            spins, seed=21, sweep0=0, n_sweeps=400, measure_every=0, chain_ids=ids,
            periodic=False, precision=PAPER)
    bits = ((spins.reshape(n_chains, 9) > 0).astype(np.int64) << np.arange(9)).sum(1)
    obs = np.bincount(bits, minlength=512).astype(float)
    assert _chi2_p(obs, q_model) > 1e-3
    assert _chi2_p(obs, exact) < 1e-6


def test_paper_mode_uses_two_uniforms_per_word(orc):
    """One hidden decision per 16-bit half: with every threshold at 1/2 (beta
    = 0, h = 0) a unit is +1 iff its half-word is below 2^15, so the spins
    after one sweep are the top bits of the named halves of the tag-1 words."""
    L, n = 4, 6
    ids = np.arange(n, dtype=np.uint32)
    spins = orc.init_spins(L, ids, seed=5)
    orc.run(L, {"J": [1.0], "Jp": [1.0], "h": [0.0], "beta": [0.0]}, np.zeros(n, np.int32), spins,
            seed=5, sweep0=0, n_sweeps=1, measure_every=0, chain_ids=ids, precision=PAPER)
    W = 2
    for c in range(n):
        for R in range(L):
            for C in range(L):
                x = 2 * (R & 1) + (C & 1)
                word = orc.philox([(R >> 1) * W + (C >> 1), 0, c, 1], [5, 0])[1 + (x >> 1)]
                u16 = (word >> 16) if (x & 1) else (word & 0xFFFF)
                assert spins[c, R, C] == (1 if u16 < 0x8000 else -1), (c, R, C)
