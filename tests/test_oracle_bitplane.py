"""Pins of the oracle's bit-plane uniforms (ORC_RNG_BITPLANE): the uniforms of
a group of 32 chains at one node are the bit-transpose of shared Philox
words, most significant plane first, so that a word-parallel comparison can
stop once all 32 chains are decided.

Fixed independently of the oracle's own assembly: with J = J' = 0 every spin
update is a single comparison against the field threshold, so each spin after
one sweep is read straight off the named Philox words (computed here from the
Philox function, not the oracle's bit-plane code); and the chain's law on a
periodic L=4 lattice (the histogram of (N_J, N_J', M) against enumeration of
all 2^16 states), which a plane shared by two nodes would bias."""
import numpy as np
import pytest

from test_oracle_paper_precision import _chi2_p

TAG = 256
PAPER = 1


def planes_uniform(orc, seed, cell, sweep, chain, node):
    """u of `chain` at `node`: bit chain % 32 of plane b is bit 31 - b of u."""
    u = 0
    for j in range(8):
        words = orc.philox([cell, sweep, chain // 32, TAG + 8 * node + j], [seed & 0xFFFFFFFF, seed >> 32])
        for i in range(4):
            u |= ((int(words[i]) >> (chain % 32)) & 1) << (31 - (4 * j + i))
    return u


@pytest.mark.parametrize("beta,h", [(0.7, 0.45), (0.0, 0.0), (2.0, -0.3125)])
def test_spins_follow_their_bit_planes(orc, beta, h):
    L, n, seed = 6, 70, 12345
    ids = np.arange(n, dtype=np.uint32)
    spins = orc.init_spins(L, ids, seed)
    params = {"J": [0.0], "Jp": [0.0], "h": [h], "beta": [beta]}
    _, tv = orc.tables(L, 0.0, 0.0, h, beta)
    t = int(tv.reshape(-1)[0])
    assert (tv == t).all()                      # no coupling: one visible threshold
    orc.run(L, params, np.zeros(n, np.int32), spins, seed, 0, 1, 0, chain_ids=ids, rng=orc.RNG_BITPLANE)
    W = L // 2
    for c in range(n):
        for R in range(L):
            for C in range(L):
                x = 2 * (R & 1) + (C & 1)
                u = planes_uniform(orc, seed, (R // 2) * W + C // 2, 0, c, 10 + x)
                assert spins[c, R, C] == (1 if u < t else -1), (c, R, C)


def test_bitplane_differs_from_the_lane_streams(orc):
    L, n, seed = 6, 64, 9
    params = {"J": [1.0], "Jp": [1.5], "h": [0.5], "beta": [0.8]}
    ids = np.arange(n, dtype=np.uint32)
    a, b = orc.init_spins(L, ids, seed), orc.init_spins(L, ids, seed)
    orc.run(L, params, np.zeros(n, np.int32), a, seed, 0, 3, 0, chain_ids=ids)
    orc.run(L, params, np.zeros(n, np.int32), b, seed, 0, 3, 0, chain_ids=ids, rng=orc.RNG_BITPLANE)
    assert not np.array_equal(a, b)
    with pytest.raises(ValueError):             # bit planes carry the exact 32-bit thresholds only
        orc.run(L, params, np.zeros(n, np.int32), b, seed, 0, 1, 0, chain_ids=ids, precision=PAPER,
                rng=orc.RNG_BITPLANE)


@pytest.mark.slow
@pytest.mark.parametrize("J,Jp,h,beta", [(1.0, 1.5, 0.6875, 0.4), (-0.5, 1.0, 0.25, 0.6)])
def test_bitplane_chain_samples_boltzmann_L4(orc, J, Jp, h, beta):
    """Periodic L=4: final (N_J, N_J', M) of 12000 chains after 120 sweeps
    against the enumerated law of exp(-beta H)."""
    L, N, n = 4, 16, 12000
    x = np.arange(1 << N)
    V = (((x[:, None] >> np.arange(N)) & 1) * 2 - 1).astype(np.int8).reshape(-1, L, L)
    c = np.array([orc.counts(v, L) for v in V])
    E = J * c[:, 0] + Jp * c[:, 1] - h * c[:, 2]
    w = np.exp(-beta * (E - E.min()))
    keys, inv = np.unique(c, axis=0, return_inverse=True)
    p = np.bincount(inv.reshape(-1), weights=w) / w.sum()
    ids = np.arange(n, dtype=np.uint32)
    spins = orc.init_spins(L, ids, 77)
    orc.run(L, {"J": [J], "Jp": [Jp], "h": [h], "beta": [beta]}, np.zeros(n, np.int32), spins, 77, 0, 120, 0,
            chain_ids=ids, rng=orc.RNG_BITPLANE)
    got = np.array([orc.counts(v, L) for v in spins])
    idx = {tuple(k): i for i, k in enumerate(keys)}
    obs = np.bincount([idx[tuple(g)] for g in got], minlength=len(keys)).astype(float)
    assert _chi2_p(obs, p) > 1e-3


def test_bitplane_tempering_without_swaps_is_the_plain_chain(orc):
    """Replica exchange whose first swap round lies beyond the run leaves every
    replica on its rung, so each replica is the plain bit-plane chain of its
    index: the ladder plumbing of the bit-plane mode against the pinned sampler."""
    L, n = 6, 64
    betas = list(0.3 * (10.0 ** (np.arange(32) / 31.0)))
    params = dict(J=[1.0] * 32, Jp=[1.5] * 32, h=[0.5] * 32, beta=betas)
    cp = np.tile(np.arange(32, dtype=np.int32), 2)
    ids = np.arange(n, dtype=np.uint32)
    a, b = orc.init_spins(L, ids, 8), orc.init_spins(L, ids, 8)
    sob = np.tile(np.arange(32, dtype=np.int32), (2, 1))
    orc.run_pt(L, params, cp, a, sob, 8, 0, 12, 0, swap_every=100, rng=orc.RNG_BITPLANE)
    orc.run(L, params, cp, b, 8, 0, 12, 0, chain_ids=ids, rng=orc.RNG_BITPLANE)
    assert np.array_equal(a, b)
    c = orc.init_spins(L, ids, 8)                # and the swaps change the trajectory once they start
    orc.run_pt(L, params, cp, c, np.tile(np.arange(32, dtype=np.int32), (2, 1)), 8, 0, 12, 0, swap_every=3,
               rng=orc.RNG_BITPLANE)
    assert not np.array_equal(a, c)
