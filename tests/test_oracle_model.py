"""Pins of the oracle's lattice, weights and threshold tables against closed
forms and the SS geometry (arXiv 2511.20911, Eq. 1, Eqs. 4-7, Eqs. 9-10)."""
import itertools
import math

import numpy as np
import pytest
from scipy.special import expit

from ss_geometry import ss_counts_batch, ss_pairs


@pytest.mark.parametrize("L", [4, 6, 8, 18])
def test_closed_form_counts(orc, L):
    N = L * L
    up = np.ones((L, L), np.int8)
    assert orc.counts(up, L) == (2 * N, N // 2, N)                 # FM
    R, C = np.indices((L, L))
    neel = np.where((R + C) % 2 == 0, 1, -1).astype(np.int8)
    assert orc.counts(neel, L) == (-2 * N, N // 2, 0)              # Neel: diagonals same sublattice
    stripes = np.where(R % 2 == 0, 1, -1).astype(np.int8)
    assert orc.counts(stripes, L) == (0, -N // 2, 0)               # row stripes
    for s in range(N):                                             # every site: 4 nn + 1 diagonal
        v = up.copy().reshape(-1)
        v[s] = -1
        assert orc.counts(v.reshape(L, L), L) == (2 * N - 8, N // 2 - 2, N - 2)


@pytest.mark.parametrize("L", [4, 6])
def test_bond_adjacency_is_shastry_sutherland(orc, L):
    """Pair flips recover the full J and J' adjacency, compared with the SS
    geometry (square lattice + orthogonal dimers on alternating plaquettes)."""
    N = L * L
    nn, dia = ss_pairs(L)
    AJ = np.zeros((N, N), int)
    AD = np.zeros((N, N), int)
    for a, b in nn:
        AJ[a, b] += 1
        AJ[b, a] += 1
    for a, b in dia:
        AD[a, b] += 1
        AD[b, a] += 1
    for s1, s2 in itertools.combinations(range(N), 2):
        v = np.ones(N, np.int8)
        v[s1] = v[s2] = -1
        nJ, nJp, _ = orc.counts(v.reshape(L, L), L)
        # flipping both: each bond to the pair loses 2, a bond inside the pair is unchanged
        assert (2 * N - nJ) == 2 * (4 + 4 - 2 * AJ[s1, s2]), (s1, s2)
        assert (N // 2 - nJp) == 2 * (1 + 1 - 2 * AD[s1, s2]), (s1, s2)
    assert (AD.sum(1) == 1).all() and (AJ.sum(1) == 4).all()


def test_open_L3_bond_count(orc):
    up = np.ones((3, 3), np.int8)
    assert orc.counts(up, 3, periodic=False) == (12, 2, 9)       # 3x3 open: 12 nn, 2 dimers
    assert orc.degrees(3, periodic=False) == (4, 1)
    assert orc.degrees(6) == (4, 1)


def test_random_counts_match_geometry(orc):
    rng = np.random.default_rng(5)
    for L in (4, 6, 10):
        st = rng.choice(np.array([-1, 1], np.int8), size=(20, L * L))
        ref = ss_counts_batch(st, L)
        for i in range(20):
            assert orc.counts(st[i].reshape(L, L), L) == (ref[0][i], ref[1][i], ref[2][i])


@pytest.mark.parametrize("beta,J", [(0.3, 1.0), (2.0, 1.0), (2.0, -1.5), (5.0, 2.0), (0.0, 1.0),
                                    (10.0, 1.5), (1.0, 0.0), (0.7, -0.25)])
def test_weight_closed_form(orc, beta, J):
    a, s = orc.weight(beta, J)
    K = -beta * J
    # cosh(2a) = exp(2|K|)  (Eq. 5 solves exp(K v v') = C sum_h exp(a h (v + s v')))
    assert math.isclose(math.cosh(2 * a), math.exp(2 * abs(K)), rel_tol=1e-13)
    assert s == (1 if K >= 0 else -1)
    # the aligned/anti-aligned ratio of 2cosh(a(v + s v')) is exp(2K)
    r = math.cosh(a * (1 + s)) / math.cosh(a * (1 - s))
    assert math.isclose(r, math.exp(2 * K), rel_tol=1e-12)


def test_threshold_bounds(orc):
    ys = np.concatenate([np.linspace(-30, 30, 601), [0.0, 1e-9, -1e-9, 50.0, -50.0, 700.0]])
    for y in ys:
        t = orc.threshold(y)
        p = expit(y)
        if t < 2**32 - 1:
            assert abs(t / 2**32 - p) <= 2.0**-33 * (1 + 1e-9), y
        else:
            assert p >= 1 - 2.0**-32 * 1.5
    assert orc.threshold(0.0) == 2**31


@pytest.mark.parametrize("pt", [(1.0, 1.0, 0.5, 2.0), (1.0, 2.0, 4.0, 5.0), (1.0, 0.5, 0.0, 0.1),
                                (-1.0, 1.5, -2.0, 0.8)])
def test_tables_match_conditionals(orc, pt):
    J, Jp, h, beta = pt
    th, tv = orc.tables(6, J, Jp, h, beta)
    aJ, _ = orc.weight(beta, J)
    aP, _ = orc.weight(beta, Jp)
    for cls, a in ((0, aJ), (1, aP)):
        for m in range(-2, 3):
            p = expit(2 * a * m)
            assert abs(int(th[cls, m + 2]) / 2**32 - p) <= 2.0**-33 + 2.0**-32 * (p > 1 - 2**-32)
    for nJ in range(-4, 5):
        for nP in range(-1, 2):
            p = expit(2 * (beta * h + aJ * nJ + aP * nP))
            t = int(tv[nJ + 4, nP + 1])
            assert abs(t / 2**32 - p) <= 2.0**-33 + 2.0**-32 * (t == 2**32 - 1)


def test_quantize(orc):
    assert orc.quantize(1.0) == 16 and orc.quantize(-0.5) == -8 and orc.quantize(4.0 / 15) == 4
    with pytest.raises(ValueError):
        orc.quantize(200.0)


def _hidden_units(L, periodic, bonds):
    """(site1, site2, cls) of every hidden unit: the stride-2 windows of the
    wrapper module (periodic copy or zero padding -> None)."""
    W = (L + 1) // 2
    out = []
    for i in range(W):
        for j in range(W):
            for (r1, c1, r2, c2, cls) in bonds:
                def site(r, c):
                    R, C = 2 * i + r, 2 * j + c
                    if R >= L or C >= L:
                        if not periodic:
                            return None
                        R, C = R % L, C % L
                    return R * L + C
                out.append((site(r1, c1), site(r2, c2), cls))
    return out


@pytest.mark.parametrize("L,periodic,J,Jp,h,beta", [(3, False, 1.0, 1.5, 0.6875, 1.3),
                                                    (3, True, 1.0, 1.5, 0.6875, 1.3),
                                                    (4, True, 1.0, 1.0, 0.5, 2.0),
                                                    (4, True, -0.5, 2.0, -1.25, 0.9)])
def test_marginal_identity_enumeration(orc, L, periodic, J, Jp, h, beta):
    """Eq. (3): sum_h P_RBM(v, h) must be proportional to exp(-beta H(v)) for
    all 2^N spin states, with H on the same bond multiset as the RBM."""
    bonds = orc.canonical_bonds()
    units = _hidden_units(L, periodic, bonds)
    N = L * L
    w = {0: orc.weight(beta, J), 1: orc.weight(beta, Jp)}
    x = np.arange(1 << N, dtype=np.int64)
    V = ((x[:, None] >> np.arange(N)) & 1) * 2 - 1
    logmarg = beta * h * V.sum(1).astype(float)
    for s1, s2, cls in units:
        a, s = w[cls]
        m = (V[:, s1] if s1 is not None else 0) + s * (V[:, s2] if s2 is not None else 0)
        logmarg = logmarg + np.log(2 * np.cosh(a * m))
    H = np.empty(len(V))
    for idx in range(len(V)):
        nJ, nJp, M = orc.counts(V[idx].astype(np.int8).reshape(L, L), L, periodic=periodic)
        H[idx] = J * nJ + Jp * nJp - h * M
    diff = logmarg + beta * H
    assert diff.max() - diff.min() < 1e-10
