"""Pins of the oracle on rectangular lattices with a boundary per axis and an
odd-column field (Sec. III: laterally confined strips with open boundaries
along one axis; appendix: separate odd- and even-column visible biases).

Fixed independently of the oracle's window code: a periodic rectangle of even
sides is still the SS lattice (closed-form counts); opening one axis removes
exactly the bonds that cross that seam; the marginal identity of Eq. (3) with
a column-dependent field; and the sampler's histogram on a small strip."""
import numpy as np
import pytest
from scipy.stats import chi2

from test_oracle_paper_precision import _chi2_p


@pytest.mark.parametrize("Lr,Lc", [(4, 6), (6, 4), (8, 10), (6, 12)])
def test_periodic_rectangle_is_shastry_sutherland(orc, Lr, Lc):
    N = Lr * Lc
    fm = np.ones((Lr, Lc), np.int8)
    assert orc.counts(fm, (Lr, Lc)) == (2 * N, N // 2, N)
    neel = np.fromfunction(lambda r, c: 1 - 2 * ((r + c) % 2), (Lr, Lc)).astype(np.int8)
    assert orc.counts(neel, (Lr, Lc)) == (-2 * N, N // 2, 0)
    assert orc.degrees((Lr, Lc)) == (4, 1)


def _seam_terms(v, Lr, Lc):
    """Bonds of the periodic SS rectangle that cross the column seam (between
    column Lc-1 and column 0): every row's horizontal J bond, and the J'
    dimers '/' of the plaquettes (2i+1, Lc-1)-(2i+2, Lc) that wrap."""
    nJ = sum(int(v[R, Lc - 1]) * int(v[R, 0]) for R in range(Lr))
    nP = sum(int(v[(2 * i + 1) % Lr, 0]) * int(v[(2 * i + 2) % Lr, Lc - 1]) for i in range(Lr // 2))
    return nJ, nP


def _row_seam_terms(v, Lr, Lc):
    nJ = sum(int(v[Lr - 1, C]) * int(v[0, C]) for C in range(Lc))
    nP = sum(int(v[0, (2 * j + 1) % Lc]) * int(v[Lr - 1, (2 * j + 2) % Lc]) for j in range(Lc // 2))
    return nJ, nP


@pytest.mark.parametrize("Lr,Lc", [(4, 6), (6, 12), (8, 4)])
def test_open_axis_removes_exactly_the_seam_bonds(orc, Lr, Lc):
    rng = np.random.default_rng(Lr * 31 + Lc)
    for _ in range(20):
        v = rng.choice(np.array([-1, 1], np.int8), size=(Lr, Lc))
        pj, pp, pm = orc.counts(v, (Lr, Lc), periodic=(True, True))
        sj, sp = _seam_terms(v, Lr, Lc)
        assert orc.counts(v, (Lr, Lc), periodic=(True, False)) == (pj - sj, pp - sp, pm)
        rj, rp = _row_seam_terms(v, Lr, Lc)
        assert orc.counts(v, (Lr, Lc), periodic=(False, True)) == (pj - rj, pp - rp, pm)


def _units(Lr, Lc, pr, pc, bonds):
    Wr, Wc = (Lr + 1) // 2, (Lc + 1) // 2
    out = []
    for i in range(Wr):
        for j in range(Wc):
            for (r1, c1, r2, c2, cls) in bonds:
                def site(r, c):
                    R, C = 2 * i + r, 2 * j + c
                    if R >= Lr:
                        if not pr:
                            return None
                        R %= Lr
                    if C >= Lc:
                        if not pc:
                            return None
                        C %= Lc
                    return R * Lc + C
                out.append((site(r1, c1), site(r2, c2), cls))
    return out


@pytest.mark.parametrize("Lr,Lc,pr,pc", [(4, 3, True, False), (3, 4, False, True), (4, 4, True, False)])
def test_marginal_identity_with_odd_column_field(orc, Lr, Lc, pr, pc):
    """Eq. (3) with the visible bias beta h on even columns and beta h_odd on
    odd ones: sum_h P(v, h) is proportional to exp(-beta H(v)),
    H = J N_J + J' N_J' - h M_even - h_odd M_odd."""
    J, Jp, h, h_odd, beta = 1.0, 1.5, 0.6875, -1.25, 0.9
    N = Lr * Lc
    w = {0: orc.weight(beta, J), 1: orc.weight(beta, Jp)}
    x = np.arange(1 << N, dtype=np.int64)
    V = ((x[:, None] >> np.arange(N)) & 1) * 2 - 1
    odd = (np.arange(N) % Lc) % 2 == 1
    logmarg = beta * (h * V[:, ~odd].sum(1) + h_odd * V[:, odd].sum(1)).astype(float)
    for s1, s2, cls in _units(Lr, Lc, pr, pc, orc.canonical_bonds()):
        a, s = w[cls]
        m = (V[:, s1] if s1 is not None else 0) + s * (V[:, s2] if s2 is not None else 0)
        logmarg = logmarg + np.log(2 * np.cosh(a * m))
    H = np.empty(len(V))
    for idx in range(len(V)):
        nJ, nJp, _ = orc.counts(V[idx].astype(np.int8).reshape(Lr, Lc), (Lr, Lc), periodic=(pr, pc))
        H[idx] = J * nJ + Jp * nJp - h * V[idx, ~odd].sum() - h_odd * V[idx, odd].sum()
    diff = logmarg + beta * H
    assert diff.max() - diff.min() < 1e-10


@pytest.mark.slow
def test_strip_sampler_with_odd_column_field(orc):
    """30000 chains on a 4 x 3 strip (rows periodic, columns open) with
    different fields on even and odd columns: final states against the
    enumerated exp(-beta H) / Z; a sampler that ignored h_odd would fail."""
    Lr, Lc, n = 4, 3, 30000
    J, Jp, h, h_odd, beta = 1.0, 1.5, 0.6875, -1.25, 0.8
    N = Lr * Lc
    x = np.arange(1 << N)
    V = (((x[:, None] >> np.arange(N)) & 1) * 2 - 1).astype(np.int8)
    odd = (np.arange(N) % Lc) % 2 == 1
    c = np.array([orc.counts(V[i].reshape(Lr, Lc), (Lr, Lc), periodic=(True, False)) for i in range(len(V))])

    def law(ho):
        E = J * c[:, 0] + Jp * c[:, 1] - h * V[:, ~odd].sum(1) - ho * V[:, odd].sum(1)
        wgt = np.exp(-beta * (E - E.min()))
        return wgt / wgt.sum()

    ids = np.arange(n, dtype=np.uint32) + 5 * n
    spins = orc.init_spins((Lr, Lc), ids, 31)
    orc.run((Lr, Lc), {"J": [J], "Jp": [Jp], "h": [h], "h_odd": [h_odd], "beta": [beta]},
            np.zeros(n, np.int32), spins, 31, 0, 300, 0, chain_ids=ids, periodic=(True, False))
    bits = ((spins.reshape(n, N) > 0).astype(np.int64) << np.arange(N)).sum(1)
    obs = np.bincount(bits, minlength=1 << N).astype(float)
    assert _chi2_p(obs, law(h_odd)) > 1e-3
    assert _chi2_p(obs, law(h)) < 1e-6
