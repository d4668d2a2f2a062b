"""Pins of the oracle's learned block proposal: back-propagated gradients
against finite differences, the block energy difference against full
energies, and exact stationarity of the Metropolis-Hastings block move."""
import numpy as np
import pytest

from ss_geometry import ss_counts_batch


def _examples(orc, k, n, seed, L=8):
    rng = np.random.default_rng(seed)
    inputs, targets = [], []
    for _ in range(n):
        v = rng.choice(np.array([-1, 1], np.int8), size=(L, L))
        bR, bC = rng.integers(0, L, 2)
        inputs.append(orc.patch_input(v, int(bR), int(bC), k, 1.7, 2.75))
        targets.append(np.array([v[(bR + a) % L, (bC + b) % L] for a in range(k) for b in range(k)],
                                np.int8))
    return np.array(inputs), np.array(targets)


def test_gradient_matches_finite_differences(orc):
    k = 4
    w = orc.random_net(1)
    inputs, targets = _examples(orc, k, 3, 2)
    loss, grad = orc.net_loss_grad(k, w, inputs, targets)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(864, 60, replace=False), 864 + np.arange(16),
                          880 + rng.choice(2304, 80, replace=False), 3184 + np.arange(16),
                          3200 + rng.choice(144, 40, replace=False), [3344]])
    eps = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += eps
        wm[i] -= eps
        fd = (orc.net_loss_grad(k, wp, inputs, targets)[0] -
              orc.net_loss_grad(k, wm, inputs, targets)[0]) / (2 * eps)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, grad[i])


def test_forward_is_translation_equivariant_and_ignores_the_block(orc):
    """q depends only on spins outside the block: changing block spins leaves
    the logits unchanged; shifting the lattice by the SS unit cell (2, 2)
    shifts the patch (parity planes unchanged)."""
    k, L = 4, 12
    w = orc.random_net(5)
    rng = np.random.default_rng(6)
    v = rng.choice(np.array([-1, 1], np.int8), size=(L, L))
    z = orc.net_forward(k, w, orc.patch_input(v, 3, 5, k, 2.0, 3.0))
    v2 = v.copy()
    v2[3:7, 5:9] *= -1
    assert np.array_equal(z, orc.net_forward(k, w, orc.patch_input(v2, 3, 5, k, 2.0, 3.0)))
    vs = np.roll(v, (2, 2), axis=(0, 1))
    assert np.allclose(z, orc.net_forward(k, w, orc.patch_input(vs, 5, 7, k, 2.0, 3.0)), atol=1e-12)


def test_block_delta_e_matches_full_energy(orc):
    rng = np.random.default_rng(7)
    for L in (4, 6, 10):
        for _ in range(30):
            v = rng.choice(np.array([-1, 1], np.int8), size=(L, L))
            k = int(rng.integers(1, 5)) if L > 4 else 2
            bR, bC = rng.integers(0, L, 2)
            nb = rng.choice(np.array([-1, 1], np.int8), size=k * k)
            v2 = v.copy()
            for a in range(k):
                for b in range(k):
                    v2[(bR + a) % L, (bC + b) % L] = nb[a * k + b]
            J, Jp, h = 1.0, 1.5, 0.6875
            e = [16 * (J * x + Jp * y - h * m) for x, y, m in
                 zip(*ss_counts_batch(np.stack([v.reshape(-1), v2.reshape(-1)]), L))]
            assert orc.block_delta_e(v, int(bR), int(bC), nb, J, Jp, h) == round(e[1] - e[0])


@pytest.mark.parametrize("origin,use_bf16", [((0, 0), False), ((1, 1), True), ((2, 1), False)])
def test_mh_block_move_is_exactly_stationary(orc, origin, use_bf16):
    """L=4 periodic, 2x2 block, random net: sum_x pi(x) K(x -> y) = pi(y) over
    all 2^16 states, with pi from the SS energies of the test's own geometry."""
    L, k = 4, 2
    J, Jp, h, beta = 1.0, 1.5, 0.3125, 0.7
    w = orc.random_net(11, scale=0.15)
    x = np.arange(1 << 16, dtype=np.int64)
    V = (((x[:, None] >> np.arange(16)) & 1) * 2 - 1).astype(np.int8)
    nJ, nP, M = ss_counts_batch(V, L)
    E = J * nJ + Jp * nP - h * M
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    rows = orc.mh_rows(V.reshape(-1, L, L), origin[0], origin[1], k, w, J, Jp, h, beta, use_bf16)
    assert np.allclose(rows.sum(1), 1.0, atol=1e-12) and (rows >= -1e-15).all()
    sites = [((origin[0] + a) % L) * L + (origin[1] + b) % L for a in range(k) for b in range(k)]
    base = x.copy()
    for s in sites:
        base &= ~(1 << s)
    target = np.zeros_like(rows, dtype=np.int64)
    for b in range(1 << (k * k)):
        t = base.copy()
        for j, s in enumerate(sites):
            t |= ((b >> j) & 1) << s
        target[:, b] = t
    flow = np.zeros(1 << 16)
    np.add.at(flow, target.reshape(-1), (pi[:, None] * rows).reshape(-1))
    assert np.abs(flow - pi).max() < 1e-14, np.abs(flow - pi).max()
    # a real move happens: the net does not propose the current block surely
    assert (1 - rows[np.arange(len(rows)), ((V[:, sites] > 0) << np.arange(4)).sum(1)]).mean() > 0.05


def _pass_setup(orc, L=12, n=24, seed=31):
    rng = np.random.default_rng(seed)
    params = dict(J=[1.0, 1.0], Jp=[1.0, 1.5], h=[3.0, 0.5], beta=[0.6, 1.3])
    cp = rng.integers(0, 2, n).astype(np.int32)
    spins = rng.choice(np.array([-1, 1], np.int8), size=(n, L, L))
    return params, cp, spins


def test_pass_matches_the_pinned_transition_kernel(orc):
    """Each record of a pass is one draw of the block move whose exact kernel
    orc_mh_row enumerates (and which the L=4 test above pins by exact
    stationarity): for the proposed block y != x, q(y) min(1, exp(log alpha))
    equals the kernel entry K(x -> y); the origin, current block and dE agree
    with the lattice."""
    L = 12
    params, cp, spins = _pass_setup(orc, L)
    w = orc.random_net(17, scale=0.15)
    rec = orc.prop_pass(spins.copy(), params, cp, w, seed=5, pass_index=3)
    assert rec.shape == (1, len(cp))
    for c in range(8):
        r = rec[0, c]
        p = cp[c]
        bR, bC = int(r["bR"]), int(r["bC"])
        cur = sum(1 << s for s in range(16) if spins[c, (bR + s // 4) % L, (bC + s % 4) % L] > 0)
        assert int(r["cur_bits"]) == cur
        nb = np.array([1 if (int(r["new_bits"]) >> s) & 1 else -1 for s in range(16)], np.int8)
        assert int(r["dE"]) == orc.block_delta_e(spins[c], bR, bC, nb, params["J"][p],
                                                 params["Jp"][p], params["h"][p])
        if int(r["new_bits"]) == cur:
            continue
        pr = r["thr"].astype(np.float64) / 2.0 ** 32
        bits = (int(r["new_bits"]) >> np.arange(16)) & 1
        q_new = np.prod(np.where(bits == 1, pr, 1 - pr))
        k = orc.mh_rows(spins[c][None], bR, bC, 4, w, params["J"][p], params["Jp"][p],
                        params["h"][p], params["beta"][p], use_bf16=True)[0]
        ours = q_new * min(1.0, np.exp(r["log_alpha"]))
        assert abs(ours - k[int(r["new_bits"])]) <= 1e-12 * k[int(r["new_bits"])] + 1e-300, (c, ours)


def test_pass_draws_and_accepts_follow_their_laws(orc):
    """With the logits fixed, each site of a proposal is +1 with probability
    t_s / 2^32 independently of the other sites, and a move is accepted with
    probability min(1, exp(log alpha)): binomial checks of every site and
    every pair of sites over 2000 chains x 16 passes (a Philox word shared by
    two sites fails the pair check)."""
    from scipy.stats import chi2
    L, n, passes = 12, 2000, 16
    params, cp, spins = _pass_setup(orc, L, n, seed=4)
    rng = np.random.default_rng(8)
    logits = rng.normal(0.0, 1.5, (1, n, 16))
    ones = np.zeros(16)
    pair = np.zeros((16, 16))              # sites s and s' both +1
    acc, exp_acc, var_acc = 0, 0.0, 0.0
    p_exp = None
    for ps in range(passes):
        rec = orc.prop_pass(spins.copy(), params, cp, None, seed=9, pass_index=ps, logits=logits)[0]
        bits = ((rec["new_bits"][:, None] >> np.arange(16)) & 1).astype(np.float64)
        ones += bits.sum(0)
        pair += bits.T @ bits
        pr = rec["thr"].astype(np.float64) / 2.0 ** 32
        if p_exp is None:
            p_exp = pr
        assert np.array_equal(pr, p_exp)   # same logits -> same thresholds
        a = np.minimum(1.0, np.exp(rec["log_alpha"]))
        acc += int(rec["accept"].sum())
        exp_acc += a.sum()
        var_acc += (a * (1 - a)).sum()
    e1 = p_exp.sum(0) * passes
    v1 = (p_exp * (1 - p_exp)).sum(0) * passes
    stat = ((ones - e1) ** 2 / v1).sum()
    assert chi2.sf(stat, 16) > 1e-3, stat
    iu = np.triu_indices(16, 1)
    pp = p_exp[:, :, None] * p_exp[:, None, :]
    e2 = pp.sum(0)[iu] * passes
    v2 = (pp * (1 - pp)).sum(0)[iu] * passes
    stat2 = ((pair[iu] - e2) ** 2 / v2).sum()
    assert chi2.sf(stat2, len(e2)) > 1e-3, stat2
    assert abs(acc - exp_acc) < 4 * np.sqrt(var_acc), (acc, exp_acc, var_acc)


def test_pass_applies_exactly_the_accepted_moves(orc):
    """apply = 1 writes the proposed block of every accepted record and
    nothing else; each chain's energy changes by the sum of its accepted dE
    (full SS energies of the test's own geometry, two blocks per side at
    L = 18 so the moves of a pass must not interfere)."""
    L = 18
    params, cp, spins = _pass_setup(orc, L, n=40, seed=6)
    w = orc.random_net(2, scale=0.1)
    before = spins.copy()
    rec = orc.prop_pass(spins, params, cp, w, seed=3, pass_index=11, apply=True)
    assert rec.shape == (4, 40)
    assert rec["accept"].any() and not rec["accept"].all()
    expect = before.copy()
    for b in range(4):
        for c in range(40):
            r = rec[b, c]
            if r["accept"]:
                for s in range(16):
                    expect[c, (r["bR"] + s // 4) % L, (r["bC"] + s % 4) % L] = \
                        1 if (int(r["new_bits"]) >> s) & 1 else -1
    assert np.array_equal(spins, expect)
    q = lambda x: round(16 * x)
    for c in range(40):
        p = cp[c]
        (a0, b0, m0), (a1, b1, m1) = [tuple(x[0] for x in ss_counts_batch(st.reshape(1, -1), L))
                                      for st in (before[c], spins[c])]
        e0 = q(params["J"][p]) * a0 + q(params["Jp"][p]) * b0 - q(params["h"][p]) * m0
        e1 = q(params["J"][p]) * a1 + q(params["Jp"][p]) * b1 - q(params["h"][p]) * m1
        assert e1 - e0 == int(rec["dE"][:, c][rec["accept"][:, c] == 1].sum())
    # origins: two per side, spaced L / 2 apart
    assert len(set(rec["bR"][:, 0])) == 2 and len(set(rec["bC"][:, 0])) == 2
    assert (rec["bR"][2, 0] - rec["bR"][0, 0]) % L == 9 and (rec["bC"][1, 0] - rec["bC"][0, 0]) % L == 9
