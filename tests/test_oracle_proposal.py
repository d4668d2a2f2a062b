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
