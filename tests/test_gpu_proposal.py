"""The learned block proposal on the GPU against the oracle: logits of the
tensor-core net vs the oracle's bf16 forward, the exact integer energy change
of every proposed move, training gradients vs the oracle's back-propagation,
the mixed sampler's observables vs plain Gibbs, and what the trained net gains
in effective samples per sweep over plain Gibbs and over the untrained net."""
import numpy as np
import pytest

import paper_2511_20911_gb300 as crbm
from paper_2511_20911_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def bits_to_block(bits):
    return np.array([1 if (int(bits) >> s) & 1 else -1 for s in range(16)], np.int8)


@pytest.mark.parametrize("L", [12, 18])
def test_pass_logits_and_exact_energy_change(orc, L):
    rng = np.random.default_rng(L)
    params = dict(J=[1.0, 1.0, -0.5], Jp=[1.0, 1.5, 2.0], h=[3.0, 0.5, -1.0], beta=[2.0, 0.7, 1.3])
    n = 70
    cp = rng.integers(0, 3, n).astype(np.int32)
    s = crbm.Sampler(L, params, n, chain_param=cp, seed=3, measure_every=0)
    s.sweep(5)
    p = crbm.Proposal(seed=1)
    w = orc.random_net(21, scale=0.15)
    p.weights = w
    rec = p.inspect(s)
    spins = s.get_spins()
    worst = 0.0
    for word in range(rec.shape[0]):
        for b in range(rec.shape[1]):
            for lane in range(32):
                c = 32 * word + lane
                if c >= n:
                    continue
                r = rec[word, b, lane]
                pt = cp[c]
                bR, bC = int(r["bR"]), int(r["bC"])
                cur = np.array([spins[c, (bR + a // 4) % L, (bC + a % 4) % L] for a in range(16)])
                assert np.array_equal(bits_to_block(r["cur_bits"]), cur)
                dE = orc.block_delta_e(spins[c], bR, bC, bits_to_block(r["new_bits"]),
                                       params["J"][pt], params["Jp"][pt], params["h"][pt])
                assert int(r["dE"]) == dE, (word, b, lane)
                inp = orc.patch_input(spins[c], bR, bC, 4, orc.bf16(params["beta"][pt]),
                                      orc.bf16(params["h"][pt]))
                ref = orc.net_forward(4, w, inp, use_bf16=True)
                err = np.abs(r["logit"] - ref) / (0.05 + 0.02 * np.abs(ref))
                worst = max(worst, float(err.max()))
    assert worst <= 1.0, worst


@pytest.mark.parametrize("L,n", [(12, 600), (18, 300)])
def test_pass_matches_the_oracle_element_wise(orc, L, n):
    """Every record of a pass, every chain of every word (the last one
    ragged), against the oracle's pass (orc_prop_pass) on the same spins:
    block origins and current blocks exactly; the GPU's thresholds within
    fp32 rounding of those the oracle derives from the GPU's logits; with the
    GPU's thresholds fed to the oracle, the proposed blocks (the Philox draws
    and their comparisons) and the exact dE bit for bit and log alpha to fp32
    accuracy; then, after the pass itself runs, every block whose accept test
    is not within 1e-3 of its boundary equals the oracle's result (beta = 0.6
    is not a bfloat16 value: the test must use the exact beta)."""
    rng = np.random.default_rng(L + 1)
    params = dict(J=[1.0, 1.0, -0.5], Jp=[1.0, 1.5, 2.0], h=[3.0, 0.5, -1.0], beta=[2.0, 0.6, 0.25])
    cp = rng.integers(0, 3, n).astype(np.int32)
    s = crbm.Sampler(L, params, n, chain_param=cp, seed=3, measure_every=0)
    s.sweep(7)
    p = crbm.Proposal(seed=1)
    w = orc.random_net(21, scale=0.15)
    p.weights = w
    g = p.inspect(s)                                       # [word][block][lane]
    g = g.transpose(1, 0, 2).reshape(g.shape[1], -1)[:, :n]  # [block][chain]
    spins = s.get_spins()
    seed, pass_index = 3, 0
    o_net = orc.prop_pass(spins.copy(), params, cp, w, seed, pass_index)
    o_lg = orc.prop_pass(spins.copy(), params, cp, None, seed, pass_index,
                         logits=g["logit"].astype(np.float64))
    o_thr = orc.prop_pass(spins.copy(), params, cp, None, seed, pass_index,
                          logits=g["logit"].astype(np.float64), thr=g["thr"])
    assert g.shape == o_net.shape == (max(1, L // 8) ** 2, n)
    for f in ("bR", "bC", "cur_bits"):
        assert np.array_equal(g[f].astype(np.int64), o_net[f].astype(np.int64)), f
    err = np.abs(g["logit"] - o_net["logit"]) / (0.05 + 0.02 * np.abs(o_net["logit"]))
    assert err.max() <= 1.0, err.max()
    tg, to = g["thr"].astype(np.float64), o_lg["thr"].astype(np.float64)
    assert (np.abs(tg - to) <= 4096 + tg * 2.0 ** -20).all(), np.abs(tg - to).max()
    assert np.array_equal(g["new_bits"], o_thr["new_bits"])
    assert np.array_equal(g["dE"].astype(np.int64), o_thr["dE"])
    la_err = np.abs(g["log_alpha"] - o_thr["log_alpha"])
    assert (la_err <= 2e-4 + 1e-5 * np.abs(o_thr["log_alpha"])).all(), la_err.max()
    # the pass itself: accept decisions away from the boundary
    after = spins.copy()
    orc.prop_pass(after, params, cp, None, seed, pass_index, apply=True,
                  logits=g["logit"].astype(np.float64), thr=g["thr"])
    p.passes(s, 1)
    got = s.get_spins()
    la, lu = o_thr["log_alpha"], np.log(o_thr["u_accept"])
    clear = (la > 1e-3) | (np.abs(la - lu) > 1e-3)
    assert clear.mean() > 0.99 and 0 < o_thr["accept"].mean() < 1
    for b in range(g.shape[0]):
        for c in range(n):
            r = o_thr[b, c]
            sites = [((r["bR"] + t // 4) % L, (r["bC"] + t % 4) % L) for t in range(16)]
            blk = np.array([got[c][x] for x in sites])
            if clear[b, c]:
                assert np.array_equal(blk, np.array([after[c][x] for x in sites])), (b, c)
            else:
                assert np.array_equal(blk, np.array([after[c][x] for x in sites])) or \
                    np.array_equal(blk, np.array([spins[c][x] for x in sites]))
    outside = np.ones((n, L, L), bool)
    for b in range(g.shape[0]):
        r = o_thr[b, 0]
        for t in range(16):
            outside[:, (r["bR"] + t // 4) % L, (r["bC"] + t % 4) % L] = False
    assert np.array_equal(got[outside], spins[outside])


@pytest.mark.parametrize("L,n_orc", [(18, 4096), (48, 4096)])
def test_pass_full_size(orc, L, n_orc):
    """The pass at the bench's full size and launch configuration (4096
    chains at the evaluation points J'/J = 1, h = 3, beta in {1.5, 2, 3}; the
    persistent grid of the bench) against the oracle's pass on the first
    n_orc chains (all of them): block origins, current blocks, the proposed
    blocks (with the GPU's thresholds) and dE exactly, logits and log alpha
    within tolerance, and after the pass runs every block whose accept test is
    clear of its boundary."""
    ew = workloads.proposal_eval_workload(L)
    s = crbm.Sampler(**dict(ew, measure_every=0))
    s.sweep(20)
    p = crbm.Proposal(seed=1)
    w = orc.random_net(5, scale=0.15)
    p.weights = w
    g = p.inspect(s)                                                   # [word][block][lane]
    g = g.transpose(1, 0, 2).reshape(g.shape[1], -1)[:, :n_orc]        # [block][chain]
    spins = np.ascontiguousarray(s.get_spins()[:n_orc])
    params, cp, seed = ew["params"], ew["chain_param"][:n_orc], ew["seed"]
    assert len(set(cp.tolist())) >= 2
    o_net = orc.prop_pass(spins.copy(), params, cp, w, seed, 0)
    for f in ("bR", "bC", "cur_bits"):
        assert np.array_equal(g[f].astype(np.int64), o_net[f].astype(np.int64)), f
    err = np.abs(g["logit"] - o_net["logit"]) / (0.05 + 0.02 * np.abs(o_net["logit"]))
    assert err.max() <= 1.0, err.max()
    o_thr = orc.prop_pass(spins.copy(), params, cp, None, seed, 0,
                          logits=g["logit"].astype(np.float64), thr=g["thr"])
    assert np.array_equal(g["new_bits"], o_thr["new_bits"])
    assert np.array_equal(g["dE"].astype(np.int64), o_thr["dE"])
    la_err = np.abs(g["log_alpha"] - o_thr["log_alpha"])
    assert (la_err <= 2e-4 + 1e-5 * np.abs(o_thr["log_alpha"])).all(), la_err.max()
    after = spins.copy()
    orc.prop_pass(after, params, cp, None, seed, 0, apply=True,
                  logits=g["logit"].astype(np.float64), thr=g["thr"])
    p.passes(s, 1)
    got = s.get_spins()[:n_orc]
    la, lu = o_thr["log_alpha"], np.log(o_thr["u_accept"])
    clear = (la > 1e-3) | (np.abs(la - lu) > 1e-3)
    assert clear.mean() > 0.99 and 0 < o_thr["accept"].mean() < 1
    for b in range(g.shape[0]):
        r = o_thr[b, 0]
        rows = (int(r["bR"]) + np.arange(16) // 4) % L
        cols = (int(r["bC"]) + np.arange(16) % 4) % L
        blk_got, blk_after, blk_before = got[:, rows, cols], after[:, rows, cols], spins[:, rows, cols]
        same_after = (blk_got == blk_after).all(1)
        assert same_after[clear[b]].all(), b
        assert (same_after | (blk_got == blk_before).all(1)).all(), b
        got[:, rows, cols] = 0
        after[:, rows, cols] = 0
    assert np.array_equal(got, after)  # nothing outside the blocks moved


def test_training_gradient_matches_oracle(orc):
    rng = np.random.default_rng(4)
    L, n = 12, 24
    spins = rng.choice(np.array([-1, 1], np.int8), size=(n, L, L))
    origins = rng.integers(0, L, (n, 2)).astype(np.int32)
    bh = np.stack([rng.uniform(0.5, 3.0, n), rng.uniform(-1, 4, n)], 1)
    bh = np.vectorize(orc.bf16)(bh).astype(np.float32)
    w = orc.random_net(8, scale=0.2)
    p = crbm.Proposal(seed=2)
    p.weights = w
    loss, grad = p.loss_grad(spins, origins, bh)
    inputs = np.array([orc.patch_input(spins[e], int(origins[e, 0]), int(origins[e, 1]), 4,
                                       float(bh[e, 0]), float(bh[e, 1])) for e in range(n)])
    targets = np.array([[spins[e, (origins[e, 0] + a // 4) % L, (origins[e, 1] + a % 4) % L]
                         for a in range(16)] for e in range(n)], np.int8)
    wb = np.vectorize(orc.bf16)(w.astype(np.float32).astype(np.float64))
    l_ref, g_ref = orc.net_loss_grad(4, wb, inputs, targets, use_bf16=True)
    assert abs(loss - l_ref) <= 2e-3 * abs(l_ref)
    scale = np.abs(g_ref).max()
    assert np.linalg.norm(grad - g_ref) <= 2e-2 * np.linalg.norm(g_ref)
    assert np.abs(grad - g_ref).max() <= 2e-2 * scale


def test_training_lowers_the_loss_and_moves_are_accepted():
    w = workloads.proposal_training_workload(n_chains=2048)
    s = crbm.Sampler(**w)
    s.sweep(300)
    p = crbm.Proposal(seed=5)
    losses = p.train(s, steps=250, batch=4096, lr=1e-2, sweeps_between=2)
    assert losses[-20:].mean() < 0.6 * losses[:3].mean(), (losses[:3], losses[-20:])
    p.passes(s, 20)
    proposed, accepted = p.stats()
    # a factorised proposal cannot capture correlations inside the block: about
    # a fifth of the moves are accepted after a few hundred steps near the plateau
    assert proposed > 0 and accepted / proposed > 0.08, (proposed, accepted)


def test_mixed_sampler_matches_plain_gibbs():
    """Exact MH keeps the Boltzmann law: energy and magnetisation per spin of
    Gibbs + block moves agree with plain Gibbs within 3 standard errors
    (standard errors from the spread of independent chain means)."""
    L, n = 12, 2048
    params = dict(J=[1.0], Jp=[1.0], h=[1.0], beta=[0.6])
    res = []
    for mixed in (False, True):
        s = crbm.Sampler(L, params, n, seed=11 + mixed, measure_every=1, series_len=1200)
        p = crbm.Proposal(seed=9)
        p.weights = np.asarray(p.weights) * 1.0
        if mixed:
            p.train(s, steps=30, batch=1024, lr=3e-3, sweeps_between=3)
            s.reset_observables()
            p.sweep_mixed(s, 1200)
            prop, acc = p.stats()
            assert acc > 0
        else:
            s.sweep(90)
            s.reset_observables()
            s.sweep(1200)
        ser = s.series()[200:].astype(np.float64)            # [T][chain][3]
        E = (ser[..., 0] + ser[..., 1] - ser[..., 2]) / (L * L)
        M = ser[..., 2] / (L * L)
        res.append([(x.mean(0).mean(), x.mean(0).std(ddof=1) / np.sqrt(n)) for x in (E, M)])
    for (m0, s0), (m1, s1) in zip(res[0], res[1]):
        assert abs(m0 - m1) < 3 * np.hypot(s0, s1), (m0, m1, s0, s1)


def test_mixed_every_is_sweeps_then_a_pass():
    """sweep_mixed(n, every) = groups of `every` sweeps (the last one
    shorter), each followed by one pass: bit-identical to the same calls made
    one by one (the passes are keyed on the pass count)."""
    params = dict(J=[1.0], Jp=[1.5], h=[0.5], beta=[1.2])
    a = crbm.Sampler(12, params, 96, seed=4, measure_every=1)
    b = crbm.Sampler(12, params, 96, seed=4, measure_every=1)
    p = crbm.Proposal(seed=2)
    p.sweep_mixed(a, 11, every=4)
    for n in (4, 4, 3):
        b.sweep(n)
        p.passes(b, 1)
    assert np.array_equal(a.get_spins(), b.get_spins())
    assert np.array_equal(a.observables(), b.observables())
    with pytest.raises(crbm.CrbmError):
        p.sweep_mixed(a, 4, every=0)


def test_trained_network_gains_effective_samples_per_sweep():
    """What the trained network adds over the method without it: from one
    equilibrated L=18 state (J'/J = 1, h = 3, beta = 2, near the 1/3 plateau),
    Gibbs + one pass of trained block moves per sweep gives more effective
    samples of the energy per sweep than plain Gibbs, and far more accepted
    moves than the same net untrained.  (Per second it does not pay: a pass
    costs about a dozen Gibbs sweeps; the bench line states that ratio.)"""
    from paper_2511_20911_gb300 import analysis
    src = crbm.Sampler(**workloads.proposal_training_workload(n_chains=2048))
    src.sweep(300)
    trained = crbm.Proposal(seed=5)
    trained.train(src, steps=250, batch=4096, lr=1e-2, sweeps_between=2)
    untrained = crbm.Proposal(seed=5)
    T = 1000
    ew = workloads.proposal_eval_workload(18, n_chains=1024, betas=(2.0,))
    base = crbm.Sampler(**dict(ew, measure_every=1, series_len=T))
    base.sweep(6000)
    ck = base.save()
    ess, acc = {}, {}
    for name, prop in (("plain", None), ("untrained", untrained), ("trained", trained)):
        s = crbm.Sampler(**dict(ew, measure_every=1, series_len=T))
        s.load(ck)
        s.reset_observables()
        if prop is None:
            s.sweep(T)
        else:
            p0 = prop.stats()
            prop.sweep_mixed(s, T)
            p1 = prop.stats()
            acc[name] = (p1[1] - p0[1]) / max(1, p1[0] - p0[0])
        ser = s.series().transpose(1, 0, 2).astype(np.float64)   # [chain][T][3]
        E = ser[..., 0] + ser[..., 1] - 3.0 * ser[..., 2]
        ess[name] = float(analysis.effective_samples(E).sum())
    assert ess["trained"] > 1.2 * ess["plain"], ess
    assert acc["trained"] > 2.0 * acc["untrained"], acc


def test_proposal_rejects_unsupported_contexts():
    p = crbm.Proposal(seed=1)
    ok = dict(J=[1.0], Jp=[1.0], h=[0.5], beta=[1.0])
    for s in (crbm.Sampler(9, ok, 32), crbm.Sampler(10, ok, 32, periodic=False),
              crbm.Sampler(20, ok, 64, layout=crbm.CRBM_LAYOUT_STREAM)):
        with pytest.raises(crbm.CrbmError) as e:
            p.passes(s, 1)
        assert e.value.code == crbm.CRBM_EUNSUPPORTED
