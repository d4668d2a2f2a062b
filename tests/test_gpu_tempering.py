"""Parallel tempering on the GPU against the oracle, bit for bit: spins per
replica slot, the replica permutation, and per-rung sums and series."""
import numpy as np
import pytest

import paper_2511_20911_gb300 as crbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def ladder(n_lad, lo=0.2, hi=10.0, J=1.0, Jp=1.5, h=1.0, jitter=None):
    """n_lad ladders of 32 geometric betas in [lo, hi]; parameter point
    32 l + k is rung k of ladder l."""
    betas = []
    for l in range(n_lad):
        b = lo * (hi / lo) ** (np.arange(32) / 31.0)
        if jitter is not None:
            b = b * (1.0 + jitter * l)
        betas.extend(b.tolist())
    n = len(betas)
    params = dict(J=[J] * n, Jp=[Jp] * n, h=[h] * n, beta=betas)
    return params, np.arange(n, dtype=np.int32)


def run_pt_pair(orc, L, n_lad, seed, splits, swap_every, measure_every, periodic=True,
                jitter=None, series_len=0, layout=crbm.CRBM_LAYOUT_AUTO, precision=crbm.CRBM_PRECISION_EXACT):
    params, cp = ladder(n_lad, jitter=jitter)
    n = 32 * n_lad
    s = crbm.Sampler(L, params, n, chain_param=cp, seed=seed, periodic=periodic,
                     measure_every=measure_every, series_len=series_len, swap_every=swap_every,
                     layout=layout, precision=precision)
    spins = orc.init_spins(L, np.arange(n, dtype=np.uint32), seed)
    sob = np.tile(np.arange(32, dtype=np.int32), (n_lad, 1))
    sums, oser = None, None
    t = 0
    for k in splits:
        s.sweep(k)
        sums, ser = orc.run_pt(L, params, cp, spins, sob, seed, t, k, measure_every, swap_every,
                               periodic=periodic, sums=sums, series_cap=series_len, precision=precision)
        if ser is not None:
            oser = ser if oser is None else np.where(ser != 0, ser, oser)
        t += k
        assert np.array_equal(s.get_spins(), spins), f"spins after {t} sweeps"
        assert np.array_equal(s.permutation().reshape(n_lad, 32), sob), f"permutation after {t}"
    if measure_every:
        assert np.array_equal(s.observables(), sums)
    if series_len:
        assert np.array_equal(s.series().transpose(1, 0, 2), oser)
    return s, sob


@pytest.mark.parametrize("L,periodic,n_lad", [(6, True, 2), (12, True, 3), (9, True, 2),
                                               (7, False, 1), (18, True, 1)])
def test_tempering_bitexact(orc, L, periodic, n_lad):
    s, sob = run_pt_pair(orc, L, n_lad, 40 + L, splits=[7, 23], swap_every=3, measure_every=2,
                         periodic=periodic, series_len=15)
    assert (sob != np.arange(32)).any()


@pytest.mark.parametrize("L,n_lad,precision", [(8, 2, 0), (12, 3, 0), (34, 1, 0), (12, 2, 1)])
def test_tempering_streamed_bitexact(orc, L, n_lad, precision):
    """Replica exchange in the streamed layout: a ladder is a 32-chain half of
    a 64-chain group (an odd ladder count leaves a padding half-word), the
    kernels read each slot's rung column, and the post-sweep step (counts,
    per-rung measurement, exchange round) runs as one warp per ladder; spins
    per slot, the permutation and per-rung sums and series against the
    oracle, in exact and paper precision, over ragged 16 x 16-cell tiles."""
    s, _ = run_pt_pair(orc, L, n_lad, 40 + L + n_lad, splits=[7, 13], swap_every=2, measure_every=3,
                       series_len=8, layout=crbm.CRBM_LAYOUT_STREAM,
                       precision=crbm.CRBM_PRECISION_PAPER if precision else crbm.CRBM_PRECISION_EXACT)
    assert s.layout == crbm.CRBM_LAYOUT_STREAM


def test_tempering_per_ladder_betas(orc):
    """Each ladder has its own beta sequence, hence its own swap tables."""
    run_pt_pair(orc, 8, 3, 5, splits=[20], swap_every=2, measure_every=5, jitter=0.3)


def test_tempering_checkpoint_resume():
    params, cp = ladder(2)
    a = crbm.Sampler(6, params, 64, chain_param=cp, seed=9, swap_every=2, series_len=30)
    a.sweep(11)
    ck = a.save()
    a.sweep(13)
    b = crbm.Sampler(6, params, 64, chain_param=cp, seed=9, swap_every=2, series_len=30)
    b.load(ck)
    b.sweep(13)
    assert np.array_equal(a.get_spins(), b.get_spins())
    assert np.array_equal(a.permutation(), b.permutation())
    assert np.array_equal(a.observables(), b.observables())


def test_tempering_validation():
    params, cp = ladder(1)
    bad_beta = dict(params, beta=params["beta"][::-1])
    bad_h = dict(params, h=[1.0] * 31 + [2.0])
    for kw, code in ((dict(params=bad_beta, n_chains=32), crbm.CRBM_EINVAL),
                     (dict(params=bad_h, n_chains=32), crbm.CRBM_EINVAL),
                     (dict(params=params, n_chains=31, chain_param=cp[:31]), crbm.CRBM_EINVAL),
                     (dict(params=params, n_chains=32, layout=crbm.CRBM_LAYOUT_STREAM, rng=crbm.CRBM_RNG_BITPLANE),
                      crbm.CRBM_EUNSUPPORTED)):
        kw.setdefault("chain_param", cp)
        with pytest.raises(crbm.CrbmError) as e:
            crbm.Sampler(8, swap_every=2, **kw)
        assert e.value.code == code, kw


@pytest.mark.slow
def test_full_tempering_batch_sampled_ladders(orc):
    """The mixed-size tempering batch at full size (L in {6,9,12,18,24,48} x 8
    ladders of 32 rungs, one graph-captured batch launch with the largest
    words split over thread-block clusters, as the benchmark runs it): the
    first two ladders of every size checked against the oracle's replica
    exchange, spins per slot, rung permutation and per-rung sums."""
    from paper_2511_20911_gb300 import workloads
    specs = [dict(sp, measure_every=10) for sp in workloads.tempering_batch_workload()]
    samplers = [crbm.Sampler(**sp) for sp in specs]
    batch = crbm.Batch(samplers)
    assert batch.cluster > 1
    n = 30
    batch.sweep(n)
    for sp, s in zip(specs, samplers):
        L, ids = sp["L"], np.arange(64, dtype=np.uint32)
        cp = np.asarray(sp["chain_param"], np.int32)[:64]
        spins = orc.init_spins(L, ids, sp["seed"])
        sob = np.tile(np.arange(32, dtype=np.int32), (2, 1))
        sums, _ = orc.run_pt(L, sp["params"], cp, spins, sob, sp["seed"], 0, n, 10, sp["swap_every"])
        assert np.array_equal(s.get_spins()[:64], spins), L
        assert np.array_equal(s.permutation().reshape(-1, 32)[:2], sob), L
        assert np.array_equal(s.observables()[:64], sums), L
    batch.close()
