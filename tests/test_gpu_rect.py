"""Rectangular lattices, a boundary per axis and an odd-column field on the
GPU against the oracle, bit for bit: tables, spins, sums and series; the
laterally confined 18 x 12 strip of Sec. III among them.  Rectangles with even
sides, periodic along both axes, run on the canonical shared-memory sweep
(also split into bands over a cluster in a batch) and on the streamed sweep;
the rest on the generic sweep."""
import numpy as np
import pytest

import paper_2511_20911_gb300 as crbm
from paper_2511_20911_gb300 import workloads

pytestmark = pytest.mark.gpu
OPEN, PERIODIC = crbm.CRBM_BC_OPEN, crbm.CRBM_BC_PERIODIC


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    crbm.load_library()


def run_pair(orc, L, Lc, pr, pc, params, n, seed, splits, measure_every=2, series_len=8, swap_every=0,
             precision=0):
    cp = (np.arange(n) % len(params["J"])).astype(np.int32)
    s = crbm.Sampler(L, params, n, chain_param=cp, seed=seed, periodic=pr, L_cols=Lc,
                     periodic_cols=PERIODIC if pc else OPEN, measure_every=measure_every,
                     series_len=series_len, precision=precision)
    assert s.get_spins().shape == (n, L, Lc)
    ids = np.arange(n, dtype=np.uint32)
    spins = orc.init_spins((L, Lc), ids, seed)
    assert np.array_equal(s.get_spins(), spins), "initial spins"
    sums, oser, t = None, None, 0
    for k in splits:
        s.sweep(k)
        sums, ser, _ = orc.run((L, Lc), params, cp, spins, seed, t, k, measure_every, chain_ids=ids,
                               periodic=(pr, pc), sums=sums, series_cap=series_len, precision=precision)
        if ser is not None:
            oser = ser if oser is None else np.where(ser != 0, ser, oser)
        t += k
        assert np.array_equal(s.get_spins(), spins), f"spins after {t} sweeps"
    assert np.array_equal(s.observables(), sums)
    if series_len:
        assert np.array_equal(s.series().transpose(1, 0, 2), oser)
    return s


@pytest.mark.parametrize("L,Lc,pr,pc", [(6, 10, True, True), (18, 12, True, False), (12, 18, False, True),
                                        (7, 10, True, True), (9, 5, False, False), (10, 3, True, True)])
def test_rectangles_bitexact(orc, L, Lc, pr, pc):
    rng = np.random.default_rng(L * 100 + Lc)
    params = workloads.random_params(rng, 3)
    s = run_pair(orc, L, Lc, pr, pc, params, 45, 3 + L + Lc, splits=[3, 14])
    assert s.layout == crbm.CRBM_LAYOUT_SMEM


@pytest.mark.parametrize("L,Lc", [(18, 12), (12, 30), (40, 8), (4, 16)])
@pytest.mark.parametrize("precision", [crbm.CRBM_PRECISION_EXACT, crbm.CRBM_PRECISION_PAPER])
def test_periodic_rectangles_on_the_canonical_sweep(orc, L, Lc, precision):
    """Even sides, periodic along both axes: the ten SS filters' fast path
    (per-cell records over W x Wc cells), in both precisions."""
    rng = np.random.default_rng(L * 31 + Lc + precision)
    params = workloads.random_params(rng, 3)
    s = run_pair(orc, L, Lc, True, True, params, 70, 7 + L + Lc, splits=[4, 9], precision=precision)
    assert s.layout == crbm.CRBM_LAYOUT_SMEM


@pytest.mark.parametrize("cluster", [2, 8])
def test_periodic_rectangle_split_over_a_cluster(orc, cluster, monkeypatch):
    """A 24 x 16 periodic rectangle split into bands of cell rows over a
    thread-block cluster, beside a square member, against its twin and the
    oracle."""
    monkeypatch.setenv("CRBM_BATCH_CLUSTER", str(cluster))
    rng = np.random.default_rng(70 + cluster)
    specs = [dict(L=24, L_cols=16, params=workloads.random_params(rng, 2), n_chains=64, seed=21,
                  measure_every=3),
             dict(L=20, params=workloads.random_params(rng, 2), n_chains=32, seed=22, measure_every=3)]
    for sp in specs:
        sp["chain_param"] = (np.arange(sp["n_chains"]) % 2).astype(np.int32)
    batched = [crbm.Sampler(**sp) for sp in specs]
    twins = [crbm.Sampler(**sp) for sp in specs]
    batch = crbm.Batch(batched)
    assert batch.cluster == cluster
    for n in (5, 7):
        batch.sweep(n)
        for t in twins:
            t.sweep(n)
    for a, b in zip(batched, twins):
        assert np.array_equal(a.get_spins(), b.get_spins())
        assert np.array_equal(a.observables(), b.observables())
    batch.close()
    sp = specs[0]
    ids = np.arange(sp["n_chains"], dtype=np.uint32)
    spins = orc.init_spins((24, 16), ids, sp["seed"])
    sums, _, _ = orc.run((24, 16), sp["params"], sp["chain_param"], spins, sp["seed"], 0, 12, 3, chain_ids=ids)
    assert np.array_equal(batched[0].get_spins(), spins)
    assert np.array_equal(batched[0].observables(), sums)


@pytest.mark.parametrize("L,Lc,pr,pc", [(8, 6, True, False), (7, 9, False, False), (6, 6, True, True)])
def test_odd_column_field_bitexact(orc, L, Lc, pr, pc):
    rng = np.random.default_rng(L * 7 + Lc)
    params = workloads.random_params(rng, 2)
    params["h_odd"] = list(np.round(rng.uniform(-3, 3, 2) * 16) / 16)
    s = run_pair(orc, L, Lc, pr, pc, params, 40, 11, splits=[5, 9])
    tabs, (dj, djp) = s.tables()
    for p in range(2):
        th, tv, tvo = orc.tables((L, Lc), params["J"][p], params["Jp"][p], params["h"][p], params["beta"][p],
                                 periodic=(pr, pc), h_odd=params["h_odd"][p])
        assert np.array_equal(tabs[p], np.concatenate([th.reshape(-1), tv.reshape(-1), tvo.reshape(-1)]))


def test_strip_in_a_batch_matches_its_twin(orc):
    """The laterally confined strip (18 rows periodic, 12 columns open) and a
    square member in one batched launch stay bit-identical to twins advanced
    alone."""
    rng = np.random.default_rng(5)
    specs = [dict(L=18, L_cols=12, periodic=True, periodic_cols=OPEN, params=workloads.random_params(rng, 2),
                  n_chains=64, seed=9, measure_every=4),
             dict(L=12, params=workloads.random_params(rng, 2), n_chains=32, seed=10, measure_every=4)]
    for sp in specs:
        sp["chain_param"] = (np.arange(sp["n_chains"]) % 2).astype(np.int32)
    batched = [crbm.Sampler(**sp) for sp in specs]
    twins = [crbm.Sampler(**sp) for sp in specs]
    batch = crbm.Batch(batched)
    for n in (6, 11):
        batch.sweep(n)
        for t in twins:
            t.sweep(n)
    for a, b in zip(batched, twins):
        assert np.array_equal(a.get_spins(), b.get_spins())
        assert np.array_equal(a.observables(), b.observables())
    batch.close()


@pytest.mark.parametrize("L,Lc", [(18, 12), (12, 40), (40, 12), (36, 34), (4, 16)])
@pytest.mark.parametrize("mode", ["exact", "paper", "bitplane"])
def test_periodic_rectangles_streamed(orc, L, Lc, mode):
    """The streamed layout on even periodic rectangles: tiles of 16 x 16
    cells over W x Wc cells (one tile or several, ragged along either axis;
    the spin and hidden halos wrapping once or by the modulo), a ragged last
    64-chain group, in exact precision, paper precision and with bit-plane
    uniforms, against the oracle and against the SMEM layout."""
    rng = np.random.default_rng(L * 53 + Lc + len(mode))
    params = workloads.random_params(rng, 3)
    n = 70
    cp = rng.integers(0, 3, n).astype(np.int32)
    precision = crbm.CRBM_PRECISION_PAPER if mode == "paper" else crbm.CRBM_PRECISION_EXACT
    rng_mode = crbm.CRBM_RNG_BITPLANE if mode == "bitplane" else crbm.CRBM_RNG_LANE
    seed = 11 + L + Lc
    kw = dict(chain_param=cp, seed=seed, L_cols=Lc, measure_every=2, series_len=4, precision=precision,
              rng=rng_mode)
    s = crbm.Sampler(L, params, n, layout=crbm.CRBM_LAYOUT_STREAM, **kw)
    assert s.layout == crbm.CRBM_LAYOUT_STREAM
    ids = np.arange(n, dtype=np.uint32)
    spins = orc.init_spins((L, Lc), ids, seed)
    assert np.array_equal(s.get_spins(), spins), "initial spins"
    sums, oser, t = None, None, 0
    orng = orc.RNG_BITPLANE if mode == "bitplane" else orc.RNG_LANE
    for k in (3, 4):
        s.sweep(k)
        sums, ser, _ = orc.run((L, Lc), params, cp, spins, seed, t, k, 2, chain_ids=ids, sums=sums,
                               series_cap=4, precision=precision, rng=orng)
        oser = ser if oser is None else np.where(ser != 0, ser, oser)
        t += k
        assert np.array_equal(s.get_spins(), spins), f"spins after {t} sweeps"
    assert np.array_equal(s.observables(), sums)
    assert np.array_equal(s.series().transpose(1, 0, 2), oser)
    m = crbm.Sampler(L, params, n, layout=crbm.CRBM_LAYOUT_SMEM, **kw)
    m.sweep(7)
    assert np.array_equal(m.get_spins(), s.get_spins())
    assert np.array_equal(m.observables(), s.observables())


def test_rectangle_validation():
    ok = dict(J=[1.0], Jp=[1.0], h=[0.5], beta=[2.0])
    for kw, code in ((dict(L_cols=2), crbm.CRBM_EINVAL), (dict(periodic_cols=5), crbm.CRBM_EINVAL),
                     (dict(L_cols=8, sq_every=2), crbm.CRBM_EINVAL),
                     (dict(periodic_cols=OPEN, sq_every=2), crbm.CRBM_EINVAL),
                     (dict(L_cols=8, periodic_cols=OPEN, layout=crbm.CRBM_LAYOUT_STREAM),
                      crbm.CRBM_EUNSUPPORTED)):
        with pytest.raises(crbm.CrbmError) as e:
            crbm.Sampler(6, ok, 32, **kw)
        assert e.value.code == code, kw
    ladder = dict(J=[1.0] * 32, Jp=[1.0] * 32, h=[0.5] * 32, h_odd=[1.0] * 32,
                  beta=list(0.5 + 0.1 * np.arange(32)))
    with pytest.raises(crbm.CrbmError) as e:
        crbm.Sampler(6, ladder, 32, chain_param=np.arange(32), swap_every=2)
    assert e.value.code == crbm.CRBM_EUNSUPPORTED
    prop = crbm.Proposal(seed=1)                  # block proposals: square lattices only
    with pytest.raises(crbm.CrbmError) as e:
        prop.passes(crbm.Sampler(8, ok, 32, L_cols=12), 1)
    assert e.value.code == crbm.CRBM_EUNSUPPORTED


@pytest.mark.slow
def test_strip_workload_sampled_chains(orc):
    """The laterally confined strip workload at full size (18 periodic rows of
    12 open columns, 2304 chains over 6 (beta, h) points): 32 chains spread
    over every word against the oracle, and its S(q) from the sampled spins."""
    from paper_2511_20911_gb300 import analysis
    w = workloads.strip_workload()
    s = crbm.Sampler(w["L"], w["params"], w["n_chains"], chain_param=w["chain_param"], seed=w["seed"],
                     periodic=w["periodic"], L_cols=w["L_cols"], periodic_cols=w["periodic_cols"],
                     measure_every=w["measure_every"])
    n = 30
    s.sweep(n)
    ids = np.linspace(0, w["n_chains"] - 1, 32).astype(np.uint32)
    spins = orc.init_spins((w["L"], w["L_cols"]), ids, w["seed"])
    sums, _, _ = orc.run((w["L"], w["L_cols"]), w["params"], w["chain_param"][ids], spins, w["seed"], 0, n,
                         w["measure_every"], chain_ids=ids, periodic=(True, False))
    got = s.get_spins()
    assert np.array_equal(got[ids], spins)
    assert np.array_equal(s.observables()[ids], sums)
    sq = analysis.structure_factor(got)
    assert sq.shape == (w["L"], w["L_cols"]) and abs(sq.mean() - 1.0) < 1e-9   # sum rule: mean_q S = 1
