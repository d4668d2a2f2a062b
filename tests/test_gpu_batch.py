"""Batched launches and the autotuner.  A batch advances every member by one
kernel launch (graph-captured); each member must stay bit-identical to a twin
context advanced on its own.  Autotuning must not touch the chains."""
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


def members():
    rng = np.random.default_rng(12)
    pt = workloads.tempering_batch_workload(sizes=(9, 12), ladders=2)
    specs = [dict(L=6, params=workloads.random_params(rng, 3), n_chains=64,
                  chain_param=rng.integers(0, 3, 64).astype(np.int32), seed=1, measure_every=2,
                  series_len=20),
             dict(L=7, params=workloads.random_params(rng, 2), n_chains=40, periodic=False,
                  chain_param=rng.integers(0, 2, 40).astype(np.int32), seed=2, measure_every=3),
             dict(L=8, params=workloads.random_params(rng, 2), n_chains=33,
                  chain_param=rng.integers(0, 2, 33).astype(np.int32), seed=3, measure_every=0,
                  sq_every=4)]
    for m in pt:
        specs.append(dict(m, measure_every=5, series_len=10))
    return specs


def make(spec):
    return crbm.Sampler(**spec)


def same(a, b):
    assert a.sweep_count == b.sweep_count
    assert np.array_equal(a.get_spins(), b.get_spins())
    assert np.array_equal(a.observables(), b.observables())
    assert np.array_equal(a.permutation(), b.permutation())
    if a.series_len:
        assert np.array_equal(a.series(), b.series())
    if a.sq_every:
        assert np.array_equal(a.correlations()[0], b.correlations()[0])


def test_batch_matches_individual_sweeps():
    specs = members()
    batched = [make(s) for s in specs]
    twins = [make(s) for s in specs]
    batch = crbm.Batch(batched)
    assert batch.threads >= 32
    plan = [("batch", 5), ("batch", 8), ("solo", 3), ("batch", 8), ("batch", 2)]
    for kind, n in plan:
        if kind == "batch":
            batch.sweep(n)
        else:                              # a member moved outside the batch: clocks re-uploaded
            batched[1].sweep(n)
            batched[3].sweep(n)
            twins[1].sweep(n)
            twins[3].sweep(n)
            continue
        for t in twins:
            t.sweep(n)
    for a, b in zip(batched, twins):
        same(a, b)
    batch.close()


@pytest.mark.parametrize("cluster", [2, 4, 8])
def test_batch_cluster_split_matches_individual_sweeps(cluster, monkeypatch):
    """Words split into bands over a thread-block cluster (boundary rows
    exchanged through distributed shared memory, measurement and replica
    exchange on rank 0) stay bit-identical to the whole-word sweep."""
    monkeypatch.setenv("CRBM_BATCH_CLUSTER", str(cluster))
    rng = np.random.default_rng(40 + cluster)
    pt = workloads.tempering_batch_workload(sizes=(12, 24), ladders=1)
    specs = [dict(m, measure_every=5, series_len=12) for m in pt]
    specs += [dict(L=18, params=workloads.random_params(rng, 3), n_chains=70,
                   chain_param=rng.integers(0, 3, 70).astype(np.int32), seed=7, measure_every=3, series_len=20),
              dict(L=9, params=workloads.random_params(rng, 2), n_chains=32,
                   chain_param=rng.integers(0, 2, 32).astype(np.int32), seed=8, measure_every=4),
              dict(L=16, params=workloads.random_params(rng, 2), n_chains=40,
                   chain_param=rng.integers(0, 2, 40).astype(np.int32), seed=9, measure_every=0, sq_every=5)]
    batched = [make(s) for s in specs]
    twins = [make(s) for s in specs]
    batch = crbm.Batch(batched)
    assert batch.cluster == cluster
    for n in (7, 13, 25, 120):
        batch.sweep(n)
        for t in twins:
            t.sweep(n)
    for a, b in zip(batched, twins):
        same(a, b)
    batch.close()


@pytest.mark.parametrize("cluster", [1, 8])
def test_batch_with_paper_precision_and_bitplane_members(cluster, monkeypatch):
    """Paper-precision members (canonical and generic) and bit-plane members
    (whole words, one per CTA; the bit-plane ladder with replica exchange)
    beside exact members split over a cluster and a generic member, in one
    launch: every member bit-identical
    to a twin advanced on its own (the twins' sweeps are pinned to the oracle
    elsewhere); a batch holding only exact members keeps the kernel without
    the other bodies."""
    monkeypatch.setenv("CRBM_BATCH_CLUSTER", str(cluster))
    rng = np.random.default_rng(60 + cluster)
    ladder = workloads.tempering_batch_workload(sizes=(8,), ladders=2)[0]
    specs = [dict(L=10, params=workloads.random_params(rng, 3), n_chains=64,
                  chain_param=rng.integers(0, 3, 64).astype(np.int32), seed=21, measure_every=2, series_len=12,
                  precision=crbm.CRBM_PRECISION_PAPER),
             dict(L=12, params=workloads.random_params(rng, 2), n_chains=50,
                  chain_param=rng.integers(0, 2, 50).astype(np.int32), seed=22, measure_every=3, series_len=12,
                  rng=crbm.CRBM_RNG_BITPLANE),
             dict(ladder, measure_every=5, series_len=10, rng=crbm.CRBM_RNG_BITPLANE),
             dict(L=24, params=workloads.random_params(rng, 2), n_chains=40,
                  chain_param=rng.integers(0, 2, 40).astype(np.int32), seed=23, measure_every=4, series_len=12),
             dict(L=9, params=workloads.random_params(rng, 2), n_chains=32,
                  chain_param=rng.integers(0, 2, 32).astype(np.int32), seed=24, measure_every=4),
             dict(L=7, params=workloads.random_params(rng, 2), n_chains=45, periodic=False,
                  chain_param=rng.integers(0, 2, 45).astype(np.int32), seed=25, measure_every=3, series_len=12,
                  precision=crbm.CRBM_PRECISION_PAPER)]
    batched = [make(s) for s in specs]
    twins = [make(s) for s in specs]
    batch = crbm.Batch(batched)
    assert batch.cluster == cluster
    for n in (5, 11, 30):
        batch.sweep(n)
        for t in twins:
            t.sweep(n)
    for a, b in zip(batched, twins):
        same(a, b)
    batch.close()


def test_batch_validation():
    spec = members()[0]
    a, b = make(spec), make(spec)
    s = crbm.Sampler(20, dict(J=[1.0], Jp=[1.0], h=[0.5], beta=[1.0]), 64,
                     layout=crbm.CRBM_LAYOUT_STREAM)
    for group in ([a, a], [a, s]):
        with pytest.raises(crbm.CrbmError) as e:
            crbm.Batch(group)
        assert e.value.code == crbm.CRBM_EINVAL


def test_autotune_keeps_chains_and_writes_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("CRBM_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    spec = members()[3]                     # a tempering member
    a, b = make(spec), make(spec)
    a.sweep(7)
    b.sweep(7)
    w = a.autotune(20)
    assert w in (2, 4, 6, 8, 10, 12, 14, 16) and a.warps == w
    a.sweep(9)
    b.sweep(9)
    same(a, b)
    text = (tmp_path / "tune.txt").read_text()
    assert text.strip().endswith(f" {w}")
    c = make(spec)                          # same shape on the same GPU: taken from the cache
    assert c.warps == w


def test_batch_autotune_keeps_state():
    """The batch autotuner probes CTA shapes on the members' own state and puts
    it back: spins, counters, sums, series, correlations, permutations, launch
    counts and first-hit records (targets set just before, so the probes do
    record hits) are as before, and the tuned batch continues bit-identically
    to twins advanced on their own."""
    specs = members()
    batched = [make(s) for s in specs]
    twins = [make(s) for s in specs]
    batch = crbm.Batch(batched)
    batch.sweep(6)
    for t in twins:
        t.sweep(6)
    big = np.full(len(specs[0]["params"]["J"]), 10 ** 9, np.int64)   # reached at the next measurement
    batched[0].set_targets(big)
    twins[0].set_targets(big)
    launches = [m.launch_count for m in batched]
    threads = batch.autotune(20)
    assert threads in [32 * w for w in (8, 12, 16, 20, 24, 28, 32)] and batch.threads == threads
    assert [m.launch_count for m in batched] == launches
    assert (batched[0].first_hits() == -1).all()
    for a, b in zip(batched, twins):
        same(a, b)
    batch.sweep(5)
    for t in twins:
        t.sweep(5)
    for a, b in zip(batched, twins):
        same(a, b)
    hits = batched[0].first_hits()
    assert np.array_equal(hits, twins[0].first_hits()) and (hits == 8).all()
    with pytest.raises(crbm.CrbmError) as e:
        batch.autotune(0)
    assert e.value.code == crbm.CRBM_EINVAL
    batch.close()


def test_batch_sees_targets_set_after_capture():
    """Targets set on a member after the batch captured its graph (the same
    sweep count, so the graph would otherwise be replayed) are recorded."""
    specs = members()[:2]
    batched = [make(s) for s in specs]
    twin = make(specs[0])
    batch = crbm.Batch(batched)
    batch.sweep(4)
    twin.sweep(4)
    big = np.full(len(specs[0]["params"]["J"]), 10 ** 9, np.int64)
    batched[0].set_targets(big)
    twin.set_targets(big)
    batch.sweep(4)
    twin.sweep(4)
    hits = batched[0].first_hits()
    assert np.array_equal(hits, twin.first_hits()) and (hits == 6).all()
    batch.close()


def test_batch_wide_ctas_match_individual_sweeps(monkeypatch):
    """CTAs of more than 512 threads run the kernel's 1024-thread instantiation
    (64 registers a thread); smaller ones the 512-thread one.  Both stay
    bit-identical to twins advanced on their own."""
    specs = members()
    monkeypatch.setenv("CRBM_WARPS", "24")
    batched = [make(s) for s in specs]
    monkeypatch.delenv("CRBM_WARPS")
    twins = [make(s) for s in specs]
    batch = crbm.Batch(batched)
    assert batch.threads == 768
    for n in (5, 8):
        batch.sweep(n)
        for t in twins:
            t.sweep(n)
    for a, b in zip(batched, twins):
        same(a, b)
    batch.close()
