"""GPU path (through the C ABI) against the oracle, element by element.

Plain Gibbs is deterministic given the Philox keying and the threshold tables,
so the bar is bit-exact: identical spins after every call, identical integer
observable sums and time series.  S(q) is FP64 post-processing of exact
integer sums and must agree to 1e-12 relative.
"""
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
    crbm.load_library()


def run_pair(orc, L, params, n_chains, chain_param, seed, splits, measure_every=1,
             periodic=True, bonds=None, series_len=0, sq_every=0, check_ids=None,
             layout=crbm.CRBM_LAYOUT_AUTO):
    s = crbm.Sampler(L, params, n_chains, chain_param=chain_param, seed=seed, periodic=periodic,
                     bonds=bonds, measure_every=measure_every, series_len=series_len,
                     sq_every=sq_every, layout=layout)
    ids = np.arange(n_chains, dtype=np.uint32) if check_ids is None else np.asarray(check_ids, np.uint32)
    cp = np.asarray(chain_param, np.int32)[ids]
    ospins = orc.init_spins(L, ids, seed)
    assert np.array_equal(s.get_spins()[ids], ospins), "initial spins"
    sums = None
    t = 0
    series_cap = series_len
    oseries = None
    osq = None
    for n in splits:
        s.sweep(n)
        sums, ser, osq = orc.run(L, params, cp, ospins, seed, t, n, measure_every, chain_ids=ids,
                                 periodic=periodic, bonds=bonds, sums=sums, series_cap=series_cap,
                                 sq_every=sq_every, sq=osq)
        if ser is not None:
            oseries = ser if oseries is None else np.where(ser != 0, ser, oseries)
        t += n
        g = s.get_spins()[ids]
        assert np.array_equal(g, ospins), f"spins differ after sweep {t}"
    if measure_every:
        assert np.array_equal(s.observables()[ids], sums), "observable sums"
    if series_len:
        gser = s.series()[:, ids, :]                 # [T][chain][3]
        assert np.array_equal(gser.transpose(1, 0, 2), oseries), "time series"
    return s, ospins, sums, osq


def test_philox_device_matches_oracle(orc):
    rng = np.random.default_rng(11)
    x = rng.integers(0, 2**32, size=(5000, 6), dtype=np.uint64).astype(np.uint32)
    x[:3] = [[0] * 6, [0xFFFFFFFF] * 6, [3, 1, 4, 1, 5, 9]]
    out = crbm.crbm_philox(x)
    for i in range(0, 5000, 7):
        assert list(out[i]) == orc.philox(x[i, :4], x[i, 4:]), i


def test_philox_stream_probe_matches_oracle(orc):
    """The throughput probe computes what it claims: thread t's XOR over
    calls i of the oracle's Philox((i, t, i ^ t, 0x9E3779B9), seed)."""
    import torch
    nb, th, calls, seed = 2, 64, 5, 0x1234567890ABCDEF
    sink = torch.zeros(nb * th, dtype=torch.int32, device="cuda")
    crbm.crbm_philox_stream(sink, nb, th, calls, seed)
    torch.cuda.synchronize()
    got = sink.cpu().numpy().view(np.uint32)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for t in range(nb * th):
        acc = 0
        for i in range(calls):
            for x in orc.philox((i, t, i ^ t, 0x9E3779B9), key):
                acc ^= x
        assert got[t] == acc, t


@pytest.mark.parametrize("L,periodic", [(6, True), (18, True), (3, True), (3, False), (9, True),
                                        (10, False)])
def test_tables_match_oracle(orc, L, periodic):
    rng = np.random.default_rng(L)
    params = workloads.random_params(rng, 7)
    params["beta"][0] = 0.0
    params["beta"][1] = 10.0
    s = crbm.Sampler(L, params, 40, chain_param=np.arange(40) % 7, periodic=periodic)
    tabs, (dj, djp) = s.tables()
    assert (dj, djp) == orc.degrees(L, periodic)
    for p in range(7):
        th, tv = orc.tables(L, params["J"][p], params["Jp"][p], params["h"][p],
                            params["beta"][p], periodic=periodic)
        assert np.array_equal(tabs[p, :10], th.reshape(-1))
        assert np.array_equal(tabs[p, 10:], tv.reshape(-1))


def test_small_workload_bitexact(orc):
    w = workloads.small_workload()
    run_pair(orc, w["L"], w["params"], w["n_chains"], w["chain_param"], w["seed"],
             splits=[1, 99, 200], measure_every=1, series_len=300)


def test_grid_L18_ragged_bitexact(orc):
    w = workloads.grid_workload(chains_per_point=1, n_beta=4, n_h=5)   # 60 chains: ragged word
    run_pair(orc, 18, w["params"], w["n_chains"], w["chain_param"], 77, splits=[7, 33],
             measure_every=5, series_len=8)


@pytest.mark.parametrize("L,periodic", [(3, True), (3, False), (5, False), (7, True), (9, True),
                                        (10, False), (4, False), (12, True)])
def test_generic_lattices_bitexact(orc, L, periodic):
    rng = np.random.default_rng(100 + L)
    params = workloads.random_params(rng, 3)
    n = 45
    run_pair(orc, L, params, n, rng.integers(0, 3, n), 5 + L, splits=[3, 17], measure_every=2,
             periodic=periodic, series_len=10)


@pytest.mark.parametrize("bonds", [
    [(0, 0, 0, 1, 0), (1, 0, 1, 1, 0), (0, 0, 1, 0, 0), (0, 1, 1, 1, 0)],          # square lattice
    [(0, 0, 0, 1, 0), (0, 1, 0, 2, 0), (1, 0, 1, 1, 0), (1, 1, 1, 2, 0), (0, 0, 1, 0, 0),
     (1, 0, 2, 0, 0), (0, 1, 1, 1, 0), (1, 1, 2, 1, 0), (0, 0, 1, 1, 1), (1, 2, 2, 1, 1),
     (0, 1, 1, 0, 1), (0, 0, 2, 2, 0), (2, 0, 0, 2, 1)],                               # 13 filters
    [(0, 0, 1, 1, 1)],                                                               # one filter
])
def test_custom_filters_bitexact(orc, bonds):
    rng = np.random.default_rng(len(bonds))
    params = workloads.random_params(rng, 2)
    for L, periodic in ((6, True), (7, False)):
        run_pair(orc, L, params, 33, rng.integers(0, 2, 33), 9, splits=[11], measure_every=3,
                 periodic=periodic, bonds=bonds)


@pytest.mark.parametrize("L,interleaved", [(8, False), (6, False), (9, False), (36, False), (4, False),
                                           (18, False), (32, False), (18, True), (10, True), (22, False),
                                           (26, True)])
def test_structure_factor_matches_oracle(orc, L, interleaved):
    """S(q) against the oracle: even sides up to 32 take the bit-transposed
    accumulation (lane = chain, one warp reduction per parameter point), odd
    and larger sides the word-parallel one; interleaved parameter points give
    lane masks that are not runs of lanes."""
    n = 70
    rng = np.random.default_rng(8 + L + 100 * interleaved)
    params = workloads.random_params(rng, 3)
    cp = rng.integers(0, 3, n).astype(np.int32)
    if not interleaved:
        cp = np.sort(cp)
    s, _, _, osq = run_pair(orc, L, params, n, cp, 4, splits=[9, 12], measure_every=0,
                            sq_every=3)
    sq = s.structure_factor()
    corr, ns = s.correlations()
    for p in range(3):
        ref = osq[cp == p].sum(0) / ns[p]
        assert ns[p] == (cp == p).sum() * 7
        assert np.allclose(sq[p], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        assert corr[p, 0, 0] == ns[p] * L * L                     # C(0) = N per sample


def test_set_spins_then_sweep(orc):
    L, n, seed = 6, 50, 21
    rng = np.random.default_rng(2)
    params = workloads.random_params(rng, 2)
    cp = rng.integers(0, 2, n).astype(np.int32)
    s = crbm.Sampler(L, params, n, chain_param=cp, seed=seed)
    v0 = workloads.random_spins(rng, n, L)
    s.set_spins(v0)
    assert np.array_equal(s.get_spins(), v0)
    s.sweep(25)
    ref = v0.copy()
    orc.run(L, params, cp, ref, seed, 0, 25, 0)
    assert np.array_equal(s.get_spins(), ref)


def test_checkpoint_resume_bitexact():
    w = workloads.small_workload()
    a = crbm.Sampler(6, w["params"], 64, chain_param=w["chain_param"], seed=1, series_len=40)
    a.sweep(20)
    ck = a.save()
    a.sweep(20)
    b = crbm.Sampler(6, w["params"], 64, chain_param=w["chain_param"], seed=1, series_len=40)
    b.load(ck)
    assert b.sweep_count == 20
    b.sweep(20)
    assert np.array_equal(a.get_spins(), b.get_spins())
    assert np.array_equal(a.observables(), b.observables())
    assert np.array_equal(a.series(), b.series())


def test_host_side_errors():
    ok = dict(J=[1.0], Jp=[1.0], h=[0.5], beta=[2.0])
    bad = [dict(L=2, params=ok, n_chains=4), dict(L=6, params=dict(ok, beta=[-1.0]), n_chains=4),
           dict(L=6, params=dict(ok, J=[500.0]), n_chains=4),
           dict(L=6, params=dict(ok, h=[float("nan")]), n_chains=4),
           dict(L=6, params=ok, n_chains=0),
           dict(L=6, params=ok, n_chains=4, chain_param=[0, 0, 1, 0]),
           dict(L=6, params=ok, n_chains=4, bonds=[(0, 0, 0, 0, 0)]),
           dict(L=6, params=ok, n_chains=4, bonds=[(0, 0, 3, 0, 0)]),
           dict(L=7, params=ok, n_chains=4, periodic=False, sq_every=1)]
    for kw in bad:
        with pytest.raises(crbm.CrbmError) as e:
            crbm.Sampler(**kw)
        assert e.value.code == crbm.CRBM_EINVAL, kw
    s = crbm.Sampler(6, ok, 4)
    with pytest.raises(crbm.CrbmError):
        s.sweep(-1)
    with pytest.raises(crbm.CrbmError):
        s.set_spins(np.zeros((4, 6, 6), np.int8))


def test_set_spins_checks_values_on_the_device():
    """crbm_set_spins checks its input on the device (four bytes per load and
    the tail one at a time) and packs only when every value is +1 or -1: an
    invalid byte at the start, in the middle or in the tail is rejected with
    CRBM_EINVAL and leaves the chains as they were."""
    ok = dict(J=[1.0], Jp=[1.0], h=[0.5], beta=[1.0])
    s = crbm.Sampler(5, ok, 3, periodic=False, seed=4)      # 75 spin bytes: 18 words and a 3-byte tail
    before = s.get_spins()
    for pos, val in ((0, 0), (37, 2), (74, -3), (73, 127)):
        bad = before.copy().reshape(-1)
        bad[pos] = val
        with pytest.raises(crbm.CrbmError) as e:
            s.set_spins(bad.reshape(before.shape))
        assert e.value.code == crbm.CRBM_EINVAL
        assert np.array_equal(s.get_spins(), before), pos
    s.set_spins(-before)
    assert np.array_equal(s.get_spins(), -before)


def test_device_memory_exhaustion_returns_enomem(orc):
    """A context whose device state exceeds the GPU's memory (L=4096 streamed,
    32768 chains: 69 GB of packed spins, then 550 GB of int8 staging) fails
    with CRBM_ENOMEM from the failed cudaMalloc, before any kernel is
    launched; its earlier allocations are released and the device stays
    usable (a small run afterwards is bit-exact against the oracle)."""
    import torch
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ok = dict(J=[1.0], Jp=[1.0], h=[0.5], beta=[1.0])
    with pytest.raises(crbm.CrbmError) as e:
        crbm.Sampler(4096, ok, 32768, layout=crbm.CRBM_LAYOUT_STREAM)
    assert e.value.code == crbm.CRBM_ENOMEM, e.value
    assert "cudaMalloc" in str(e.value)
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (64 << 20), (free0, free1)
    run_pair(orc, 6, ok, 64, np.zeros(64, np.int32), seed=5, splits=[3, 2])


@pytest.mark.slow
def test_full_grid_workload_sampled_chains(orc):
    """The L=18 grid at full size (12288 chains, the benchmark's launch), with
    64 chains spread over every word checked one by one against the oracle."""
    w = workloads.grid_workload()
    ids = np.linspace(0, w["n_chains"] - 1, 64).astype(np.uint32)
    run_pair(orc, 18, w["params"], w["n_chains"], w["chain_param"], w["seed"], splits=[10, 20],
             measure_every=10, check_ids=ids)


@pytest.mark.parametrize("L,n", [(8, 70), (20, 64), (36, 130), (34, 33)])
def test_stream_layout_bitexact(orc, L, n):
    """Two-phase HBM layout (64-chain words, 16x16-cell tiles with halos),
    including ragged tiles and a ragged last 64-chain group."""
    rng = np.random.default_rng(L * 7 + n)
    params = workloads.random_params(rng, 3)
    cp = rng.integers(0, 3, n).astype(np.int32)
    s, spins, sums, _ = run_pair(orc, L, params, n, cp, 11, splits=[2, 5], measure_every=2,
                                 series_len=4, layout=crbm.CRBM_LAYOUT_STREAM)
    assert s.layout == crbm.CRBM_LAYOUT_STREAM
    m = crbm.Sampler(L, params, n, chain_param=cp, seed=11, measure_every=2,
                     layout=crbm.CRBM_LAYOUT_SMEM)
    m.sweep(7)
    assert np.array_equal(m.get_spins(), spins)
    assert np.array_equal(m.observables(), sums)


@pytest.mark.slow
def test_stream_workload_L384_sampled_chains(orc):
    """The L=384 workload at full size (3072 chains, the benchmark's launch):
    16 chains spread over all words checked against the oracle."""
    w = workloads.stream_workload()
    ids = np.linspace(0, w["n_chains"] - 1, 16).astype(np.uint32)
    run_pair(orc, 384, w["params"], w["n_chains"], w["chain_param"], w["seed"], splits=[1, 2],
             measure_every=1, check_ids=ids)


def test_stream_rejects_unsupported():
    ok = dict(J=[1.0], Jp=[1.0], h=[0.5], beta=[2.0])
    for kw in (dict(L=9), dict(L=10, periodic=False), dict(L=10, sq_every=1)):
        with pytest.raises(crbm.CrbmError) as e:
            crbm.Sampler(params=ok, n_chains=4, layout=crbm.CRBM_LAYOUT_STREAM, **kw)
        assert e.value.code == crbm.CRBM_EUNSUPPORTED


@pytest.mark.parametrize("warps,precision", [("4", 0), ("12", 0), ("13", 0), ("32", 0), ("12", 1), ("16", 1)])
def test_persistent_cta_shapes(orc, warps, precision, monkeypatch):
    """The persistent sweep runs one instantiation for CTAs of up to 12 warps
    (80 registers a thread) and another for larger ones (64): every shape
    bit-exact against the oracle (exact precision) or against a 12-warp twin
    (paper precision), with S(q) samples and measurements inside the chunks."""
    monkeypatch.setenv("CRBM_WARPS", warps)
    L, n = 18, 70
    rng = np.random.default_rng(int(warps) + 7 * precision)
    params = workloads.random_params(rng, 3)
    cp = rng.integers(0, 3, n).astype(np.int32)
    if precision == 0:
        s, _, _, _ = run_pair(orc, L, params, n, cp, 5, splits=[9, 24], measure_every=2, series_len=6,
                              sq_every=4)
        assert s.warps == int(warps)
        return
    s = crbm.Sampler(L, params, n, chain_param=cp, seed=5, measure_every=2, sq_every=4,
                     precision=crbm.CRBM_PRECISION_PAPER)
    monkeypatch.setenv("CRBM_WARPS", "12")
    ref = crbm.Sampler(L, params, n, chain_param=cp, seed=5, measure_every=2, sq_every=4,
                       precision=crbm.CRBM_PRECISION_PAPER)
    assert s.warps == int(warps) and ref.warps == 12
    for k in (9, 24):
        s.sweep(k)
        ref.sweep(k)
    assert np.array_equal(s.get_spins(), ref.get_spins())
    assert np.array_equal(s.observables(), ref.observables())
    assert np.array_equal(s.correlations()[0], ref.correlations()[0])
