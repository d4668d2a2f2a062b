"""Bit-plane uniforms (CRBM_RNG_BITPLANE) on the GPU against the oracle's
ORC_RNG_BITPLANE mode, bit for bit: spins, sums and series on square lattices
and rectangles (ragged 32-chain words, signs of J and J' both ways, staged and
global node records, several CTA shapes), the streamed layout (ragged tiles,
against the oracle and the SMEM layout), the full L=18 grid and L=384 lattice
on sampled chains in the launches the benchmark times, and the contexts that
refuse the mode."""
import numpy as np
import pytest

import paper_2511_20911_gb300 as crbm
from paper_2511_20911_gb300 import workloads

pytestmark = pytest.mark.gpu
BP = crbm.CRBM_RNG_BITPLANE


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    crbm.load_library()


def run_pair(orc, shape, params, n, cp, seed, splits, measure_every=2, series_len=0, check_ids=None,
             layout=crbm.CRBM_LAYOUT_SMEM):
    L, Lc = shape if isinstance(shape, tuple) else (shape, shape)
    s = crbm.Sampler(L, params, n, chain_param=cp, seed=seed, measure_every=measure_every,
                     series_len=series_len, L_cols=Lc if Lc != L else 0, rng=BP, layout=layout)
    assert s.layout == layout
    ids = np.arange(n, dtype=np.uint32) if check_ids is None else np.asarray(check_ids, np.uint32)
    cpi = np.asarray(cp, np.int32)[ids]
    spins = orc.init_spins((L, Lc), ids, seed)
    sums, oser, t = None, None, 0
    for k in splits:
        s.sweep(k)
        sums, ser, _ = orc.run((L, Lc), params, cpi, spins, seed, t, k, measure_every, chain_ids=ids, sums=sums,
                               series_cap=series_len, rng=orc.RNG_BITPLANE)
        if ser is not None:
            oser = ser if oser is None else np.where(ser != 0, ser, oser)
        t += k
        assert np.array_equal(s.get_spins()[ids], spins), f"spins after {t} sweeps"
    if measure_every:
        assert np.array_equal(s.observables()[ids], sums)
    if series_len:
        assert np.array_equal(s.series()[:, ids, :].transpose(1, 0, 2), oser)
    return s


@pytest.mark.parametrize("L,n", [(4, 40), (6, 64), (10, 33), (18, 70), (20, 96)])
def test_bitplane_bitexact(orc, L, n):
    rng = np.random.default_rng(L * 17 + n)
    params = workloads.random_params(rng, 4)
    run_pair(orc, L, params, n, rng.integers(0, 4, n).astype(np.int32), 3 + L, splits=[3, 14],
             series_len=10)


@pytest.mark.parametrize("shape", [(18, 12), (8, 30)])
def test_bitplane_rectangles_bitexact(orc, shape):
    rng = np.random.default_rng(shape[0] * 41 + shape[1])
    params = workloads.random_params(rng, 3)
    n = 50
    run_pair(orc, shape, params, n, rng.integers(0, 3, n).astype(np.int32), 8, splits=[4, 9])


@pytest.mark.parametrize("warps", ["1", "5", "16", "32"])
def test_bitplane_cta_shapes(orc, warps, monkeypatch):
    """One warp (every node loop runs many rounds), five (ragged last round),
    sixteen and thirty-two (most warps idle in the visible half-step at L=12,
    one CTA per SM)."""
    monkeypatch.setenv("CRBM_WARPS", warps)
    rng = np.random.default_rng(int(warps))
    params = workloads.random_params(rng, 2)
    run_pair(orc, 12, params, 64, (np.arange(64) % 2).astype(np.int32), 21, splits=[5, 6])


def test_bitplane_records_from_global_memory(orc):
    """L=96: the node records (about 200 KB) do not fit beside the lattice in
    shared memory and are read through L1."""
    rng = np.random.default_rng(96)
    params = workloads.random_params(rng, 2)
    run_pair(orc, 96, params, 40, (np.arange(40) % 2).astype(np.int32), 4, splits=[2, 2], measure_every=1)


@pytest.mark.parametrize("L,n", [(8, 70), (40, 64), (34, 130)])
def test_bitplane_stream_bitexact(orc, L, n):
    """Streamed layout: 16 x 16-cell tiles (ragged at W = 20 and 17), hidden
    words bit-sliced in HBM, a ragged last 64-chain group; against the oracle
    and against the SMEM layout."""
    rng = np.random.default_rng(L * 29 + n)
    params = workloads.random_params(rng, 3)
    cp = rng.integers(0, 3, n).astype(np.int32)
    s = run_pair(orc, L, params, n, cp, 13 + L, splits=[2, 5], series_len=4, layout=crbm.CRBM_LAYOUT_STREAM)
    m = crbm.Sampler(L, params, n, chain_param=cp, seed=13 + L, measure_every=2, rng=BP,
                     layout=crbm.CRBM_LAYOUT_SMEM)
    m.sweep(7)
    assert np.array_equal(m.get_spins(), s.get_spins())
    assert np.array_equal(m.observables(), s.observables())


@pytest.mark.slow
def test_bitplane_stream_L384_sampled_chains(orc):
    """The L=384 workload at full size (3072 chains) with bit-plane uniforms,
    as the benchmark's streamed bit-plane line runs it: 16 chains over all
    words."""
    w = workloads.stream_workload()
    ids = np.linspace(0, w["n_chains"] - 1, 16).astype(np.uint32)
    run_pair(orc, 384, w["params"], w["n_chains"], w["chain_param"], w["seed"], splits=[1, 2],
             measure_every=1, check_ids=ids, layout=crbm.CRBM_LAYOUT_STREAM)


@pytest.mark.slow
def test_bitplane_full_grid_sampled_chains(orc):
    """The L=18 grid at full size (12288 chains over 768 points) as the
    benchmark's bit-plane line runs it: 64 chains spread over every word."""
    w = workloads.grid_workload()
    ids = np.linspace(0, w["n_chains"] - 1, 64).astype(np.uint32)
    run_pair(orc, 18, w["params"], w["n_chains"], w["chain_param"], w["seed"], splits=[10, 20],
             measure_every=10, check_ids=ids)


@pytest.mark.parametrize("L,n_lad,signs", [(8, 2, (1.0, 1.5)), (12, 3, (-1.0, 0.5))])
def test_bitplane_tempering_bitexact(orc, L, n_lad, signs):
    """Replica exchange with bit-plane uniforms: slot l of a ladder draws as
    chain 32 w + l and reads the threshold planes of the rung it holds (the
    planes are re-permuted after every swap round); spins, permutation and
    sums against the oracle, with both coupling signs."""
    J, Jp = signs
    betas = 0.2 * (50.0 ** (np.arange(32) / 31.0))
    params = dict(J=[J] * 32, Jp=[Jp] * 32, h=[0.75] * 32, beta=list(betas))
    cp = np.tile(np.arange(32, dtype=np.int32), n_lad)
    s = crbm.Sampler(L, params, 32 * n_lad, chain_param=cp, seed=6, measure_every=2, swap_every=3, rng=BP)
    spins = orc.init_spins(L, np.arange(32 * n_lad, dtype=np.uint32), 6)
    sob = np.tile(np.arange(32, dtype=np.int32), (n_lad, 1))
    sums = None
    t = 0
    for k in (10, 17):
        s.sweep(k)
        sums, _ = orc.run_pt(L, params, cp, spins, sob, 6, t, k, 2, 3, sums=sums, rng=orc.RNG_BITPLANE)
        t += k
        assert np.array_equal(s.get_spins(), spins), f"spins after {t} sweeps"
        assert np.array_equal(s.permutation().reshape(n_lad, 32), sob)
    assert np.array_equal(s.observables(), sums)
    assert (sob != np.arange(32)).any()


def test_bitplane_differs_from_lane_uniforms():
    params = dict(J=[1.0], Jp=[1.5], h=[0.5], beta=[0.8])
    a = crbm.Sampler(12, params, 64, seed=3)
    b = crbm.Sampler(12, params, 64, seed=3, rng=BP)
    assert np.array_equal(a.get_spins(), b.get_spins())   # same initial spins
    a.sweep(3)
    b.sweep(3)
    assert not np.array_equal(a.get_spins(), b.get_spins())
    with pytest.raises(crbm.CrbmError) as e:                # a checkpoint keeps its uniform source
        a.load(b.save())
    assert e.value.code == crbm.CRBM_EINVAL


def test_bitplane_where_unsupported():
    ok = dict(J=[1.0], Jp=[1.0], h=[0.5], beta=[2.0])
    for kw in (dict(L=9), dict(L=10, periodic=False),
               dict(L=20, L_cols=12, periodic_cols=crbm.CRBM_BC_OPEN, layout=crbm.CRBM_LAYOUT_STREAM),
               dict(L=10, precision=crbm.CRBM_PRECISION_PAPER), dict(L=10, sq_every=2)):
        with pytest.raises(crbm.CrbmError) as e:
            crbm.Sampler(params=ok, n_chains=32, rng=BP, **kw)
        assert e.value.code == crbm.CRBM_EUNSUPPORTED, kw
    ladder = dict(J=[1.0] * 32, Jp=[1.0] * 32, h=[0.5] * 32, beta=list(0.5 + 0.1 * np.arange(32)))
    with pytest.raises(crbm.CrbmError) as e:
        crbm.Sampler(8, ladder, 32, chain_param=np.arange(32), swap_every=2, rng=BP,
                     layout=crbm.CRBM_LAYOUT_STREAM)
    assert e.value.code == crbm.CRBM_EUNSUPPORTED
    with pytest.raises(crbm.CrbmError) as e:
        crbm.Sampler(8, ok, 32, rng=7)
    assert e.value.code == crbm.CRBM_EINVAL
    a = crbm.Sampler(8, ok, 32, rng=BP)
    with pytest.raises(crbm.CrbmError) as e:    # a batch member twice
        crbm.Batch([a, a])
    assert e.value.code == crbm.CRBM_EINVAL
    with pytest.raises(crbm.CrbmError) as e:
        crbm.Proposal(seed=1).passes(a, 1)
    assert e.value.code == crbm.CRBM_EUNSUPPORTED
