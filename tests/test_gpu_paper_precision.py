"""The paper-precision mode (CRBM_PRECISION_PAPER) on the GPU against the
oracle's, bit for bit: host tables, spins, sums and series, replica exchange,
the streamed layout (which draws the tag-1 call twice), and the full L=18
grid and L=384 lattice in the launches the benchmark times."""
import numpy as np
import pytest

import paper_2511_20911_gb300 as crbm
from paper_2511_20911_gb300 import workloads

pytestmark = pytest.mark.gpu
PAPER = crbm.CRBM_PRECISION_PAPER


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    crbm.load_library()


def run_pair(orc, L, params, n_chains, chain_param, seed, splits, measure_every=1, series_len=0,
             check_ids=None, sq_every=0, layout=crbm.CRBM_LAYOUT_AUTO):
    s = crbm.Sampler(L, params, n_chains, chain_param=chain_param, seed=seed, measure_every=measure_every,
                     series_len=series_len, sq_every=sq_every, precision=PAPER, layout=layout)
    ids = np.arange(n_chains, dtype=np.uint32) if check_ids is None else np.asarray(check_ids, np.uint32)
    cp = np.asarray(chain_param, np.int32)[ids]
    spins = orc.init_spins(L, ids, seed)
    sums, oser, t = None, None, 0
    for n in splits:
        s.sweep(n)
        sums, ser, _ = orc.run(L, params, cp, spins, seed, t, n, measure_every, chain_ids=ids, sums=sums,
                               series_cap=series_len, precision=PAPER)
        if ser is not None:
            oser = ser if oser is None else np.where(ser != 0, ser, oser)
        t += n
        assert np.array_equal(s.get_spins()[ids], spins), f"spins after {t} sweeps"
    if measure_every:
        assert np.array_equal(s.observables()[ids], sums)
    if series_len:
        assert np.array_equal(s.series()[:, ids, :].transpose(1, 0, 2), oser)
    return s


@pytest.mark.parametrize("L", [6, 18])
def test_paper_tables_match_oracle(orc, L):
    rng = np.random.default_rng(L + 300)
    params = workloads.random_params(rng, 6)
    s = crbm.Sampler(L, params, 40, chain_param=np.arange(40) % 6, precision=PAPER)
    tabs, (dj, djp) = s.tables()
    for p in range(6):
        th, tv = orc.tables(L, params["J"][p], params["Jp"][p], params["h"][p], params["beta"][p],
                            precision=1)
        assert np.array_equal(tabs[p, :10], th.reshape(-1))
        assert np.array_equal(tabs[p, 10:], tv.reshape(-1))


@pytest.mark.parametrize("L,n", [(6, 64), (18, 70), (10, 33)])
def test_paper_precision_bitexact(orc, L, n):
    rng = np.random.default_rng(L * 11 + n)
    params = workloads.random_params(rng, 3)
    run_pair(orc, L, params, n, rng.integers(0, 3, n).astype(np.int32), 17 + L, splits=[3, 17],
             measure_every=2, series_len=12)


@pytest.mark.parametrize("L,n", [(8, 70), (40, 64), (34, 130)])
def test_paper_precision_stream_bitexact(orc, L, n):
    """Streamed layout in paper precision: ragged 16x16-cell tiles (W = 20,
    17) and a ragged last 64-chain group, against the oracle and against the
    shared-memory layout, which keeps the tag-1 words instead of drawing them
    again."""
    rng = np.random.default_rng(L * 13 + n)
    params = workloads.random_params(rng, 3)
    cp = rng.integers(0, 3, n).astype(np.int32)
    s = run_pair(orc, L, params, n, cp, 5 + L, splits=[2, 5], measure_every=2, series_len=4,
                 layout=crbm.CRBM_LAYOUT_STREAM)
    assert s.layout == crbm.CRBM_LAYOUT_STREAM
    m = crbm.Sampler(L, params, n, chain_param=cp, seed=5 + L, measure_every=2, precision=PAPER,
                     layout=crbm.CRBM_LAYOUT_SMEM)
    m.sweep(7)
    assert np.array_equal(m.get_spins(), s.get_spins())
    assert np.array_equal(m.observables(), s.observables())


@pytest.mark.slow
def test_paper_precision_stream_L384_sampled_chains(orc):
    """The L=384 workload at full size (3072 chains) in paper precision, as
    the benchmark's streamed paper line runs it: 16 chains over all words."""
    w = workloads.stream_workload()
    ids = np.linspace(0, w["n_chains"] - 1, 16).astype(np.uint32)
    run_pair(orc, 384, w["params"], w["n_chains"], w["chain_param"], w["seed"], splits=[1, 2],
             measure_every=1, check_ids=ids)


def test_paper_precision_tempering_bitexact(orc):
    L, n_lad = 8, 2
    betas = 0.2 * (50.0 ** (np.arange(32) / 31.0))
    params = dict(J=[1.0] * 32, Jp=[1.5] * 32, h=[1.0] * 32, beta=list(betas))
    cp = np.tile(np.arange(32, dtype=np.int32), n_lad)
    s = crbm.Sampler(L, params, 32 * n_lad, chain_param=cp, seed=4, measure_every=2, swap_every=3,
                     precision=PAPER)
    spins = orc.init_spins(L, np.arange(32 * n_lad, dtype=np.uint32), 4)
    sob = np.tile(np.arange(32, dtype=np.int32), (n_lad, 1))
    s.sweep(25)
    sums, _ = orc.run_pt(L, params, cp, spins, sob, 4, 0, 25, 2, 3, precision=PAPER)
    assert np.array_equal(s.get_spins(), spins)
    assert np.array_equal(s.permutation().reshape(n_lad, 32), sob)
    assert np.array_equal(s.observables(), sums)
    assert (sob != np.arange(32)).any()


@pytest.mark.slow
def test_paper_precision_full_grid_sampled_chains(orc):
    """The L=18 grid at full size (12288 chains) in paper precision, as the
    benchmark's paper line runs it: 64 chains spread over every word."""
    w = workloads.grid_workload()
    ids = np.linspace(0, w["n_chains"] - 1, 64).astype(np.uint32)
    run_pair(orc, 18, w["params"], w["n_chains"], w["chain_param"], w["seed"], splits=[10, 20],
             measure_every=10, check_ids=ids)


THIRTEEN = [(0, 0, 0, 1, 0), (0, 1, 0, 2, 0), (1, 0, 1, 1, 0), (1, 1, 1, 2, 0), (0, 0, 1, 0, 0),
            (1, 0, 2, 0, 0), (0, 1, 1, 1, 0), (1, 1, 2, 1, 0), (0, 0, 1, 1, 1), (1, 2, 2, 1, 1),
            (0, 1, 1, 0, 1), (0, 0, 2, 2, 0), (2, 0, 0, 2, 1)]


@pytest.mark.parametrize("shape,periodic,bonds", [
    (9, True, None), (7, False, None), ((18, 12), (True, False), None), ((9, 5), (False, False), None),
    ((10, 3), (True, True), None),
    (6, True, [(0, 0, 0, 1, 0), (1, 0, 1, 1, 0), (0, 0, 1, 0, 0), (0, 1, 1, 1, 0)]),
    (7, False, [(0, 0, 1, 1, 1)])])
def test_paper_precision_on_the_generic_sweep(orc, shape, periodic, bonds):
    """Odd sides, open axes, laterally confined strips and custom filter lists
    of at most ten filters in paper precision (the generic SMEM sweep: filter k
    draws half k & 1 of word k >> 1 of tag 0, filters 8 and 9 of word 0 of tag
    1, spin x half x & 1 of word 1 + (x >> 1) of tag 1): spins, sums and
    series against the oracle, bit for bit."""
    L, Lc = shape if isinstance(shape, tuple) else (shape, shape)
    pr, pc = periodic if isinstance(periodic, tuple) else (periodic, periodic)
    rng = np.random.default_rng(L * 7 + Lc + (0 if bonds is None else len(bonds)))
    params = workloads.random_params(rng, 3)
    n = 45
    cp = rng.integers(0, 3, n).astype(np.int32)
    seed = 31 + L + Lc
    s = crbm.Sampler(L, params, n, chain_param=cp, seed=seed, periodic=pr, L_cols=Lc,
                     periodic_cols=crbm.CRBM_BC_PERIODIC if pc else crbm.CRBM_BC_OPEN, measure_every=2,
                     series_len=8, precision=PAPER, bonds=bonds)
    assert s.layout == crbm.CRBM_LAYOUT_SMEM
    ids = np.arange(n, dtype=np.uint32)
    spins = orc.init_spins((L, Lc), ids, seed)
    assert np.array_equal(s.get_spins(), spins)
    sums, oser, t = None, None, 0
    for k in (3, 9):
        s.sweep(k)
        sums, ser, _ = orc.run((L, Lc), params, cp, spins, seed, t, k, 2, chain_ids=ids, periodic=(pr, pc),
                               bonds=bonds, sums=sums, series_cap=8, precision=PAPER)
        oser = ser if oser is None else np.where(ser != 0, ser, oser)
        t += k
        assert np.array_equal(s.get_spins(), spins), f"spins after {t} sweeps"
    assert np.array_equal(s.observables(), sums)
    assert np.array_equal(s.series().transpose(1, 0, 2), oser)


def test_paper_precision_where_unsupported():
    ok = dict(J=[1.0], Jp=[1.0], h=[0.5], beta=[2.0])
    for kw in (dict(L=6, bonds=THIRTEEN), dict(L=9, layout=crbm.CRBM_LAYOUT_STREAM)):
        with pytest.raises(crbm.CrbmError) as e:
            crbm.Sampler(params=ok, n_chains=32, precision=PAPER, **kw)
        assert e.value.code == crbm.CRBM_EUNSUPPORTED, kw
    with pytest.raises(crbm.CrbmError) as e:
        crbm.Sampler(6, ok, 32, precision=7)
    assert e.value.code == crbm.CRBM_EINVAL
    a = crbm.Sampler(6, ok, 32, precision=PAPER)
    b = crbm.Sampler(6, ok, 32)
    with pytest.raises(crbm.CrbmError) as e:    # a batch member twice
        crbm.Batch([a, a])
    assert e.value.code == crbm.CRBM_EINVAL
    prop = crbm.Proposal(seed=1)
    with pytest.raises(crbm.CrbmError) as e:
        prop.passes(a, 1)
    assert e.value.code == crbm.CRBM_EUNSUPPORTED
    with pytest.raises(crbm.CrbmError) as e:       # a checkpoint keeps its precision
        b.load(a.save())
    assert e.value.code == crbm.CRBM_EINVAL
