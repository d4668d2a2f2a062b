"""crbm_sweep_stream_noalloc, the streamed sweep that allocates nothing.

It exists for callers that cannot call cudaMalloc (code running under another
framework's allocator or memory pool, or a service whose device memory is
fixed at start-up): they pass their own device spins, and the sweep's scratch
comes from a fixed array in the library.  Here its result, called twice in a
row through the C ABI, must equal the context-based streamed sweep bit for
bit.  Collected last on purpose: a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

import paper_2511_20911_gb300 as crbm
from paper_2511_20911_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def pack_stream(spins):
    """[n][L][L] int8 +-1 -> streamed layout u32 [ceil(n/64)][L*L][2]."""
    n, L, _ = spins.shape
    G = (n + 63) // 64
    bits = np.zeros((G * 64, L * L), np.uint64)
    bits[:n] = spins.reshape(n, -1) > 0
    words = (bits.reshape(G, 2, 32, L * L) << np.arange(32, dtype=np.uint64)[None, None, :, None]).sum(2)
    return np.ascontiguousarray(words.astype(np.uint32).transpose(0, 2, 1))


def unpack_stream(words, n, L):
    G = words.shape[0]
    w = words.transpose(0, 2, 1).astype(np.uint64)                     # [G][2][N]
    bits = (w[:, :, None, :] >> np.arange(32, dtype=np.uint64)[None, None, :, None]) & 1
    return np.where(bits.reshape(G * 64, L, L)[:n] == 1, 1, -1).astype(np.int8)


def make_params(L, params, n, cp, seed, stream, precision=0):
    keep = {k: np.ascontiguousarray(params[k], np.float64) for k in ("J", "Jp", "h", "beta")}
    keep["cp"] = np.ascontiguousarray(cp, np.int32)
    p = crbm.crbm_params()
    p.L, p.periodic, p.bonds, p.n_bonds = L, 1, None, 0
    for name in ("J", "Jp", "h", "beta"):
        setattr(p, name, keep[name].ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    p.n_params = len(keep["J"])
    p.chain_param = keep["cp"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p.n_chains, p.seed = n, seed
    p.precision = precision
    p.stream = ctypes.c_void_p(int(stream)) if stream else None
    return p, keep


@pytest.mark.parametrize("precision", [crbm.CRBM_PRECISION_EXACT, crbm.CRBM_PRECISION_PAPER])
def test_noalloc_stream_sweep_matches_context(torch_cuda, precision):
    torch = torch_cuda
    lib = crbm.load_library()
    L, n, seed = 20, 70, 31
    rng = np.random.default_rng(5)
    params = workloads.random_params(rng, 3)
    cp = rng.integers(0, 3, n).astype(np.int32)
    ctx = crbm.Sampler(L, params, n, chain_param=cp, seed=seed, measure_every=0,
                       layout=crbm.CRBM_LAYOUT_STREAM, precision=precision)
    dev = torch.from_numpy(pack_stream(ctx.get_spins()).view(np.int32)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    p, _keep = make_params(L, params, n, cp, seed, stream, precision)
    t = 0
    for n_sweeps in (3, 4):                      # two calls in a row, continuing the counter
        rc = lib.crbm_sweep_stream_noalloc(ctypes.byref(p), ctypes.c_void_p(dev.data_ptr()), t, n_sweeps)
        assert rc == crbm.CRBM_OK
        torch.cuda.synchronize()
        ctx.sweep(n_sweeps)
        t += n_sweeps
        got = unpack_stream(dev.cpu().numpy().view(np.uint32), n, L)
        assert np.array_equal(got, ctx.get_spins()), f"after {t} sweeps"


def test_noalloc_rejects_oversize_and_bad_arguments(torch_cuda):
    """Host-side checks, each with a spin buffer of the full size the call
    names (the requests are refused before any GPU work)."""
    torch = torch_cuda
    lib = crbm.load_library()
    w = workloads.stream_workload()
    n = 4096                                     # L=384: far beyond the fixed scratch
    p, _keep = make_params(384, w["params"], n, np.zeros(n, np.int32), 1, 0)
    big = torch.zeros(64 * 384 * 384 * 2, dtype=torch.int32, device="cuda")
    ptr = ctypes.c_void_p(big.data_ptr())
    assert lib.crbm_sweep_stream_noalloc(ctypes.byref(p), ptr, 0, 1) == crbm.CRBM_EUNSUPPORTED
    p.L = 21
    assert lib.crbm_sweep_stream_noalloc(ctypes.byref(p), ptr, 0, 1) == crbm.CRBM_EINVAL
    p.L = 20
    assert lib.crbm_sweep_stream_noalloc(ctypes.byref(p), ptr, -1, 1) == crbm.CRBM_EINVAL
    assert lib.crbm_sweep_stream_noalloc(ctypes.byref(p), None, 0, 1) == crbm.CRBM_EINVAL
    for field, bad in (("precision", 7), ("L_cols", 12), ("periodic_cols", crbm.CRBM_BC_OPEN),
                       ("periodic_cols", 5), ("rng", crbm.CRBM_RNG_BITPLANE)):
        old = getattr(p, field)
        setattr(p, field, bad)
        assert lib.crbm_sweep_stream_noalloc(ctypes.byref(p), ptr, 0, 1) == crbm.CRBM_EINVAL, field
        setattr(p, field, old)
