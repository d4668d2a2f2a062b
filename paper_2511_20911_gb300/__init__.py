"""Python binding of the GB300 CRBM block-Gibbs sampler (include/crbm.h).

Argument marshalling only: every step of the sampling path runs in the CUDA
kernels of ``libcrbm.so``.  PyTorch is used for the CUDA stream (the current
torch stream is handed to the library); the library owns its device memory.
There is no CPU fallback: if the compiled library is missing this module
raises on first use.

Method: Brahma et al., arXiv 2511.20911 -- the Shastry–Sutherland Ising
lattice (Eq. 1) mapped onto a convolutional RBM (Eqs. 3-8) and sampled by
block Gibbs sweeps (Eqs. 9-10).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB, build

CRBM_OK, CRBM_EINVAL, CRBM_ENOMEM, CRBM_ECUDA, CRBM_ETIMEOUT, CRBM_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
CRBM_NSUM = 11
CRBM_LAYOUT_AUTO, CRBM_LAYOUT_SMEM, CRBM_LAYOUT_STREAM = 0, 1, 2
CRBM_PRECISION_EXACT, CRBM_PRECISION_PAPER = 0, 1
CRBM_BC_AS_ROWS, CRBM_BC_PERIODIC, CRBM_BC_OPEN = 0, 1, 2
CRBM_RNG_LANE, CRBM_RNG_BITPLANE = 0, 1
CRBM_SMEM_MAX_L = 96
SUM_FIELDS = ("n", "NJ", "NJp", "M", "absM", "NJ2", "NJp2", "M2", "NJ_NJp", "NJ_M", "NJp_M")

# Names of every entry point include/crbm.h declares.
ABI_FUNCTIONS = (
    "crbm_create", "crbm_destroy", "crbm_sweep", "crbm_sweep_count", "crbm_observables",
    "crbm_series", "crbm_correlations", "crbm_structure_factor", "crbm_reset_observables",
    "crbm_get_spins", "crbm_set_spins", "crbm_get_tables", "crbm_get_permutation", "crbm_layout",
    "crbm_launch_count", "crbm_autotune", "crbm_warps", "crbm_set_targets", "crbm_first_hits", "crbm_batch_create", "crbm_batch_sweep",
    "crbm_batch_threads", "crbm_batch_autotune", "crbm_batch_cluster", "crbm_batch_last_error", "crbm_batch_destroy",
    "crbm_proposal_create", "crbm_proposal_destroy", "crbm_proposal_set_weights",
    "crbm_proposal_get_weights", "crbm_proposal_train", "crbm_proposal_loss_grad",
    "crbm_proposal_pass", "crbm_sweep_mixed", "crbm_sweep_mixed_every", "crbm_proposal_inspect",
    "crbm_proposal_stats",
    "crbm_proposal_last_error",
    "crbm_save", "crbm_load", "crbm_philox", "crbm_philox_stream", "crbm_sweep_stream_noalloc",
    "crbm_last_error",
)


class CrbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"crbm error {code}: {msg}")
        self.code = code


class crbm_bond(ctypes.Structure):
    _fields_ = [("r1", ctypes.c_int8), ("c1", ctypes.c_int8), ("r2", ctypes.c_int8),
                ("c2", ctypes.c_int8), ("cls", ctypes.c_uint8)]


class crbm_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("periodic", ctypes.c_int32),
                ("bonds", ctypes.POINTER(crbm_bond)), ("n_bonds", ctypes.c_int32),
                ("J", ctypes.POINTER(ctypes.c_double)), ("Jp", ctypes.POINTER(ctypes.c_double)),
                ("h", ctypes.POINTER(ctypes.c_double)), ("beta", ctypes.POINTER(ctypes.c_double)),
                ("n_params", ctypes.c_int32), ("chain_param", ctypes.POINTER(ctypes.c_int32)),
                ("n_chains", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("measure_every", ctypes.c_int32), ("series_len", ctypes.c_int32),
                ("sq_every", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("swap_every", ctypes.c_int32), ("stream", ctypes.c_void_p), ("precision", ctypes.c_int32),
                ("L_cols", ctypes.c_int32), ("periodic_cols", ctypes.c_int32),
                ("h_odd", ctypes.POINTER(ctypes.c_double)), ("rng", ctypes.c_int32)]


_lib = None


def load_library(path: str | None = None):
    """Load libcrbm.so (building it if absent and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB
    if not os.path.exists(p):
        p = build()
    lib = ctypes.CDLL(p)
    c = ctypes
    vp = c.c_void_p
    sigs = {
        "crbm_create": (c.c_int, [c.POINTER(vp), c.POINTER(crbm_params)]),
        "crbm_destroy": (None, [vp]),
        "crbm_sweep": (c.c_int, [vp, c.c_int64]),
        "crbm_sweep_count": (c.c_int64, [vp]),
        "crbm_observables": (c.c_int, [vp, c.POINTER(c.c_int64), c.c_size_t]),
        "crbm_series": (c.c_int, [vp, c.POINTER(c.c_int32), c.c_size_t]),
        "crbm_correlations": (c.c_int, [vp, c.POINTER(c.c_int64), c.c_size_t, c.POINTER(c.c_int64)]),
        "crbm_structure_factor": (c.c_int, [vp, c.POINTER(c.c_double), c.c_size_t]),
        "crbm_reset_observables": (c.c_int, [vp]),
        "crbm_get_spins": (c.c_int, [vp, c.POINTER(c.c_int8), c.c_size_t]),
        "crbm_set_spins": (c.c_int, [vp, c.POINTER(c.c_int8), c.c_size_t]),
        "crbm_get_tables": (c.c_int, [vp, c.POINTER(c.c_uint32), c.c_size_t, c.POINTER(c.c_int32)]),
        "crbm_get_permutation": (c.c_int, [vp, c.POINTER(c.c_int32), c.c_size_t]),
        "crbm_layout": (c.c_int, [vp]),
        "crbm_autotune": (c.c_int, [vp, c.c_int64, c.POINTER(c.c_int32)]),
        "crbm_warps": (c.c_int, [vp]),
        "crbm_batch_create": (c.c_int, [c.POINTER(vp), c.POINTER(vp), c.c_int32]),
        "crbm_batch_sweep": (c.c_int, [vp, c.c_int64]),
        "crbm_batch_threads": (c.c_int, [vp]),
        "crbm_batch_autotune": (c.c_int, [vp, c.c_int64, c.POINTER(c.c_int32)]),
        "crbm_batch_cluster": (c.c_int, [vp]),
        "crbm_set_targets": (c.c_int, [vp, c.POINTER(c.c_int64), c.c_int32]),
        "crbm_first_hits": (c.c_int, [vp, c.POINTER(c.c_int64), c.c_size_t]),
        "crbm_batch_last_error": (c.c_char_p, [vp]),
        "crbm_batch_destroy": (None, [vp]),
        "crbm_proposal_create": (c.c_int, [c.POINTER(vp), c.c_int32, c.c_uint64]),
        "crbm_proposal_destroy": (None, [vp]),
        "crbm_proposal_set_weights": (c.c_int, [vp, c.POINTER(c.c_float), c.c_size_t]),
        "crbm_proposal_get_weights": (c.c_int, [vp, c.POINTER(c.c_float), c.c_size_t]),
        "crbm_proposal_train": (c.c_int, [vp, vp, c.c_int32, c.c_int32, c.c_float, c.c_int32,
                                          c.POINTER(c.c_float)]),
        "crbm_proposal_loss_grad": (c.c_int, [vp, c.POINTER(c.c_int8), c.c_int32, c.POINTER(c.c_int32),
                                              c.POINTER(c.c_float), c.c_int32, c.POINTER(c.c_float),
                                              c.POINTER(c.c_float)]),
        "crbm_proposal_pass": (c.c_int, [vp, vp, c.c_int64]),
        "crbm_sweep_mixed": (c.c_int, [vp, vp, c.c_int64]),
        "crbm_sweep_mixed_every": (c.c_int, [vp, vp, c.c_int64, c.c_int32]),
        "crbm_proposal_inspect": (c.c_int, [vp, vp, vp, c.c_size_t]),
        "crbm_proposal_stats": (c.c_int, [vp, c.POINTER(c.c_int64), c.POINTER(c.c_int64)]),
        "crbm_proposal_last_error": (c.c_char_p, []),
        "crbm_launch_count": (c.c_int64, [vp]),
        "crbm_save": (c.c_int, [vp, vp, c.POINTER(c.c_size_t)]),
        "crbm_load": (c.c_int, [vp, vp, c.c_size_t]),
        "crbm_philox": (c.c_int, [c.POINTER(c.c_uint32), c.POINTER(c.c_uint32), c.c_size_t]),
        "crbm_philox_stream": (c.c_int, [vp, c.c_int32, c.c_int32, c.c_int32, c.c_uint64, vp]),
        "crbm_sweep_stream_noalloc": (c.c_int, [c.POINTER(crbm_params), vp, c.c_int64, c.c_int64]),
        "crbm_last_error": (c.c_char_p, [vp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc, ctx=None):
    if rc != CRBM_OK:
        msg = load_library().crbm_last_error(ctx)
        raise CrbmError(rc, msg.decode() if msg else "")


def current_stream_handle():
    """The raw cudaStream_t of torch's current stream (0 if torch has no CUDA)."""
    import torch
    if not torch.cuda.is_available():
        raise CrbmError(CRBM_ECUDA, "no CUDA device: the sampler runs only on the GPU")
    return torch.cuda.current_stream().cuda_stream


class Sampler:
    """One context of include/crbm.h: chains of L x L spins at parameter points.

    params: dict with equal-length sequences J, Jp, h, beta (one entry per
    parameter point); chain_param maps each chain to a point.
    """

    def __init__(self, L, params, n_chains, chain_param=None, seed=1, periodic=True,
                 bonds=None, measure_every=1, series_len=0, sq_every=0,
                 layout=CRBM_LAYOUT_AUTO, swap_every=0, stream=None, precision=0, L_cols=0,
                 periodic_cols=CRBM_BC_AS_ROWS, rng=CRBM_RNG_LANE):
        lib = load_library()
        self.L, self.n_chains = int(L), int(n_chains)
        self.L_cols = int(L_cols) if L_cols else self.L
        self._J = np.ascontiguousarray(params["J"], np.float64)
        self._Jp = np.ascontiguousarray(params["Jp"], np.float64)
        self._h = np.ascontiguousarray(params["h"], np.float64)
        self._beta = np.ascontiguousarray(params["beta"], np.float64)
        self._h_odd = (None if params.get("h_odd") is None
                       else np.ascontiguousarray(params["h_odd"], np.float64))
        self.n_params = len(self._J)
        self.series_len, self.sq_every = int(series_len), int(sq_every)
        self._cp = None if chain_param is None else np.ascontiguousarray(chain_param, np.int32)
        if self._cp is not None and len(self._cp) != self.n_chains:
            raise CrbmError(CRBM_EINVAL, "chain_param must have n_chains entries")
        self._bonds = None
        if bonds is not None:
            self._bonds = (crbm_bond * len(bonds))(*[crbm_bond(*b) for b in bonds])
        if stream is None:
            stream = current_stream_handle()
        p = crbm_params()
        p.L, p.periodic = self.L, int(bool(periodic))
        p.bonds = self._bonds if self._bonds is not None else None
        p.n_bonds = len(bonds) if bonds is not None else 0
        p.J, p.Jp = _ptr(self._J, ctypes.c_double), _ptr(self._Jp, ctypes.c_double)
        p.h, p.beta = _ptr(self._h, ctypes.c_double), _ptr(self._beta, ctypes.c_double)
        p.n_params = self.n_params
        p.chain_param = _ptr(self._cp, ctypes.c_int32) if self._cp is not None else None
        p.n_chains = self.n_chains
        p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        p.measure_every, p.series_len, p.sq_every = int(measure_every), self.series_len, self.sq_every
        p.layout = int(layout)
        p.swap_every = int(swap_every)
        p.stream = ctypes.c_void_p(int(stream)) if stream else None
        p.precision = int(precision)
        p.L_cols, p.periodic_cols = int(L_cols), int(periodic_cols)
        p.h_odd = _ptr(self._h_odd, ctypes.c_double) if self._h_odd is not None else None
        p.rng = int(rng)
        self.precision, self.rng = int(precision), int(rng)
        h = ctypes.c_void_p()
        _check(lib.crbm_create(ctypes.byref(h), ctypes.byref(p)))
        self._ctx = h
        self._lib = lib

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.crbm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n_sweeps):
        _check(self._lib.crbm_sweep(self._ctx, int(n_sweeps)), self._ctx)

    @property
    def sweep_count(self):
        return int(self._lib.crbm_sweep_count(self._ctx))

    @property
    def launch_count(self):
        return int(self._lib.crbm_launch_count(self._ctx))

    @property
    def layout(self):
        return int(self._lib.crbm_layout(self._ctx))

    def observables(self, out=None):
        """Per-chain sums [n_chains][CRBM_NSUM]; `out` (C-contiguous int64 of that
        shape, e.g. in pinned memory) receives them in place when given."""
        if out is None:
            out = np.zeros((self.n_chains, CRBM_NSUM), np.int64)
        elif out.dtype != np.int64 or out.shape != (self.n_chains, CRBM_NSUM) or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous int64 array of shape (n_chains, CRBM_NSUM)")
        _check(self._lib.crbm_observables(self._ctx, _ptr(out, ctypes.c_int64), out.size), self._ctx)
        return out

    def series(self):
        out = np.zeros((self.series_len, self.n_chains, 3), np.int32)
        _check(self._lib.crbm_series(self._ctx, _ptr(out, ctypes.c_int32), out.size), self._ctx)
        return out

    def correlations(self):
        out = np.zeros((self.n_params, self.L, self.L), np.int64)
        ns = np.zeros(self.n_params, np.int64)
        _check(self._lib.crbm_correlations(self._ctx, _ptr(out, ctypes.c_int64), out.size,
                                           _ptr(ns, ctypes.c_int64)), self._ctx)
        return out, ns

    def structure_factor(self):
        out = np.zeros((self.n_params, self.L, self.L), np.float64)
        _check(self._lib.crbm_structure_factor(self._ctx, _ptr(out, ctypes.c_double), out.size),
               self._ctx)
        return out

    def set_targets(self, e_target):
        """Target energy per parameter point (1/16 units); clears the first-hit records."""
        t = np.ascontiguousarray(e_target, np.int64)
        _check(self._lib.crbm_set_targets(self._ctx, _ptr(t, ctypes.c_int64), len(t)), self._ctx)

    def first_hits(self):
        """Per chain, the first sweep count after which its energy reached the target (-1: not yet)."""
        out = np.zeros(self.n_chains, np.int64)
        _check(self._lib.crbm_first_hits(self._ctx, _ptr(out, ctypes.c_int64), out.size), self._ctx)
        return out

    def reset_observables(self):
        _check(self._lib.crbm_reset_observables(self._ctx), self._ctx)

    def get_spins(self, out=None):
        if out is None:
            out = np.zeros((self.n_chains, self.L, self.L_cols), np.int8)
        _check(self._lib.crbm_get_spins(self._ctx, _ptr(out, ctypes.c_int8), out.size), self._ctx)
        return out

    def set_spins(self, spins):
        a = np.ascontiguousarray(spins, np.int8)
        _check(self._lib.crbm_set_spins(self._ctx, _ptr(a, ctypes.c_int8), a.size), self._ctx)

    def autotune(self, probe_sweeps=200):
        """Time the SMEM sweep's CTA shapes on scratch copies; returns the warps kept."""
        best = ctypes.c_int32(0)
        _check(self._lib.crbm_autotune(self._ctx, int(probe_sweeps), ctypes.byref(best)), self._ctx)
        return best.value

    @property
    def warps(self):
        return int(self._lib.crbm_warps(self._ctx))

    def permutation(self):
        """[n_chains] int32: entry 32 l + k = slot of ladder l holding rung k."""
        out = np.zeros(self.n_chains, np.int32)
        _check(self._lib.crbm_get_permutation(self._ctx, _ptr(out, ctypes.c_int32), out.size), self._ctx)
        return out

    def tables(self):
        dims = np.zeros(2, np.int32)
        _check(self._lib.crbm_get_tables(self._ctx, None, 0, _ptr(dims, ctypes.c_int32)), self._ctx)
        dj, djp = int(dims[0]), int(dims[1])
        ntab = 10 + (2 if self._h_odd is not None else 1) * (2 * dj + 1) * (2 * djp + 1)
        out = np.zeros((self.n_params, ntab), np.uint32)
        _check(self._lib.crbm_get_tables(self._ctx, _ptr(out, ctypes.c_uint32), out.size, None),
               self._ctx)
        return out, (dj, djp)

    def save(self):
        n = ctypes.c_size_t(0)
        _check(self._lib.crbm_save(self._ctx, None, ctypes.byref(n)), self._ctx)
        buf = np.zeros(n.value, np.uint8)
        _check(self._lib.crbm_save(self._ctx, buf.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)),
               self._ctx)
        return buf

    def load(self, buf):
        b = np.ascontiguousarray(buf, np.uint8)
        _check(self._lib.crbm_load(self._ctx, b.ctypes.data_as(ctypes.c_void_p), b.size), self._ctx)


class Batch:
    """Several Samplers advanced by one graph-captured kernel launch
    (crbm_batch_*).  Keep the members alive while the batch exists."""

    def __init__(self, samplers):
        lib = load_library()
        self.members = list(samplers)
        arr = (ctypes.c_void_p * len(self.members))(*[s._ctx.value for s in self.members])
        h = ctypes.c_void_p()
        rc = lib.crbm_batch_create(ctypes.byref(h), arr, len(self.members))
        if rc != CRBM_OK:
            raise CrbmError(rc, (lib.crbm_batch_last_error(None) or b"").decode())
        self._b, self._lib = h, lib

    def sweep(self, n_sweeps):
        rc = self._lib.crbm_batch_sweep(self._b, int(n_sweeps))
        if rc != CRBM_OK:
            raise CrbmError(rc, (self._lib.crbm_batch_last_error(self._b) or b"").decode())

    @property
    def threads(self):
        return int(self._lib.crbm_batch_threads(self._b))

    def autotune(self, probe_sweeps=200):
        """Time the batched launch's CTA shapes (crbm_batch_autotune; the
        members' state is put back); returns the threads per CTA kept."""
        best = ctypes.c_int32(0)
        rc = self._lib.crbm_batch_autotune(self._b, int(probe_sweeps), ctypes.byref(best))
        if rc != CRBM_OK:
            raise CrbmError(rc, (self._lib.crbm_batch_last_error(self._b) or b"").decode())
        return best.value

    @property
    def cluster(self):
        """CTAs per thread-block cluster of the batched launch (1: none)."""
        return int(self._lib.crbm_batch_cluster(self._b))

    def close(self):
        if getattr(self, "_b", None):
            self._lib.crbm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NET_PARAMS = 3345
PASS_RECORD = np.dtype([("logit", np.float32, 16), ("dE", np.int32), ("cur_bits", np.uint32),
                        ("new_bits", np.uint32), ("log_alpha", np.float32), ("bR", np.int32),
                        ("bC", np.int32), ("thr", np.uint32, 16)])


class Proposal:
    """Learned 4x4 block proposal (crbm_proposal_*): a conv net trained on the
    GPU on the sampler's own configurations, used in exact MH block moves."""

    def __init__(self, seed=0, block=4):
        lib = load_library()
        h = ctypes.c_void_p()
        self._lib = lib
        self._chk(lib.crbm_proposal_create(ctypes.byref(h), int(block), int(seed)))
        self._p = h

    def _chk(self, rc):
        if rc != CRBM_OK:
            raise CrbmError(rc, (self._lib.crbm_proposal_last_error() or b"").decode())

    def close(self):
        if getattr(self, "_p", None):
            self._lib.crbm_proposal_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def weights(self):
        w = np.zeros(NET_PARAMS, np.float32)
        self._chk(self._lib.crbm_proposal_get_weights(self._p, _ptr(w, ctypes.c_float), w.size))
        return w

    @weights.setter
    def weights(self, w):
        w = np.ascontiguousarray(w, np.float32)
        self._chk(self._lib.crbm_proposal_set_weights(self._p, _ptr(w, ctypes.c_float), w.size))

    def train(self, sampler, steps, batch=2048, lr=3e-3, sweeps_between=2):
        losses = np.zeros(max(1, steps), np.float32)
        self._chk(self._lib.crbm_proposal_train(self._p, sampler._ctx, int(steps), int(batch), float(lr),
                                                int(sweeps_between), _ptr(losses, ctypes.c_float)))
        return losses[:steps]

    def loss_grad(self, spins, origins, beta_h):
        s = np.ascontiguousarray(spins, np.int8)
        o = np.ascontiguousarray(origins, np.int32)
        bh = np.ascontiguousarray(beta_h, np.float32)
        grad = np.zeros(NET_PARAMS, np.float32)
        loss = ctypes.c_float()
        self._chk(self._lib.crbm_proposal_loss_grad(self._p, _ptr(s, ctypes.c_int8), s.shape[-1],
                                                    _ptr(o, ctypes.c_int32), _ptr(bh, ctypes.c_float),
                                                    len(o), ctypes.byref(loss), _ptr(grad, ctypes.c_float)))
        return loss.value, grad

    def passes(self, sampler, n):
        self._chk(self._lib.crbm_proposal_pass(sampler._ctx, self._p, int(n)))

    def sweep_mixed(self, sampler, n, every=1):
        """n Gibbs sweeps with one pass of block moves after every `every` sweeps."""
        if every == 1:
            self._chk(self._lib.crbm_sweep_mixed(sampler._ctx, self._p, int(n)))
        else:
            self._chk(self._lib.crbm_sweep_mixed_every(sampler._ctx, self._p, int(n), int(every)))

    def inspect(self, sampler):
        nb1 = max(1, sampler.L // 8)
        n_words = (sampler.n_chains + 31) // 32
        out = np.zeros(n_words * nb1 * nb1 * 32, PASS_RECORD)
        self._chk(self._lib.crbm_proposal_inspect(sampler._ctx, self._p,
                                                  out.ctypes.data_as(ctypes.c_void_p), out.size))
        return out.reshape(n_words, nb1 * nb1, 32)

    def stats(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._chk(self._lib.crbm_proposal_stats(self._p, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value


def crbm_philox(inputs):
    """Device Philox-4x32-10 on rows (c0, c1, c2, c3, k0, k1) -> rows of 4 words."""
    a = np.ascontiguousarray(inputs, np.uint32).reshape(-1, 6)
    out = np.zeros((len(a), 4), np.uint32)
    _check(load_library().crbm_philox(_ptr(a, ctypes.c_uint32), _ptr(out, ctypes.c_uint32), len(a)))
    return out


def crbm_philox_stream(sink, n_blocks, threads, calls, seed=0, stream=None):
    """Philox throughput probe on a device uint32 tensor sink[n_blocks *
    threads] (see include/crbm.h); asynchronous on `stream` (torch stream,
    default: the current one)."""
    import torch
    assert sink.dtype == torch.int32 or sink.dtype == torch.uint32
    assert sink.is_cuda and sink.numel() >= n_blocks * threads
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(load_library().crbm_philox_stream(ctypes.c_void_p(sink.data_ptr()), int(n_blocks), int(threads),
                                             int(calls), ctypes.c_uint64(seed), ctypes.c_void_p(st.cuda_stream)))


# C-ABI names, for callers that prefer the flat interface.
def crbm_create(L, params, n_chains, **kw):
    return Sampler(L, params, n_chains, **kw)


def crbm_sweep(s: Sampler, n):
    s.sweep(n)


def crbm_observables(s: Sampler):
    return s.observables()


def crbm_destroy(s: Sampler):
    s.close()
