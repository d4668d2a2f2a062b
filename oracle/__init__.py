"""The oracle: TEST INFRASTRUCTURE ONLY.

A plain, slow CPU restatement (scalar C, double precision) of block Gibbs
sampling of the convolutional RBM that encodes the Shastry–Sutherland Ising
lattice (arXiv 2511.20911, Sec. II.A–II.B).  Only ``tests/``, the smoke check
and the benchmark's CPU-baseline / reference legs may import this package.  It
shares no code with ``paper_2511_20911_gb300``: both sides implement the same
readings of the paper (bond list, weights, tables, Philox keying) separately.

This module only marshals numpy arrays into ``crbm_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crbm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

NSUM = 11
TAG_VIS, TAG_INIT, TAG_SWAP = 4, 5, 6
PRECISION_EXACT, PRECISION_PAPER = 0, 1
RNG_LANE, RNG_BITPLANE = 0, 1      # RNG_BITPLANE: ORC_RNG_BITPLANE in crbm_oracle.h
TAG_BITPLANE = 256


def build(force: bool = False) -> str:
    """Compile crbm_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    srcs = [_SRC, os.path.join(_HERE, "crbm_oracle.h")]
    srcs = [s for s in srcs if os.path.exists(s)]
    if not force and os.path.exists(_LIB):
        if all(os.path.getmtime(_LIB) >= os.path.getmtime(s) for s in srcs):
            return _LIB
    cfiles = [s for s in srcs if s.endswith(".c")]
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp] + cfiles + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class Bond(ctypes.Structure):
    _fields_ = [("r1", ctypes.c_int8), ("c1", ctypes.c_int8), ("r2", ctypes.c_int8),
                ("c2", ctypes.c_int8), ("cls", ctypes.c_uint8)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_threshold.restype = ctypes.c_uint32
        _lib.orc_threshold.argtypes = [ctypes.c_double]
        _lib.orc_lut16.restype = ctypes.c_uint32
        _lib.orc_lut16.argtypes = [ctypes.c_int32]
        _lib.orc_q54.restype = ctypes.c_int32
        _lib.orc_q54.argtypes = [ctypes.c_double]
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def bonds_array(bonds=None):
    """ctypes array of bonds; None -> the canonical SS unit cell."""
    if bonds is None:
        bonds = canonical_bonds()
    arr = (Bond * len(bonds))()
    for i, b in enumerate(bonds):
        arr[i] = Bond(*b)
    return arr, len(bonds)


def canonical_bonds():
    arr = (Bond * 10)()
    n = lib().orc_canonical_bonds(arr)
    return [(arr[i].r1, arr[i].c1, arr[i].r2, arr[i].c2, arr[i].cls) for i in range(n)]


def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [o[i] for i in range(4)]


def weight(beta, J):
    a = ctypes.c_double()
    s = ctypes.c_int()
    lib().orc_weight(ctypes.c_double(beta), ctypes.c_double(J), ctypes.byref(a), ctypes.byref(s))
    return a.value, s.value


def threshold(y):
    return int(lib().orc_threshold(float(y)))


def q54(x):
    """Paper precision: nearest multiple of 1/16 within +-511/16, in 1/16 units."""
    return int(lib().orc_q54(float(x)))


def lut16(acc):
    """Paper precision: 16-bit sigmoid table entry of an accumulator value (1/16
    units), in the upper half of a 32-bit threshold."""
    return int(lib().orc_lut16(int(acc)))


def quantize(x):
    q = ctypes.c_int32()
    if lib().orc_quantize(ctypes.c_double(x), ctypes.byref(q)):
        raise ValueError(f"coupling {x} out of Q.4 range")
    return q.value


def shape(L, periodic=True):
    """(Lr, Lc, pr, pc) from L = int or (rows, cols) and periodic = bool or
    (rows axis, cols axis)."""
    Lr, Lc = (int(L), int(L)) if np.isscalar(L) else (int(L[0]), int(L[1]))
    pr, pc = ((bool(periodic),) * 2) if np.isscalar(periodic) else (bool(periodic[0]), bool(periodic[1]))
    return Lr, Lc, int(pr), int(pc)


def degrees(L, periodic=True, bonds=None):
    arr, nb = bonds_array(bonds)
    dj, djp = ctypes.c_int(), ctypes.c_int()
    Lr, Lc, pr, pc = shape(L, periodic)
    if lib().orc_degrees_rect(Lr, Lc, pr, pc, arr, nb, ctypes.byref(dj), ctypes.byref(djp)):
        raise ValueError("bad model")
    return dj.value, djp.value


def tables(L, J, Jp, h, beta, periodic=True, bonds=None, precision=PRECISION_EXACT, h_odd=None):
    """(Th[2][5], Tv[2DJ+1][2DJp+1]) uint32 for one parameter point; with
    h_odd, also the odd-column visible table as a third element."""
    arr, nb = bonds_array(bonds)
    dj, djp = degrees(L, periodic, bonds)
    Lr, Lc, pr, pc = shape(L, periodic)
    th = np.zeros(10, np.uint32)
    tv = np.zeros((2 * dj + 1) * (2 * djp + 1), np.uint32)
    tvo = np.zeros_like(tv)
    rc = lib().orc_tables_rect(Lr, Lc, pr, pc, arr, nb, ctypes.c_double(J), ctypes.c_double(Jp),
                               ctypes.c_double(h), ctypes.c_double(h if h_odd is None else h_odd),
                               ctypes.c_double(beta), int(precision), _p(th, ctypes.c_uint32),
                               _p(tv, ctypes.c_uint32), _p(tvo, ctypes.c_uint32))
    if rc:
        raise ValueError("bad parameters")
    shp = (2 * dj + 1, 2 * djp + 1)
    if h_odd is None:
        return th.reshape(2, 5), tv.reshape(shp)
    return th.reshape(2, 5), tv.reshape(shp), tvo.reshape(shp)


def init_spins(L, chain_ids, seed):
    ids = np.ascontiguousarray(chain_ids, dtype=np.uint32)
    Lr, Lc, _, _ = shape(L)
    out = np.zeros((len(ids), Lr, Lc), np.int8)
    lib().orc_init_rect(Lr, Lc, _p(ids, ctypes.c_uint32), len(ids), ctypes.c_uint64(seed),
                        _p(out, ctypes.c_int8))
    return out


def counts(spins, L, periodic=True, bonds=None):
    """Exact (N_J, N_J', M) of one configuration [Lr][Lc] of +-1."""
    arr, nb = bonds_array(bonds)
    v = np.ascontiguousarray(spins, dtype=np.int8)
    Lr, Lc, pr, pc = shape(L, periodic)
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib().orc_counts_rect(Lr, Lc, pr, pc, arr, nb, _p(v, ctypes.c_int8), ctypes.byref(a),
                          ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


def run(L, params, chain_param, spins, seed, sweep0, n_sweeps, measure_every=1,
        chain_ids=None, periodic=True, bonds=None, sums=None, series_cap=0, sq_every=0,
        sq=None, precision=PRECISION_EXACT, rng=RNG_LANE):
    """Advance ``spins`` [n_chains][L][L] (int8 +-1, modified in place).

    params: dict of equal-length sequences J, Jp, h, beta.
    rng: RNG_LANE (one Philox stream per chain) or RNG_BITPLANE (uniforms from
    bit-plane words shared by each group of 32 chains).
    Returns (sums [n_chains][11] int64, series or None, sq or None).
    """
    arr, nb = bonds_array(bonds)
    J = np.ascontiguousarray(params["J"], np.float64)
    Jp = np.ascontiguousarray(params["Jp"], np.float64)
    h = np.ascontiguousarray(params["h"], np.float64)
    h_odd = None if params.get("h_odd") is None else np.ascontiguousarray(params["h_odd"], np.float64)
    beta = np.ascontiguousarray(params["beta"], np.float64)
    cp = np.ascontiguousarray(chain_param, np.int32)
    n = len(cp)
    Lr, Lc, pr, pc = shape(L, periodic)
    assert spins.dtype == np.int8 and spins.flags.c_contiguous and spins.shape == (n, Lr, Lc)
    ids = np.arange(n, dtype=np.uint32) if chain_ids is None else np.ascontiguousarray(
        chain_ids, np.uint32)
    if sums is None:
        sums = np.zeros((n, NSUM), np.int64)
    series = np.zeros((n, series_cap, 3), np.int32) if series_cap > 0 else None
    if sq_every > 0 and sq is None:
        sq = np.zeros((n, Lr, Lc), np.float64)
    rc = lib().orc_run_rect(Lr, Lc, pr, pc, arr, nb, _p(J, ctypes.c_double), _p(Jp, ctypes.c_double),
                       _p(h, ctypes.c_double), _p(h_odd, ctypes.c_double), _p(beta, ctypes.c_double), len(J),
                       _p(cp, ctypes.c_int32), _p(ids, ctypes.c_uint32), n, ctypes.c_uint64(seed),
                       ctypes.c_int64(sweep0), ctypes.c_int64(n_sweeps), int(measure_every),
                       _p(spins, ctypes.c_int8), _p(sums, ctypes.c_int64),
                       _p(series, ctypes.c_int32), ctypes.c_int64(series_cap), int(sq_every),
                       _p(sq, ctypes.c_double) if sq_every > 0 else None,
                       int(precision) | (0x10 if rng == RNG_BITPLANE else 0))
    if rc:
        raise ValueError(f"orc_run failed ({rc})")
    return sums, series, sq


def set_threads(n):
    lib().orc_set_threads(int(n))


def get_threads():
    return int(lib().orc_get_threads())


def run_pt(L, params, chain_param, spins, slot_of_beta, seed, sweep0, n_sweeps, measure_every=1,
           swap_every=10, periodic=True, bonds=None, sums=None, series_cap=0,
           precision=PRECISION_EXACT, rng=RNG_LANE):
    """Parallel tempering on ladders of 32 chains (see orc_run_pt).  Advances
    ``spins`` (per slot) and ``slot_of_beta`` [n_ladders][32] in place; sums
    and series rows are per rung (chain index 32 l + k)."""
    arr, nb = bonds_array(bonds)
    J = np.ascontiguousarray(params["J"], np.float64)
    Jp = np.ascontiguousarray(params["Jp"], np.float64)
    h = np.ascontiguousarray(params["h"], np.float64)
    beta = np.ascontiguousarray(params["beta"], np.float64)
    cp = np.ascontiguousarray(chain_param, np.int32)
    n = len(cp)
    Lr, Lc, pr, pc = shape(L, periodic)
    assert spins.dtype == np.int8 and spins.flags.c_contiguous and spins.shape == (n, Lr, Lc)
    assert slot_of_beta.dtype == np.int32 and slot_of_beta.flags.c_contiguous
    if sums is None:
        sums = np.zeros((n, NSUM), np.int64)
    series = np.zeros((n, series_cap, 3), np.int32) if series_cap > 0 else None
    rc = lib().orc_run_pt_rect(Lr, Lc, pr, pc, arr, nb, _p(J, ctypes.c_double),
                          _p(Jp, ctypes.c_double), _p(h, ctypes.c_double),
                          _p(beta, ctypes.c_double), len(J), _p(cp, ctypes.c_int32), n,
                          ctypes.c_uint64(seed), ctypes.c_int64(sweep0), ctypes.c_int64(n_sweeps),
                          int(measure_every), int(swap_every), _p(spins, ctypes.c_int8),
                          _p(slot_of_beta, ctypes.c_int32), _p(sums, ctypes.c_int64),
                          _p(series, ctypes.c_int32), ctypes.c_int64(series_cap),
                          int(precision) | (0x10 if rng == RNG_BITPLANE else 0))
    if rc:
        raise ValueError(f"orc_run_pt failed ({rc})")
    return sums, series


def swap_threshold(x):
    f = lib().orc_swap_threshold
    f.restype = ctypes.c_uint32
    f.argtypes = [ctypes.c_double]
    return int(f(float(x)))


NET_PARAMS = 3345


def bf16(x):
    f = lib().orc_bf16
    f.restype = ctypes.c_double
    f.argtypes = [ctypes.c_double]
    return float(f(float(x)))


def patch_input(spins, bR, bC, k, beta, h):
    L = spins.shape[-1]
    v = np.ascontiguousarray(spins, np.int8)
    P = k + 6
    out = np.zeros((6, P, P), np.float64)
    lib().orc_patch_input(L, _p(v, ctypes.c_int8), bR, bC, k, ctypes.c_double(beta),
                          ctypes.c_double(h), _p(out, ctypes.c_double))
    return out


def net_forward(k, w, inp, use_bf16=False):
    w = np.ascontiguousarray(w, np.float64)
    inp = np.ascontiguousarray(inp, np.float64)
    out = np.zeros(k * k, np.float64)
    if lib().orc_net_forward(k, _p(w, ctypes.c_double), _p(inp, ctypes.c_double), int(use_bf16),
                             _p(out, ctypes.c_double)):
        raise ValueError("orc_net_forward failed")
    return out


def net_loss_grad(k, w, inputs, targets, use_bf16=False):
    w = np.ascontiguousarray(w, np.float64)
    inputs = np.ascontiguousarray(inputs, np.float64)
    targets = np.ascontiguousarray(targets, np.int8)
    n = len(targets)
    grad = np.zeros(NET_PARAMS, np.float64)
    loss = ctypes.c_double()
    if lib().orc_net_loss_grad(k, _p(w, ctypes.c_double), _p(inputs, ctypes.c_double),
                               _p(targets, ctypes.c_int8), n, int(use_bf16), ctypes.byref(loss),
                               _p(grad, ctypes.c_double)):
        raise ValueError("orc_net_loss_grad failed")
    return loss.value, grad


def block_delta_e(spins, bR, bC, newblock, J, Jp, h):
    L = spins.shape[-1]
    v = np.ascontiguousarray(spins, np.int8)
    nb = np.ascontiguousarray(newblock, np.int8).reshape(-1)
    k = int(round(np.sqrt(nb.size)))
    f = lib().orc_block_delta_e
    f.restype = ctypes.c_int64
    return int(f(L, _p(v, ctypes.c_int8), bR, bC, k, _p(nb, ctypes.c_int8), quantize(J),
                 quantize(Jp), quantize(h)))


def mh_rows(states, bR, bC, k, w, J, Jp, h, beta, use_bf16=False):
    v = np.ascontiguousarray(states, np.int8)
    n, L = v.shape[0], v.shape[-1]
    w = np.ascontiguousarray(w, np.float64)
    out = np.zeros((n, 1 << (k * k)), np.float64)
    if lib().orc_mh_rows(L, _p(v, ctypes.c_int8), n, bR, bC, k, _p(w, ctypes.c_double),
                         ctypes.c_double(J), ctypes.c_double(Jp), ctypes.c_double(h),
                         ctypes.c_double(beta), int(use_bf16), _p(out, ctypes.c_double)):
        raise ValueError("orc_mh_rows failed")
    return out


def random_net(seed, scale=0.3):
    """Random parameters in the documented order (W1, b1, W2, b2, W3, b3)."""
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, scale, NET_PARAMS)
    w[864:880] *= 0.1
    w[3184:3200] *= 0.1
    return w


PASS_REC = np.dtype([("logit", np.float64, 16), ("thr", np.uint32, 16), ("draw", np.uint32, 16),
                     ("bR", np.int32),
                     ("bC", np.int32), ("cur_bits", np.uint32), ("new_bits", np.uint32),
                     ("dE", np.int64), ("log_alpha", np.float64), ("u_accept", np.float64),
                     ("accept", np.int32), ("pad", np.int32)])


def prop_pass(spins, params, chain_param, w, seed, pass_index, apply=False, logits=None, thr=None):
    """One pass of learned block moves (see orc_prop_pass): records
    [n_blocks][n_chains] of PASS_REC; with apply, accepted blocks are written
    into ``spins`` [n_chains][L][L] in place.  logits: optional
    [n_blocks][n_chains][16] used instead of the net; thr: optional
    [n_blocks][n_chains][16] thresholds used instead of the logits' ones."""
    assert spins.dtype == np.int8 and spins.flags.c_contiguous
    n, L = spins.shape[0], spins.shape[-1]
    J = np.ascontiguousarray(params["J"], np.float64)
    Jp = np.ascontiguousarray(params["Jp"], np.float64)
    h = np.ascontiguousarray(params["h"], np.float64)
    beta = np.ascontiguousarray(params["beta"], np.float64)
    cp = np.ascontiguousarray(chain_param, np.int32)
    w = np.ascontiguousarray(w, np.float64)
    nb1 = max(1, L // 8)
    rec = np.zeros((nb1 * nb1, n), PASS_REC)
    lg = None if logits is None else np.ascontiguousarray(logits, np.float64)
    if lg is not None:
        assert lg.shape == (nb1 * nb1, n, 16)
    th = None if thr is None else np.ascontiguousarray(thr, np.uint32)
    if th is not None:
        assert th.shape == (nb1 * nb1, n, 16)
    f = lib().orc_prop_pass
    f.restype = ctypes.c_int
    rc = f(L, _p(spins, ctypes.c_int8), n, _p(J, ctypes.c_double), _p(Jp, ctypes.c_double),
           _p(h, ctypes.c_double), _p(beta, ctypes.c_double), _p(cp, ctypes.c_int32),
           _p(w, ctypes.c_double), _p(lg, ctypes.c_double), _p(th, ctypes.c_uint32),
           ctypes.c_uint64(seed),
           ctypes.c_uint32(pass_index), int(bool(apply)), rec.ctypes.data_as(ctypes.c_void_p))
    if rc < 0:
        raise ValueError(f"orc_prop_pass failed ({rc})")
    return rec


def structure_factor(spins):
    """S(q) [Lr][Lc] of one configuration (orc_structure_factor)."""
    v = np.ascontiguousarray(spins, np.int8)
    Lr, Lc = v.shape
    out = np.zeros((Lr, Lc), np.float64)
    lib().orc_structure_factor(Lr, Lc, _p(v, ctypes.c_int8), _p(out, ctypes.c_double))
    return out
