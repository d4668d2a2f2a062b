"""Seeded synthetic workloads (parameter grids, chain assignments, spin
configurations) shared by the tests and the benchmark.

Holds no arithmetic of the sampling method: only the shapes and parameter
values of the paper's workloads (arXiv 2511.20911: 18x18 periodic lattices,
J1 = 1, J2/J1 in [0, 3], h in [-8, 8]; lattice sizes 6x6 ... 18x18).
"""
from __future__ import annotations

import numpy as np


def q4(x):
    """Round to the nearest multiple of 1/16 (the Q.4 grid of the couplings)."""
    return np.round(np.asarray(x, np.float64) * 16.0) / 16.0


def small_workload():
    """L=6 periodic, J=J'=1, h=0.5, beta=2, 64 chains, seed 1, 10^4 sweeps."""
    return dict(L=6, params=dict(J=[1.0], Jp=[1.0], h=[0.5], beta=[2.0]), n_chains=64,
                chain_param=np.zeros(64, np.int32), seed=1, n_sweeps=10_000)


def grid_workload(chains_per_point=16, n_beta=16, n_h=16, ratios=(0.5, 1.0, 2.0)):
    """L=18 periodic: J'/J in `ratios` x n_beta beta linear in [0.1, 5] x n_h h
    linear in [0, 4] (on the 1/16 grid) x chains_per_point chains, J = 1.
    Chains of one parameter point are contiguous."""
    betas = np.linspace(0.1, 5.0, n_beta)
    hs = q4(np.linspace(0.0, 4.0, n_h))
    J, Jp, h, beta = [], [], [], []
    for r in ratios:
        for b in betas:
            for x in hs:
                J.append(1.0)
                Jp.append(float(r))
                h.append(float(x))
                beta.append(float(b))
    n_p = len(J)
    cp = np.repeat(np.arange(n_p, dtype=np.int32), chains_per_point)
    return dict(L=18, params=dict(J=J, Jp=Jp, h=h, beta=beta), n_chains=len(cp),
                chain_param=cp, seed=2025)


def random_params(rng, n):
    """n random parameter points on the Q.4 grid (signs of J, J' both ways)."""
    return dict(J=list(q4(rng.uniform(-2, 2, n))), Jp=list(q4(rng.uniform(-3, 3, n))),
                h=list(q4(rng.uniform(-4, 4, n))), beta=list(rng.uniform(0.05, 3.0, n)))


def random_spins(rng, n_chains, L):
    return rng.choice(np.array([-1, 1], np.int8), size=(n_chains, L, L))


def stream_workload():
    """L=384 periodic, J=J'=1, beta=1, h in {0, 1, 2} x 1024 chains (3072
    chains), spins and hidden units in HBM; 10^4 sweeps."""
    return dict(L=384, params=dict(J=[1.0] * 3, Jp=[1.0] * 3, h=[0.0, 1.0, 2.0], beta=[1.0] * 3),
                n_chains=3072, chain_param=np.repeat(np.arange(3, dtype=np.int32), 1024), seed=384,
                n_sweeps=10_000)


def tempering_batch_workload(sizes=(6, 9, 12, 18, 24, 48), ladders=8, b_lo=0.2, b_hi=10.0):
    """Mixed lattice sizes, each with `ladders` replica-exchange ladders of 32
    geometric beta in [b_lo, b_hi] (256 chains per size), J=1, J'=1.5, h=1,
    swaps every 10 sweeps; 10^5 sweeps."""
    betas = list(b_lo * (b_hi / b_lo) ** (np.arange(32) / 31.0))
    params = dict(J=[1.0] * 32, Jp=[1.5] * 32, h=[1.0] * 32, beta=betas)
    members = []
    for L in sizes:
        members.append(dict(L=L, params=params, n_chains=32 * ladders,
                            chain_param=np.tile(np.arange(32, dtype=np.int32), ladders),
                            seed=1000 + L, swap_every=10))
    return members


def proposal_training_workload(L=18, n_chains=4096, betas=(1.5, 2.0, 2.5, 3.0),
                               hs=(2.5, 2.75, 3.0, 3.25, 3.5)):
    """Training configurations for the block proposal: J'/J = 1, beta in
    [1.5, 3], h around the 1/3 magnetisation plateau (J2 = J1, h near 3)."""
    pts = [(b, h) for b in betas for h in hs]
    params = dict(J=[1.0] * len(pts), Jp=[1.0] * len(pts), h=[h for _, h in pts],
                  beta=[b for b, _ in pts])
    return dict(L=L, params=params, n_chains=n_chains,
                chain_param=(np.arange(n_chains) * len(pts) // n_chains).astype(np.int32),
                seed=55, measure_every=0)


def proposal_eval_workload(L, n_chains=4096, betas=(1.5, 2.0, 3.0), h=3.0):
    """Evaluation points of the block proposal: J'/J = 1, h = 3, beta in
    {1.5, 2, 3}."""
    params = dict(J=[1.0] * len(betas), Jp=[1.0] * len(betas), h=[h] * len(betas),
                  beta=list(betas))
    return dict(L=L, params=params, n_chains=n_chains,
                chain_param=(np.arange(n_chains) * len(betas) // n_chains).astype(np.int32),
                seed=77)


def strip_workload(hs=(3.0, 4.5), betas=(1.0, 2.0, 4.0), chains_per_point=256, rows=18, width=12):
    """Laterally confined SS strip (Sec. III): `rows` periodic rows of `width`
    spins with open edges across the width, J = 1, J'/J = 1.5 (the spin-liquid
    cut of the paper: an ordered up-up-down state below h = 3.5, a classical
    spin liquid above), h and beta on a small grid."""
    pts = [(b, h) for h in hs for b in betas]
    params = dict(J=[1.0] * len(pts), Jp=[1.5] * len(pts), h=[q4(h) for _, h in pts],
                  beta=[b for b, _ in pts])
    n = chains_per_point * len(pts)
    return dict(L=rows, L_cols=width, periodic=True, periodic_cols=2, params=params, n_chains=n,
                chain_param=(np.arange(n) // chains_per_point).astype(np.int32), seed=12, measure_every=10)


def phase_scan_workload(jp_values=None, h_values=None, L=18, rungs=32, beta_min=0.25, beta_max=8.0, seed=909):
    """The ground-state phase diagram scan (Sec. III, next to the paper's
    time-to-solution points): J = 1, J'/J over [0, 3] in steps of 1/4 and h
    over [-8, 8] in steps of 1/2 (all on the Q.4 grid), one replica-exchange
    ladder of `rungs` chains per point, beta geometric in [beta_min,
    beta_max].  Chain 32 p + k is rung k of point p; each chain has its own
    parameter point (its rung's beta)."""
    jp = np.arange(0.0, 3.0001, 0.25) if jp_values is None else np.asarray(jp_values, np.float64)
    hs = np.arange(-8.0, 8.0001, 0.5) if h_values is None else np.asarray(h_values, np.float64)
    betas = beta_min * (beta_max / beta_min) ** (np.arange(rungs) / (rungs - 1))
    points = [(1.0, q4(a), q4(x)) for a in jp for x in hs]
    params = dict(J=[], Jp=[], h=[], beta=[])
    for J, a, x in points:
        params["J"] += [J] * rungs
        params["Jp"] += [a] * rungs
        params["h"] += [x] * rungs
        params["beta"] += [float(b) for b in betas]
    n = len(points) * rungs
    return dict(L=L, params=params, n_chains=n, chain_param=np.arange(n, dtype=np.int32), swap_every=10,
                measure_every=2, seed=seed, points=points, rungs=rungs, n_jp=len(jp), n_h=len(hs))
