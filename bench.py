"""Benchmark of the GB300 CRBM block-Gibbs sampler (one JSON line on stdout).

Default workload: the L=18 periodic Shastry–Sutherland grid -- J'/J in
{0.5, 1, 2} x 16 beta in [0.1, 5] x 16 h in [0, 4] x 16 chains = 12288 chains,
couplings on the Q.4 grid, SMEM-resident lattices.  A step is one crbm_sweep
call of --sweeps-per-step sweeps over every chain (hidden then visible
half-step, observables every 10 sweeps), inputs resident in HBM.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

N > 1 (torchrun): every rank runs an independent replica with its own chains
(no data-path collective); value = all ranks' spin-updates / max rank time.
--impl reference times the CPU oracle (the reference arm) on host cores.
"""
from __future__ import annotations

import argparse
import functools
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin-updates/s and ESS/s (energy, m) per GB300 vs plain Gibbs; roofline %"
UNIT = "spin-updates/s"
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
# The path is bound by 32-bit integer multiplies: every node decision needs a
# Philox-4x32-10 word, and one Philox call (4 words) is 10 rounds x two
# 32x32->64 products = 40 multiply lane-operations (low and high halves).  The
# GB300 SM retires 64 integer-multiply lanes per clock, so the ceiling is
# 152 SM x 64 x 2070 MHz = 20.1 T multiply-ops/s = 5.03e11 Philox calls/s.
IMUL_LANES_PER_SM_CLK = 64
MUL_OPS_PER_CALL = 40
CALLS_PER_CELL = 4          # 3 hidden calls (10 filters) + 1 visible call (4 spins) per cell
CALLS_PER_CELL_PAPER = 2    # paper precision: 16-bit uniforms, two per Philox word (14 of 16 used)
CALLS_PER_CELL_PAPER_STREAM = 3  # streamed paper precision: the visible half-step draws the tag-1 call again
# DRAM bytes (read + write) of the timed unit, from one ncu capture of the
# kernels as they stand (commands in the named profiles/ summaries): one bench
# launch of k_sweep_canon_persistent (2000 sweeps of the L=18 grid), and one
# streamed sweep of the L=384 lattice (k_stream_hidden + k_stream_visible).
MEASURED_TRAFFIC = {
    "grid": (8.73e6 + 0.84e6, "per launch; profiles/launches_L18_grid.md"),
    "grid_sq": (10.91e6 + 0.87e6, "per launch with S(q) every 100 sweeps; profiles/launches_L18_grid.md"),
    "stream": (56.74e6 + 392.31e6 + 454.82e6 + 48.83e6, "per sweep (two launches); profiles/k_stream_L384.md"),
    "grid_paper": (8.34e6 + 0.78e6, "per launch; profiles/k_sweep_canon_persistent_L18_grid_paper.md"),
    "grid_paper_sq": (10.46e6 + 0.77e6,
                      "per launch with S(q) every 100 sweeps; profiles/k_sweep_canon_persistent_L18_grid_paper.md"),
    "stream_paper": (56.76e6 + 390.29e6 + 454.76e6 + 45.71e6, "per sweep (two launches); profiles/k_stream_L384.md"),
    "grid_bitplane": (2.48e6 + 0.78e6, "per launch; profiles/k_sweep_bitplane_L18_grid.md"),
    "stream_bitplane": (56.88e6 + 82.96e6 + 141.80e6 + 29.02e6, "per sweep (two launches); profiles/k_stream_bp_L384.md"),
}


@functools.lru_cache(maxsize=None)
def bitplane_expected_calls(n_nodes):
    """Expected Philox calls (lane-calls) of one bit-plane half-step over
    n_nodes nodes of one 32-chain word.  Every node draws two calls of four
    planes; the nodes with a comparison still open after them go to a
    straggler list, taken 32 at a time, and a group of stragglers draws calls
    while any of its comparisons is open.  Each plane decides an undecided
    comparison with probability 1/2, so it is still open after 4 m planes with
    probability 2^-4m, independently; the number of stragglers is binomial.
    (A node past the list's capacity, a quarter of the half-step, finishes in
    place; its probability is negligible and not modelled.)"""
    def node_open(m):                         # any of the node's 32 chains open after m calls
        return -math.expm1(32.0 * math.log1p(-(2.0 ** (-4 * m))))
    p2 = node_open(2)
    cond = [node_open(2 + m) / p2 for m in range(6)]   # open after m more calls, given open after 2

    def group_calls(g):                       # lane-calls of a group of g stragglers
        return g * sum(1.0 if c >= 1.0 else -math.expm1(g * math.log1p(-c)) for c in cond)

    n = int(n_nodes)
    total = 2.0 * n
    lq, lp = math.log1p(-p2), math.log(p2)
    for k in range(1, n + 1):
        lpmf = math.lgamma(n + 1) - math.lgamma(k + 1) - math.lgamma(n - k + 1) + k * lp + (n - k) * lq
        if lpmf < -60.0 and k > n * p2:
            break
        pmf = math.exp(lpmf)
        if pmf == 0.0:
            continue
        total += pmf * sum(group_calls(min(32, k - b)) for b in range(0, k, 32))
    return total


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid", choices=["grid", "stream", "batch", "proposal", "tts", "phase"])
    ap.add_argument("--sweeps-per-step", type=int, default=None)
    ap.add_argument("--measure-every", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-lines", action="store_true",
                    help="grid workload: skip the L=384 streamed line printed inside the same JSON line")
    ap.add_argument("--sq-every", type=int, default=None,
                    help="structure-factor accumulation every K sweeps (grid default 100, the grid "
                         "workload's estimator; 0 = off)")
    ap.add_argument("--precision", default="exact", choices=["exact", "paper"],
                    help="paper: the FPGA's 10-bit weights, 16-bit sigmoid table and 16-bit uniforms "
                         "(grid and stream workloads)")
    ap.add_argument("--rng", default="lane", choices=["lane", "bitplane"],
                    help="bitplane: uniforms from bit-plane words shared by the 32 chains of a word, compared "
                         "most significant bit first (grid workload)")
    ap.add_argument("--warps", type=int, default=0,
                    help="grid and batch workloads: CTAs of this many warps instead of the autotuners' choice "
                         "(0), so that a profile captures one known shape")
    args = ap.parse_args()
    if args.rng == "bitplane" and (args.workload not in ("grid", "stream", "phase") or args.precision != "exact"):
        ap.error("--rng bitplane runs the grid, stream and phase workloads in exact precision")
    if args.precision == "paper" and args.workload not in ("grid", "stream"):
        ap.error("--precision paper runs the grid and stream workloads only")
    return args


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        rank = int(os.environ["RANK"])
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
        dist.init_process_group("nccl")
        return rank, ws
    return 0, 1


class ClockSampler:
    """nvidia-smi clock/throttle samples every 50 ms while running (a timed region of a quarter of a
    second still gets several)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.t.join(timeout=2)

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 7 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 7 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 7 for i in range(4)
                          if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(sm)}


def replica_seed(seed, rank):
    """Seed of rank `rank`'s replica: every rank samples its own chains."""
    return seed + 1000003 * rank


def max_over_ranks(t_local, ws):
    """Largest of the ranks' timed seconds (the job's time); the tensor lives
    on the device for NCCL and on the host for gloo."""
    if ws == 1:
        return t_local
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([t_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, ws, t_max):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (replicas do equal work)."""
    return units_per_rank * ws / t_max


def workload_config(name, rank):
    from paper_2511_20911_gb300 import workloads
    w = workloads.grid_workload() if name == "grid" else workloads.stream_workload()
    w["seed"] = replica_seed(w["seed"], rank)
    return w


DEFAULT_SWEEPS = {"grid": 2000, "stream": 20, "batch": 500, "proposal": 250, "tts": 200000, "phase": 4000}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline(w, seconds, precision=0, rng=0, one_core=True):
    """The oracle as it stands, OpenMP over chains on every host core, on a
    bounded sample of the same workload (a spread subset of its chains); then
    the same on one core for a third of the time."""
    import oracle
    oracle.build()
    n_all = w["n_chains"]
    L = w["L"]
    cores = os.cpu_count() or 1

    def run(n_ch, n_sw):
        ids = np.linspace(0, n_all - 1, n_ch).astype(np.uint32)
        cp = np.asarray(w["chain_param"], np.int32)[ids]
        sp = oracle.init_spins(L, ids, w["seed"])
        t = time.perf_counter()
        oracle.run(L, w["params"], cp, sp, w["seed"], 0, n_sw, 10, chain_ids=ids, precision=precision, rng=rng)
        return time.perf_counter() - t

    def timed(threads, n_ch, budget):
        oracle.set_threads(threads)
        sw0 = 20 if L <= 64 else 1
        dt = run(n_ch, sw0)
        while dt < 0.2 and sw0 < (1 << 20):   # calibrate on at least 0.2 s of work
            sw0 *= 4
            dt = run(n_ch, sw0)
        n_sw = max(sw0, int(sw0 * budget / max(dt, 1e-3)))
        dt = run(n_ch, n_sw)
        return n_ch * n_sw * L * L / dt, n_ch, n_sw, dt

    small = L <= 64
    value, n_ch, n_sw, dt = timed(cores, 16 * cores if small else cores, seconds)
    out = {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
           "cpu_model": cpu_model(), "seconds": dt,
           "sample": f"{n_ch} of the {n_all} chains (spread over all parameter points), "
                     f"{n_sw} sweeps, measure every 10, {dt:.1f} s wall"}
    if one_core:
        v1, n1, s1, d1 = timed(1, 16 if small else 1, seconds / 3)
        out["one_core"] = {"value": v1, "unit": UNIT,
                           "sample": f"{n1} chains, {s1} sweeps, one thread, {d1:.1f} s wall"}
    oracle.set_threads(cores)
    return out


def run_reference(args, rank, ws):
    """Reference arm: the CPU oracle timed on the host cores."""
    if rank != 0:
        return
    if args.workload not in ("grid", "stream"):
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle's timed leg covers the grid and "
                                                               f"stream workloads, not {args.workload}"}))
        return
    w = workload_config(args.workload, 0)
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    prec, rng = (1 if args.precision == "paper" else 0), (1 if args.rng == "bitplane" else 0)
    for _ in range(args.warmup):
        cpu_baseline(w, min(per_step, 2.0), prec, rng, one_core=False)
    vals = [cpu_baseline(w, per_step, prec, rng, one_core=False) for _ in range(args.steps)]
    v = float(np.mean([x["value"] for x in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    n_ch = int(cb["sample"].split()[0])
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean([x["seconds"] for x in vals])) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
        "data": "synthetic", "config": config_dict(w, args), "cpu_baseline": cb,
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def config_dict(w, args, workload=None):
    workload = workload or args.workload
    if workload == "grid":
        desc = ("L=18 periodic SS grid: J'/J in {0.5,1,2} x 16 beta in [0.1,5] x 16 h in [0,4] "
                "x 16 chains, SMEM-resident")
    else:
        desc = ("L=384 periodic SS lattice: J=J'=1, beta=1, h in {0,1,2} x 1024 chains, 64-chain "
                "words, spins and hidden units in HBM (two launches per sweep)")
    if getattr(args, "precision", "exact") == "paper":
        desc += ("; paper precision: Q5.4 weights and bias, 12-bit accumulator, 16-bit sigmoid table "
                 "and 16-bit uniforms (two per Philox word)")
    if getattr(args, "rng", "lane") == "bitplane":
        desc += ("; bit-plane uniforms: shared plane words per 32-chain word, compared most significant "
                 "bit first with early exit (word-parallel kernel, one thread per node)")
    return {"workload": desc, "L": w["L"], "n_chains": w["n_chains"],
            "n_params": len(w["params"]["J"]), "sweeps_per_step": args.sweeps_per_step,
            "measure_every": args.measure_every,
            "layout": "smem (persistent, dynamically scheduled)" if workload == "grid" else "stream",
            "l2": "flushed between steps (256 MiB write outside the step events)",
            "parallelism": f"replicas x{args.gpus}"}


# The paper's time-to-solution phases (Sec. III, "Hardware Acceleration") and
# the times it prints for its FPGA (lattice sizes not stated in the text).
TTS_PHASES = (("FM", 1.0, 1.0, 7.0, 33e-9), ("dimer", 1.0, 2.5, 0.0, 5e-6), ("Neel", 1.0, 1.0, 0.0, 200e-6),
              ("1/3 plateau", 1.0, 0.5, 4.0, 120e-3))
# beta range of each phase's replica-exchange ladders (geometric, 32 rungs): the paper tunes its
# temperatures per phase too.  The 1/3 plateau freezes into domain walls above beta ~ 5 and is never
# reached by rungs up to beta = 8 at L = 18; a ladder over [2, 5] reaches it in every run of 2x10^5 sweeps.
TTS_LADDERS = ((0.25, 8.0), (0.25, 8.0), (0.25, 8.0), (2.0, 5.0))


def run_tts(args, rank, ws):
    """Time to solution at the paper's four phase points, L in {6, 12, 18}.
    Per point, 32 independent replica-exchange ladders of 32 rungs (beta
    geometric in the phase's range of TTS_LADDERS, swaps every 2 sweeps) and, for comparison, 1024
    independent chains at fixed beta = 4; every chain's first sweep at its
    point's brute-force supercell ground-state energy is recorded on the
    device (measured every sweep).  A run is a ladder (first hit of any rung)
    or a fixed-beta chain; TTS_99 = T log(0.01) / log(1 - p_gnd) in sweeps,
    and in seconds of this GPU's sweep time for the whole context (every run
    of the context advances together)."""
    import torch
    import paper_2511_20911_gb300 as crbm
    from paper_2511_20911_gb300 import analysis
    S = args.sweeps_per_step
    R, ladders, beta_fixed = 32, 32, 4.0
    ladder_betas = [lo * (hi / lo) ** (np.arange(R) / (R - 1)) for lo, hi in TTS_LADDERS]
    rows, total_updates, total_s = [], 0, 0.0
    with ClockSampler(torch.cuda.current_device()) as clk:
        for L in (6, 12, 18):
            e_gs = [analysis.ground_state_energy(L, J, Jp, h)[0] for _, J, Jp, h, _ in TTS_PHASES]
            for mode in ("tempering", "fixed"):
                if mode == "tempering":
                    params = dict(J=[], Jp=[], h=[], beta=[])
                    for (_, J, Jp, h, _), betas in zip(TTS_PHASES, ladder_betas):
                        for _ in range(ladders):
                            params["J"] += [J] * R
                            params["Jp"] += [Jp] * R
                            params["h"] += [h] * R
                            params["beta"] += [float(b) for b in betas]
                    n = len(params["J"])
                    cp = np.arange(n, dtype=np.int32)
                    point_of_chain = np.arange(n) // (ladders * R)
                    s = crbm.Sampler(L, params, n, chain_param=cp, seed=replica_seed(31 + L, rank), measure_every=1,
                                     swap_every=2, layout=crbm.CRBM_LAYOUT_SMEM)
                    s.set_targets(np.repeat(np.asarray(e_gs, np.int64), ladders * R))
                else:
                    params = dict(J=[p[1] for p in TTS_PHASES], Jp=[p[2] for p in TTS_PHASES],
                                  h=[p[3] for p in TTS_PHASES], beta=[beta_fixed] * len(TTS_PHASES))
                    n = ladders * R * len(TTS_PHASES)
                    cp = (np.arange(n) // (ladders * R)).astype(np.int32)
                    point_of_chain = cp
                    s = crbm.Sampler(L, params, n, chain_param=cp, seed=replica_seed(21 + L, rank), measure_every=1,
                                     layout=crbm.CRBM_LAYOUT_SMEM)
                    s.set_targets(e_gs)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record()
                s.sweep(S)
                b.record()
                torch.cuda.synchronize()
                sec = a.elapsed_time(b) / 1e3
                total_s += sec
                total_updates += n * L * L * S
                hits = s.first_hits()
                if mode == "tempering":   # a run is a ladder: its first rung to reach the ground state
                    h = hits.reshape(-1, R)
                    runs = np.where((h >= 0).any(1), np.where(h >= 0, h, np.iinfo(np.int64).max).min(1), -1)
                    run_point = point_of_chain[::R]
                else:
                    runs, run_point = hits, point_of_chain
                for k, (name, J, Jp, h_, paper) in enumerate(TTS_PHASES):
                    pg, T, tts = analysis.time_to_solution(runs[run_point == k], S)
                    rows.append({"phase": name, "L": L, "mode": mode, "J": J, "Jp": Jp, "h": h_,
                                 "beta": list(TTS_LADDERS[k]) if mode == "tempering" else beta_fixed,
                                 "runs": int((run_point == k).sum()), "p_gnd": pg, "T_sweeps": T,
                                 "tts99_sweeps": tts, "tts99_s": None if tts is None else tts * sec / S,
                                 "context_s_per_sweep": sec / S, "paper_fpga_s": paper,
                                 "e_gs_per_spin": e_gs[k] / 16.0 / (L * L)})
                s.close()
    t_total = max_over_ranks(total_s, ws)
    out = {"metric": METRIC, "value": replica_value(total_updates, ws, t_total), "unit": UNIT, "n_gpus": ws,
           "steps": 1, "warmup": 0, "ms_per_step": t_total * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": {"workload": "time to solution at the paper's FM, dimer, Neel and 1/3-plateau points, "
                                  f"L in {{6,12,18}}: {ladders} replica-exchange ladders of {R} rungs (beta "
                                  f"geometric in [0.25, 8]; [2, 5] for the 1/3 plateau; swaps every 2 sweeps) per "
                                  f"point, and {ladders * R} "
                                  f"chains at fixed beta = {beta_fixed} per point; {S} sweeps; ground states by "
                                  "brute force over even supercells of <= 16 sites",
                      "parallelism": f"replicas x{ws}"},
           "clocks": clk.summary(),
           "tts": rows,
           "note": "tts99_s = TTS_99 in sweeps x this GPU's time per sweep of the whole context (all runs of "
                   "the context advance together); a tempering run is a 32-rung ladder; paper_fpga_s is the "
                   "FPGA time the paper prints for the phase"}
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_phase(args, rank, ws):
    """Ground-state phase diagram scan at L=18: 429 points (J'/J in [0, 3],
    h in [-8, 8]) x one 32-rung replica-exchange ladder each (beta in
    [0.25, 8]), every rung's first sweep at the point's brute-force supercell
    ground-state energy recorded on the device.  A point is solved when any
    of its rungs reaches that energy; the point's phase is the supercell
    ground state's (FM, Neel, dimer, 1/3 or 1/2 plateau)."""
    import torch
    import paper_2511_20911_gb300 as crbm
    from paper_2511_20911_gb300 import analysis, workloads
    S = args.sweeps_per_step
    w = workloads.phase_scan_workload()
    L, R, N = w["L"], w["rungs"], w["L"] ** 2
    s = crbm.Sampler(L, w["params"], w["n_chains"], chain_param=w["chain_param"], seed=replica_seed(w["seed"], rank),
                     measure_every=w["measure_every"], swap_every=w["swap_every"], layout=crbm.CRBM_LAYOUT_SMEM,
                     rng=crbm.CRBM_RNG_BITPLANE if args.rng == "bitplane" else crbm.CRBM_RNG_LANE)
    e_gs, labels = [], []
    for J, Jp, h in w["points"]:
        E, (a, b), pattern = analysis.ground_state_energy(L, J, Jp, h)
        nJ, nP, M = (int(x[0]) * (N // (a * b)) for x in analysis.ss_counts(pattern[None]))
        e_gs.append(E)
        labels.append(analysis.phase_label(nJ, nP, M, N))
    s.set_targets(np.repeat(np.asarray(e_gs, np.int64), R))
    with ClockSampler(torch.cuda.current_device()) as clk:
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a_ev.record()
        s.sweep(S)
        b_ev.record()
        torch.cuda.synchronize()
    sec = max_over_ranks(a_ev.elapsed_time(b_ev) / 1e3, ws)
    hits = s.first_hits().reshape(len(w["points"]), R)
    first = np.where((hits >= 0).any(1), np.where(hits >= 0, hits, np.iinfo(np.int64).max).min(1), -1)
    by_phase = {}
    for lab, f in zip(labels, first):
        d = by_phase.setdefault(lab, {"points": 0, "solved": 0, "first_hit_sweeps": []})
        d["points"] += 1
        if f >= 0:
            d["solved"] += 1
            d["first_hit_sweeps"].append(int(f))
    for d in by_phase.values():
        f = d.pop("first_hit_sweeps")
        d["median_first_hit_sweep"] = float(np.median(f)) if f else None
    short = {"FM": "F", "Neel": "N", "dimer": "D", "1/3 plateau": "3", "1/2 plateau": "2"}
    rows = []
    for i in range(w["n_jp"]):
        row = ""
        for j in range(w["n_h"]):
            k = i * w["n_h"] + j
            c = short.get(labels[k], "?")
            row += c if first[k] >= 0 else c.lower() if c.isalpha() else "."
        rows.append(f"J'={w['points'][i * w['n_h']][1]:.2f} " + row)
    out = {"metric": METRIC, "value": replica_value(w["n_chains"] * N * S, ws, sec), "unit": UNIT, "n_gpus": ws,
           "steps": 1, "warmup": 0, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": {"workload": "ground-state phase scan: L=18, J=1, J'/J in [0,3] step 1/4, h in [-8,8] step 1/2 "
                                  f"(429 points) x 32-rung replica-exchange ladders (beta 0.25..8, swaps every "
                                  f"{w['swap_every']} sweeps), {S} sweeps, ground states by brute force over even "
                                  "supercells of <= 16 sites" + ("; bit-plane uniforms" if args.rng == "bitplane"
                                                                  else ""), "parallelism": f"replicas x{ws}"},
           "clocks": clk.summary(),
           "phase_scan": {"points": len(first), "solved": int((first >= 0).sum()), "by_phase": by_phase,
                          "map": rows,
                          "map_key": "rows J'/J, columns h = -8..8; F FM, N Neel, D dimer, 3 1/3 plateau, "
                                     "2 1/2 plateau (supercell ground state); lower case or '.': not reached"}}
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_batch(args, rank, ws, quiet=False):
    """Mixed L in {6,9,12,18,24,48} x 8 tempering ladders of 32 betas, all
    members advanced by one graph-captured launch per step."""
    import torch
    import paper_2511_20911_gb300 as crbm
    from paper_2511_20911_gb300 import workloads
    specs = workloads.tempering_batch_workload()
    S = args.sweeps_per_step if args.workload == "batch" else DEFAULT_SWEEPS["batch"]
    K, W = args.steps, args.warmup
    members = []
    env_warps = os.environ.get("CRBM_WARPS")
    if args.warps > 0:
        os.environ["CRBM_WARPS"] = str(args.warps)  # every member, read when it is created
    try:
        for sp in specs:
            sp = dict(sp, seed=replica_seed(sp["seed"], rank), measure_every=args.measure_every)
            m = crbm.Sampler(**sp)
            if args.warps <= 0:
                m.autotune(50)
            members.append(m)
    finally:
        if args.warps > 0:
            if env_warps is None:
                del os.environ["CRBM_WARPS"]
            else:
                os.environ["CRBM_WARPS"] = env_warps
    batch = crbm.Batch(members)
    if args.warps <= 0:
        batch.autotune(200)  # the batched launch's own CTA shape (members' state put back)
    else:
        assert batch.threads == 32 * args.warps, (batch.threads, args.warps)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(W):
        batch.sweep(S)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    if ws > 1:
        torch.distributed.barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for k in range(K):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            batch.sweep(S)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    t_total = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, ws)
    per_sweep = sum(sp["n_chains"] * sp["L"] ** 2 for sp in specs)
    value = replica_value(per_sweep * S * K, ws, t_total)
    calls = sum(4 * ((sp["L"] + 1) // 2) ** 2 * sp["n_chains"] for sp in specs) * S
    achieved = MUL_OPS_PER_CALL * calls / (t_total / K) / 1e12
    peak = SM_COUNT * IMUL_LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    # end to end with host buffers: spins in, one batched step, observables out
    host = [m.get_spins() for m in members]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m, hsp in zip(members, host):
        m.set_spins(hsp)
    batch.sweep(S)
    obs = [m.observables() for m in members]
    e2e_t = time.perf_counter() - t0
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
           "ms_per_step": t_total / K * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": {"workload": "mixed L in {6,9,12,18,24,48} x 8 replica-exchange ladders of 32 "
                                  "geometric beta in [0.2,10], J'/J=1.5, h=1, swaps every 10 sweeps, "
                                  "one graph-captured launch per step",
                      "n_chains": sum(sp["n_chains"] for sp in specs), "sweeps_per_step": S,
                      "threads_per_cta": batch.threads, "threads_autotuned": args.warps <= 0,
                      "warps_tuned": [m.warps for m in members],
                      "l2": "flushed between steps (256 MiB write outside the step events)",
                      "parallelism": f"replicas x{ws}"},
           "sweeps_per_s": S * K / t_total,
           "clocks": clk.summary(),
           "e2e": {"value": per_sweep * S / e2e_t, "unit": UNIT,
                   "h2d_bytes_per_step": int(sum(h.nbytes for h in host)),
                   "d2h_bytes_per_step": int(sum(o.nbytes for o in obs))},
           # each step replays one captured graph of two kernels: the batched sweep and the clock update
           "gpu_launches": 2 * K,
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                        "frac": achieved / peak, "traffic": None}}
    for m in members:
        m.close()
    if rank == 0 and not quiet:
        print(json.dumps(out))
    return out


PASS_FLOP_PER_BLOCK = 2 * (64 * 16 * 54 + 36 * 16 * 144 + 16 * 144)  # the net's MACs x 2 per 4x4 block


def proposal_arm(s, prop, every, chunk, target_se, max_chunks, cp, L, stream, min_chunks=4):
    """Advance sampler ``s`` in chunks of ``chunk`` sweeps (plain Gibbs when
    ``every`` is None, else Gibbs with a block-move pass after every ``every``
    sweeps) until the standard error of the mean energy per spin is at most
    ``target_se`` at every beta point (and at least ``min_chunks`` chunks, so
    the autocorrelation estimates rest on enough samples), or ``max_chunks``.  Per chunk and
    chain: the mean, and the effective samples of E and m by Sokal windowing
    (c = 5) on the chunk's series (chunks are much longer than the
    autocorrelation times); SE of a point = pooled sigma / sqrt(sum of ESS).
    Returns the GPU seconds of the sweeps and passes, sweeps run, and per point
    the SE of e and m, the ESS of E and m and the mean e."""
    import torch
    from paper_2511_20911_gb300 import analysis
    N = L * L
    G = int(cp.max()) + 1
    sums = {k: np.zeros(G) for k in ("essE", "essM", "sE", "sE2", "sM", "sM2", "n")}
    sec, chunks = 0.0, 0
    p0 = prop.stats() if prop is not None else None
    se_e = np.full(G, np.inf)
    while chunks < max_chunks:  # at least min_chunks, then until the target error
        s.reset_observables()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        if every is None:
            s.sweep(chunk)
        else:
            prop.sweep_mixed(s, chunk, every=every)
        b.record(stream)
        torch.cuda.synchronize()
        sec += a.elapsed_time(b) / 1e3
        chunks += 1
        ser = s.series().transpose(1, 0, 2).astype(np.float64)     # [chain][T][3]
        E = (ser[..., 0] + ser[..., 1] - 3.0 * ser[..., 2]) / N     # e per spin (J = J' = 1, h = 3)
        M = ser[..., 2] / N
        essE = analysis.effective_samples(E, burn_frac=0.0)
        essM = analysis.effective_samples(M, burn_frac=0.0)
        for g in range(G):
            m = cp == g
            sums["essE"][g] += essE[m].sum()
            sums["essM"][g] += essM[m].sum()
            sums["sE"][g] += E[m].sum()
            sums["sE2"][g] += (E[m] ** 2).sum()
            sums["sM"][g] += M[m].sum()
            sums["sM2"][g] += (M[m] ** 2).sum()
            sums["n"][g] += E[m].size
        varE = sums["sE2"] / sums["n"] - (sums["sE"] / sums["n"]) ** 2
        varM = sums["sM2"] / sums["n"] - (sums["sM"] / sums["n"]) ** 2
        se_e = np.sqrt(np.maximum(varE, 0) / np.maximum(sums["essE"], 1e-300))
        se_m = np.sqrt(np.maximum(varM, 0) / np.maximum(sums["essM"], 1e-300))
        if chunks >= min_chunks and (se_e <= target_se).all():
            break
    out = {"seconds": sec, "sweeps": chunks * chunk, "reached": bool((se_e <= target_se).all()),
           "se_e": se_e.tolist(), "se_m": se_m.tolist(), "ess_E": sums["essE"].tolist(),
           "ess_m": sums["essM"].tolist(), "e_per_spin": (sums["sE"] / sums["n"]).tolist(),
           "m_per_spin": (sums["sM"] / sums["n"]).tolist(),
           "ess_per_s_E": (sums["essE"] / sec).tolist(), "ess_per_s_m": (sums["essM"] / sec).tolist()}
    if prop is not None:
        p1 = prop.stats()
        out["accept"] = (p1[1] - p0[1]) / max(1, p1[0] - p0[0])
    return out


def run_proposal(args, rank, ws, sizes=((18, 20000), (48, 60000)), everys=(1, 4, 8), quiet=False):
    """Learned block proposal: train it on the GPU on configurations the
    sampler generates (L=18, J'/J=1, beta in [1.5,3], h in [2.5,3.5]); then, at
    L=18 and L=48 (J'/J=1, h=3, beta in {1.5,2,3}, 4096 chains, from one
    equilibrated state), run plain Gibbs and Gibbs + block moves (a pass after
    every 1, 4 or 8 sweeps) each until the standard error of the energy per
    spin is <= 1e-4 at every beta, and compare effective samples per second
    (and the time to that error).  Also times the pass kernel alone against
    the measured bf16 tensor peak."""
    import torch
    import paper_2511_20911_gb300 as crbm
    from paper_2511_20911_gb300 import workloads
    chunk = args.sweeps_per_step
    target = 1e-4
    stream = torch.cuda.current_stream()
    tw = workloads.proposal_training_workload()
    src = crbm.Sampler(**tw)
    src.sweep(500)
    prop = crbm.Proposal(seed=2024 + rank)
    t0 = time.perf_counter()
    losses = prop.train(src, steps=400, batch=4096, lr=1e-2, sweeps_between=2)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    results, kernel = [], {}
    peak = measured_peaks().get("bf16_tflops") or 1900.8
    with ClockSampler(torch.cuda.current_device()) as clk:
        for L, burn in sizes:
            ew = workloads.proposal_eval_workload(L)
            cp = np.asarray(ew["chain_param"])
            base = crbm.Sampler(**dict(ew, measure_every=1, series_len=chunk))
            base.sweep(burn)
            ck = base.save()
            # the pass alone: CUDA events around 200 passes
            pk = crbm.Sampler(**dict(ew, measure_every=1, series_len=chunk))
            pk.load(ck)
            prop.passes(pk, 5)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            prop.passes(pk, 200)
            b.record(stream)
            torch.cuda.synchronize()
            pass_s = a.elapsed_time(b) / 1e3 / 200
            a.record(stream)
            pk.sweep(200)
            b.record(stream)
            torch.cuda.synchronize()
            sweep_s = a.elapsed_time(b) / 1e3 / 200
            flop = PASS_FLOP_PER_BLOCK * max(1, L // 8) ** 2 * ew["n_chains"]
            kernel[f"L{L}"] = {"pass_us": pass_s * 1e6, "sweep_us": sweep_s * 1e6,
                               "pass_in_sweeps": pass_s / sweep_s, "flop_per_pass": flop,
                               "tflops": flop / pass_s / 1e12, "frac_of_bf16_peak": flop / pass_s / 1e12 / peak}
            pk.close()
            arms = {}
            for name, every in [("plain", None)] + [(f"every{k}", k) for k in everys]:
                s = crbm.Sampler(**dict(ew, measure_every=1, series_len=chunk))
                s.load(ck)
                arms[name] = proposal_arm(s, None if every is None else prop, every, chunk, target, 80, cp, L,
                                          stream)
                s.close()
            row = {"L": L, "beta": ew["params"]["beta"], "h": 3.0, "burn_in_sweeps": burn, "arms": arms}
            for name in arms:
                if name == "plain":
                    continue
                row[f"ess_per_s_gain_E_{name}"] = [m / p for m, p in zip(arms[name]["ess_per_s_E"],
                                                                           arms["plain"]["ess_per_s_E"])]
                row[f"ess_per_s_gain_m_{name}"] = [m / p for m, p in zip(arms[name]["ess_per_s_m"],
                                                                           arms["plain"]["ess_per_s_m"])]
                row[f"time_to_se_ratio_{name}"] = (arms["plain"]["seconds"] / arms[name]["seconds"]
                                                   if arms[name]["reached"] and arms["plain"]["reached"] else None)
            results.append(row)
            base.close()
    best = max((g for r in results for k, v in r.items() if k.startswith("ess_per_s_gain_E_") for g in v),
               default=None)
    k18 = kernel.get("L18", next(iter(kernel.values())))
    line = {"metric": METRIC, "value": best, "unit": "ESS/s of E, mixed / plain Gibbs (best arm and beta)",
            "n_gpus": ws, "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16+u32", "data": "synthetic",
            "config": {"workload": "learned 4x4 block proposal (3x3 conv net 6-16-16-1, bf16/fp32, tcgen05) + "
                                   "Gibbs vs plain Gibbs, J'/J=1, h=3, beta in {1.5,2,3}, L in {18,48}, 4096 "
                                   "chains, from one equilibrated state, each arm run until SE(E)/N <= 1e-4",
                       "chunk_sweeps": chunk, "train_steps": 400, "train_batch": 4096},
            "train": {"seconds": train_s, "loss_first": float(losses[:5].mean()),
                      "loss_last": float(losses[-20:].mean())},
            "pass_kernel": kernel,
            "roofline": {"bound": "tensor", "achieved": k18["tflops"], "peak": peak, "unit": "TFLOP/s",
                         "frac": k18["tflops"] / peak, "traffic": None,
                         "note": "k_prop_pass at L=18, 4096 chains: the net's algorithmic FLOPs (0.28 MFLOP per "
                                 "4x4 block) per pass over the CUDA-event time of one pass; peak = measured bf16 "
                                 "burst (MEASURED_PEAKS.json)"},
            "clocks": clk.summary(),
            "results": results}
    if rank == 0 and not quiet:
        print(json.dumps(line))
    return line


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def philox_peak(dev, sm_max_mhz):
    """Measured integer-multiply ceiling: the library's Philox throughput probe
    (crbm_philox_stream, 20 wide products per call, none shareable) on 8 CTAs
    of 256 threads per SM, best of 5 timed launches after 2 warm-ups."""
    import torch
    import paper_2511_20911_gb300 as crbm
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    nb, th, calls = sms * 8, 256, 4096
    sink = torch.zeros(nb * th, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    best = None
    for k in range(7):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        crbm.crbm_philox_stream(sink, nb, th, calls, seed=k)
        b.record(st)
        torch.cuda.synchronize()
        if k >= 2:
            t = a.elapsed_time(b) / 1e3
            best = t if best is None else min(best, t)
    rate = nb * th * calls / best
    derived = sms * IMUL_LANES_PER_SM_CLK * sm_max_mhz * 1e6
    return {"philox_calls_per_s": rate, "mul_ops_per_s": rate * MUL_OPS_PER_CALL, "sms": sms,
            "derived_mul_ops_per_s": derived, "probe": f"crbm_philox_stream {nb}x{th} threads x {calls} calls, "
                                                      "best of 5 launches"}


def measure_sampler(args, workload, rank, ws, with_e2e=True, sq_every=0):
    """One timed line of the grid (L=18, SMEM) or stream (L=384, HBM) workload:
    W warm-up steps, K timed steps of S sweeps with CUDA events on the
    library's stream, L2 flushed between steps, clocks sampled meanwhile."""
    import torch
    import paper_2511_20911_gb300 as crbm
    from paper_2511_20911_gb300 import analysis

    dev = torch.cuda.current_device()
    w = workload_config(workload, rank)
    S = args.sweeps_per_step if workload == args.workload else DEFAULT_SWEEPS[workload]
    K, W = args.steps, args.warmup
    n_meas = S * K // args.measure_every
    layout = crbm.CRBM_LAYOUT_SMEM if workload == "grid" else crbm.CRBM_LAYOUT_STREAM
    paper = args.precision == "paper"
    bitplane = args.rng == "bitplane"
    fixed_warps = args.warps if workload == "grid" and args.warps > 0 else 0
    env_warps = os.environ.get("CRBM_WARPS")
    if fixed_warps:
        os.environ["CRBM_WARPS"] = str(fixed_warps)  # read when the context is created
    try:
        s = crbm.Sampler(w["L"], w["params"], w["n_chains"], chain_param=w["chain_param"], seed=w["seed"],
                         measure_every=args.measure_every, series_len=n_meas, layout=layout, sq_every=sq_every,
                         precision=crbm.CRBM_PRECISION_PAPER if paper else crbm.CRBM_PRECISION_EXACT,
                         rng=crbm.CRBM_RNG_BITPLANE if bitplane else crbm.CRBM_RNG_LANE)
    finally:
        if fixed_warps:
            if env_warps is None:
                del os.environ["CRBM_WARPS"]
            else:
                os.environ["CRBM_WARPS"] = env_warps
    if fixed_warps:
        assert s.warps == fixed_warps, (s.warps, fixed_warps)
    # CTA shape, on scratch copies
    tuned_warps = s.autotune(200) if workload == "grid" and not fixed_warps else None
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(W):
        s.sweep(S)
    torch.cuda.synchronize()
    s.reset_observables()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    launches0 = s.launch_count
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for k in range(K):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            s.sweep(S)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches = s.launch_count - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = max_over_ranks(sum(step_ms) / 1e3, ws)
    spin_updates = w["n_chains"] * w["L"] ** 2 * S * K
    value = replica_value(spin_updates, ws, t_total)

    # effective samples of E and m over the timed steps
    ser = s.series()                                   # [T][chain][3]
    p = w["params"]
    cp = np.asarray(w["chain_param"])
    Jc, Jpc, hc = (np.asarray(p[k])[cp] for k in ("J", "Jp", "h"))
    E = analysis.energy_series(ser.transpose(1, 0, 2), Jc[:, None], Jpc[:, None], hc[:, None])
    Mx = ser[:, :, 2].T.astype(np.float64)
    if ser.shape[0] >= 20:
        ess_E = float(analysis.effective_samples(E).sum())
        ess_m = float(analysis.effective_samples(Mx).sum())
    else:                      # too few measurements in the timed steps for a windowed estimate
        ess_E = ess_m = float("nan")
    sq_info = None
    if sq_every:
        sq = s.structure_factor()                      # [n_params][L][L]
        _, ns = s.correlations()
        sq_info = {"every_sweeps": sq_every, "samples_per_point": int(np.min(ns)),
                   "note": "per-point S(q) = (1/N)<|sum_r s_r e^{iq.r}|^2> accumulated on the device "
                           "inside the timed steps",
                   "max_S_over_N": float(sq[:, :, :].max() / w["L"] ** 2)}

    e2e = None
    if with_e2e:
        # end to end through the C ABI with host buffers in pinned memory: set
        # spins (H2D), sweep, read observables (D2H), every step
        spins_h = torch.from_numpy(s.get_spins()).pin_memory().numpy()
        obs_h = torch.zeros((w["n_chains"], crbm.CRBM_NSUM), dtype=torch.int64).pin_memory().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_steps = max(1, K // 2)
        for k in range(e2e_steps):
            s.set_spins(spins_h)
            s.sweep(S)
            s.observables(out=obs_h)
        e2e_t = time.perf_counter() - t0
        e2e = {"value": w["n_chains"] * w["L"] ** 2 * S * e2e_steps * ws / e2e_t, "unit": UNIT,
               "h2d_bytes_per_step": int(spins_h.nbytes), "d2h_bytes_per_step": int(obs_h.nbytes)}

    cpc = CALLS_PER_CELL
    if paper:
        cpc = CALLS_PER_CELL_PAPER if workload == "grid" else CALLS_PER_CELL_PAPER_STREAM
    calls = cpc * (w["L"] // 2) ** 2 * w["n_chains"] * S
    if bitplane:   # expected calls of the early-exit comparison (hidden nodes, then spins)
        Wc = w["L"] // 2
        if workload == "grid":   # one CTA per word: its nodes in groups of 32
            n_words = (w["n_chains"] + 31) // 32
            per_word = bitplane_expected_calls(10 * Wc * Wc) + bitplane_expected_calls(w["L"] ** 2)
        else:                    # 64-chain groups of two words; 16 x 16-cell tiles
            n_words = 2 * ((w["n_chains"] + 63) // 64)
            per_word = 0.0
            for ti in range(0, Wc, 16):
                for tj in range(0, Wc, 16):
                    cells = min(16, Wc - ti) * min(16, Wc - tj)
                    per_word += bitplane_expected_calls(10 * cells) + bitplane_expected_calls(4 * cells)
        calls = per_word * n_words * S
        cpc = calls / ((w["L"] // 2) ** 2 * w["n_chains"] * S)
    if workload == "grid":   # one launch per step: spins in and out once
        hbm_bytes = w["n_chains"] * w["L"] ** 2 / 8 * 2
    else:                    # per sweep: spins read + written, hidden written + read
        hbm_bytes = w["n_chains"] * w["L"] ** 2 * 7 / 8 * S
    ck = clk.summary()
    sm_max = ck["sm_max_mhz"] or SM_MAX_MHZ
    pk = philox_peak(dev, sm_max)
    achieved = MUL_OPS_PER_CALL * calls / (t_total / K) / 1e12
    peak = pk["derived_mul_ops_per_s"] / 1e12
    traffic = MEASURED_TRAFFIC.get(workload + ("_paper" if paper else "") + ("_bitplane" if bitplane else "") +
                                   ("_sq" if sq_every else ""))
    cfg = config_dict(w, args, workload)
    cfg["sweeps_per_step"] = S
    if sq_every:
        cfg["sq_every"] = sq_every
    if tuned_warps:
        cfg["warps_per_cta_autotuned"] = tuned_warps
    if fixed_warps:
        cfg["warps_per_cta"] = fixed_warps
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": t_total / K * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": cfg,
        "ess_per_s": {"energy": None if ess_E != ess_E else ess_E * ws / t_total,
                      "m": None if ess_m != ess_m else ess_m * ws / t_total,
                      "method": "Sokal windowing c=5 on per-chain series (every "
                                f"{args.measure_every} sweeps), first 10% discarded, summed over chains"},
        "node_updates_per_s": value * 3.5,
        "clocks": ck,
        "gpu_launches": int(launches),
        "hbm": {"algorithmic_gbs": hbm_bytes / (t_total / K) / 1e9, "peak_gbs": 6790.0,
                "note": "0.25 B (SMEM layout: spins in and out once per launch) or 0.875 B "
                        "(streamed: spins 2 bits + hidden 5 bits per spin-update) of algorithmic traffic"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak,
                     "peak_measured": pk["mul_ops_per_s"] / 1e12,
                     "frac_of_measured": achieved / (pk["mul_ops_per_s"] / 1e12),
                     "peak_probe": pk["probe"],
                     "traffic": traffic[0] if traffic else None,
                     "traffic_unit": "bytes " + traffic[1] if traffic else None,
                     "note": f"integer-multiply ceiling: {pk['sms']} SM x 64 lanes/clk x {sm_max:.0f} MHz "
                             "(peak) and the library's Philox throughput probe (peak_measured); 40 "
                             "multiply ops per Philox-4x32-10 call, "
                             f"{cpc:.3g} calls per chain-cell-sweep" + (" (expected count of the bit-plane "
                             "early exit)" if bitplane else ""),
                     "philox_calls_per_s": calls / (t_total / K)},
    }
    if e2e:
        out["e2e"] = e2e
    if sq_info:
        out["structure_factor"] = sq_info
    s.close()
    del flush
    torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.sweeps_per_step is None:
        args.sweeps_per_step = DEFAULT_SWEEPS[args.workload]
    rank, ws = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, ws)
        return
    if args.workload == "batch":
        run_batch(args, rank, ws)
        return
    if args.workload == "proposal":
        run_proposal(args, rank, ws)
        return
    if args.workload == "tts":
        run_tts(args, rank, ws)
        return
    if args.workload == "phase":
        run_phase(args, rank, ws)
        return
    import torch
    sq_every = 100 if args.workload == "grid" and args.sq_every is None else (args.sq_every or 0)
    if args.rng == "bitplane" or args.workload != "grid":
        sq_every = 0            # correlations: lane uniforms, SMEM layout
    out = measure_sampler(args, args.workload, rank, ws, with_e2e=True, sq_every=sq_every)
    if args.workload == "grid" and not args.no_extra_lines:
        keys = ("value", "unit", "ms_per_step", "steps", "warmup", "config", "clocks", "gpu_launches", "hbm",
                "roofline")
        out["lines"] = {}
        sub = measure_sampler(args, "stream", rank, ws, with_e2e=False)
        out["lines"]["stream_L384"] = {k: sub[k] for k in keys}
        if args.precision == "exact" and args.rng == "lane":
            # the other modes of the grid workload, the tempering batch and the learned
            # proposal (L=18), so that one bench run measures every line
            for name, prec, rng in (("grid_paper_precision", "paper", "lane"), ("grid_bitplane", "exact", "bitplane")):
                sub = measure_sampler(argparse.Namespace(**dict(vars(args), precision=prec, rng=rng)), "grid",
                                      rank, ws, with_e2e=False)
                out["lines"][name] = {k: sub[k] for k in keys}
            sub = run_batch(args, rank, ws, quiet=True)
            out["lines"]["tempering_batch"] = {k: sub[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup",
                                                                 "config", "clocks", "gpu_launches", "roofline")}
            sub = run_proposal(argparse.Namespace(**dict(vars(args), sweeps_per_step=DEFAULT_SWEEPS["proposal"])),
                               rank, ws, sizes=((18, 20000),), everys=(1, 8), quiet=True)
            out["lines"]["learned_proposal_L18"] = {k: sub[k] for k in ("value", "unit", "config", "pass_kernel",
                                                                        "roofline", "clocks", "results")}
    if rank == 0 and not args.no_cpu_baseline:
        w = workload_config(args.workload, 0)
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds, 1 if args.precision == "paper" else 0,
                                           1 if args.rng == "bitplane" else 0)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
