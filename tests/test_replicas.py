"""Host logic of the multi-GPU replica path (bench.py --gpus N) on CPU ranks:
world size 2 over gloo.  Each rank gets its own seed, the job time is the
largest rank time, and the whole-job value counts every rank's units.  No
data-path collective exists: the chains of different ranks never meet."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        t_local = 1.0 + 0.5 * rank            # rank 1 is the slower one
        t_max = bench.max_over_ranks(t_local, ws)
        grid = bench.workload_config("grid", rank)
        stream = bench.workload_config("stream", rank)
        out[rank] = (t_max, grid["seed"], stream["seed"], bench.replica_value(1000, ws, t_max))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replica_logic():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == pytest.approx(1.5)      # max over ranks
    assert res[0][1] != res[1][1] and res[0][2] != res[1][2]  # independent replicas
    assert res[0][3] == pytest.approx(2000 / 1.5)             # all ranks' units / slowest time


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.replica_seed(7, 0) == 7


def test_bitplane_expected_calls_matches_a_simulation():
    """The bit-plane roofline counts the expected Philox calls of the early
    exit: per warp of up to 32 nodes x 32 chains, calls of four planes while
    any comparison is open.  A direct simulation of that comparison (random
    uniforms and thresholds, bits drawn plane by plane) must give the same
    mean call count."""
    import numpy as np
    import bench
    rng = np.random.default_rng(3)
    for lanes in (32, 10):
        trials, calls = 4000, 0
        for _ in range(trials):
            u = rng.integers(0, 2**32, size=(lanes, 32), dtype=np.uint64)
            t = rng.integers(0, 2**32, size=(lanes, 32), dtype=np.uint64)
            diff = u ^ t                                   # first differing bit decides
            first = np.where(diff == 0, 32, 31 - np.floor(np.log2(np.maximum(diff, 1))).astype(int))
            planes = int(first.max()) + 1                  # planes until every comparison is decided
            calls += min(8, (planes + 3) // 4)
        expect = bench.bitplane_expected_calls(lanes) / lanes
        assert abs(calls / trials - expect) < 0.03, (lanes, calls / trials, expect)


def test_bitplane_expected_calls_with_half_thresholds():
    """Hidden units with m = 0 have the threshold exactly 2^31.  Such a
    comparison is decided on the first plane only when the uniform's top bit
    is 0; otherwise it stays open until the uniform's first further 1 bit, so
    it too closes with probability 1/2 per plane and the model needs no
    correction for them: a direct simulation with half (or most) of the
    thresholds at 2^31 gives the same mean call count."""
    import numpy as np
    import bench
    rng = np.random.default_rng(5)
    for f in (0.5, 0.9):
        trials, calls = 4000, 0
        for _ in range(trials):
            u = rng.integers(0, 2**32, size=(32, 32), dtype=np.uint64)
            t = rng.integers(0, 2**32, size=(32, 32), dtype=np.uint64)
            t[rng.random((32, 32)) < f] = 2**31
            diff = u ^ t
            first = np.where(diff == 0, 32, 31 - np.floor(np.log2(np.maximum(diff, 1))).astype(int))
            planes = int(first.max()) + 1
            calls += min(8, max(2, (planes + 3) // 4))   # the hidden half-step draws two calls first
        expect = bench.bitplane_expected_calls(32) / 32
        assert abs(calls / trials - expect) < 0.03, (f, calls / trials, expect)
