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


def _straggler_calls(first):
    """Lane-calls of the straggler scheme for one half-step, given per node
    and chain the first plane (0-based) at which the comparison is decided:
    two calls per node, then the nodes needing more, 32 at a time, each group
    drawing calls until its slowest node is decided."""
    import numpy as np
    need = np.minimum(8, (first.max(axis=1) + 1 + 3) // 4)   # calls each node needs
    extra = need[need > 2] - 2
    calls = 2 * len(need)
    for b in range(0, len(extra), 32):
        grp = extra[b:b + 32]
        calls += len(grp) * int(grp.max())
    return calls


def _first_planes(u, t):
    import numpy as np
    diff = u ^ t                                   # the first differing bit decides
    return np.where(diff == 0, 32, 31 - np.floor(np.log2(np.maximum(diff, 1))).astype(int))


def test_bitplane_expected_calls_matches_a_simulation():
    """The bit-plane roofline counts the expected Philox calls of the
    comparison as the kernels run it: two calls of four planes for every node,
    then the nodes with an open comparison (any of their 32 chains) from a
    straggler list, 32 at a time, each group drawing calls while any of its
    comparisons is open.  A direct simulation (random uniforms and thresholds,
    bits compared plane by plane) must give the same mean call count."""
    import numpy as np
    import bench
    rng = np.random.default_rng(3)
    for nodes, trials in ((32, 3000), (810, 300), (10, 3000)):
        calls = 0
        for _ in range(trials):
            u = rng.integers(0, 2**32, size=(nodes, 32), dtype=np.uint64)
            t = rng.integers(0, 2**32, size=(nodes, 32), dtype=np.uint64)
            calls += _straggler_calls(_first_planes(u, t))
        expect = bench.bitplane_expected_calls(nodes) / nodes
        assert abs(calls / trials / nodes - expect) < 0.01, (nodes, calls / trials / nodes, expect)


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
        trials, calls, nodes = 300, 0, 810
        for _ in range(trials):
            u = rng.integers(0, 2**32, size=(nodes, 32), dtype=np.uint64)
            t = rng.integers(0, 2**32, size=(nodes, 32), dtype=np.uint64)
            t[rng.random((nodes, 32)) < f] = 2**31
            calls += _straggler_calls(_first_planes(u, t))
        expect = bench.bitplane_expected_calls(nodes) / nodes
        assert abs(calls / trials / nodes - expect) < 0.01, (f, calls / trials / nodes, expect)
