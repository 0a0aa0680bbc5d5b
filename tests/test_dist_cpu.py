"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the
barrier, the max over ranks of the timed region and the whole-job sums that
turn per-rank replicas into one number (weak scaling, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    d = bench.Dist()
    d.barrier()
    t = d.max(1.0 + rank)                 # slowest rank sets the time
    cycles = d.sum(10.0 * (rank + 1))     # units processed by all ranks
    from paper_2012_10091_gb300 import workloads as W
    w = W.burgers_large(seed=d.rank)      # each replica draws its own inputs
    q.put((rank, t, cycles, float(W.initial_fine_model(w)[0])))
    d.close()


def test_two_rank_replicas_reduce_on_host():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]
    assert [o[2] for o in out] == [30.0, 30.0]
    assert out[0][3] != out[1][3]          # independent replicas


def test_batched_problems_shard_over_ranks():
    """The 96 independent problems are split over ranks with no overlap, every
    problem owned once, and the forecast work balanced within 2 %."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_2012_10091_gb300 import workloads as W
    ws = W.ns2d_batch(96, seed=0)
    for world in (1, 2, 4, 8):
        parts = [bench.shard_problems(ws, world, r) for r in range(world)]
        owned = sorted(i for p in parts for i in p)
        assert owned == list(range(len(ws)))
        loads = [sum(bench.problem_work(ws[i]) for i in p) for p in parts]
        assert max(loads) <= 1.02 * min(loads)


def test_batched_workload_recipe():
    """Coarse sides, ensemble sizes and observation counts of the batched
    workload stay in their stated sets and ranges, drawn reproducibly."""
    from paper_2012_10091_gb300 import workloads as W
    ws = W.ns2d_batch(96, seed=0)
    assert len(ws) == 96
    assert {w.nc for w in ws} == {64, 96, 128, 192}
    assert {w.ne for w in ws} == {16, 32, 64, 128}
    assert all(w.nf == 4 * w.nc and w.ny % 2 == 0 and 256 <= w.ny <= 2048 for w in ws)
    assert len({w.seed for w in ws}) == 96
    assert [w.name for w in W.ns2d_batch(96, seed=0)] == [w.name for w in ws]
