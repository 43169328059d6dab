"""The N > 1 host path of bench.py on CPU: two gloo ranks (127.0.0.1), each with its own scene replica
(weak scaling, no data-path collective); the whole-job value sums the ranks' units and divides by the
slowest rank's time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2005_06773_gb300 import scenarios as S
        value, total, t_max = bench.aggregate(1000.0 * (rank + 1), 0.5 + rank, world, "cpu")
        sc = S.intersection11(bench.replica_seed(rank))
        q.put((rank, value, total, t_max, sc.n_tests(), float(sc.objects[0].x0), float(sc.objects[0].y0)))
    finally:
        dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(2):
            r = q.get(timeout=120)
            out[r[0]] = r
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert sorted(out) == [0, 1]
    for r in (0, 1):
        _, value, total, t_max, n_tests, _, _ = out[r]
        assert total == 3000.0 and t_max == 1.5 and value == pytest.approx(2000.0)
    assert out[0][4] == out[1][4]                        # same workload shape per rank
    assert (out[0][5], out[0][6]) != (out[1][5], out[1][6])   # independent placements


def test_single_rank_aggregation_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(500.0, 0.25, 1, "cpu") == (2000.0, 500.0, 0.25)
