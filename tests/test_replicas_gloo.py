"""The N > 1 (replicas) path of bench.py on CPU: two gloo ranks.  Each rank
runs its own replica; the job's time is the slowest rank's and its rate is
all ranks' work over that time.  The reference arm does its work on rank 0
only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r measured (10 + r) ms for the metric and (20 + 3 r) ms in total
    metric_ms, total_ms = bench.replica_max(dist, "cpu", 10.0 + rank, 20.0 + 3 * rank)
    value = bench.replica_value(world, 2.0e12, metric_ms)
    out.put((rank, metric_ms, total_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, metric_ms, total_ms, value in res:
        assert metric_ms == 11.0 and total_ms == 23.0          # both ranks see the maxima
        assert value == pytest.approx(2 * 2.0e12 / 11.0e-3 / 1e12)


def test_single_process_aggregation_is_the_identity():
    import bench
    assert bench.replica_max(None, "cpu", 5.0, 7.0) == [5.0, 7.0]
    assert bench.replica_value(1, 1.0e12, 1000.0) == pytest.approx(1.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench
    sys_argv = sys.argv
    try:
        sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"]
        args = bench.parse()
    finally:
        sys.argv = sys_argv
    bench.run_reference(args, rank=1)                         # other ranks: no work, no output
    assert capsys.readouterr().out == ""
