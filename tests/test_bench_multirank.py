"""The N > 1 logic of bench.py on CPU: two gloo ranks (independent replicas,
no collective on the data path) agree on the slowest rank's time, the
whole-job throughput counts every rank's pixels, each rank detects its own
image, and the reference arm runs on rank 0 only."""
import json
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_ms = [120.0, 150.0][rank]  # rank 1 is the slow one
    slowest = bench.max_over_ranks(t_ms, dist, "cpu")
    rate = bench.whole_job_rate(world, 10, 1920 * 1200, slowest)
    q.put((rank, slowest, rate, bench.replica_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    if not torch.distributed.is_available():
        pytest.skip("torch.distributed unavailable")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [150.0, 150.0]
    # 2 ranks x 10 steps x 2.304 Mpx in 150 ms
    assert got[0][2] == pytest.approx(2 * 10 * 2.304 / 0.150)
    assert got[0][3] != got[1][3]


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_rate(1, 4, 1e6, 2000.0) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps = 1
        warmup = 0
        gpus = 2
    assert bench.run_reference(A, 1, 2) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_line(capsys, oracle_mod):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps = 1
        warmup = 0
        gpus = 1
    # a tiny bounded sample keeps this quick: the budget is per step
    bench_budget = bench.oracle_sample_rate
    try:
        bench.oracle_sample_rate = lambda img, budget, **kw: bench_budget(img, 0.05, **kw)
        assert bench.run_reference(A, 0, 1) == 0
    finally:
        bench.oracle_sample_rate = bench_budget
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0

