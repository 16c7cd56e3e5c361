"""The multi-rank host logic of the benchmark on CPU, two gloo ranks.

Every rank embeds its own replica of the workload (the path does not shard),
so the job time is the slowest rank's and the whole-job value counts every
rank's work over that time; the oracle arm runs on rank 0 alone."""
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank total times of 3 steps: 300 ms on rank 0, 450 ms on rank 1
        total = bench.max_over_ranks(300.0 + 150.0 * rank, world)
        value = bench.job_value(2.0e9, world, 3, total)
        dist.barrier()
    finally:
        dist.destroy_process_group()
    q.put((rank, total, value))


def test_two_gloo_ranks_take_slowest_time_and_sum_work():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0]
    got = sorted(q.get() for _ in range(world))
    for rank, total, value in got:
        assert total == 450.0
        # 2 ranks x 3 steps x 2e9 entries in 0.45 s
        assert abs(value - 2 * 3 * 2.0e9 / 0.45) < 1e-3 * value


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_value(1e6, 1, 4, 2000.0) == 2e6


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"],
                       env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
