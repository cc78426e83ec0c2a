"""Host logic of multi-GPU runs on CPU ranks (gloo, world size 2).

The path does not shard: `bench.py --gpus N` runs N replicas of the same workload, one per
rank, reduces the timed region's duration to its maximum over ranks, reports the
units of all replicas over that time, and prints from rank 0 only. These tests run
that host logic on two CPU processes."""
import multiprocessing as mp
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=2)
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow replica
    ms = bench.max_over_ranks(local_ms, 2, "cpu")
    dist.barrier()
    q.put((rank, ms, bench.whole_job_rate(40, 2, ms)))
    dist.destroy_process_group()


def test_timed_region_is_the_slowest_rank_and_value_counts_every_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [150.0, 150.0]
    # 40 units per rank, 2 ranks, 150 ms -> 533.3 units/s for the whole job
    assert all(abs(o[2] - 80 / 0.150) < 1e-9 for o in out)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_rate(20, 1, 500.0) == 40.0


def test_reference_arm_prints_on_rank_zero_only():
    """Under torchrun every rank but 0 exits 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
