"""Host logic of bench.py's multi-GPU path, on CPU with two gloo ranks: every rank advances its own
grid (replicas, no exchange), the timed region is the slowest rank's, and the reported rate counts
the cell-updates of all ranks.  The reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = bench.max_over_ranks(times[rank], dist)
    rate = bench.whole_job_rate(100, 10, 3, dist.get_world_size(), m)
    out.put((rank, m, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [120.0, 150.0]
    ps = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in res:
        assert m == 150.0
        assert rate == pytest.approx(100 * 10 * 3 * 2 / 0.150)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.whole_job_rate(8, 2, 5, 1, 1000.0) == pytest.approx(80.0)
    assert bench.launch_key(bench.parse_launch("twopass:32x8:z32:cpasync")) == "twopass:32x8:z32:cpasync"


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
