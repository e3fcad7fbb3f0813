"""Host logic of the N > 1 benchmark path on CPU: two processes over gloo
(the GPU path runs independent replicas with no collective on the data
path; the only exchange is the max over ranks of the step time)."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(torch, 10.0 + 3.0 * rank, torch.device("cpu"))
    dist.barrier()
    q.put((rank, ms, bench.job_value(world, 1000, ms)))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_processes():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    # both ranks see the slowest rank's time; the job rate counts both replicas
    assert [g[1] for g in got] == [13.0, 13.0]
    assert all(abs(g[2] - 2 * 1000 / 0.013) < 1e-6 for g in got)


def test_single_process_time_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, 7.5, torch.device("cpu")) == 7.5
    assert bench.job_value(1, 500, 250.0) == 2000.0


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
