"""The multi-rank (replica) logic of bench.py on CPU with the gloo backend,
world size 2: the whole-job value uses the slowest rank's time, and the
reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]
    value, t = bench.combine_ranks(local_ms, 1e12, world, dist)
    q.put((rank, value, t))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_uses_max_time_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, t in out:
        assert t == 250.0
        # two replicas x 1e12 flop in 0.25 s
        assert abs(value - 2 * 1e12 / 0.25 / 1e9) < 1e-6


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


@pytest.mark.slow
def test_reference_arm_prints_one_line():
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--atoms", "50000"], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0


def test_build_waves_bound_host_memory():
    """The ranks of a multi-GPU bench build their operators in waves small
    enough for the host's memory: all at once for small operators, fewer at a
    time as the operator grows, never zero."""
    import bench
    assert bench._build_waves(1, 1_000_000) == 1
    assert bench._build_waves(8, 1000) == 8
    assert bench._build_waves(8, 10 ** 12) == 1
    w = bench._build_waves(8, 1_000_000)
    assert 1 <= w <= 8
