"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the path runs independent
replicas, so the only exchange is the max-over-ranks of the timed region, and the reference arm
runs on rank 0 alone."""
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


def _worker(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local = 10.0 * (rank + 1)                   # rank 1 is the slower replica
    mx = bench.reduce_max_ms(local, torch.device("cpu"))
    q.put((rank, mx, bench.aggregate_rate(5, ws, mx)))
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [20.0, 20.0]          # both ranks see the slowest replica
    assert out[0][2] == pytest.approx(2 * 5 / 0.020)    # 2 replicas x 5 steps in 20 ms


def test_reference_arm_runs_on_rank0_only():
    """--impl reference under a 2-rank launch: rank 0 prints one JSON line, rank 1 exits 0 silently."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r1 = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                         "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=600)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
