"""N > 1 replicas (bench.py --gpus N): each rank simulates its own network
with no data-path communication; the whole-job figure is the sum of events
over ranks divided by the max time over ranks.  Checked with 2 gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, ev = bench.aggregate(10.0 + rank * 5.0, 1000.0 * (rank + 1))
    q.put((rank, ms, ev))
    dist.destroy_process_group()


def test_two_replicas_aggregate():
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
    assert out == [(0, 15.0, 3000.0), (1, 15.0, 3000.0)]


def test_single_process_is_identity():
    import bench

    assert bench.aggregate(3.5, 42.0) == (3.5, 42.0)


def test_reference_arm_under_torchrun_prints_once():
    """bench.py --impl reference launched as the N-GPU job is: rank 0 alone
    times the oracle and prints one line (n_gpus = N); the other rank exits 0
    without work."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), os.path.join(root, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "4", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.lstrip().startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 4
