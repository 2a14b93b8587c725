"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks (replicas only --
no data-path collective; one all-reduce of the timing, max over ranks)."""
import os
import socket
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        t = bench.max_over_ranks(1.5 + rank, torch.device("cpu"), ws)
        q.put((rank, t, bench.replica_throughput(100, ws, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
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
    # the slower replica (2.5 s) sets the time; the job rendered 2 x 100 frames
    assert got == [(0, 2.5, 80.0), (1, 2.5, 80.0)]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0, torch.device("cpu"), 1) == 3.0
    assert bench.replica_throughput(50, 1, 2.0) == 25.0


def test_reference_arm_other_ranks_exit_silently():
    """Under torchrun only rank 0 times the oracle; the others exit 0 at once."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
