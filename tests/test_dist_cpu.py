"""The multi-process (torchrun) path of bench.py on CPU with gloo, world size
2: replicas time their own workload and the job takes the slowest rank's
time; the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys
from pathlib import Path


ROOT = Path(__file__).resolve().parent.parent


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, str(ROOT))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        t = bench.max_over_ranks(1.5 + rank, dist)  # rank 1 is the slow one
        v = bench.job_value(100.0, ws, t)
        q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [t for _, t, _ in out] == [2.5, 2.5]
    assert all(abs(v - 200.0 / 2.5) < 1e-12 for _, _, v in out)


def test_single_process_helpers():
    sys.path.insert(0, str(ROOT))
    import bench

    assert bench.max_over_ranks(3.25, None) == 3.25
    assert bench.job_value(10.0, 1, 2.0) == 5.0


def test_reference_arm_nonzero_rank_exits_quietly():
    """Under torchrun only rank 0 runs and prints the reference arm."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
