"""The multi-GPU path of the bench is replicas only (independent problems per rank, no
data-path collective): the whole-job rate is the units of all ranks over the slowest
rank's time.  Its host logic runs here as two gloo ranks on the CPU; the reference arm
on a non-zero rank exits without work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TIMES_MS = [12.5, 17.25]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.replica_max(TIMES_MS[rank], dist, device="cpu")))
    finally:
        dist.destroy_process_group()


def test_replica_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: max(TIMES_MS), 1: max(TIMES_MS)}


def test_replica_rate_is_whole_job():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_rate(1000.0, 2, 17.25) == pytest.approx(2000.0 / 0.01725)
    assert bench.replica_max(3.0) == 3.0


def test_reference_arm_on_other_ranks_does_no_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
