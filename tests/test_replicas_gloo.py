"""The N > 1 path of bench.py (independent replicas, no data-path
collective): each rank times its own replica, the job takes the slowest
rank's time, and the value counts the iterations of every rank.  Run as two
gloo processes on the CPU."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [1.0 + rank, 2.0 - 0.5 * rank]          # rank 1 is slower on the first timing
    slow = bench.slowest_rank(local)
    value = bench.replica_throughput(steps=5, world=world, slowest_secs=slow[0])
    out[rank] = (slow, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert res[0][0] == [2.0, 2.0] and res[1][0] == [2.0, 2.0]
    assert res[0][1] == pytest.approx(world * 5 / 2.0)
    assert res[0][1] == res[1][1]


@pytest.mark.slow
def test_reference_arm_prints_on_rank0_only():
    import json
    import subprocess
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "0"]
    for rank in (1, 0):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
        r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600)
        assert r.returncode == 0, r.stderr
        if rank == 1:
            assert r.stdout.strip() == ""
        else:
            line = json.loads(r.stdout.strip().splitlines()[-1])
            assert line["impl"] == "reference" and line["value"] > 0
            assert line["cpu_baseline"]["kind"] == "oracle"
            assert line["e2e"]["h2d_bytes_per_step"] == 0
