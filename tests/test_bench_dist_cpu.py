"""The multi-process path of bench.py on CPU with the gloo backend (world size 2): max-over-ranks timing,
whole-job throughput of independent replicas, and the reference arm printing on rank 0 only."""

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


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as tdist

    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    vals = bench.dist_max([1.0 + rank, 10.0 - rank, 0.5 * rank])
    out.put((rank, vals))
    tdist.barrier()
    tdist.destroy_process_group()


def test_dist_max_and_job_throughput_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [2.0, 10.0, 0.5]
    sys.path.insert(0, ROOT)
    import bench
    # 2 replicas x 1e6 DOF x 10 steps in 100 ms (slowest rank) = 200 MDOF/s
    assert abs(bench.job_mdofs(2, 1_000_000, 10, 100.0) - 200.0) < 1e-9


def test_reference_arm_non_zero_rank_prints_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
