"""The multi-GPU path of the benchmark is replicas only (each rank runs the whole workload;
no data-path collective): the slowest rank's time and the whole-job value, checked with
two gloo ranks on the CPU, and the reference arm's rank > 0 exiting without work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        torch.distributed.barrier()
        t = bench.max_over_ranks(1.0 + rank, ws, "cpu")     # rank 1 is the slower one
        v = bench.job_value(1000, 20, ws, t)
        out.put((rank, t, v))
        torch.distributed.barrier()
    finally:
        torch.distributed.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_units():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 2.0                              # max over ranks
        assert v == 1000 * 20 * 2 / 2.0              # both ranks' units over the slowest time


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
