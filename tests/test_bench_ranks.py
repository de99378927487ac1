"""The benchmark's multi-rank (replica) path on CPU: two gloo ranks.

Under torchrun every rank runs an independent replica of the step; the only
collective is the max over ranks of the timed seconds, and the whole-job rate
is world x units / slowest.  The reference arm runs on rank 0 alone.
"""
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r took (r + 1) * 1.5 s for 1000 units
        rate, slowest = bench.replica_throughput((rank + 1) * 1.5, 1000, world)
        out[rank] = (rate, slowest)
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    world = 2
    with mp.get_context("spawn").Manager() as m:   # no fork of this process
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rate, slowest in res.values():
        # every rank sees the slowest rank's time, and the job rate it implies
        assert slowest == 3.0
        assert rate == pytest.approx(1000 * world / 3.0, rel=1e-12)


def test_replica_throughput_single_rank_is_local():
    import bench
    rate, slowest = bench.replica_throughput(2.0, 500, 1)
    assert (rate, slowest) == (250.0, 2.0)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
