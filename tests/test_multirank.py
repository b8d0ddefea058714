"""Multi-process host logic of the benchmark on the CPU (gloo, two ranks).

Instances are independent, so ranks run replicas with no collective on the
data path; the only exchange is the timing reduction (slowest rank) behind
the whole-job value.  Under torchrun the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    m = bench.max_over_ranks(10.0 + 3.0 * rank)
    v = bench.weak_scaling_value(world, 50000, 100, m)
    q.put((rank, m, v, bench.rank_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_to_the_slowest():
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
    assert [o[1] for o in out] == [13.0, 13.0]          # both see the slowest rank
    assert out[0][2] == out[1][2] == pytest.approx(2 * 50000 * 100 / 13e-3)
    assert out[0][3] != out[1][3]                        # independent replicas


def test_single_process_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.5) == 4.5
    assert bench.weak_scaling_value(1, 1000, 10, 2.0) == pytest.approx(5e6)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
