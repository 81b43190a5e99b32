"""The N > 1 path of the benchmark (replicas only: every rank advances its own
replica, no data-path collective) exercised with two gloo ranks on the CPU:
the max-over-ranks timing rule, the aggregate throughput, distinct per-rank
seeds, and that only rank 0 of the reference arm prints."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    import lbm_inputs
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    t_local = [0.8, 1.3][rank]
    t_max = bench.reduce_max(t_local, dist, "cpu")
    value = bench.aggregate_mlups(1000, 50, world, t_max)
    f = lbm_inputs.fields_box2d(16, 8, seed=bench.replica_seed(2, rank))
    q.put((rank, t_max, value, float(f["u_g"].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_timing_and_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [1.3, 1.3]
    assert res[0][2] == pytest.approx(2 * 1000 * 50 / 1.3 / 1e6)
    assert res[0][3] != res[1][3]  # different replica seeds


def test_reference_arm_prints_on_rank0_only(tmp_path):
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
