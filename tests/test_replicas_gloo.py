"""The N > 1 path of bench.py on CPU: two ranks over gloo.

The solver does not shard across GPUs, so N ranks run independent
replicas.  What crosses ranks is bookkeeping only: the barriers around the
timed region, the maximum of the ranks' times, and the whole-job rate (all
ranks' point-steps over the slowest rank's time).  The reference arm runs
on rank 0 alone; the other ranks return without work.
"""
import json
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


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    T = bench.Timer(torch, dist, world, None, device="cpu")
    T.barrier()
    local_ms = 100.0 + 25.0 * rank          # rank 1 is the slower replica
    t_max = T.max(local_ms)
    T.barrier()
    rate = bench.whole_job_rate(1000, 4, world, t_max)
    # the reference arm: rank 0 alone does work; here only rank 1 calls it,
    # which must return at once without touching the oracle
    ref = None
    if rank != 0:
        ref = bench.reference_arm(None)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"t_max": t_max, "rate": rate, "ref": ref, "oracle_loaded": "oracle.oracle" in sys.modules}, f)


def test_two_replicas_take_the_slowest_time_and_sum_the_work(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(os.path.join(str(tmp_path), "rank%d.json" % r))) for r in range(world)]
    for r in res:
        assert r["t_max"] == 125.0                           # max over ranks, seen by every rank
        assert r["rate"] == pytest.approx(1000 * 4 * 2 / 0.125)  # all ranks' work / slowest time
    assert res[1]["ref"] is None and not res[1]["oracle_loaded"]
