"""bench.py's multi-rank path on the CPU: two gloo ranks, as torchrun launches them.

The benchmark runs independent replicas (each rank solves its own seeded copy
of the workload; nothing is exchanged on the data path), so what the ranks share
is host logic: distinct seeds per rank, the timed interval taken as the maximum
over ranks, the whole-job rate from it, and the reference arm running on rank 0
only.  These are checked here with world size 2 over gloo on 127.0.0.1.
"""
import os
import socket
import types

import pytest

import bench
from paper_2006_14952_gb300 import workloads as W


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        wsz, rk, _ = bench.dist_env()
        local_seconds = [3.0, 5.0][rank]
        slowest = bench.max_over_ranks(local_seconds)
        cfg = bench.replica_config(W.CONFIGS["uniform-32k"], rk, wsz)
        seeds = [None] * ws
        dist.all_gather_object(seeds, cfg.seed)
        out[rank] = (slowest, tuple(seeds), bench.whole_job_rate(wsz, cfg.n, 4, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time_and_solve_distinct_replicas():
    import torch.multiprocessing as mp

    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 5.0  # every rank reports the slowest rank's time
    assert res[0][1] == res[1][1] and res[0][1][0] != res[0][1][1]  # one seed per rank
    n = W.CONFIGS["uniform-32k"].n
    assert res[0][2] == res[1][2] == pytest.approx(2 * n * 4 / 5.0)  # both ranks' units / slowest time


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(2.5) == 2.5
    cfg = W.CONFIGS["uniform-32k"]
    assert bench.replica_config(cfg, 0, 1) is cfg
    assert bench.whole_job_rate(1, 1000, 5, 0.5) == 10000


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = types.SimpleNamespace(steps=1, warmup=0)
    assert bench.run_reference(args, W.CONFIGS["uniform-32k"]) is None
    assert capsys.readouterr().out == ""
