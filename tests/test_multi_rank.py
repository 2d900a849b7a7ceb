"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

The scheme shards by independent problems (weak scaling): every rank advances
its own seeded instance, and the only collectives are the barrier and the
max-over-ranks of the elapsed time.  These tests run that logic as two gloo
processes, with no GPU.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=ws)
    try:
        w, r, lr = bench.dist_env()
        assert (w, r, lr) == (ws, rank, rank)
        ms_local = 10.0 + 5.0 * rank           # rank 1 is the slow one
        dist.barrier()
        ms = bench.max_over_ranks(ms_local, torch.device("cpu"), ws)
        value = bench.job_value(1000, 4, ws, ms)
        P, U0 = bench.rank_problem(rank)
        out.put((rank, ms, value, float(P.V.sum()), float(U0[0, 0])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_and_sum_the_work():
    ws, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, V0, u0), (r1, ms1, v1, V1, u1) = res
    assert ms0 == ms1 == 15.0                               # max over ranks
    assert v0 == v1 == pytest.approx(1000 * 4 * 2 / 15e-3)  # whole-job units / job time
    assert V0 != V1 and u0 != u1                            # independent seeded instances


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"steps": 1, "warmup": 3, "gpus": 2})()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_single_rank_defaults():
    assert bench.max_over_ranks(7.5, None, 1) == 7.5
    assert bench.job_value(10, 3, 1, 1000.0) == pytest.approx(30.0)
    P0, _ = bench.rank_problem(0)
    assert P0.n == 64 ** 3 and P0.p == 128 and np.isfinite(P0.V).all()
