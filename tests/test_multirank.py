"""The multi-GPU path of bench.py is replicas: every rank runs the whole
workload on its own GPU with no collective in the data path, timings are
the slowest rank's (a MAX all-reduce), and the job's value is N times the
work over that time.  Checked here with two gloo ranks on the CPU; the
reference arm runs on rank 0 only."""
from __future__ import annotations

import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        r, w, _ = bench.dist_env()
        mine = [3.0, 7.5][rank]              # this rank's step time, seconds
        slowest = bench.max_over_ranks(mine, w, device="cpu")
        out.put((r, w, slowest, bench.whole_job_value(w, 2.0e9, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_scale_the_work():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for _, world, slowest, value in got:
        assert world == 2 and slowest == 7.5
        assert value == pytest.approx(2 * 2.0e9 / 7.5 / 1e9)


def test_one_rank_needs_no_process_group():
    bench = _bench()
    assert bench.max_over_ranks(4.25, 1) == 4.25
    assert bench.whole_job_value(1, 3.0e9, 1.5) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    bench = _bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("Args", (), {"matrices": "stencil27", "steps": 1, "warmup": 0, "scale": "full",
                             "betas": "4x8"})()
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
