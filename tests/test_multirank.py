"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): replicas with no data-path
collective, timings reduced by max over ranks, the whole-job value, and the reference arm printed by
rank 0 alone."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r's step and e2e times; the slowest rank sets each
        step_s, e2e_s = bench.max_over_ranks(dist, [1.0 + rank, 5.0 - rank], "cpu")
        dist.barrier()
        q.put((rank, step_s, e2e_s, bench.whole_job_value(100, world, step_s)))
    finally:
        dist.destroy_process_group()


def test_timings_reduce_by_max_over_two_gloo_ranks():
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
    assert [o[1:] for o in out] == [(2.0, 5.0, 100.0)] * 2  # max of (1, 2) and (5, 4); 2 x 100 / 2


def test_single_rank_passes_timings_through():
    assert bench.max_over_ranks(None, [0.5, 0.7], "cpu") == [0.5, 0.7]
    assert bench.whole_job_value(1000, 1, 0.5) == 2000


class _Args:
    steps, warmup = 1, 0
    workload, lattice, strings = bench.HEADLINE, None, None


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    monkeypatch.setattr(bench, "cpu_oracle_sample", lambda spec, dt, n_images=8: (1.0, 4, 0.25))
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(_Args, rank=1, world=2)
    assert buf.getvalue() == ""
    with redirect_stdout(buf):
        bench.run_reference(_Args, rank=0, world=2)
    line = json.loads(buf.getvalue())
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] == pytest.approx(line["e2e"]["value"])
