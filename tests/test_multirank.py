"""The N > 1 host logic of bench.py on CPU: two gloo ranks (the GPU job launches one
process per GPU and reduces over NCCL in the same way).  Each rank runs its own copy of
the workload, so the job's time is the slowest rank's and its throughput counts every
rank's rows; the reference arm runs on rank 0 only."""
import importlib.util
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        b = _bench()
        slowest = b.max_over_ranks(times[rank], world, torch.device("cpu"))
        dist.barrier()
        out.put((rank, slowest, b.job_rows_per_s(world, 1000, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank_and_count_all_rows():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    times = [0.25, 0.5]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rows_per_s in got:
        assert slowest == 0.5
        assert rows_per_s == pytest.approx(2 * 1000 / 0.5)


def _shard_rank(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2511_09376_gb300 import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        b = _bench()
        ens, _, B = synth.make("tiny")
        lo, hi = b.shard_rows(B.shape[0], rank, world)
        counts = torch.from_numpy(oracle.bg_hist(ens, B[lo:hi]).astype(np.int64))
        dist.all_reduce(counts)  # the one exchange of the sharded background
        out.put((rank, lo, hi, bool(np.array_equal(counts.numpy(), oracle.bg_hist(ens, B).astype(np.int64)))))
    finally:
        dist.destroy_process_group()


def test_sharded_background_counts_sum_to_the_whole():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(lo, hi) for _, lo, hi, _ in got] == [(0, 100), (100, 200)]
    assert all(ok for *_, ok in got)


def test_single_rank_needs_no_process_group():
    b = _bench()
    assert b.max_over_ranks(0.125, 1, None) == 0.125
    assert b.job_rows_per_s(1, 3000, 0.5) == 6000


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    b = _bench()
    called = []
    monkeypatch.setattr(b, "run_reference", lambda *a, **k: called.append(a) or {"impl": "reference"})
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        b.main()
    assert called == [] and buf.getvalue() == ""
    monkeypatch.setenv("RANK", "0")
    with redirect_stdout(buf):
        b.main()
    assert len(called) == 1 and '"impl": "reference"' in buf.getvalue()
