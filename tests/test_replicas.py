"""The N > 1 path of bench.py on CPU: replicas (one independent lattice per rank) share
only the timing barrier and the maximum of the timings, and the job's value is the
updates of all ranks over the slowest rank's time.  Two gloo ranks stand in for the GPUs;
the reference arm runs on rank 0 alone."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    w, r, local = bench.dist_env()
    dist = bench.init_replicas(w, "gloo")
    dist.barrier()
    t = bench.max_over_ranks(10.0 + 5.0 * r, dist)  # the slower rank takes 15 ms
    out.put((r, w, local, t, bench.whole_job_mlups(w, 4096 * 4096, 100, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

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
    assert [x[:3] for x in res] == [(0, 2, 0), (1, 2, 1)]
    assert all(x[3] == 15.0 for x in res)
    # 2 ranks x 4096^2 cells x 100 steps in 15 ms
    assert res[0][4] == pytest.approx(2 * 4096 * 4096 * 100 / 15e-3 / 1e6)


def test_single_process_needs_no_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    sys.path.insert(0, ROOT)
    import bench

    assert bench.dist_env() == (1, 0, 0)
    assert bench.init_replicas(1) is None
    assert bench.max_over_ranks(3.5, None) == 3.5


def _args(**kw):
    import argparse

    a = argparse.Namespace(gpus=2, steps=1, warmup=0, impl="reference")
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(_args()) == 0
    assert buf.getvalue() == ""
    monkeypatch.setenv("RANK", "0")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(_args()) == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "MLUPS"
    import oracle

    assert line["e2e"]["h2d_bytes_per_step"] == 0
    # the oracle runs its row sweeps on every host core (one thread without OpenMP)
    want = oracle.host_cores() if oracle.lib().orc_have_openmp() else 1
    assert line["cpu_baseline"]["cores"] == want
    assert oracle.get_threads() == 1  # and leaves the serial default in force
