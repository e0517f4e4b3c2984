"""The benchmark's multi-process host logic on CPU (gloo, world size 2): every rank runs an
independent replica, the job's time is the slowest rank's, its rate the units of all ranks
over that time; the reference arm prints from rank 0 only."""
import io
import os
import socket
import contextlib

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, local, w = bench.env_rank()
    ms = 10.0 + 20.0 * rank                       # rank 1 is the slow one
    m = bench.max_over_ranks(ms, w, torch.device("cpu"))
    out[rank] = (r, local, w, m, bench.whole_job_rate(1000, w, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    # spawn, not fork: in a full test run CUDA is already initialised in this process
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        r, local, w, m, rate = res[rank]
        assert (r, local, w) == (rank, rank, 2)
        assert m == 30.0
        assert rate == pytest.approx(2 * 1000 / 0.030)


def test_single_process_defaults():
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        os.environ.pop(k, None)
    assert bench.env_rank() == (0, 0, 1)
    assert bench.max_over_ranks(5.0, 1, None) == 5.0


def test_reference_arm_prints_only_on_rank_0(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    import argparse
    a = argparse.Namespace(gpus=2, steps=1, warmup=0, tol=1e-11)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(a)
    assert buf.getvalue() == ""
