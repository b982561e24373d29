"""The multi-rank host logic of bench.py (replicas, one system per rank, no data-path
collective) with world size 2 on the gloo backend, on the CPU: rank setup, the barrier,
the max-over-ranks time, the whole-job throughput, and the reference arm that only
rank 0 runs."""
import io
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


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist
    r, w, loc = bench.dist_setup(world, backend="gloo")
    assert (r, w, loc) == (rank, world, rank)
    bench.barrier(w)
    ms = 100.0 + 50.0 * rank                      # the slower rank decides the job's time
    ms_max = bench.max_over_ranks(w, ms)
    value = bench.job_throughput(3000, w, ms_max)
    # the reference arm: rank 0 alone runs it; the others return at once, printing nothing
    buf = io.StringIO()
    rc = None
    if rank != 0:
        class A:   # arguments are never read on a non-zero rank
            pass
        with redirect_stdout(buf):
            rc = bench.run_reference(A())
    out[rank] = (ms_max, value, rc, buf.getvalue())
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    assert res[0][1] == res[1][1] == pytest.approx(2 * 3000 / 0.150)
    assert res[1][2] == 0 and res[1][3] == ""


def test_world_size_must_match_gpus(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "0")
    with pytest.raises(SystemExit):
        bench.dist_setup(1, backend="gloo")


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1, 12.5) == 12.5
    assert bench.job_throughput(1000, 1, 500.0) == pytest.approx(2000.0)
