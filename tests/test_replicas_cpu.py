"""The replica path of bench.py on CPU: two gloo ranks (one process each) agree
on the job's time (the slowest rank's) and on the whole-job throughput.  The
GPU runs the same code with NCCL, one lattice per rank and no data-path
collective."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local_ms = 100.0 + 25.0 * rank  # rank 1 is the slow one
    total = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (total, bench.job_mlups(1000, 10, ws, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_job_throughput():
    ws = 2
    # spawn, not fork: earlier tests in this process may have started OpenMP
    # threads (the oracle), and a fork of a threaded process can deadlock
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0] == res[1]
    total, mlups = res[0]
    assert total == 125.0
    assert mlups == pytest.approx(ws * 1000 * 10 / 0.125 / 1e6)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_mlups(2_097_152, 8, 1, 1.0) == pytest.approx(2_097_152 * 8 / 1e-3 / 1e6)
