"""The multi-rank path of bench.py on CPU: world_size-2 gloo ranks, each with
its own elapsed time and units; the whole-job rate sums the units and divides
by the slowest rank's time (replicas, no data-path collective)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench._dist() == (ws, rank, rank)
        ms = [250.0, 400.0][rank]          # rank 1 is the slow one
        units = [100.0, 300.0][rank]
        rate, ms_max = bench._job_rate(units, ms, ws, torch.device("cpu"))
        out.put((rank, rate, ms_max))
    finally:
        dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, rate, ms_max in res:
        assert ms_max == 400.0
        assert rate == pytest.approx(400.0 / 0.4)   # (100 + 300) units over the slowest rank's 0.4 s


def test_job_rate_single_rank():
    import bench
    rate, ms_max = bench._job_rate(500.0, 250.0, 1, torch.device("cpu"))
    assert ms_max == 250.0 and rate == pytest.approx(2000.0)
