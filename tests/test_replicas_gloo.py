"""The multi-rank path of bench.py (independent replicas, one per GPU) on CPU ranks with gloo:
the slowest rank's times set the whole-job numbers, on every rank alike."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = 10.0 + 5.0 * rank                 # rank 1 is slower on the device
    e2e = 2.0 - 0.5 * rank                 # rank 0 is slower end to end
    res = bench.aggregate_replicas(ms, e2e, ws, cells=1000, steps=4, device="cpu")
    out[rank] = torch.tensor(res, dtype=torch.float64)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(ws):
        ms_max, e2e_max, value, e2e_value = out[r].tolist()
        assert ms_max == 15.0 and e2e_max == 2.0
        assert value == pytest.approx(ws * 1000 * 4 / 15e-3)
        assert e2e_value == pytest.approx(ws * 1000 * 4 / 2.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert not dist.is_initialized()
    ms_max, e2e_max, value, e2e_value = bench.aggregate_replicas(8.0, 1.0, 1, 1000, 4, "cpu")
    assert (ms_max, e2e_max) == (8.0, 1.0) and value == pytest.approx(1000 * 4 / 8e-3)
