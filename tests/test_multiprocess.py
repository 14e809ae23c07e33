"""The N > 1 path of bench.py on CPU: replicas only, timing aggregated as the
maximum over ranks (two gloo ranks on 127.0.0.1)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.aggregate_ms(10.0 + 5.0 * rank, dist)
    w, r, _ = bench.dist_env()
    out[rank] = ms
    dist.barrier()
    dist.destroy_process_group()


def test_step_time_is_max_over_two_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == 15.0 and out[1] == 15.0


def test_single_process_passthrough():
    import bench
    assert bench.aggregate_ms(3.5, None) == 3.5
