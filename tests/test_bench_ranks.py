"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas) report
the slowest rank's time and the summed work, as the driver's N-GPU runs do
over NCCL."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
    res = bench.aggregate_ranks(ms, 2 * ms, 1e9 * (rank + 1), 2e9 * (rank + 1), device="cpu")
    out[rank] = res
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_sum_work():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms, e2e_ms, work, e2e_work = out[r]
        assert ms == 150.0 and e2e_ms == 300.0
        assert work == 3e9 and e2e_work == 6e9


def test_single_process_is_identity():
    import bench
    assert bench.aggregate_ranks(1.0, 2.0, 3.0, 4.0) == (1.0, 2.0, 3.0, 4.0)
