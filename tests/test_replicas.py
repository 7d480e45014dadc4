"""Two-rank gloo test (CPU) of the replica timing bookkeeping used by
bench.py --gpus N: max over ranks of the time, sum of the interactions."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1812_00367_gb300.replicas import combine_timing
    ms, inter = combine_timing(100.0 + 50.0 * rank, 1e9 * (rank + 1))
    q.put((rank, ms, inter))
    dist.destroy_process_group()


def test_combine_timing_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, inter in res:
        assert ms == 150.0 and inter == 3e9


def test_combine_timing_single_process_is_identity():
    from paper_1812_00367_gb300.replicas import combine_timing
    assert combine_timing(12.5, 7.0) == (12.5, 7.0)
