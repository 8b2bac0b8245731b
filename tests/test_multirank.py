"""The N > 1 logic of bench.py on CPU: two gloo ranks get disjoint scan ids
(independent scans, weak scaling) and the job time / work reduce to the
maximum time and the summed work.  No GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    warm, steps = bench.shard_scan_ids(rank, steps=5, warmup=2)
    ms, units = bench.reduce_timing(10.0 * (rank + 1), 100.0 + rank, world)
    out.put((rank, warm, steps, ms, units))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ids = [set(r[1]) | set(r[2]) for r in res]
    assert not (ids[0] & ids[1])                     # no scan id traced twice
    assert all(len(r[2]) == 5 and len(r[1]) == 2 for r in res)
    for r in res:
        assert r[3] == pytest.approx(20.0)           # max over ranks
        assert r[4] == pytest.approx(201.0)          # sum over ranks
