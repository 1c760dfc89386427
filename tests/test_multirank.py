"""The benchmark's cross-rank steps on CPU ranks (gloo, world size 2).

The hot path shards into independent replicas, one per GPU; the only
cross-rank operations are a barrier and a MAX all-reduce of the step time.
"""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [2.5, 4.0][rank]
        dist.barrier()
        q.put((rank, bench.max_over_ranks(ms), bench.max_over_ranks(-ms)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 4.0, -2.5), (1, 4.0, -2.5)]


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
