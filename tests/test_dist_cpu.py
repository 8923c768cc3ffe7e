"""The multi-GPU plumbing (cell sharding, max-over-ranks timing) on CPU with
the gloo backend, world size 2 (no GPU, no collective on the data path)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_2103_14890_gb300 import dist as bzdist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bzdist.rank_env()
        b, e = bzdist.shard(1001, r, w)
        t = bzdist.max_over_ranks(1.5 + r)          # per-rank "step time"
        dist.barrier()
        q.put((r, w, lr, b, e, t))
    finally:
        dist.destroy_process_group()


def test_shard_covers_all_cells():
    from paper_2103_14890_gb300 import dist as bzdist
    for n in (0, 1, 7, 65536, 100003):
        for world in (1, 2, 3, 8):
            ranges = [bzdist.shard(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        bzdist.shard(10, 2, 2)


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, b0, e0, t0), (r1, w1, l1, b1, e1, t1) = out
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert (b0, e0, b1, e1) == (0, 501, 501, 1001)
    assert t0 == t1 == 2.5                           # max over the two ranks
