"""The multi-process path on CPU: world_size-2 gloo process groups. Each rank
counts the matches whose first attribute lies in its own range (here with
the CPU oracle; on GPUs each rank runs the library on its replica), the
ranks exchange one (count, checksum) sum per query, and the result equals
the unsharded count. Also the max-over-ranks step-time reduction."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1802_03760_b300.shard import shard_range

M64 = (1 << 64) - 1


def test_shard_ranges_partition():
    for n in (1, 7, 1000, 1 << 20):
        for world in range(1, 9):
            rs = [shard_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(h - l for l, h in rs) - min(h - l for l, h in rs) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import oracle
    from paper_1802_03760_b300.inputs import QUERIES, er_edges
    from paper_1802_03760_b300.shard import max_over_ranks, reduce_counts, shard_range

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s, d = er_edges(400, 6000, seed=5)
    og = oracle.Graph(400, s, d)
    names = ["triangle", "diamond", "4-cycle"]
    lo, hi = shard_range(400, rank, world)
    mine = [og.count(oracle.Query(*QUERIES[nm]), first_range=(lo, hi)) for nm in names]
    c, h = reduce_counts([x[0] for x in mine], [x[1] for x in mine])
    t = max_over_ranks(10.0 * (rank + 1))
    if rank == 0:
        full = [og.count(oracle.Query(*QUERIES[nm])) for nm in names]
        out.put((list(zip(c, h)), full, t))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_rank_sharded_count_equals_full_count():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, full, tmax = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == full
    assert tmax == 20.0
