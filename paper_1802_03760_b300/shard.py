"""Host-side splitting of a count over several GPUs (one process per GPU).

A static count is additive over disjoint ranges of the first attribute's
value (each match has exactly one first value), so every rank can count the
matches whose first attribute lies in its own contiguous range, on its own
replica of the indices (every worker holds the whole graph, Section 4.2),
and the only exchange is one sum of (count, checksum) per query at the end.
"""
from __future__ import annotations

M64 = (1 << 64) - 1


def shard_range(n: int, rank: int, world: int):
    """Contiguous first-attribute range [lo, hi) of rank among world ranks over [0, n)."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def reduce_counts(counts, checksums):
    """Sums per-query counts and checksums (mod 2^64) over all ranks of the
    default process group; returns python ints on every rank."""
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    c = torch.tensor([int(x) for x in counts], dtype=torch.int64, device=dev)
    # checksums travel as their two's-complement int64 bit patterns; the sum wraps mod 2^64
    h = torch.tensor([int(x) - (1 << 64) if int(x) >= (1 << 63) else int(x) for x in checksums],
                     dtype=torch.int64, device=dev)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    dist.all_reduce(h, op=dist.ReduceOp.SUM)
    return [int(x) for x in c.tolist()], [int(x) & M64 for x in h.tolist()]


def max_over_ranks(value: float) -> float:
    """The maximum of a per-rank float (step times) over the default process group."""
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
