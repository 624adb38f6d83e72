"""Table-sharded FLINNG query, for an index larger than one GPU.

Every rank holds the same groups (the same points and group permutations)
but a disjoint, contiguous range of the L hash tables. A cell's count is the
number of tables whose bucket list holds it (Sec. 5), so it is the sum of the
ranks' partial counts: one sum all-reduce of the B*R count vector per query
gives the whole index's counts, and any rank can then run Alg. 3's decode on
them (flinng_query_counts). Sharding by points instead would change the
cells, and with them the method's results.
"""
from __future__ import annotations


def table_range(L: int, world: int, rank: int) -> tuple[int, int]:
    """Tables [l0, l1) of this rank: contiguous ranges whose sizes differ by
    at most one."""
    if not (0 <= rank < world) or L < world:
        raise ValueError("need 0 <= rank < world <= L")
    base, extra = divmod(L, world)
    l0 = rank * base + min(rank, extra)
    return l0, l0 + base + (1 if rank < extra else 0)


def allreduce_counts(counts, dist):
    """Sum of every rank's partial counts (returned on every rank). Summed in
    int32, returned as int16 holding the uint16 counts (totals stay <= 4095)."""
    import torch
    t = counts.to(torch.int32)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.to(torch.int16)


def sharded_query(shard, qb_shard, dist, max_count: int, k_max: int, k=None):
    """One query batch on this rank. shard: this rank's index (an
    ``flinng.Index`` built over its tables); qb_shard: the batch's buckets of
    those tables (nq x (l1 - l0), on the device); max_count: the total number
    of tables. Returns (ids, scores), identical on every rank."""
    partial = shard.counts(qb_shard)
    return shard.query_counts(allreduce_counts(partial, dist), k_max, max_count, k=k)
