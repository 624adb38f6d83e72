"""Table sharding with a sum all-reduce of per-cell counts, on two gloo
processes (CPU): the ranks' partial counts (the oracle's reverse-index walk
over each rank's tables) summed by the collective, then decoded (the oracle's
Alg. 3), equal the whole index's query."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, L, R, B, W, NQ, K = 600, 24, 3, 40, 4, 20, 15


def _data():
    rng = np.random.default_rng(42)
    buckets = rng.integers(0, 1 << W, size=(N, L)).astype(np.uint32)
    qb = rng.integers(0, 1 << W, size=(NQ, L)).astype(np.uint32)
    qb[:5] = buckets[:5]                                # some queries equal indexed points
    return buckets, qb


class _OracleShard:
    """The oracle over one rank's tables, with the two calls sharded_query uses."""

    def __init__(self, buckets, gid, l0, l1):
        from oracle import oracle as O
        self.O = O
        self.off, self.cells = O.build_csr(buckets[:, l0:l1], gid, B, W)
        self.moff, self.mem = O.members(gid, B)
        self.nl = l1 - l0

    def counts(self, qb):
        import torch
        c = np.stack([self.O.counts(self.off, self.cells, self.nl, W, row, B * R) for row in qb])
        return torch.from_numpy(c.astype(np.int32))

    def query_counts(self, counts, k_max, max_count, k=None):
        c = counts.numpy().astype(np.uint16)
        out = [self.O.alg3(np.minimum(row, max_count), self.moff, self.mem, N, R, B, k_max) for row in c]
        return np.stack([o[0] for o in out]), np.stack([o[1] for o in out])


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2106_11565_gb300 import sharded, workloads as WL
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    buckets, qb = _data()
    gid = O.groups(WL.group_permutations(7, R, N), B)
    l0, l1 = sharded.table_range(L, world, rank)
    shard = _OracleShard(buckets, gid, l0, l1)
    ids, sc = sharded.sharded_query(shard, qb[:, l0:l1], dist, L, K)
    out.put((rank, ids, sc))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_table_range_partitions_the_tables():
    sys.path.insert(0, ROOT)
    from paper_2106_11565_gb300 import sharded
    for L_, w in ((24, 2), (25, 4), (7, 7), (4095, 8)):
        rs = [sharded.table_range(L_, w, r) for r in range(w)]
        assert rs[0][0] == 0 and rs[-1][1] == L_
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        sizes = [b - a for a, b in rs]
        assert max(sizes) - min(sizes) <= 1


def test_sharded_counts_allreduce_equals_whole_index_gloo():
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2106_11565_gb300 import workloads as WL
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(world)), key=lambda t: t[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    buckets, qb = _data()
    gid = O.groups(WL.group_permutations(7, R, N), B)
    o = O.OracleIndex("jaccard", R, B, L, 1, W)
    o.N, o.buckets, o.gid = N, buckets, gid
    o.off, o.cells = O.build_csr(buckets, gid, B, W)
    o.moff, o.mem = O.members(gid, B)
    ids, sc = o.query_buckets(qb, K)
    for _, rids, rsc in res:
        assert np.array_equal(rids, ids) and np.array_equal(rsc, sc)
