"""Table-sharded query on one GPU: two indices over the same groups, each
holding half of the tables (built from column slices of the full index's
buckets). Their partial counts sum to the full index's counts, and
flinng_query_counts on the summed counts returns the full index's query,
bit for bit, also when the total exceeds 255 tables (16-bit decode)."""
import numpy as np
import pytest

from paper_2106_11565_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2106_11565_gb300 import _build, flinng
    _build.build()
    return flinng


def u32(a):
    if hasattr(a, "is_cuda"):
        a = a.cpu().numpy()
    a = np.asarray(a)
    return a.view(np.uint32) if a.dtype == np.int32 else (a.view(np.uint16) if a.dtype == np.int16 else a)


@pytest.mark.parametrize("L,K,W,B,R", [(32, 2, 17, 1000, 2), (300, 1, 12, 250, 3), (64, 1, 3, 60, 4)])
def test_sharded_counts_and_decode_equal_full_index(F, L, K, W, B, R):
    import torch
    from paper_2106_11565_gb300 import sharded
    N, nq = 4000, 80
    g = WL.genomic_reads(90 + L, ref_len=200_000, n_reads=N, read_len=300, n_queries=nq)
    pts, q = (g["off"], g["elems"]), (g["q_off"], g["q_elems"])
    perm = WL.group_permutations(90 + L, R, N)
    full = F.Index("jaccard", R, B, L, K, capacity=N, params=WL.doph_params(90 + L, L, K), W=W)
    full.build(pts, perm)
    bk = full.hash(pts)[0]                      # N x L buckets of every point
    qb = full.hash(q)[0]                        # nq x L
    parts = [sharded.table_range(L, 2, r) for r in range(2)]
    shards = []
    for l0, l1 in parts:
        sh = F.Index("jaccard", R, B, l1 - l0, K, capacity=N, params=WL.doph_params(1, l1 - l0, K), W=W)
        sh.build_buckets(np.ascontiguousarray(bk[:, l0:l1]), perm)
        shards.append(sh)
    want = full.counts(qb).astype(np.int64)
    got = sum(sh.counts(np.ascontiguousarray(qb[:, l0:l1])).astype(np.int64)
              for sh, (l0, l1) in zip(shards, parts))
    assert np.array_equal(got, want)
    ids, sc = full.query_buckets(qb, 50)
    # host buffers
    hid, hsc = shards[0].query_counts(got.astype(np.uint16), 50, L)
    assert np.array_equal(u32(hid), u32(ids)) and np.array_equal(hsc, sc)
    # device buffers, the other shard, ragged k
    k = np.random.default_rng(L).integers(0, 51, size=nq).astype(np.uint32)
    kid, ksc = full.query_buckets(qb, 50, k=k)
    dc = torch.from_numpy(got.astype(np.int16)).cuda()
    did, dsc = shards[1].query_counts(dc, 50, L, k=torch.from_numpy(k.view(np.int32)).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(u32(did), u32(kid)) and np.array_equal(u32(dsc), ksc)
    # the sharded step through the helper (no process group: one rank holds both sums)
    sid, ssc = sharded.sharded_query(shards[0], torch.from_numpy(np.ascontiguousarray(qb[:, parts[0][0]:parts[0][1]])
                                                                 .view(np.int32)).cuda(),
                                     None, L, 50)
    # with one rank the all-reduce is the identity: the decode sees shard 0's counts only
    pid, psc = shards[0].query_counts(shards[0].counts(np.ascontiguousarray(qb[:, parts[0][0]:parts[0][1]])), 50, L)
    assert np.array_equal(u32(sid), u32(pid)) and np.array_equal(u32(ssc), psc)


def test_query_counts_rejects_bad_max_count(F):
    w = WL.srp_projections(5, 4 * 4, 8)
    ix = F.Index("cosine", 1, 4, 4, 4, capacity=16, params=w, dim=8)
    with pytest.raises(F.FlinngError) as e:
        ix.query_counts(np.zeros((1, 4), np.uint16), 4, 0)
    assert e.value.code == F.ERR_INVALID_ARG
    with pytest.raises(F.FlinngError):
        ix.query_counts(np.zeros((1, 4), np.uint16), 4, 5000)
