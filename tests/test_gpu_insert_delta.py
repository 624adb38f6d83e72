"""Inserts that merge only the slots gaining cells (batches with n * R <=
8192) against the oracle's insert: after every batch of a sequence the
exported CSR, the group ids, per-cell counts (which read the cell bitmaps of
heavy slots) and top-k equal the oracle's. The sequence mixes batch sizes
(one point, a few, hundreds, the largest delta batch) with a batch above the
limit (the full merge), on indices whose lists are mostly light, mostly heavy,
and near the heavy threshold, so that slots become heavy during inserts and
heavy slots gain cells."""
import numpy as np
import pytest

from oracle import oracle as O
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
    return np.asarray(a).view(np.uint32) if a.dtype == np.int32 else np.asarray(a)


def check(ix, o, q, qb, k=15):
    ex = ix.export()
    assert np.array_equal(ex["gid"], o.gid)
    assert np.array_equal(ex["off"], o.off)
    assert np.array_equal(ex["cells"], o.cells)
    cnt = u32(ix.counts(qb))
    for i in range(0, qb.shape[0], 7):
        assert np.array_equal(cnt[i], O.counts_direct(o.buckets, o.gid, o.B, qb[i]))
    ids, sc = ix.query(q, k)
    oids, osc = o.query(q, k)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)


def sets_slice(pts, lo, hi):
    off, el = pts
    return (off[lo:hi + 1] - off[lo]).astype(np.uint64), np.ascontiguousarray(el[off[lo]:off[hi]])


# W = 4: every list heavy; W = 7: lists near the threshold max(B R / 16, 32)
@pytest.mark.parametrize("W", [4, 7, 14])
def test_jaccard_insert_sequence(F, W):
    R, B, L, K = 2, 300, 12, 2
    sizes = [1500, 1, 7, 300, 1500, 4096, 5000, 250]    # build, then inserts (5000 * R > 8192: full merge)
    N = sum(sizes)
    pts = WL.random_sets(70 + W, N, 5000, 20, 200)
    q = WL.random_sets(71 + W, 60, 5000, 20, 200)
    dp = WL.doph_params(72 + W, L, K)
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    o = O.OracleIndex("jaccard", R, B, L, K, W, doph=dp)
    qv = O.doph(q[0], q[1], L * K, dp["doph_a"], dp["doph_b"], dp["doph_seed"])
    qb = O.minhash_buckets(qv, L, K, dp["bucket_a"], dp["bucket_c"], W)
    lo = 0
    heavy_seen = []
    for step, n in enumerate(sizes):
        part = sets_slice(pts, lo, lo + n)
        perm = WL.group_permutations(73 + W, R, n, batch=step)
        if step == 0:
            ix.build(part, perm)
            o.build(part, perm)
        else:
            ix.insert(part, perm)
            o.insert(part, perm)
        lo += n
        check(ix, o, q, qb)
        lens = np.diff(o.off.astype(np.int64))
        heavy_seen.append(int((lens >= max(B * R // 16, 32)).sum()))
    if W == 4:
        assert heavy_seen[0] > 0
    if W == 7:
        assert heavy_seen[-1] > heavy_seen[0] > 0       # slots became heavy during the inserts
    ix.close()


def test_wide_keys(F):
    """W + log2(B R) > 31: the batch's keys are sorted as 64-bit words."""
    R, B, L, K, W = 2, 4096, 4, 2, 22
    sizes = [3000, 5, 1200]
    N = sum(sizes)
    pts = WL.random_sets(95, N, 5000, 20, 200)
    q = WL.random_sets(96, 40, 5000, 20, 200)
    dp = WL.doph_params(97, L, K)
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    o = O.OracleIndex("jaccard", R, B, L, K, W, doph=dp)
    qv = O.doph(q[0], q[1], L * K, dp["doph_a"], dp["doph_b"], dp["doph_seed"])
    qb = O.minhash_buckets(qv, L, K, dp["bucket_a"], dp["bucket_c"], W)
    lo = 0
    for step, n in enumerate(sizes):
        part = sets_slice(pts, lo, lo + n)
        perm = WL.group_permutations(98, R, n, batch=step)
        if step == 0:
            ix.build(part, perm)
            o.build(part, perm)
        else:
            ix.insert(part, perm)
            o.insert(part, perm)
        lo += n
        check(ix, o, q, qb)
    ix.close()


def test_cosine_insert_sequence_and_host_buffers(F):
    import torch
    N0, d, R, B, L, K = 2000, 32, 4, 150, 9, 6
    sizes = [N0, 3, 500, 2048, 2100]                   # 2048 * 4 = 8192: the largest delta batch
    N = sum(sizes)
    pts, _ = WL.gaussian_mixture(80, N, d, 30, 0.1)
    q, _ = WL.noisy_queries(80, pts, 50, 0.05)
    w = WL.srp_projections(80, L * K, d)
    ix = F.Index("cosine", R, B, L, K, capacity=N, params=w, dim=d)
    o = O.OracleIndex("cosine", R, B, L, K, K, srp_w=w)
    qb = O.srp_codes(q, w, L, K)
    lo = 0
    for step, n in enumerate(sizes):
        perm = WL.group_permutations(81, R, n, batch=step)
        part = pts[lo:lo + n]
        if step == 0:
            ix.build(part, perm)
            o.build(part, perm)
        elif step % 2:
            ix.insert(torch.from_numpy(part).cuda(), torch.from_numpy(perm.view(np.int32)).cuda())
            o.insert(part, perm)
        else:
            ix.insert(part, perm)
            o.insert(part, perm)
        lo += n
        check(ix, o, q, qb)
    ix.close()


def test_insert_of_points_already_present(F):
    """A batch that repeats indexed points adds their cells where the lists
    lack them (their groups are new), and nothing else."""
    R, B, L, K, W = 3, 50, 8, 1, 10
    pts = WL.random_sets(90, 400, 3000, 20, 100)
    dp = WL.doph_params(91, L, K)
    ix = F.Index("jaccard", R, B, L, K, capacity=800, params=dp, W=W)
    o = O.OracleIndex("jaccard", R, B, L, K, W, doph=dp)
    p0 = WL.group_permutations(92, R, 400)
    ix.build(pts, p0)
    o.build(pts, p0)
    again = sets_slice(pts, 100, 300)
    p1 = WL.group_permutations(92, R, 200, batch=1)
    ix.insert(again, p1)
    o.insert(again, p1)
    q = sets_slice(pts, 0, 40)
    qv = O.doph(q[0], q[1], L * K, dp["doph_a"], dp["doph_b"], dp["doph_seed"])
    qb = O.minhash_buckets(qv, L, K, dp["bucket_a"], dp["bucket_c"], W)
    check(ix, o, q, qb)
    ix.close()
