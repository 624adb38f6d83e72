"""The largest shapes the ABI allows in R and B*R: R = 8 repetitions and
B*R = 65,536 cells (cell ids up to 65,535, the last 16-bit value), through a
build, a touched-slot insert (n*R <= 8,192; 32-bit sort keys at W = 10,
64-bit at W = 17), a full-merge insert, per-cell counts and top-k with 8- and
16-bit counters (L = 4 and L = 300), against the oracle."""
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


def sets_slice(pts, lo, hi):
    off, el = pts
    return (off[lo:hi + 1] - off[lo]).astype(np.uint64), np.ascontiguousarray(el[off[lo]:off[hi]])


@pytest.mark.parametrize("L,K,W", [(4, 2, 10), (4, 2, 17), (300, 1, 6)])
def test_r8_and_65536_cells(F, L, K, W):
    R, B = 8, 8192
    sizes = [12000, 1000, 1500]            # build; 1000 * 8 = 8,000 keys: touched slots; 12,000 keys: full merge
    N = sum(sizes)
    pts = WL.random_sets(60 + W, N, 4000, 10, 120)
    q = WL.random_sets(61 + W, 40, 4000, 10, 120)
    dp = WL.doph_params(62 + W, L, K)
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    o = O.OracleIndex("jaccard", R, B, L, K, W, doph=dp)
    qv = O.doph(q[0], q[1], L * K, dp["doph_a"], dp["doph_b"], dp["doph_seed"])
    qb = O.minhash_buckets(qv, L, K, dp["bucket_a"], dp["bucket_c"], W)
    lo = 0
    for step, n in enumerate(sizes):
        part = sets_slice(pts, lo, lo + n)
        perm = WL.group_permutations(63 + W, R, n, batch=step)
        if step == 0:
            ix.build(part, perm)
            o.build(part, perm)
        else:
            ix.insert(part, perm)
            o.insert(part, perm)
        lo += n
        ex = ix.export()
        assert np.array_equal(ex["gid"], o.gid)
        assert np.array_equal(ex["off"], o.off) and np.array_equal(ex["cells"], o.cells)
        cnt = u32(ix.counts(qb))
        for i in range(0, qb.shape[0], 9):
            assert np.array_equal(cnt[i], O.counts_direct(o.buckets, o.gid, B, qb[i]))
        for mode in (F.QUERY_PLAIN, F.QUERY_FUSED):
            ix.set_query_mode(mode)
            ids, sc = ix.query(q, 40)
            oids, osc = o.query(q, 40)
            assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc), (step, mode)
    assert int(o.cells.max()) >= 60000            # cell ids in the top of the 16-bit range occur
    ix.close()
