"""Parity at the full workload sizes, in the launch form the bench times
(fused kernel through a CUDA graph, autotuned).

Genomic reads (100,000 reads, 1,000 queries): everything against the oracle.
URL strings (1,000,000 sets, 10,000 queries): the buckets of every point, the
group ids, and the counts and top-k of a sample of queries, which the oracle
computes one by one from the definition (no reverse index).
"""
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


def test_genomic_reads_full_size(F):
    seed = WL.config_seed(2)
    N, nq, R, B, L, K, W, k = 100_000, 1000, 2, 1000, 32, 2, 17, 100
    g = WL.genomic_reads(seed, 5_000_000, N, 1000, nq)
    pts, q = (g["off"], g["elems"]), (g["q_off"], g["q_elems"])
    dp = WL.doph_params(seed, L, K)
    perm = WL.group_permutations(seed, R, N)
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    ix.build(pts, perm)
    ix.tune(q, k)
    ix.set_query_mode(F.QUERY_GRAPH)
    ids, sc = ix.query(q, k)
    o = O.OracleIndex("jaccard", R, B, L, K, W, doph=dp)
    o.build(pts, perm)
    ex = ix.export()
    assert np.array_equal(ex["gid"], o.gid)
    assert np.array_equal(ex["off"], o.off) and np.array_equal(ex["cells"], o.cells)
    oids, osc = o.query(q, k)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)


def test_url_strings_full_size_sampled(F):
    seed = WL.config_seed(3)
    N, nq, R, B, L, K, W, k = 1_000_000, 10_000, 4, 5000, 64, 1, 17, 10
    g = WL.url_strings(seed, N, nq)
    pts, q = (g["off"], g["elems"]), (g["q_off"], g["q_elems"])
    dp = WL.doph_params(seed, L, K)
    perm = WL.group_permutations(seed, R, N)
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    ix.build(pts, perm)
    # buckets of every indexed point
    gb, _, _ = ix.hash(pts)
    v = O.doph(pts[0], pts[1], L * K, dp["doph_a"], dp["doph_b"], dp["doph_seed"])
    ob = O.minhash_buckets(v, L, K, dp["bucket_a"], dp["bucket_c"], W)
    del v
    assert np.array_equal(u32(gb), ob)
    # group ids
    ogid = O.groups(perm, B)
    assert np.array_equal(ix.export()["gid"], ogid)
    # all queries in the bench's form, a sample checked one by one
    ix.tune(q, k)
    ix.set_query_mode(F.QUERY_GRAPH)
    ids, sc = ix.query(q, k)
    qv = O.doph(q[0], q[1], L * K, dp["doph_a"], dp["doph_b"], dp["doph_seed"])
    qb = O.minhash_buckets(qv, L, K, dp["bucket_a"], dp["bucket_c"], W)
    moff, mem = O.members(ogid, B)
    rng = np.random.default_rng(5)
    sample = np.concatenate([[0, nq - 1], rng.choice(nq, 18, replace=False)])
    gcnt = ix.counts(np.ascontiguousarray(qb[sample]))
    for r, i in enumerate(sample):
        cnt = O.counts_direct(ob, ogid, B, qb[i])
        assert np.array_equal(gcnt[r], cnt)
        oid, osc, n = O.alg3(cnt, moff, mem, N, R, B, k)
        assert np.array_equal(u32(ids)[i], oid) and np.array_equal(sc[i], osc)


def test_embeddings_full_size_sampled(F):
    """10^7 x 4096 embeddings streamed from the seed: the device generator
    against the host generator, the SRP codes of sampled points against the
    oracle's exact signs, the group ids, and sampled queries end to end."""
    import ctypes as C

    import torch
    seed = WL.config_seed(4)
    N, d, nc, sig, qsig = 10_000_000, 4096, 1000, 0.1, 0.05
    nq, R, B, L, K, k = 10_000, 3, 20000, 64, 16, 10
    rows = np.array([0, 1, 12345, 7_654_321, N - 1])
    for r in rows:
        xd = F.generate_embeddings(seed, d, nc, sig, int(r), 1).cpu().numpy()
        assert np.array_equal(xd, WL.embed_points(seed, [r], d, nc, sig))
    qd_all = F.generate_embeddings(seed, d, nc, sig, 0, nq, queries=True, q_sigma=qsig, n_points=N)
    qrows = np.array([0, 7, 4242, nq - 1])
    assert np.array_equal(qd_all[torch.from_numpy(qrows).cuda()].cpu().numpy(),
                          WL.embed_queries(seed, qrows, N, d, nc, sig, qsig))

    w = WL.srp_projections(seed, L * K, d)
    perm = WL.group_permutations(seed, R, N)
    ix = F.Index("cosine", R, B, L, K, capacity=N, params=w, dim=d)
    all_b = torch.empty((N, L), dtype=torch.int32, device="cuda")
    ch = 32768
    xbuf = torch.empty((ch, d), dtype=torch.float32, device="cuda")
    for first in range(0, N, ch):
        n = min(ch, N - first)
        x = F.generate_embeddings(seed, d, nc, sig, first, n, out=xbuf[:n])
        fp = F.flinng_points()
        fp.x, fp.ld = x.data_ptr(), d
        F._check(ix.lib.flinng_hash(ix.h, C.byref(fp), n, all_b[first:first + n].data_ptr(), None, None, 1))
    ix.build_buckets(all_b, torch.from_numpy(perm.view(np.int32)).cuda())
    codes = all_b.cpu().numpy().view(np.uint32)
    samp = np.unique(np.concatenate([[0, N - 1], np.random.default_rng(3).choice(N, 94, replace=False)]))
    assert np.array_equal(codes[samp], O.srp_codes(WL.embed_points(seed, samp, d, nc, sig), w, L, K))
    ogid = O.groups(perm, B)
    assert np.array_equal(ix.export(cells=False)["gid"], ogid)
    ids, sc = ix.query(qd_all, k)
    moff, mem = O.members(ogid, B)
    qs = np.array([0, 4242, nq - 1])
    oqb = O.srp_codes(WL.embed_queries(seed, qs, N, d, nc, sig, qsig), w, L, K)
    gqb, _, _ = ix.hash(qd_all[torch.from_numpy(qs).cuda()].contiguous())
    assert np.array_equal(u32(gqb), oqb)
    gcnt = ix.counts(oqb)
    for r, i in enumerate(qs):
        cnt = O.counts_direct(codes, ogid, B, oqb[r])
        assert np.array_equal(gcnt[r], cnt)
        oid, osc, n = O.alg3(cnt, moff, mem, N, R, B, k)
        assert np.array_equal(u32(ids)[i], oid) and np.array_equal(sc.cpu().numpy()[i], osc)
