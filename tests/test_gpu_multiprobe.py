"""Multi-probe counting on the GPU (cosine indices): per-cell counts equal
the oracle's multi-probe definition for P = 1 .. K + 1 probes per table, on
light and heavy (bitmap) slots and a ragged B*R; queries decode those counts
exactly as Alg. 3 does in the oracle, through host and device buffers and in
every query mode; P = 1 is the single-probe index."""
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


def make(F, seed, N, d, R, B, L, K, nq):
    pts, _ = WL.gaussian_mixture(seed, N, d, 40, 0.1)
    q, _ = WL.noisy_queries(seed, pts, nq, 0.05)
    w = WL.srp_projections(seed, L * K, d)
    perm = WL.group_permutations(seed, R, N)
    ix = F.Index("cosine", R, B, L, K, capacity=N, params=w, dim=d)
    ix.build(pts, perm)
    ob = O.srp_codes(pts, w, L, K)
    gid = O.groups(perm, B)
    qb = O.srp_codes(q, w, L, K)
    return ix, q, ob, gid, qb, (pts, w, perm)


# (K = 9: mostly light lists; K = 4: 16 buckets per table, most slots heavy)
@pytest.mark.parametrize("N,R,B,L,K", [(5000, 3, 347, 20, 9), (3000, 2, 200, 7, 4)])
def test_counts_and_queries_equal_oracle(F, N, R, B, L, K):
    import torch
    nq, k = 61, 10
    ix, q, ob, gid, qb, (pts, w, perm) = make(F, 300 + K, N, 64, R, B, L, K, nq)
    moff, mem = O.members(gid, B)
    heavy_min = max(B * R // 16, 32)
    off = ix.export(cells=False)["off"]
    lens = np.diff(off.astype(np.int64))
    heavy = (lens >= heavy_min).mean()
    assert 0 < heavy < 1 and ((heavy > 0.5) if K == 4 else (heavy < 0.5))
    prev = None
    for P in sorted({1, 2, 3, K + 1}):
        ix.set_probes(P)
        cnt = u32(ix.counts(qb))
        ocnt = np.stack([O.counts_multiprobe(ob, gid, B, qb[i], P) for i in range(nq)])
        assert np.array_equal(cnt, ocnt), P
        assert cnt.max() <= L
        if prev is not None:
            assert np.all(cnt >= prev)
        prev = cnt
        # per-query k, host buffers
        kq = np.array([(i * 7) % (k + 1) for i in range(nq)], np.uint32)
        ids, sc = ix.query(q, k, k=kq)
        for i in range(nq):
            oid, osc, _ = O.alg3(ocnt[i], moff, mem, N, R, B, int(kq[i]), k_max=k)
            assert np.array_equal(u32(ids)[i], oid) and np.array_equal(sc[i], osc), (P, i)
        # device buffers, each query mode; and the buckets entry point
        for mode in (F.QUERY_PLAIN, F.QUERY_FUSED, F.QUERY_GRAPH):
            ix.set_query_mode(mode)
            dids, dsc = ix.query(torch.from_numpy(q).cuda(), k)
            bids, bsc = ix.query_buckets(torch.from_numpy(qb.view(np.int32)).cuda(), k)
            torch.cuda.synchronize()
            for i in range(nq):
                oid, osc, _ = O.alg3(ocnt[i], moff, mem, N, R, B, k)
                assert np.array_equal(u32(dids)[i], oid) and np.array_equal(dsc.cpu().numpy()[i], osc)
                assert np.array_equal(u32(bids)[i], oid) and np.array_equal(bsc.cpu().numpy()[i], osc)
        ix.set_query_mode(F.QUERY_FUSED)
    # P = 1 again: the single-probe index (fused path)
    ix.set_probes(1)
    ids, sc = ix.query(q, k)
    o = O.OracleIndex("cosine", R, B, L, K, K, srp_w=w)
    o.build(pts, perm)
    oids, osc = o.query(q, k)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)
    ix.close()


def test_probes_raise_planted_neighbour_scores(F):
    """With few long codes, probing flipped buckets reaches more tables for
    the planted neighbour: its decode score (the smallest count over its R
    cells) never drops as P grows, and rises over the batch. (The top-k
    recall need not rise: probes raise the competitors' counts too.)"""
    N, d, R, B, L, K, nq = 4000, 64, 3, 100, 4, 12, 200
    pts, _ = WL.gaussian_mixture(77, N, d, 40, 0.1)
    q, src = WL.noisy_queries(77, pts, nq, 0.15)
    w = WL.srp_projections(77, L * K, d)
    perm = WL.group_permutations(77, R, N)
    ix = F.Index("cosine", R, B, L, K, capacity=N, params=w, dim=d)
    ix.build(pts, perm)
    gid = O.groups(perm, B)
    qb = O.srp_codes(q, w, L, K)
    cells = np.arange(R)[None, :] * B + gid[src].astype(np.int64)          # nq x R
    score = []
    for P in (1, 4, K + 1):
        ix.set_probes(P)
        cnt = u32(ix.counts(qb)).astype(np.int64)
        score.append(np.take_along_axis(cnt, cells, axis=1).min(axis=1))
    assert np.all(score[1] >= score[0]) and np.all(score[2] >= score[1])
    assert score[2].sum() > score[0].sum(), [s.sum() for s in score]
    ix.close()


def test_probe_arguments_and_rejections(F):
    w = WL.srp_projections(5, 4 * 6, 16)
    ix = F.Index("cosine", 2, 10, 4, 6, capacity=100, params=w, dim=16)
    ix.set_probes(0)
    ix.set_probes(7)
    with pytest.raises(F.FlinngError) as e:
        ix.set_probes(8)                      # K + 2
    assert e.value.code == F.ERR_INVALID_ARG
    srv = F.Server(hbm_budget=ix.device_bytes + (1 << 30), n_slots=2, max_batch=64, k_max=10)
    with pytest.raises(F.FlinngError) as e:
        srv.add_index(ix)
    assert e.value.code == F.ERR_INVALID_ARG
    srv.close()
    import ctypes as C
    import torch
    x = torch.zeros((3, 16), dtype=torch.float32, device="cuda")
    fp = F.flinng_points()
    fp.x, fp.ld = x.data_ptr(), 16
    ids = torch.zeros((3, 10), dtype=torch.int32, device="cuda")
    sc = torch.zeros((3, 10), dtype=torch.int16, device="cuda")
    rc = F.load().flinng_query_noalloc(ix.h, C.byref(fp), 3, None, 10, ids.data_ptr(), sc.data_ptr())
    assert rc == F.ERR_INVALID_ARG
    ix.close()
    dp = WL.doph_params(5, 4, 2)
    jx = F.Index("jaccard", 2, 10, 4, 2, capacity=100, params=dp, W=10)
    jx.set_probes(1)
    with pytest.raises(F.FlinngError) as e:
        jx.set_probes(2)
    assert e.value.code == F.ERR_INVALID_ARG
    jx.close()
