"""GPU path vs the CPU oracle, through the C ABI.

Integer results (hash codes, MinHash values, buckets, group ids, the reverse
index, counts, top-k ids and scores) must be bit-exact. The one
floating-point quantity, the SRP projection, must be within 1e-5 of the fp64
oracle relative to ||w|| ||x|| before its sign is taken (the sign itself is
exact).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_11565_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch  # noqa: F401
    from paper_2106_11565_gb300 import _build, flinng
    _build.build()
    return flinng


def u32(a):
    if hasattr(a, "is_cuda"):
        a = a.cpu().numpy()
    return np.asarray(a).view(np.uint32) if a.dtype == np.int32 else np.asarray(a)


# ------------------------------------------------------------------ cases

def dense_case(seed, N, d, nq, R, B, L, K, n_centers=100):
    pts, _ = WL.gaussian_mixture(seed, N, d, n_centers, 0.1)
    q, _ = WL.noisy_queries(seed, pts, nq, 0.05)
    w = WL.srp_projections(seed, L * K, d)
    perm = WL.group_permutations(seed, R, N)
    return pts, q, w, perm


def sets_case(seed, N, nq, R, L, K):
    g = WL.genomic_reads(seed, ref_len=200_000, n_reads=N, read_len=300, n_queries=nq)
    dp = WL.doph_params(seed, L, K)
    perm = WL.group_permutations(seed, R, N)
    return (g["off"], g["elems"]), (g["q_off"], g["q_elems"]), dp, perm


def ragged_sets(seed, n):
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        s = int(rng.choice([0, 1, 2, 5, 31, 32, 33, 64, 200, 1000]))
        rows.append(rng.integers(0, 1 << 32, size=s, dtype=np.uint64).astype(np.uint32))
    return WL.csr_from_rows(rows)


# ------------------------------------------------------------------ hashing

@pytest.mark.parametrize("n,d,L,K", [(300, 128, 16, 12), (257, 67, 5, 7), (64, 1, 3, 20), (1, 4096, 2, 16)])
def test_srp_codes_bit_exact_and_projection_tolerance(F, n, d, L, K):
    pts, _, w, _ = dense_case(1, n, d, 1, 1, 1, L, K)
    # plant exact and near cancellations
    for i in range(0, n, 5):
        j = i % (L * K)
        if d > 1:
            pts[i, -1] = np.float32(-float(np.dot(w[j, :-1].astype(np.float64), pts[i, :-1])) / float(w[j, -1]))
    pts[n - 1] = 0.0
    ix = F.Index("cosine", 1, 1, L, K, capacity=n, params=w, dim=d)
    codes, _, proj = ix.hash(pts, proj=True)
    ocodes, oproj, _ = O.srp_codes(pts, w, L, K, want_proj=True)
    assert np.array_equal(u32(codes), ocodes)
    scale = np.linalg.norm(pts.astype(np.float64), axis=1)[:, None] * \
        np.linalg.norm(w.astype(np.float64), axis=1)[None, :]
    rel = np.abs(proj.astype(np.float64) - oproj) / np.maximum(scale, 1e-300)
    assert rel.max() <= 1e-5
    nre, nex = ix.hash_stats()
    assert nre >= n // 5 and nex >= 1       # planted zeros went to the exact path


def test_srp_device_and_host_paths_agree(F):
    import torch
    pts, _, w, _ = dense_case(2, 500, 96, 1, 1, 1, 8, 10)
    ix = F.Index("cosine", 1, 1, 8, 10, capacity=500, params=w, dim=96)
    h, _, _ = ix.hash(pts)
    dvc, _, _ = ix.hash(torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(u32(h), u32(dvc))


@pytest.mark.parametrize("L,K,W", [(32, 2, 17), (64, 1, 17), (3, 5, 9), (1, 1, 1)])
def test_doph_values_and_buckets_bit_exact(F, L, K, W):
    off, el = ragged_sets(3, 400)
    dp = WL.doph_params(3, L, K)
    ix = F.Index("jaccard", 1, 1, L, K, capacity=400, params=dp, W=W)
    b, v, _ = ix.hash((off, el), values=True)
    ov = O.doph(off, el, L * K, dp["doph_a"], dp["doph_b"], dp["doph_seed"])
    ob = O.minhash_buckets(ov, L, K, dp["bucket_a"], dp["bucket_c"], W)
    assert np.array_equal(u32(v), ov)
    assert np.array_equal(u32(b), ob)


# ------------------------------------------------------------------ index

def oracle_index(metric, R, B, L, K, W, params, pts, perm, t_min=1):
    idx = O.OracleIndex(metric, R, B, L, K, W, t_min=t_min,
                        srp_w=params if metric == "cosine" else None,
                        doph=params if metric != "cosine" else None)
    idx.build(pts, perm)
    return idx


@pytest.mark.parametrize("R,B", [(3, 100), (1, 1), (4, 7), (2, 1000)])
def test_build_reverse_index_bit_exact(F, R, B):
    N, d, L, K = 2000, 32, 6, 8
    pts, _, w, perm = dense_case(4, N, d, 1, R, B, L, K)
    ix = F.Index("cosine", R, B, L, K, capacity=N, params=w, dim=d)
    ix.build(pts, perm)
    ex = ix.export()
    o = oracle_index("cosine", R, B, L, K, K, w, pts, perm)
    assert np.array_equal(ex["gid"], o.gid)
    assert np.array_equal(ex["off"], o.off)
    assert np.array_equal(ex["cells"], o.cells)


def test_build_rejects_bad_permutation_and_capacity(F):
    pts, _, w, perm = dense_case(5, 100, 8, 1, 2, 10, 2, 4)
    ix = F.Index("cosine", 2, 10, 2, 4, capacity=100, params=w, dim=8)
    bad = perm.copy()
    bad[1, 3] = bad[1, 4]
    with pytest.raises(F.FlinngError) as e:
        ix.build(pts, bad)
    assert e.value.code == F.ERR_INVALID_ARG
    bad[1, 3] = 100
    with pytest.raises(F.FlinngError):
        ix.build(pts, bad)
    ix.build(pts, perm)
    with pytest.raises(F.FlinngError) as e:
        ix.insert(pts[:1], np.zeros((2, 1), np.uint32))
    assert e.value.code == F.ERR_CAPACITY
    assert ix.size == 100


def test_insert_equals_oracle_insert(F):
    N1, N2, d, R, B, L, K = 700, 300, 24, 3, 37, 5, 9
    pts, q, w, perm = dense_case(6, N1 + N2, d, 50, R, B, L, K)
    p1 = WL.group_permutations(6, R, N1)
    p2 = WL.group_permutations(6, R, N2, batch=1)
    ix = F.Index("cosine", R, B, L, K, capacity=N1 + N2, params=w, dim=d)
    ix.build(pts[:N1], p1)
    ix.insert(pts[N1:], p2)
    o = O.OracleIndex("cosine", R, B, L, K, K, srp_w=w)
    o.build(pts[:N1], p1)
    o.insert(pts[N1:], p2)
    ex = ix.export()
    assert np.array_equal(ex["gid"], o.gid)
    assert np.array_equal(ex["off"], o.off) and np.array_equal(ex["cells"], o.cells)
    ids, sc = ix.query(q, 20)
    oids, osc = o.query(q, 20)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)


def test_given_design_bit_exact(F):
    """Sec. 3.1: a design given outright (each point's group drawn uniformly
    and independently per repetition: unequal and empty groups), by build,
    by build then insert, and with every point in one group; the index and
    every query mode equal the oracle's. A group id >= B is refused and the
    index is left as it was."""
    import torch
    N, nq, R, B, L, K, W = 3000, 200, 3, 400, 32, 2, 15
    pts, q, dp, perm = sets_case(45, N, nq, R, L, K)
    g = WL.random_design(45, R, N, B)
    assert np.bincount(g[0], minlength=B).min() == 0 or np.bincount(g[0], minlength=B).max() > N // B + 1

    def sets(lo, hi):
        off, el = pts
        return (off[lo:hi + 1] - off[lo]).astype(np.uint64), np.ascontiguousarray(el[off[lo]:off[hi]])

    def check(ix, o):
        ex = ix.export()
        assert np.array_equal(ex["gid"], o.gid)
        assert np.array_equal(ex["off"], o.off) and np.array_equal(ex["cells"], o.cells)
        oids, osc = o.query(q, 30)
        for mode in (0, 1, 2):
            ix.set_query_mode(mode)
            ids, sc = ix.query(q, 30)
            assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc), mode

    o = O.OracleIndex("jaccard", R, B, L, K, W, doph=dp)
    o.build_groups(pts, g)
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    ix.build_groups(pts, g)
    check(ix, o)
    # build then insert, groups in device memory
    jx = F.Index("jaccard", R, B, L, K, capacity=N + 100, params=dp, W=W)
    d_off = lambda a: torch.from_numpy(a.view(np.int64)).cuda()
    d_el = lambda a: torch.from_numpy(a.view(np.int32)).cuda()
    d_g = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).cuda()
    a_off, a_el = sets(0, 1800)
    b_off, b_el = sets(1800, N)
    jx.build_groups((d_off(a_off), d_el(a_el)), d_g(g[:, :1800]))
    jx.insert_groups((d_off(b_off), d_el(b_el)), d_g(g[:, 1800:]))
    torch.cuda.synchronize()
    check(jx, o)
    # a refused group id leaves the index as it was
    bad = g[:, :10].copy()
    bad[1, 3] = B
    with pytest.raises(F.FlinngError) as e:
        jx.insert_groups(sets(0, 10), bad)
    assert e.value.code == F.ERR_INVALID_ARG
    check(jx, o)
    # every point in group 0: one cell of N members per repetition
    z = np.zeros((R, N), np.uint16)
    o2 = O.OracleIndex("jaccard", R, B, L, K, W, doph=dp)
    o2.build_groups(pts, z)
    kx = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    kx.build_groups(pts, z)
    check(kx, o2)


# ------------------------------------------------------------------ query

def test_counts_bit_exact(F):
    N, d, R, B, L, K = 3000, 64, 3, 100, 16, 12
    pts, q, w, perm = dense_case(7, N, d, 64, R, B, L, K)
    ix = F.Index("cosine", R, B, L, K, capacity=N, params=w, dim=d)
    ix.build(pts, perm)
    o = oracle_index("cosine", R, B, L, K, K, w, pts, perm)
    qb = O.srp_codes(q, w, L, K)
    got = ix.counts(qb)
    for i in range(q.shape[0]):
        assert np.array_equal(got[i], O.counts(o.off, o.cells, L, K, qb[i], B * R))


MODES = [0, 1, 2]     # flinng QUERY_PLAIN, QUERY_FUSED, QUERY_GRAPH


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("t_min", [1, 3])
def test_query_dense_bit_exact(F, t_min, mode):
    N, d, R, B, L, K = 10_000, 128, 3, 100, 16, 12      # the paper-shaped cosine config
    pts, q, w, perm = dense_case(WL.config_seed(1), N, d, 100, R, B, L, K)
    ix = F.Index("cosine", R, B, L, K, capacity=N, params=w, dim=d, t_min=t_min)
    ix.set_query_mode(mode)
    ix.build(pts, perm)
    o = oracle_index("cosine", R, B, L, K, K, w, pts, perm, t_min=t_min)
    ids, sc = ix.query(q, 10)
    oids, osc = o.query(q, 10)
    assert np.array_equal(u32(ids), oids)
    assert np.array_equal(sc, osc)


@pytest.mark.parametrize("mode", MODES)
def test_query_ragged_k_and_edge_cases(F, mode):
    N, d, R, B, L, K = 1500, 32, 2, 40, 8, 6
    pts, q, w, perm = dense_case(8, N, d, 97, R, B, L, K)
    q[5] = 0.0                    # zero query: every projection takes the exact path
    q[9, :] = pts[3]              # exact copy of an indexed point
    ix = F.Index("cosine", R, B, L, K, capacity=N, params=w, dim=d)
    ix.set_query_mode(mode)
    ix.build(pts, perm)
    o = oracle_index("cosine", R, B, L, K, K, w, pts, perm)
    rng = np.random.default_rng(8)
    k = rng.integers(0, 301, size=q.shape[0]).astype(np.uint32)
    k[:3] = [0, 1, 300]
    ids, sc = ix.query(q, 300, k=k)
    oids, osc = o.query(q, 300, k=k)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)
    # k larger than the index: every point with score >= t_min, then padding
    ids, sc = ix.query(q[:5], 1024)
    oids, osc = o.query(q[:5], 1024)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)
    # a query equal to an indexed point returns it with score L
    ids, sc = ix.query(pts[:20], 5)
    for i in range(20):
        assert sc[i, 0] == L
    with pytest.raises(F.FlinngError):
        ix.query(q, 10, k=np.full(q.shape[0], 11, np.uint32))


@pytest.mark.parametrize("mode", MODES)
def test_query_empty_index_and_empty_batch(F, mode):
    w = WL.srp_projections(9, 4 * 3, 8)
    ix = F.Index("cosine", 2, 5, 4, 3, capacity=10, params=w, dim=8)
    ix.set_query_mode(mode)
    q = np.ones((3, 8), np.float32)
    ids, sc = ix.query(q, 4)
    assert np.all(u32(ids) == 0xFFFFFFFF) and np.all(sc == 0)
    ids, sc = ix.query(np.zeros((0, 8), np.float32), 4)
    assert ids.shape == (0, 4)


@pytest.mark.parametrize("mode", MODES)
def test_query_sets_bit_exact(F, mode):
    N, nq, R, B, L, K, W = 4000, 200, 2, 1000, 32, 2, 17
    pts, q, dp, perm = sets_case(10, N, nq, R, L, K)
    # ragged query sets: empty, single element, duplicates
    qoff, qel = q
    rows = [qel[qoff[i]:qoff[i + 1]] for i in range(nq)]
    rows[0] = rows[0][:0]
    rows[1] = rows[1][:1]
    rows[2] = np.concatenate([rows[2], rows[2][:50]])
    q = WL.csr_from_rows(rows)
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    ix.set_query_mode(mode)
    ix.build(pts, perm)
    o = oracle_index("jaccard", R, B, L, K, W, dp, pts, perm)
    ex = ix.export()
    assert np.array_equal(ex["off"], o.off) and np.array_equal(ex["cells"], o.cells)
    ids, sc = ix.query(q, 100)
    oids, osc = o.query(q, 100)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)


@pytest.mark.parametrize("mode", MODES)
def test_query_device_buffers_match_host(F, mode):
    import torch
    N, nq, R, B, L, K, W = 3000, 100, 2, 300, 16, 2, 12
    pts, q, dp, perm = sets_case(11, N, nq, R, L, K)
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    ix.set_query_mode(mode)
    ix.build((torch.from_numpy(pts[0].view(np.int64)).cuda(), torch.from_numpy(pts[1].view(np.int32)).cuda()),
             torch.from_numpy(perm.view(np.int32)).cuda())
    torch.cuda.synchronize()
    hid, hsc = ix.query(q, 50)
    did, dsc = ix.query((torch.from_numpy(q[0].view(np.int64)).cuda(),
                         torch.from_numpy(q[1].view(np.int32)).cuda()), 50)
    torch.cuda.synchronize()
    assert np.array_equal(u32(hid), u32(did)) and np.array_equal(hsc, dsc.cpu().numpy())
    o = oracle_index("jaccard", R, B, L, K, W, dp, pts, perm)
    oids, osc = o.query(q, 50)
    assert np.array_equal(u32(hid), oids)


@pytest.mark.parametrize("R,B,L,K,W,k", [(4, 500, 64, 1, 17, 10), (3, 2000, 24, 2, 14, 1000), (1, 3000, 8, 3, 12, 7)])
def test_fused_equals_plain_and_oracle_sets(F, R, B, L, K, W, k):
    N, nq = 3000, 150
    pts, q, dp, perm = sets_case(12 + R, N, nq, R, L, K)
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    ix.build(pts, perm)
    ix.set_query_mode(0)
    pids, psc = ix.query(q, k)
    ix.set_query_mode(1)
    fids, fsc = ix.query(q, k)
    assert np.array_equal(pids, fids) and np.array_equal(psc, fsc)
    o = oracle_index("jaccard", R, B, L, K, W, dp, pts, perm)
    oids, osc = o.query(q, k)
    assert np.array_equal(u32(fids), oids) and np.array_equal(fsc, osc)


@pytest.mark.parametrize("d,L,K", [(1, 4, 5), (67, 6, 9), (1024, 8, 16)])
def test_fused_srp_equals_oracle(F, d, L, K):
    N, R, B = 1200, 2, 60
    pts, q, w, perm = dense_case(20 + d, N, d, 64, R, B, L, K, n_centers=10)
    q[1] = 0.0
    if d > 1:
        for i in range(2, 64, 3):         # plant near-zero projections in the queries
            j = i % (L * K)
            q[i, -1] = np.float32(-float(np.dot(w[j, :-1].astype(np.float64), q[i, :-1])) / float(w[j, -1]))
    ix = F.Index("cosine", R, B, L, K, capacity=N, params=w, dim=d)
    ix.build(pts, perm)
    ix.set_query_mode(1)
    ids, sc = ix.query(q, 15)
    o = oracle_index("cosine", R, B, L, K, K, w, pts, perm)
    oids, osc = o.query(q, 15)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)
    nre, nex = ix.hash_stats()
    assert nex >= 1


def test_graph_replay_and_tuning_keep_results(F):
    # graph mode across calls of different sizes in the same and in different
    # size classes, before and after autotuning, equals the plain form
    N, nq, R, B, L, K, W = 3000, 300, 2, 300, 32, 2, 15
    pts, q, dp, perm = sets_case(40, N, nq, R, L, K)
    qoff, qel = q
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    ix.build(pts, perm)

    def sl(lo, hi):
        return (qoff[lo:hi + 1] - qoff[lo]).astype(np.uint64), np.ascontiguousarray(qel[qoff[lo]:qoff[hi]])
    ix.set_query_mode(0)
    ref = {r: ix.query(sl(*r), 30) for r in [(0, 300), (10, 250), (5, 6), (0, 129)]}
    ix.set_query_mode(2)
    for r, (rid, rsc) in ref.items():
        ids, sc = ix.query(sl(*r), 30)
        assert np.array_equal(ids, rid) and np.array_equal(sc, rsc)
    ch = ix.tune(sl(0, 300), 30)
    assert ch["threads"] in (128, 256, 512)        # any shape the tuner knows
    for r, (rid, rsc) in list(ref.items())[::-1]:
        ids, sc = ix.query(sl(*r), 30)
        assert np.array_equal(ids, rid) and np.array_equal(sc, rsc)
    ix.set_query_mode(1)
    ids, sc = ix.query(sl(0, 300), 30)
    assert np.array_equal(ids, ref[(0, 300)][0])


def test_pinned_shapes_keep_results(F):
    # every launch shape flinng_set_tuning accepts gives the plain form's
    # results, in graph and fused modes; other values are refused
    N, nq, R, B, L, K, W = 3000, 300, 2, 300, 32, 2, 15
    pts, q, dp, perm = sets_case(42, N, nq, R, L, K)
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    ix.build(pts, perm)
    ix.set_query_mode(0)
    rid, rsc = ix.query(q, 30)
    for th in (128, 256, 512):
        for cp in (0, 1, 4):
            for cap in (0, 64, 1024, 8192):
                ix.set_tuning(nq, th, cp, cap)
                for mode in (1, 2):
                    ix.set_query_mode(mode)
                    ids, sc = ix.query(q, 30)
                    assert np.array_equal(ids, rid) and np.array_equal(sc, rsc), (th, cp, cap, mode)
    for bad in [(nq, 64, 0, 0), (nq, 1024, 0, 0), (nq, 256, 17, 0), (nq, 256, 0, 100), (nq, 256, 0, 16384),
                (0, 256, 0, 0)]:
        with pytest.raises(F.FlinngError) as e:
            ix.set_tuning(*bad)
        assert e.value.code == F.ERR_INVALID_ARG


def _pinned(a):
    import torch
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a.view({1: np.int8, 2: np.int16, 4: np.int32, 8: np.int64}[a.itemsize]))
    return t.pin_memory().numpy().view(a.dtype)


def test_pinned_host_buffers_in_place(F):
    # page-locked queries and results are read and written in place by the
    # kernels; every mix of pinned and pageable buffers gives the staged results
    N, nq, R, B, L, K, W = 3000, 300, 2, 300, 32, 2, 15
    pts, q, dp, perm = sets_case(43, N, nq, R, L, K)
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    ix.build(pts, perm)
    ix.set_query_mode(0)
    rid, rsc = ix.query(q, 30)                      # pageable: staged by copies
    pq = (_pinned(q[0]), _pinned(q[1]))
    oi, osc = _pinned(np.zeros((nq, 30), np.uint32)), _pinned(np.zeros((nq, 30), np.uint16))
    for mode in (0, 1, 2):
        ix.set_query_mode(mode)
        for qq, out in ((pq, (oi, osc)), (pq, None), (q, (oi, osc))):
            if out is not None:
                oi.fill(7)
                osc.fill(7)
            ids, sc = ix.query(qq, 30, out=out)
            if out is not None:
                assert ids is oi and sc is osc
            assert np.array_equal(ids, rid) and np.array_equal(sc, rsc), mode
    # a pinned sub-range (interior pointers) of a larger batch
    big = _pinned(np.zeros((nq + 5, 30), np.uint32))
    ids, _ = ix.query(pq, 30, out=(big[5:], _pinned(np.zeros((nq, 30), np.uint16))))
    assert np.array_equal(big[5:], rid)
    # cosine: the fused form reads pinned queries in place, the plain form stages them
    pts, qd, w, perm = dense_case(44, 2000, 64, 150, 2, 40, 8, 10)
    jx = F.Index("cosine", 2, 40, 8, 10, capacity=2000, params=w, dim=64)
    jx.build(pts, perm)
    jx.set_query_mode(0)
    cid, csc = jx.query(qd, 12)
    pqd = _pinned(qd)
    ci, cs = _pinned(np.zeros((150, 12), np.uint32)), _pinned(np.zeros((150, 12), np.uint16))
    for mode in (0, 1, 2):
        jx.set_query_mode(mode)
        ids, sc = jx.query(pqd, 12, out=(ci, cs))
        assert np.array_equal(ids, cid) and np.array_equal(sc, csc), mode
    with pytest.raises(ValueError):
        jx.query(pqd, 12, out=(ci[:, :5], cs))
    # device queries: the out tensors' dtype and layout are checked before any launch
    import torch
    dq = torch.from_numpy(qd).cuda()
    for bad in [(torch.empty((150, 12), dtype=torch.int16, device="cuda"),
                 torch.empty((150, 12), dtype=torch.int16, device="cuda")),
                (torch.empty((12, 150), dtype=torch.int32, device="cuda").t(),
                 torch.empty((150, 12), dtype=torch.int16, device="cuda"))]:
        with pytest.raises(ValueError):
            jx.query(dq, 12, out=bad)


def test_host_buckets_out_of_range_refused(F):
    # a host bucket >= 2^W is refused before anything is copied or launched
    pts, q, w, perm = dense_case(46, 300, 16, 10, 2, 10, 4, 6)
    ix = F.Index("cosine", 2, 10, 4, 6, capacity=300, params=w, dim=16)
    ix.build(pts, perm)
    qb = O.srp_codes(q, w, 4, 6)
    ids, sc = ix.query_buckets(qb, 5)
    bad = qb.copy()
    bad[3, 2] = 1 << 6
    for call in (lambda: ix.query_buckets(bad, 5), lambda: ix.counts(bad)):
        with pytest.raises(F.FlinngError) as e:
            call()
        assert e.value.code == F.ERR_INVALID_ARG
    ids2, sc2 = ix.query_buckets(qb, 5)
    assert np.array_equal(ids, ids2) and np.array_equal(sc, sc2)


def test_graph_mode_cosine_stats_reset(F):
    pts, q, w, perm = dense_case(41, 800, 40, 50, 2, 20, 6, 7)
    q[0] = 0.0
    ix = F.Index("cosine", 2, 20, 6, 7, capacity=800, params=w, dim=40)
    ix.build(pts, perm)
    ix.set_query_mode(2)
    exact = []
    for _ in range(3):
        ids, sc = ix.query(q, 8)
        exact.append(ix.hash_stats()[1])
    # the zero query's 42 projections take the exact path; counters restart per call
    assert exact[0] >= 6 * 7 and exact[0] == exact[1] == exact[2]
    o = oracle_index("cosine", 2, 20, 6, 7, 7, w, pts, perm)
    oids, osc = o.query(q, 8)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)


@pytest.mark.parametrize("mode", MODES)
def test_heavy_bucket_bitmaps(F, mode):
    # 2-bit buckets: every list is long, most slots get a cell bitmap; a few
    # 9-bit tables stay light: counts and top-k must not change
    N, d, R, B = 2500, 24, 3, 60
    pts, q, w, perm = dense_case(50, N, d, 80, R, B, 6, 2)
    ix = F.Index("cosine", R, B, 6, 2, capacity=N, params=w, dim=d)
    ix.set_query_mode(mode)
    ix.build(pts, perm)
    o = oracle_index("cosine", R, B, 6, 2, 2, w, pts, perm)
    qb = O.srp_codes(q, w, 6, 2)
    got = ix.counts(qb)
    for i in range(q.shape[0]):
        assert np.array_equal(got[i], O.counts(o.off, o.cells, 6, 2, qb[i], B * R))
    ids, sc = ix.query(q, 40)
    oids, osc = o.query(q, 40)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)
    # mixed heavy and light tables in one query
    pts2, q2, w2, perm2 = dense_case(51, N, d, 80, R, B, 10, 9)
    w2[:18] = w2[:18] * 0 + w[:1]          # tables 0-1 use one projection repeatedly: 2 buckets
    jx = F.Index("cosine", R, B, 10, 9, capacity=N, params=w2, dim=d)
    jx.set_query_mode(mode)
    jx.build(pts2, perm2)
    o2 = oracle_index("cosine", R, B, 10, 9, 9, w2, pts2, perm2)
    ids, sc = jx.query(q2, 25)
    oids, osc = o2.query(q2, 25)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L,K,W,B", [(300, 1, 17, 1000), (1024, 1, 12, 250), (600, 2, 3, 60)])
def test_wide_counts_bit_exact(F, mode, L, K, W, B):
    """More than 255 tables: 16-bit counts and 60-bit keys. Scores above 255,
    heavy buckets (W = 3: every list is long) and light ones, all modes."""
    N, nq, R = 3000, 60, 2
    pts, q, dp, perm = sets_case(70 + L, N, nq, R, L, K)
    ix = F.Index("jaccard", R, B, L, K, capacity=N, params=dp, W=W)
    ix.set_query_mode(mode)
    ix.build(pts, perm)
    o = oracle_index("jaccard", R, B, L, K, W, dp, pts, perm)
    qb = ix.hash(q)[0]
    got = ix.counts(qb)
    for i in range(0, nq, 7):
        assert np.array_equal(got[i], O.counts(o.off, o.cells, L, W, u32(qb)[i], B * R))
    ids, sc = ix.query(q, 50)
    oids, osc = o.query(q, 50)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)
    # queries equal to indexed points: score L > 255 (no false negative)
    pq = WL.csr_from_rows([pts[1][pts[0][i]:pts[0][i + 1]] for i in range(5)])
    ids, sc = ix.query(pq, 20)
    oids, osc = o.query(pq, 20)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc, osc)
    for i in range(5):
        assert sc[i, 0] == L
