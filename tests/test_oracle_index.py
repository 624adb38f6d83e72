"""Pins for the oracle's index and decode steps (CPU only).

* Alg. 1 group design: every point in exactly one cell per repetition, cell
  sizes floor(N/B) or ceil(N/B) (Sec. 3.1, doubly regular design).
* Sec. 5 reverse index: lists sorted, unique, and holding exactly the
  distinct (table, bucket, cell) triples (brute force).
* Sec. 5 counts: the reverse-index walk equals a brute-force count with no
  index.
* Alg. 3: a hand-worked example, and equality with an independent closed
  form of its output order on random tiny inputs.
* No false negative: a query equal to an indexed point gives that point
  the maximum score L and returns it.
* Reduction to exact kNN: with B = N and R = 1 the ranking converges to the
  brute-force cosine ranking as L grows.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_11565_gb300 import workloads as WL


# ------------------------------------------------------------ Alg. 1 groups

def test_groups_identity_permutation_by_hand():
    perm = np.arange(7, dtype=np.uint32)[None, :]
    gid = O.groups(perm, B=3)
    assert gid[:, 0].tolist() == [0, 1, 2, 0, 1, 2, 0]
    # a second batch continues the positions: cells keep cycling
    gid2 = np.zeros((10, 1), np.uint16)
    gid2[:7] = gid
    O.groups(np.arange(3, dtype=np.uint32)[None, :], B=3, n_old=7, gid=gid2)
    assert gid2[:, 0].tolist() == [0, 1, 2, 0, 1, 2, 0, 1, 2, 0]


@pytest.mark.parametrize("N,B,R", [(1, 1, 1), (10, 3, 2), (1000, 7, 4), (257, 256, 3)])
def test_groups_doubly_regular(N, B, R):
    perm = WL.group_permutations(1, R, N)
    gid = O.groups(perm, B)
    assert gid.shape == (N, R)
    for r in range(R):
        sizes = np.bincount(gid[:, r], minlength=B)
        assert sizes.sum() == N                       # one cell per point
        assert set(sizes.tolist()) <= {N // B, -(-N // B)}
        # position i of the permutation lands in cell i mod B
        assert np.all(gid[perm[r], r] == np.arange(N) % B)


def test_groups_rejects_non_permutation():
    with pytest.raises(ValueError):
        O.groups(np.array([[0, 0, 1]], np.uint32), B=2)


def test_members_partition_points():
    N, B, R = 300, 11, 3
    gid = O.groups(WL.group_permutations(2, R, N), B)
    moff, mem = O.members(gid, B)
    for r in range(R):
        seen = []
        for b in range(B):
            m = mem[r, moff[r, b]:moff[r, b + 1]]
            assert np.all(np.diff(m.astype(np.int64)) > 0)      # ascending ids
            assert np.all(gid[m, r] == b)
            seen.extend(m.tolist())
        assert sorted(seen) == list(range(N))


# ------------------------------------------------------------ reverse index

def _tiny_index(seed, N, L, R, B, W):
    rng = np.random.default_rng(seed)
    buckets = rng.integers(0, 1 << W, size=(N, L), dtype=np.uint64).astype(np.uint32)
    gid = O.groups(WL.group_permutations(seed, R, N), B)
    return buckets, gid


@pytest.mark.parametrize("seed,N,L,R,B,W", [(0, 50, 4, 2, 5, 3), (1, 200, 8, 3, 20, 5),
                                            (2, 1, 1, 1, 1, 1), (3, 64, 3, 4, 64, 2)])
def test_csr_holds_exactly_the_distinct_triples(seed, N, L, R, B, W):
    buckets, gid = _tiny_index(seed, N, L, R, B, W)
    off, cells = O.build_csr(buckets, gid, B, W)
    triples = {(l, int(buckets[x, l]), r * B + int(gid[x, r]))
               for x in range(N) for l in range(L) for r in range(R)}
    assert off[-1] == len(cells) == len(triples)
    got = set()
    for l in range(L):
        for h in range(1 << W):
            lst = cells[off[(l << W) + h]:off[(l << W) + h + 1]].astype(np.int64)
            assert np.all(np.diff(lst) > 0)                      # sorted, unique
            got |= {(l, h, int(c)) for c in lst}
    assert got == triples


@pytest.mark.parametrize("seed", range(5))
def test_counts_equal_brute_force(seed):
    N, L, R, B, W = 120, 6, 3, 10, 3
    buckets, gid = _tiny_index(seed, N, L, R, B, W)
    off, cells = O.build_csr(buckets, gid, B, W)
    rng = np.random.default_rng(100 + seed)
    q = rng.integers(0, 1 << W, size=L).astype(np.uint32)
    cnt = O.counts(off, cells, L, W, q, B * R)
    # brute force, no index: a cell counts table l once if any member of
    # the cell has the query's bucket in table l
    brute = np.zeros(B * R, np.int64)
    for r in range(R):
        for b in range(B):
            mem = np.nonzero(gid[:, r] == b)[0]
            for l in range(L):
                brute[r * B + b] += bool(np.any(buckets[mem, l] == q[l]))
    assert np.array_equal(cnt.astype(np.int64), brute)
    assert cnt.max() <= L


# ------------------------------------------------------------ Alg. 3

def test_alg3_hand_worked():
    # N = 6 points, B = 2, R = 2.
    # rep 0, identity permutation: cell 0 = {0,2,4}, cell 1 = {1,3,5}
    # rep 1, permutation [0,2,1,3,4,5]: positions 0,2,4 hold points 0,1,4
    #   -> cell 2 (= 1*B + 0) = {0,1,4}; cell 3 = {2,3,5}
    perm = np.array([[0, 1, 2, 3, 4, 5], [0, 2, 1, 3, 4, 5]], np.uint32)
    gid = O.groups(perm, B=2)
    moff, mem = O.members(gid, 2)
    cnt = np.array([3, 1, 2, 2], np.uint8)
    # visit order: cell 0 (3), cell 2 (2), cell 3 (2), cell 1 (1)
    #  cell 0: 0,2,4 -> 1 each; cell 2: 0 -> 2 emit, 1 -> 1, 4 -> 2 emit
    #  cell 3: 2 -> 2 emit, 3 -> 1, 5 -> 1; cell 1: 1, 3, 5 emit
    ids, sc, n = O.alg3(cnt, moff, mem, 6, 2, 2, k=4, t_min=1)
    assert ids.tolist() == [0, 4, 2, 1] and sc.tolist() == [2, 2, 2, 1] and n == 4
    ids, sc, n = O.alg3(cnt, moff, mem, 6, 2, 2, k=6, t_min=2, k_max=6)
    assert ids.tolist() == [0, 4, 2] + [0xFFFFFFFF] * 3 and n == 3
    ids, sc, n = O.alg3(cnt, moff, mem, 6, 2, 2, k=0, t_min=1, k_max=2)
    assert n == 0 and ids.tolist() == [0xFFFFFFFF] * 2


def closed_key_order(cnt, gid, B, k, t_min):
    """Alg. 3's output written as one sort: a point is emitted when the last
    of its R cells in the visiting order is visited, i.e. its cell of least
    count (ties: the largest cell id); points emitted from the same cell come
    in id order. Key = (-score, last cell, id)."""
    N, R = gid.shape
    keys = []
    for x in range(N):
        cs = [r * B + int(gid[x, r]) for r in range(R)]
        score = min(int(cnt[c]) for c in cs)
        last = max(c for c in cs if cnt[c] == score)
        if score >= t_min:
            keys.append((-score, last, x))
    keys.sort()
    return [x for _, _, x in keys[:k]], [-s for s, _, _ in keys[:k]]


@pytest.mark.parametrize("seed", range(40))
def test_alg3_equals_closed_key(seed):
    rng = np.random.default_rng(seed)
    N = int(rng.integers(1, 65))
    R = int(rng.integers(1, 5))
    B = int(rng.integers(1, N + 1))
    L = int(rng.integers(1, 9))
    gid = O.groups(WL.group_permutations(seed, R, N), B)
    moff, mem = O.members(gid, B)
    cnt = rng.integers(0, L + 1, size=B * R).astype(np.uint8)
    for k in (1, 3, N, N + 5):
        for t_min in (1, 2, L):
            ids, sc, n = O.alg3(cnt, moff, mem, N, R, B, k=k, t_min=t_min)
            e_ids, e_sc = closed_key_order(cnt, gid, B, k, t_min)
            assert ids[:n].tolist() == e_ids and sc[:n].tolist() == e_sc
            assert np.all(ids[n:] == 0xFFFFFFFF)


# ------------------------------------------------------------ whole index

def _dense_index(seed, N, d, R, B, L, K, n_centers=10):
    pts, _ = WL.gaussian_mixture(seed, N, d, n_centers, 0.1)
    w = WL.srp_projections(seed, L * K, d)
    idx = O.OracleIndex("cosine", R, B, L, K, K, srp_w=w)
    idx.build(pts, WL.group_permutations(seed, R, N))
    return idx, pts


def test_no_false_negative():
    idx, pts = _dense_index(4, 400, 16, 3, 20, 8, 6)
    qsrc = np.arange(0, 400, 7)
    qb = idx.hash(pts[qsrc])
    # score L for the point itself (its R cells see all L tables)
    for q, x in zip(qb, qsrc):
        cnt = O.counts(idx.off, idx.cells, idx.L, idx.W, q, idx.B * idx.R)
        assert min(int(cnt[r * idx.B + idx.gid[x, r]]) for r in range(idx.R)) == idx.L
    # returned whenever k covers every point of score L
    k_max = 400
    ids, sc = idx.query_buckets(qb, k_max)
    for i, x in enumerate(qsrc):
        n_top = int(np.sum(sc[i] == idx.L))
        assert x in ids[i, :n_top].tolist()
        assert np.all(sc[i, :n_top] == idx.L)


def test_reduction_to_exact_knn_with_one_point_per_cell():
    # B = N, R = 1: each cell holds one point, its count is the number of
    # tables in which the point collides with the query, whose expectation
    # is L * s^K with s = 1 - theta/pi; ranking by count tends to ranking
    # by cosine as L grows (well-separated tiny data).
    rng = np.random.default_rng(8)
    N, d, K = 24, 16, 4
    q = rng.standard_normal(d)
    q /= np.linalg.norm(q)
    angles = np.linspace(0.05, 1.6, N)
    pts = []
    for a in angles:
        v = rng.standard_normal(d)
        v -= v.dot(q) * q
        v /= np.linalg.norm(v)
        pts.append(np.cos(a) * q + np.sin(a) * v)
    pts = np.array(pts, np.float32)
    exact = list(np.argsort(angles)[:5])
    recalls = []
    for L in (8, 64, 240):          # counts are 8-bit: L <= 255
        w = WL.srp_projections(L, L * K, d)
        idx = O.OracleIndex("cosine", 1, N, L, K, K, srp_w=w)
        idx.build(pts, WL.group_permutations(L, 1, N))
        ids, _ = idx.query(q[None, :].astype(np.float32), 5)
        recalls.append(len(set(ids[0].tolist()) & set(exact)) / 5)
    assert recalls[-1] == 1.0
    assert recalls[0] <= recalls[-1]


def test_insert_equals_build_of_union():
    # inserting a second batch (fresh permutation, positions continuing)
    # gives the same index as Alg. 1 applied to the concatenated positions
    pts, _ = WL.gaussian_mixture(9, 300, 8, 5, 0.1)
    w = WL.srp_projections(9, 4 * 5, 8)
    a = O.OracleIndex("cosine", 2, 7, 4, 5, 5, srp_w=w)
    a.build(pts[:200], WL.group_permutations(9, 2, 200))
    p2 = WL.group_permutations(9, 2, 100, batch=1)
    a.insert(pts[200:], p2)
    # the same assignment written by hand: batch-2 position i -> cell (200+i) mod B
    for r in range(2):
        for i in range(100):
            assert a.gid[200 + p2[r, i], r] == (200 + i) % 7
    b_off, b_cells = O.build_csr(a.buckets, a.gid, 7, 5)
    assert np.array_equal(a.off, b_off) and np.array_equal(a.cells, b_cells)


@pytest.mark.parametrize("seed", range(3))
def test_counts_direct_equals_index_walk(seed):
    N, L, R, B, W = 300, 7, 3, 13, 4
    buckets, gid = _tiny_index(seed, N, L, R, B, W)
    off, cells = O.build_csr(buckets, gid, B, W)
    rng = np.random.default_rng(200 + seed)
    for _ in range(5):
        q = rng.integers(0, 1 << W, size=L).astype(np.uint32)
        assert np.array_equal(O.counts(off, cells, L, W, q, B * R), O.counts_direct(buckets, gid, B, q))


@pytest.mark.parametrize("seed", range(10))
def test_alg3_equals_closed_key_wide_counts(seed):
    """Counts above 255 (L up to 4095 tables): the literal Alg. 3 and the
    closed key still agree, so 16-bit counts order cells exactly."""
    rng = np.random.default_rng(1000 + seed)
    N = int(rng.integers(1, 65))
    R = int(rng.integers(1, 5))
    B = int(rng.integers(1, N + 1))
    L = int(rng.choice([256, 300, 1024, 4095]))
    gid = O.groups(WL.group_permutations(seed, R, N), B)
    moff, mem = O.members(gid, B)
    cnt = rng.integers(0, L + 1, size=B * R).astype(np.uint16)
    cnt[rng.integers(0, B * R)] = L
    for k in (1, 3, N):
        for t_min in (1, 256, L):
            ids, sc, n = O.alg3(cnt, moff, mem, N, R, B, k=k, t_min=t_min)
            e_ids, e_sc = closed_key_order(cnt, gid, B, k, t_min)
            assert ids[:n].tolist() == e_ids and sc[:n].tolist() == e_sc


def test_counts_wide_equal_direct_definition():
    """L = 300 tables: the reverse-index walk and the index-free definition
    give the same counts, above 255 where every table collides."""
    seed, N, L, K, R, B = 5, 200, 300, 1, 2, 10
    rng = np.random.default_rng(seed)
    buckets = rng.integers(0, 4, size=(N, L)).astype(np.uint32)   # 2-bit buckets: dense collisions
    gid = O.groups(WL.group_permutations(seed, R, N), B)
    off, cells = O.build_csr(buckets, gid, B, 2)
    for i in range(5):
        qb = buckets[i]
        c1 = O.counts(off, cells, L, 2, qb, B * R)
        c2 = O.counts_direct(buckets, gid, B, qb)
        assert np.array_equal(c1, c2)
        assert c1.max() == L and c1.dtype == np.uint16


# ------------------------------------------------------------ other designs
#
# Sec. 3.1: the framework takes any non-adaptive design. With one test per
# point and repetition given outright, groups are of any size (some empty),
# and the count, CSR and Alg. 3 steps must still follow their definitions.

def test_design_groups_by_hand():
    g = np.array([[2, 0, 2, 2], [1, 1, 0, 1]], np.uint16)      # R = 2, n = 4, B = 3
    gid = O.design_groups(g, B=3)
    assert gid.tolist() == [[2, 1], [0, 1], [2, 0], [2, 1]]
    moff, mem = O.members(gid, 3)
    # repetition 0: group 0 = {1}, group 1 = {}, group 2 = {0, 2, 3}
    assert moff[0].tolist() == [0, 1, 1, 4] and mem[0, :4].tolist() == [1, 0, 2, 3]
    with pytest.raises(ValueError):
        O.design_groups(np.array([[0, 3]], np.uint16), B=3)


def test_design_equal_to_alg1_gives_the_same_index():
    # Alg. 1's own groups, given outright, rebuild the permutation's index
    idx, pts = _dense_index(6, 300, 16, 3, 20, 8, 6)
    perm_gid = idx.gid
    jdx = O.OracleIndex("cosine", 3, 20, 8, 6, 6, srp_w=idx.srp_w)
    jdx.build_groups(pts, perm_gid.T)
    assert np.array_equal(jdx.off, idx.off) and np.array_equal(jdx.cells, idx.cells)
    q = pts[::13]
    assert all(np.array_equal(a, b) for a, b in zip(jdx.query(q, 20), idx.query(q, 20)))


@pytest.mark.parametrize("seed", range(6))
def test_irregular_design_counts_equal_brute_force(seed):
    N, L, R, B, W = 150, 6, 3, 12, 3
    rng = np.random.default_rng(200 + seed)
    buckets = rng.integers(0, 1 << W, size=(N, L), dtype=np.uint64).astype(np.uint32)
    gid = O.design_groups(WL.random_design(seed, R, N, B), B)
    assert np.any(np.bincount(gid[:, 0], minlength=B) != N // B)   # not doubly regular
    off, cells = O.build_csr(buckets, gid, B, W)
    q = rng.integers(0, 1 << W, size=L).astype(np.uint32)
    cnt = O.counts(off, cells, L, W, q, B * R)
    brute = np.zeros(B * R, np.int64)
    for r in range(R):
        for b in range(B):
            mem = np.nonzero(gid[:, r] == b)[0]
            for l in range(L):
                brute[r * B + b] += bool(np.any(buckets[mem, l] == q[l]))
    assert np.array_equal(cnt.astype(np.int64), brute)


@pytest.mark.parametrize("seed", range(30))
def test_irregular_design_alg3_equals_closed_key(seed):
    rng = np.random.default_rng(500 + seed)
    N = int(rng.integers(1, 65))
    R = int(rng.integers(1, 5))
    B = int(rng.integers(1, N + 3))            # B may exceed N: empty groups
    L = int(rng.integers(1, 9))
    if seed % 5 == 0:
        g = np.zeros((R, N), np.uint16)        # every point in one group
    else:
        g = WL.random_design(seed, R, N, B)
    gid = O.design_groups(g, B)
    moff, mem = O.members(gid, B)
    cnt = rng.integers(0, L + 1, size=B * R).astype(np.uint8)
    for k in (1, 3, N, N + 5):
        for t_min in (1, 2, L):
            ids, sc, n = O.alg3(cnt, moff, mem, N, R, B, k=k, t_min=t_min)
            e_ids, e_sc = closed_key_order(cnt, gid, B, k, t_min)
            assert ids[:n].tolist() == e_ids and sc[:n].tolist() == e_sc
            assert np.all(ids[n:] == 0xFFFFFFFF)


def test_insert_groups_equals_build_of_union():
    pts, _ = WL.gaussian_mixture(8, 500, 12, 10, 0.1)
    w = WL.srp_projections(8, 5 * 7, 12)
    g = WL.random_design(8, 2, 500, 25)
    a = O.OracleIndex("cosine", 2, 25, 5, 7, 7, srp_w=w)
    a.build_groups(pts, g)
    b = O.OracleIndex("cosine", 2, 25, 5, 7, 7, srp_w=w)
    b.build_groups(pts[:200], g[:, :200])
    b.insert_groups(pts[200:], g[:, 200:])
    assert np.array_equal(a.off, b.off) and np.array_equal(a.cells, b.cells)
    assert np.array_equal(a.moff, b.moff) and np.array_equal(a.mem, b.mem)
