"""flinng_query_noalloc, the query entry point for callers that cannot
allocate device memory (fixed HBM budgets, allocation-free serving loops,
caller-owned memory pools): it must return exactly what flinng_query returns,
call after call, although every call reuses the same fixed scratch array, and
it must allocate nothing, even for a batch larger than any the index has seen.

Called through the C ABI with device buffers, on two calls in a row with
different batches, for a MinHash index, an fp32 cosine index and a BF16X2
(tensor-core) cosine index. Integer outputs, so the comparison is exact (the
tolerance of all top-k parity tests).
"""
import ctypes as C

import numpy as np
import pytest

from paper_2106_11565_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _call(F, ix, pts_dev, nq, k_max, ids, sc):
    fp, n, dev, keep = ix._points(pts_dev)
    assert dev == 1 and n == nq
    return F.load().flinng_query_noalloc(ix.h, C.byref(fp), nq, None, k_max, ids.data_ptr(),
                                         None if sc is None else sc.data_ptr())


def _noalloc(F, ix, pts_dev, nq, k_max):
    import torch
    ids = torch.full((nq, k_max), 7, dtype=torch.int32, device="cuda")
    sc = torch.full((nq, k_max), 7, dtype=torch.int16, device="cuda")
    rc = _call(F, ix, pts_dev, nq, k_max, ids, sc)
    assert rc == F.OK, F.load().flinng_last_error()
    torch.cuda.synchronize()
    return ids.cpu().numpy(), sc.cpu().numpy()


def _sets_dev(off, el):
    import torch
    return (torch.from_numpy(off.view(np.int64)).cuda(), torch.from_numpy(el.view(np.int32)).cuda())


def _slice_sets(qoff, qel, lo, hi):
    off = (qoff[lo:hi + 1] - qoff[lo]).astype(np.uint64)
    return off, np.ascontiguousarray(qel[qoff[lo]:qoff[hi]])


def _lib():
    from paper_2106_11565_gb300 import _build
    from paper_2106_11565_gb300 import flinng as F
    _build.build()
    return F


def test_noalloc_matches_flinng_query_on_consecutive_calls():
    import torch
    F = _lib()

    # MinHash index over genomic reads
    g = WL.genomic_reads(31, 200_000, 3000, 300, 300)
    dp = WL.doph_params(31, 32, 2)
    ix = F.Index("jaccard", 2, 300, 32, 2, capacity=3000, params=dp, W=16)
    ix.build((g["off"], g["elems"]), WL.group_permutations(31, 2, 3000))
    qoff, qel = g["q_off"], g["q_elems"]
    for lo, hi in [(0, 200), (120, 300)]:        # two calls in a row, different batches
        off, el = _slice_sets(qoff, qel, lo, hi)
        ids, sc = _noalloc(F, ix, _sets_dev(off, el), hi - lo, 50)
        ref_ids, ref_sc = ix.query(_sets_dev(off, el), 50)
        torch.cuda.synchronize()
        assert np.array_equal(ids, ref_ids.cpu().numpy())
        assert np.array_equal(sc, ref_sc.cpu().numpy())
        # both entry points leave the same hash counters (none for MinHash)
        assert ix.hash_stats() == (0, 0)

    # cosine index (exercises the sign re-check list in the fixed scratch)
    pts, _ = WL.gaussian_mixture(32, 2000, 64, 20, 0.1)
    q, _ = WL.noisy_queries(32, pts, 160, 0.05)
    q[::7, -1] = 0.0
    q[3] = 0.0                                   # all-zero query: every sign goes to the exact path
    w = WL.srp_projections(32, 8 * 10, 64)
    cx = F.Index("cosine", 3, 50, 8, 10, capacity=2000, params=w, dim=64)
    cx.build(pts, WL.group_permutations(32, 3, 2000))
    for lo, hi in [(0, 160), (40, 100)]:
        qd = torch.from_numpy(np.ascontiguousarray(q[lo:hi])).cuda()
        ids, sc = _noalloc(F, cx, qd, hi - lo, 20)
        ref_ids, ref_sc = cx.query(qd, 20)
        torch.cuda.synchronize()
        assert np.array_equal(ids, ref_ids.cpu().numpy())
        assert np.array_equal(sc, ref_sc.cpu().numpy())

    # batches beyond the fixed scratch are refused, not truncated
    big = 262144 // 32 + 1
    off = np.arange(big + 1, dtype=np.uint64)
    el = np.arange(big, dtype=np.uint32)
    out = torch.empty((big, 1), dtype=torch.int32, device="cuda")
    assert _call(F, ix, _sets_dev(off, el), big, 1, out, None) == F.ERR_INVALID_ARG
    ix.close()
    cx.close()


def test_noalloc_tensor_core_cosine_index():
    """A BF16X2 index keeps its split query rows and both re-check lists in
    the same fixed array; a batch whose tensor-core staging exceeds it is
    refused although it passes the bucket and fp32 limits."""
    import torch
    F = _lib()
    d, L, K = 64, 8, 10
    pts, _ = WL.gaussian_mixture(33, 3000, d, 30, 0.1)
    q, _ = WL.noisy_queries(33, pts, 300, 0.05)
    q[5] = 0.0
    q[::11, 0] = 0.0
    w = WL.srp_projections(33, L * K, d)
    tx = F.Index("cosine", 3, 60, L, K, capacity=3000, params=w, dim=d, precision=F.PREC_BF16X2)
    tx.build(torch.from_numpy(pts).cuda(), torch.from_numpy(WL.group_permutations(33, 3, 3000).view(np.int32)).cuda())
    for lo, hi in [(0, 300), (17, 150)]:
        qd = torch.from_numpy(np.ascontiguousarray(q[lo:hi])).cuda()
        ids, sc = _noalloc(F, tx, qd, hi - lo, 25)
        ref_ids, ref_sc = tx.query(qd, 25)
        torch.cuda.synchronize()
        assert np.array_equal(ids, ref_ids.cpu().numpy())
        assert np.array_equal(sc, ref_sc.cpu().numpy())
    # about 4*d + 16*L*K + 4 = 1,540 bytes of staging per row: 4,000 rows need
    # ~6.2 MB > 5 MiB, while nq*L = 32,000 and nq*L*K*8 = 2.6 MB pass
    nq = 4000
    qd = torch.zeros((nq, d), dtype=torch.float32, device="cuda")
    out = torch.empty((nq, 1), dtype=torch.int32, device="cuda")
    assert _call(F, tx, qd, nq, 1, out, None) == F.ERR_INVALID_ARG
    assert "tensor-core scratch" in F.load().flinng_last_error().decode()
    tx.close()


def test_noalloc_allocates_nothing():
    """A batch larger than any before makes flinng_query grow its workspace
    (cudaMalloc); the same batch through flinng_query_noalloc leaves the
    index's device bytes and the device's free memory unchanged."""
    import torch
    F = _lib()
    n, nq, L = 600, 8000, 32                    # nq * L = 256,000 <= 262,144
    g = WL.genomic_reads(41, 100_000, n, 300, nq)
    dp = WL.doph_params(41, L, 2)
    perm = torch.from_numpy(WL.group_permutations(41, 2, n).view(np.int32)).cuda()

    def fresh():
        # W = 10: 32 x 1,024 slots, so the build's workspace stays far below
        # the 1 MB of query buckets a batch of 8,000 needs
        ix = F.Index("jaccard", 2, 64, L, 2, capacity=n, params=dp, W=10)
        ix.build(_sets_dev(g["off"], g["elems"]), perm)
        ix.set_query_mode(F.QUERY_PLAIN)
        torch.cuda.synchronize()
        return ix

    q_small = _sets_dev(*_slice_sets(g["q_off"], g["q_elems"], 0, 16))
    q_big = _sets_dev(g["q_off"], g["q_elems"])
    ids = torch.empty((nq, 10), dtype=torch.int32, device="cuda")
    sc = torch.empty((nq, 10), dtype=torch.int16, device="cuda")

    # flinng_query does grow for this batch (so the check below is meaningful)
    ref = fresh()
    b0 = ref.device_bytes
    ref_ids, ref_sc = ref.query(q_big, 10)
    torch.cuda.synchronize()
    assert ref.device_bytes > b0
    ref_ids, ref_sc = ref_ids.cpu().numpy(), ref_sc.cpu().numpy()
    ref.close()

    ix = fresh()
    # a small call first: loads the library's kernels and looks up the
    # scratch address, both of which may take device memory once
    assert _call(F, ix, q_small, 16, 10, ids, sc) == F.OK, F.load().flinng_last_error()
    torch.cuda.synchronize()
    b0 = ix.device_bytes
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert _call(F, ix, q_big, nq, 10, ids, sc) == F.OK, F.load().flinng_last_error()
        torch.cuda.synchronize()
        assert ix.device_bytes == b0
        assert torch.cuda.mem_get_info()[0] == free0
        assert np.array_equal(ids.cpu().numpy(), ref_ids)
        assert np.array_equal(sc.cpu().numpy(), ref_sc)
    ix.close()
