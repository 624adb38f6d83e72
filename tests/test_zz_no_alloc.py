"""flinng_query_noalloc, the query entry point for callers that cannot
allocate device memory (fixed HBM budgets, allocation-free serving loops,
caller-owned memory pools): it must return exactly what flinng_query returns,
call after call, although every call reuses the same fixed scratch array.

Called through the C ABI with device buffers, on two calls in a row with
different batches, for a MinHash index and a cosine index. Integer outputs,
so the comparison is exact (the tolerance of all top-k parity tests).
"""
import ctypes as C

import numpy as np
import pytest

from paper_2106_11565_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _noalloc(F, ix, pts_dev, nq, k_max):
    import torch
    fp, n, dev, keep = ix._points(pts_dev)
    assert dev == 1 and n == nq
    ids = torch.full((nq, k_max), 7, dtype=torch.int32, device="cuda")
    sc = torch.full((nq, k_max), 7, dtype=torch.int16, device="cuda")
    rc = F.load().flinng_query_noalloc(ix.h, C.byref(fp), nq, None, k_max, ids.data_ptr(), sc.data_ptr())
    assert rc == F.OK, F.load().flinng_last_error()
    torch.cuda.synchronize()
    return ids.cpu().numpy(), sc.cpu().numpy()


def _sets_dev(off, el):
    import torch
    return (torch.from_numpy(off.view(np.int64)).cuda(), torch.from_numpy(el.view(np.int32)).cuda())


def test_noalloc_matches_flinng_query_on_consecutive_calls():
    import torch
    from paper_2106_11565_gb300 import _build
    from paper_2106_11565_gb300 import flinng as F
    _build.build()

    # MinHash index over genomic reads
    g = WL.genomic_reads(31, 200_000, 3000, 300, 300)
    dp = WL.doph_params(31, 32, 2)
    ix = F.Index("jaccard", 2, 300, 32, 2, capacity=3000, params=dp, W=16)
    ix.build((g["off"], g["elems"]), WL.group_permutations(31, 2, 3000))
    qoff, qel = g["q_off"], g["q_elems"]
    batches = [(0, 200), (120, 300)]
    for lo, hi in batches:                       # two calls in a row, different batches
        off = (qoff[lo:hi + 1] - qoff[lo]).astype(np.uint64)
        el = np.ascontiguousarray(qel[qoff[lo]:qoff[hi]])
        ids, sc = _noalloc(F, ix, _sets_dev(off, el), hi - lo, 50)
        ref_ids, ref_sc = ix.query(_sets_dev(off, el), 50)
        torch.cuda.synchronize()
        assert np.array_equal(ids, ref_ids.cpu().numpy())
        assert np.array_equal(sc, ref_sc.cpu().numpy())

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
    fp, n, dev, keep = ix._points(_sets_dev(off, el))
    out = torch.empty((big, 1), dtype=torch.int32, device="cuda")
    rc = F.load().flinng_query_noalloc(ix.h, C.byref(fp), big, None, 1, out.data_ptr(), None)
    assert rc == F.ERR_INVALID_ARG
    ix.close()
    cx.close()
