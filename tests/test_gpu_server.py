"""Serving form: continuous batching over two resident indices.

A Poisson trace of queries (k in {1, 10, 100}, uneven set sizes) against a
MinHash index and a cosine index, interleaved with insert batches. Every
served result must equal flinng_query run alone on a replica of its index at
the same version (inserts applied before the query ran), batches must have
overlapped in time (host clock, and CUDA events on the device), and admission
must respect the HBM budget.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2106_11565_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2106_11565_gb300 import _build, flinng
    _build.build()
    return flinng


def _make(F, seed):
    g = WL.genomic_reads(seed, 400_000, 6000, 400, 800)
    dp = WL.doph_params(seed, 32, 2)
    pts, _ = WL.gaussian_mixture(seed, 5000, 96, 40, 0.1)
    qd, _ = WL.noisy_queries(seed, pts, 600, 0.05)
    w = WL.srp_projections(seed, 8 * 12, 96)

    def new_pair():
        a = F.Index("jaccard", 2, 200, 32, 2, capacity=6000, params=dp, W=16)
        a.build((g["off"][:4001], g["elems"][:g["off"][4000]]), WL.group_permutations(seed, 2, 4000))
        b = F.Index("cosine", 3, 80, 8, 12, capacity=5000, params=w, dim=96)
        b.build(pts, WL.group_permutations(seed, 3, 5000))
        return a, b
    return g, dp, pts, qd, w, new_pair


def test_serving_matches_queries_alone(F):
    seed = 77
    g, dp, pts, qd, w, new_pair = _make(F, seed)
    ia, ib = new_pair()
    srv = F.Server(hbm_budget=ia.device_bytes + ib.device_bytes + (64 << 20), n_slots=4, max_batch=64,
                   k_max=100, max_batch_elems=1 << 18)
    a_id = srv.add_index(ia)
    b_id = srv.add_index(ib)
    assert srv.device_bytes <= ia.device_bytes + ib.device_bytes + (64 << 20)
    # a third index (about 200 MB for 2M points) does not fit the budget
    extra = F.Index("cosine", 3, 80, 8, 12, capacity=2_000_000, params=w, dim=96)
    assert extra.device_bytes > (64 << 20)
    with pytest.raises(F.FlinngError) as e:
        srv.add_index(extra)
    assert e.value.code == F.ERR_OOM

    rng = np.random.default_rng(seed)
    qoff, qel = g["q_off"], g["q_elems"]
    keep = []       # every buffer a request points to stays alive here
    trace = []      # (kind, payload, k, ctypes request)
    t = 0.0
    ins_first = 4000
    for i in range(1200):
        t += rng.exponential(20e-6)
        r = F.flinng_request()
        r.arrival_s, r.kind, r.k = t, F.REQ_QUERY, int(rng.choice([1, 10, 100]))
        if i % 2 == 0:
            j = int(rng.integers(0, 800))
            s_ = np.ascontiguousarray(qel[qoff[j]:qoff[j + 1]])
            if i % 50 == 0:
                s_ = np.ascontiguousarray(s_[: int(rng.integers(0, 3))])   # empty and tiny sets
            keep.append(s_)
            r.index, r.n, r.data = a_id, len(s_), s_.ctypes.data if len(s_) else None
            trace.append(("a", s_, r.k, r))
        else:
            v = np.ascontiguousarray(qd[int(rng.integers(0, 600))])
            keep.append(v)
            r.index, r.n, r.data = b_id, 0, v.ctypes.data
            trace.append(("b", v, r.k, r))
        if i in (300, 700):                               # insert batches into the MinHash index
            n = 1000
            off = (g["off"][ins_first:ins_first + n + 1] - g["off"][ins_first]).astype(np.uint64)
            el = np.ascontiguousarray(g["elems"][g["off"][ins_first]:g["off"][ins_first + n]])
            perm = WL.group_permutations(seed, 2, n, batch=ins_first)
            fp = F.flinng_points()
            fp.off, fp.elems = off.ctypes.data, el.ctypes.data
            keep += [off, el, perm, fp]
            ri = F.flinng_request()
            ri.arrival_s, ri.kind, ri.index, ri.n, ri.on_device = t, F.REQ_INSERT, a_id, n, 0
            ri.data = C.cast(C.pointer(fp), C.c_void_p)
            ri.perm = perm.ctypes.data
            trace.append(("ins", (off, el, perm), 0, ri))
            ins_first += n
    # an insert beyond capacity is refused, the index unchanged
    fp_big = F.flinng_points()
    rb = F.flinng_request()
    rb.arrival_s, rb.kind, rb.index, rb.n = t, F.REQ_INSERT, a_id, 5000
    rb.data = C.cast(C.pointer(fp_big), C.c_void_p)
    keep.append(fp_big)
    trace.append(("big", None, 0, rb))

    arr = (F.flinng_request * len(trace))()
    for i, e in enumerate(trace):
        arr[i] = e[3]
    ids, sc, res = srv.replay(arr)
    reqs_py = trace

    # the big insert: refused for capacity
    assert res[len(reqs_py) - 1].status == F.ERR_CAPACITY
    assert ia.size == 6000

    # each query equals the query alone on a replica at its version
    ra, rb_ = new_pair()
    versions = sorted({res[i].version for i, e in enumerate(reqs_py) if e[0] == "a"})
    inserts = [e[1] for e in reqs_py if e[0] == "ins"]
    applied = 0
    for v in versions:
        while applied < v:
            off, el, perm = inserts[applied]
            ra.insert((off, el), perm)
            applied += 1
        for i, e in enumerate(reqs_py):
            if e[0] == "a" and res[i].version == v:
                s = e[1]
                o = np.array([0, len(s)], np.uint64)
                rid, rsc = ra.query((o, s if len(s) else np.zeros(0, np.uint32)), 100,
                                    k=np.array([e[2]], np.uint32))
                assert np.array_equal(ids[i], rid[0]) and np.array_equal(sc[i], rsc[0])
    for i, e in enumerate(reqs_py):
        if e[0] == "b":
            rid, rsc = rb_.query(e[1][None, :], 100, k=np.array([e[2]], np.uint32))
            assert np.array_equal(ids[i], rid[0]) and np.array_equal(sc[i], rsc[0])
    # times are ordered and batches overlapped on the device
    qs = [i for i, e in enumerate(reqs_py) if e[0] in ("a", "b")]
    for i in qs:
        assert res[i].t_admit <= res[i].t_start <= res[i].t_done
    spans = {}
    for i in qs:
        b = res[i].batch
        s0, s1 = spans.get(b, (res[i].t_start, res[i].t_done))
        spans[b] = (min(s0, res[i].t_start), max(s1, res[i].t_done))
    sp = sorted(spans.values())
    assert any(sp[j + 1][0] < sp[j][1] for j in range(len(sp) - 1)), "no two batches were in flight together"
    # the same on the device clock: CUDA events on each batch's stream slot
    # (first copy in .. results out) show batches of different slots running
    # at once on the GPU
    dev = {}
    for i in qs:
        b = res[i].batch
        assert 0.0 <= res[i].d_start <= res[i].d_done, (res[i].d_start, res[i].d_done)
        assert res[i].slot < 4
        dev[b] = (res[i].d_start, res[i].d_done, res[i].slot)
    ds = sorted(dev.values())
    overlap = [(a, b) for a, b in zip(ds, ds[1:]) if b[0] < a[1] and b[2] != a[2]]
    assert overlap, "no two batches overlapped on the device"
    assert len({v[2] for v in dev.values()}) >= 2
    assert len({res[i].version for i, e in enumerate(reqs_py) if e[0] == "a"}) >= 2
    srv.close()
