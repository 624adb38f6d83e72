"""Save and load of built indices: a loaded index returns the saved one's
export and queries bit for bit (and the oracle's), takes inserts like the
original, and a wrong or truncated file is refused."""
import os

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


def _sets(seed, N, nq, R, L, K):
    g = WL.genomic_reads(seed, ref_len=200_000, n_reads=N + 500, read_len=300, n_queries=nq)
    return g, WL.doph_params(seed, L, K)


@pytest.mark.parametrize("L,K,W,B,R", [(32, 2, 17, 1000, 2), (24, 1, 3, 60, 3), (300, 1, 12, 250, 2)])
def test_jaccard_save_load_insert(F, tmp_path, L, K, W, B, R):
    N, nq = 3000, 60
    g, dp = _sets(40 + L, N, nq, R, L, K)
    off, el = g["off"], g["elems"]
    pts = (off[:N + 1], el[:off[N]])
    q = (g["q_off"], g["q_elems"])
    perm = WL.group_permutations(40 + L, R, N)
    ix = F.Index("jaccard", R, B, L, K, capacity=N + 500, params=dp, W=W)
    ix.build(pts, perm)
    path = os.path.join(tmp_path, "ix.flinng")
    ix.save(path)
    jx = F.Index.load(path)
    assert (jx.metric, jx.R, jx.B, jx.L, jx.K, jx.W) == ("jaccard", R, B, L, K, W)
    a, b = ix.export(), jx.export()
    for key in ("off", "cells", "gid"):
        assert np.array_equal(a[key], b[key])
    for mode in (0, 1):
        ix.set_query_mode(mode)
        jx.set_query_mode(mode)
        i1, s1 = ix.query(q, 40)
        i2, s2 = jx.query(q, 40)
        assert np.array_equal(u32(i1), u32(i2)) and np.array_equal(s1, s2)
    o = O.OracleIndex("jaccard", R, B, L, K, W, doph=dp)
    o.build(pts, perm)
    oi, os_ = o.query(q, 40)
    assert np.array_equal(u32(i2), oi) and np.array_equal(s2, os_)
    # an insert into the loaded index equals the same insert into the original
    ins = (off[N:N + 501] - off[N], el[off[N]:off[N + 500]])
    iperm = WL.group_permutations(41 + L, R, 500, batch=N)
    ix.insert(ins, iperm)
    jx.insert(ins, iperm)
    i1, s1 = ix.query(q, 40)
    i2, s2 = jx.query(q, 40)
    assert np.array_equal(u32(i1), u32(i2)) and np.array_equal(s1, s2)
    assert jx.size == N + 500


@pytest.mark.parametrize("precision", [0, 1])
def test_cosine_save_load(F, tmp_path, precision):
    N, d, R, B, L, K = 4000, 128, 3, 100, 16, 12
    pts, _ = WL.gaussian_mixture(81, N, d, 60, 0.1)
    q, _ = WL.noisy_queries(81, pts, 100, 0.05)
    w = WL.srp_projections(81, L * K, d)
    perm = WL.group_permutations(81, R, N)
    ix = F.Index("cosine", R, B, L, K, capacity=N, params=w, dim=d, precision=precision)
    ix.build(pts, perm)
    path = os.path.join(tmp_path, "c.flinng")
    ix.save(path)
    jx = F.Index.load(path)
    i1, s1 = ix.query(q, 10)
    i2, s2 = jx.query(q, 10)
    assert np.array_equal(u32(i1), u32(i2)) and np.array_equal(s1, s2)
    c1, _, _ = ix.hash(q)
    c2, _, _ = jx.hash(q)
    assert np.array_equal(u32(c1), u32(c2))


def test_load_refuses_bad_files(F, tmp_path):
    bad = os.path.join(tmp_path, "bad")
    with open(bad, "wb") as f:
        f.write(b"not an index at all, just bytes" * 4)
    with pytest.raises(F.FlinngError):
        F.Index.load(bad)
    with pytest.raises(F.FlinngError):
        F.Index.load(os.path.join(tmp_path, "missing"))
    # a truncated file
    w = WL.srp_projections(3, 4 * 4, 8)
    ix = F.Index("cosine", 1, 4, 4, 4, capacity=32, params=w, dim=8)
    ix.build(np.random.default_rng(0).standard_normal((32, 8)).astype(np.float32), WL.group_permutations(3, 1, 32))
    good = os.path.join(tmp_path, "good")
    ix.save(good)
    data = open(good, "rb").read()
    cut = os.path.join(tmp_path, "cut")
    with open(cut, "wb") as f:
        f.write(data[: len(data) // 2])
    with pytest.raises(F.FlinngError):
        F.Index.load(cut)
    assert np.array_equal(F.Index.load(good).export()["cells"], ix.export()["cells"])
