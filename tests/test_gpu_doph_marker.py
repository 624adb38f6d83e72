"""DOPH bins whose minimum equals the empty marker: an element e* with
a e* + b = 2^32 - 1 (mod 2^32) hashes to the all-ones value, so its bin is
occupied although its minimum is the marker's value. The batched hash and the
fused query's per-CTA hash must treat that bin as occupied (no
densification), exactly as the oracle does; sets holding e* alone, with other
elements, and repeated."""
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


def marker_element(a: int, b: int) -> int:
    return ((0xFFFFFFFF - b) * pow(a, -1, 1 << 32)) % (1 << 32)


def test_marker_value_bins_are_occupied(F):
    R, B, L, K, W = 2, 16, 8, 4, 12
    dp = WL.doph_params(3, L, K)
    es = marker_element(dp["doph_a"], dp["doph_b"])
    assert (dp["doph_a"] * es + dp["doph_b"]) % (1 << 32) == 0xFFFFFFFF
    rng = np.random.default_rng(4)
    rows = [np.array([es], np.uint32), np.array([es, es], np.uint32)]
    for i in range(40):
        r = rng.choice(1 << 20, size=int(rng.integers(1, 60)), replace=False).astype(np.uint32)
        rows.append(np.concatenate([r, [es]]).astype(np.uint32) if i % 2 == 0 else r)
    off, el = WL.csr_from_rows(rows)
    ix = F.Index("jaccard", R, B, L, K, capacity=len(rows), params=dp, W=W)
    b, v, _ = ix.hash((off, el), values=True)
    ov = O.doph(off, el, L * K, dp["doph_a"], dp["doph_b"], dp["doph_seed"])
    assert (ov == 0xFFFFFFFF).any()                     # the marker value is a real bin minimum
    assert np.array_equal(v, ov)
    assert np.array_equal(b, O.minhash_buckets(ov, L, K, dp["bucket_a"], dp["bucket_c"], W))
    # the fused query hashes each query in its CTA: same answers as the oracle
    perm = WL.group_permutations(5, R, len(rows))
    ix.build((off, el), perm)
    o = O.OracleIndex("jaccard", R, B, L, K, W, doph=dp)
    o.build((off, el), perm)
    for mode in (F.QUERY_PLAIN, F.QUERY_FUSED):
        ix.set_query_mode(mode)
        ids, sc = ix.query((off, el), 10)
        oids, osc = o.query((off, el), 10)
        assert np.array_equal(ids.view(np.uint32), oids) and np.array_equal(sc, osc), mode
    ix.close()
