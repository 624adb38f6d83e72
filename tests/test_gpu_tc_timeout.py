"""Failure path of the tensor-core SRP pipeline's bounded waits, made to run
out without any fault: with every pipeline wait limited to a single try
(flinng_set_tc_wait(idx, 0)), waits give up while the first copies are still
in flight; the kernel stops issuing work, waits with its normal limit for the
copies and MMAs it issued, frees its tensor memory and sets the index's
timeout flag. The call that synchronises returns FLINNG_ERR_TIMEOUT, so does
every later call on that index, and the context stays usable: another index
hashes exactly afterwards."""
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


@pytest.mark.parametrize("prec", ["bf16x2", "bf16", "fp8"])
def test_pipeline_wait_gives_up_and_reports(F, prec):
    p = {"bf16x2": F.PREC_BF16X2, "bf16": F.PREC_BF16, "fp8": F.PREC_FP8}[prec]
    d, L, K, n = 256, 8, 16, 600
    pts, _ = WL.gaussian_mixture(95, n, d, 20, 0.1)
    w = WL.srp_projections(95, L * K, d)
    ocodes = O.srp_codes(pts, w, L, K)
    ix = F.Index("cosine", 1, 1, L, K, capacity=n, params=w, dim=d, precision=p)
    codes, _, _ = ix.hash(pts)
    assert np.array_equal(np.asarray(codes).view(np.uint32), ocodes)
    ix.set_tc_wait(0)                       # every pipeline wait: a single try
    with pytest.raises(F.FlinngError) as e:
        ix.hash(pts)                        # host buffers: the call synchronises
    assert e.value.code == F.ERR_TIMEOUT
    ix.set_tc_wait(2 ** 64 - 1)             # the default limit again; the flag stays
    with pytest.raises(F.FlinngError) as e:
        ix.hash(pts)
    assert e.value.code == F.ERR_TIMEOUT
    with pytest.raises(F.FlinngError) as e:
        ix.query(pts[:10], 5)
    assert e.value.code == F.ERR_TIMEOUT
    with pytest.raises(F.FlinngError) as e:
        ix.hash_counters()
    assert e.value.code == F.ERR_TIMEOUT
    ix.close()
    # the context is intact: a fresh index of the same form hashes exactly
    jx = F.Index("cosine", 1, 1, L, K, capacity=n, params=w, dim=d, precision=p)
    codes2, _, _ = jx.hash(pts)
    assert np.array_equal(np.asarray(codes2).view(np.uint32), ocodes)
    jx.close()
