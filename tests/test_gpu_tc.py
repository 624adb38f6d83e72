"""Tensor-core precision form (tcgen05, two-term bf16 split): the sign bits
must equal the oracle's exact signs; the projection before its sign must be
within 2e-2 of the fp64 oracle relative to ||w|| ||x|| (the tolerance stated
for BF16); queries through such an index equal the oracle's."""
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


def tc_bound(d):
    """Relative first-pass bound on |p~ - w.x| / (||x|| ||w||) (blocks of 64)."""
    u, up = 2.0 ** -24, 2.0 ** -22
    g = lambda m, uu: m * uu / (1 - m * uu)
    q = (1 + 2.0 ** -8) ** 2
    m = (d + 63) // 64
    return ((g(64, up) + 2.0 ** -7 * g(128, up)) * q + g(2 * m, u) * (1 + g(64, up)) * (1 + 2.0 ** -7) * q
            + 3.1 * 2.0 ** -16)


@pytest.mark.parametrize("n,d,L,K", [(300, 128, 16, 12), (130, 200, 5, 7), (1000, 4096, 8, 16), (1, 64, 2, 29)])
def test_tc_codes_exact_and_projection_tolerance(F, n, d, L, K):
    pts, _ = WL.gaussian_mixture(60 + d, n, d, 20, 0.1)
    w = WL.srp_projections(60 + d, L * K, d)
    for i in range(0, n, 7):                      # planted near-zero projections
        j = i % (L * K)
        pts[i, -1] = np.float32(-float(np.dot(w[j, :-1].astype(np.float64), pts[i, :-1])) / float(w[j, -1]))
    if n > 3:
        pts[3] = 0.0
    ix = F.Index("cosine", 1, 1, L, K, capacity=n, params=w, dim=d, precision=F.PREC_BF16X2)
    codes, _, proj = ix.hash(pts, proj=True)
    ocodes, oproj, _ = O.srp_codes(pts, w, L, K, want_proj=True)
    assert np.array_equal(u32(codes), ocodes)
    scale = np.linalg.norm(pts.astype(np.float64), axis=1)[:, None] * \
        np.linalg.norm(w.astype(np.float64), axis=1)[None, :]
    rel = np.abs(proj.astype(np.float64) - oproj) / np.maximum(scale, 1e-300)
    assert rel.max() <= 2e-2
    # the first-pass error bound the kernel decides signs with (64-wide k-blocks
    # drained into fp32, two-term split): every projection must sit inside it
    assert np.all(np.abs(proj.astype(np.float64) - oproj) <= tc_bound(d) * scale * 1.01 + 1e-30)
    cnt = ix.hash_counters()
    assert cnt["undecided"] >= n // 7   # planted projections were not decided by the tensor cores
    assert cnt["compensated"] == cnt["undecided"]
    assert cnt["fp64"] <= cnt["undecided"] and cnt["flips"] <= cnt["undecided"]
    # same codes as the fp32 path
    jx = F.Index("cosine", 1, 1, L, K, capacity=n, params=w, dim=d)
    fc, _, _ = jx.hash(pts)
    assert np.array_equal(u32(fc), u32(codes))


def test_tc_device_buffers_and_query(F):
    import torch
    N, d, R, B, L, K = 4000, 256, 3, 50, 12, 10
    pts, _ = WL.gaussian_mixture(70, N, d, 30, 0.1)
    q, _ = WL.noisy_queries(70, pts, 120, 0.05)
    w = WL.srp_projections(70, L * K, d)
    perm = WL.group_permutations(70, R, N)
    ix = F.Index("cosine", R, B, L, K, capacity=N, params=w, dim=d, precision=F.PREC_BF16X2)
    ix.build(torch.from_numpy(pts).cuda(), torch.from_numpy(perm.view(np.int32)).cuda())
    ids, sc = ix.query(torch.from_numpy(q).cuda(), 10)
    torch.cuda.synchronize()
    o = O.OracleIndex("cosine", R, B, L, K, K, srp_w=w)
    o.build(pts, perm)
    oids, osc = o.query(q, 10)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc.cpu().numpy(), osc)
    assert np.array_equal(ix.export()["cells"], o.cells)


def test_tc_rejects_unaligned_dim(F):
    w = WL.srp_projections(71, 4 * 4, 13)
    with pytest.raises(F.FlinngError) as e:
        F.Index("cosine", 1, 1, 4, 4, capacity=10, params=w, dim=13, precision=F.PREC_BF16X2)
    assert e.value.code == F.ERR_INVALID_ARG


def test_tc_flag_and_flip_rates_embedding_shape(F):
    """YFCC-shaped rows (ReLU of a Gaussian mixture, d = 4096): codes exact, the
    share of projections left to the re-checks small, flips counted."""
    import torch
    d, L, K, n = 4096, 64, 16, 2000
    seed = WL.config_seed(4)
    w = WL.srp_projections(seed, L * K, d)
    x = WL.embed_points(seed, np.arange(n), d, 1000, 0.1)
    ix = F.Index("cosine", 1, 1, L, K, capacity=n, params=w, dim=d, precision=F.PREC_BF16X2)
    codes, _, _ = ix.hash(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ocodes = O.srp_codes(x, w, L, K)
    assert np.array_equal(u32(codes), ocodes)
    cnt = ix.hash_counters()
    rate = cnt["undecided"] / (n * L * K)
    assert 0 < rate < 0.01, cnt
    assert cnt["flips"] <= cnt["undecided"]
