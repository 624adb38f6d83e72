"""Single-term tensor-core precision forms (FLINNG_PREC_BF16: one bf16 term per
operand; FLINNG_PREC_FP8: E4M3 with a power-of-two scale per row), both with
fp32 accumulation and an a-posteriori margin from each row's quantisation
residual. The sign bits must equal the oracle's exact signs; the projection
before its sign must stay within a worst-case bound derived here from the
formats alone (independent of the kernel's own margin), and within 2e-2 of the
fp64 oracle relative to ||w|| ||x|| (the tolerance stated for BF16 and FP8)
wherever the dimension is large enough for the FP8 rounding errors to average;
queries through such an index equal the oracle's."""
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


def worst_case_error(x, w, form):
    """Bound on |p~ - w.x| per (row, projection) from the formats alone:
    bf16 rounds each value within 2^-8 of itself; E4M3 within 2^-4, except
    values flushed to 0, each below 2^-6 s with s <= max|x| / 224; plus the
    fp32 accumulation over k-blocks (four units per product) and underflow."""
    x = x.astype(np.float64)
    w = w.astype(np.float64)
    nx = np.linalg.norm(x, axis=1)
    nw = np.linalg.norm(w, axis=1)
    d = x.shape[1]
    if form == "bf16":
        ex, ew = 2.0 ** -8 * nx, 2.0 ** -8 * nw
        kb = 64
    else:
        sx = np.abs(x).max(axis=1) / 224.0
        sw = np.abs(w).max(axis=1) / 224.0
        ex = 2.0 ** -4 * nx + np.sqrt(d) * 2.0 ** -6 * sx
        ew = 2.0 ** -4 * nw + np.sqrt(d) * 2.0 ** -6 * sw
        kb = 128
    g = lambda m, u: m * u / (1 - m * u)
    m = -(-d // kb)
    acc = g(kb, 2.0 ** -22) + g(m, 2.0 ** -24) * (1 + g(kb, 2.0 ** -22))
    res = nx[:, None] * ew[None, :] + ex[:, None] * nw[None, :] + 3 * ex[:, None] * ew[None, :]
    return res + acc * (nx + ex)[:, None] * (nw + ew)[None, :] + 1e-30


@pytest.mark.parametrize("form", ["bf16", "fp8"])
@pytest.mark.parametrize("n,d,L,K", [(300, 128, 16, 12), (130, 208, 5, 7), (1000, 4096, 8, 16), (1, 64, 2, 29),
                                     (257, 16, 3, 9)])
def test_single_term_codes_exact_and_projection_bounds(F, form, n, d, L, K):
    prec = F.PREC_BF16 if form == "bf16" else F.PREC_FP8
    pts, _ = WL.gaussian_mixture(80 + d, n, d, 20, 0.1)
    w = WL.srp_projections(80 + d, L * K, d)
    for i in range(0, n, 7):                      # planted near-zero projections
        j = i % (L * K)
        pts[i, -1] = np.float32(-float(np.dot(w[j, :-1].astype(np.float64), pts[i, :-1])) / float(w[j, -1]))
    if n > 3:
        pts[3] = 0.0                              # all-zero row (scale 1, every sign exact)
    if n > 5:
        pts[5, ::2] *= np.float32(1e-4)           # wide range inside one row (FP8 flushes its small half)
    ix = F.Index("cosine", 1, 1, L, K, capacity=n, params=w, dim=d, precision=prec)
    codes, _, proj = ix.hash(pts, proj=True)
    ocodes, oproj, _ = O.srp_codes(pts, w, L, K, want_proj=True)
    assert np.array_equal(u32(codes), ocodes)
    err = np.abs(proj.astype(np.float64) - oproj)
    assert np.all(err <= worst_case_error(pts, w, form) * 1.01)
    scale = np.linalg.norm(pts.astype(np.float64), axis=1)[:, None] * \
        np.linalg.norm(w.astype(np.float64), axis=1)[None, :]
    rel = err / np.maximum(scale, 1e-300)
    if form == "bf16" or d >= 128:
        assert rel.max() <= 2e-2
    cnt = ix.hash_counters()
    assert cnt["undecided"] >= n // 7            # planted projections were not decided by the tensor cores
    assert cnt["compensated"] == cnt["undecided"]
    assert cnt["fp64"] <= cnt["undecided"] and cnt["flips"] <= cnt["undecided"]
    # same codes as the fp32 path
    jx = F.Index("cosine", 1, 1, L, K, capacity=n, params=w, dim=d)
    fc, _, _ = jx.hash(pts)
    assert np.array_equal(u32(fc), u32(codes))


@pytest.mark.parametrize("form", ["bf16", "fp8"])
def test_single_term_index_query(F, form):
    import torch
    prec = F.PREC_BF16 if form == "bf16" else F.PREC_FP8
    N, d, R, B, L, K = 4000, 256, 3, 50, 12, 10
    pts, _ = WL.gaussian_mixture(90, N, d, 30, 0.1)
    q, _ = WL.noisy_queries(90, pts, 120, 0.05)
    w = WL.srp_projections(90, L * K, d)
    perm = WL.group_permutations(90, R, N)
    ix = F.Index("cosine", R, B, L, K, capacity=N, params=w, dim=d, precision=prec)
    ix.build(torch.from_numpy(pts).cuda(), torch.from_numpy(perm.view(np.int32)).cuda())
    ids, sc = ix.query(torch.from_numpy(q).cuda(), 10)
    torch.cuda.synchronize()
    o = O.OracleIndex("cosine", R, B, L, K, K, srp_w=w)
    o.build(pts, perm)
    oids, osc = o.query(q, 10)
    assert np.array_equal(u32(ids), oids) and np.array_equal(sc.cpu().numpy(), osc)
    assert np.array_equal(ix.export()["cells"], o.cells)


def test_single_term_rejects_unaligned_dim(F):
    w = WL.srp_projections(91, 4 * 4, 24)
    with pytest.raises(F.FlinngError) as e:        # FP8 rows are 16-byte multiples
        F.Index("cosine", 1, 1, 4, 4, capacity=10, params=w, dim=24, precision=F.PREC_FP8)
    assert e.value.code == F.ERR_INVALID_ARG
    w = WL.srp_projections(91, 4 * 4, 12)
    with pytest.raises(F.FlinngError) as e:
        F.Index("cosine", 1, 1, 4, 4, capacity=10, params=w, dim=12, precision=F.PREC_BF16)
    assert e.value.code == F.ERR_INVALID_ARG


def test_single_term_embedding_shape_shares(F):
    """YFCC-shaped rows (ReLU of a Gaussian mixture, d = 4096): codes exact in
    both forms; the share of projections inside the margin is reported by the
    counters and is larger for FP8 than for BF16, as the formats' precisions
    say; flips are counted."""
    import torch
    d, L, K, n = 4096, 64, 16, 1000
    seed = WL.config_seed(4)
    w = WL.srp_projections(seed, L * K, d)
    x = WL.embed_points(seed, np.arange(n), d, 1000, 0.1)
    ocodes = O.srp_codes(x, w, L, K)
    share = {}
    for form, prec in (("bf16", F.PREC_BF16), ("fp8", F.PREC_FP8)):
        ix = F.Index("cosine", 1, 1, L, K, capacity=n, params=w, dim=d, precision=prec)
        codes, _, _ = ix.hash(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(u32(codes), ocodes), form
        cnt = ix.hash_counters()
        share[form] = cnt["undecided"] / (n * L * K)
        assert cnt["flips"] <= cnt["undecided"]
        ix.close()
    assert 0 < share["bf16"] < share["fp8"] <= 1.0, share
