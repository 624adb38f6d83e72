"""Pins for the seeded generators shared by both sides (CPU only)."""
import os
from fractions import Fraction

import numpy as np

from paper_2106_11565_gb300 import workloads as WL

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox4x32_10_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = WL.philox4x32_10(*v[:6])
        assert [int(x) for x in out] == v[6:]


def _round_fp32(x: Fraction) -> np.float32:
    """Correct fp32 rounding of an exact rational (ties to even), by search."""
    c = np.float32(float(x))
    cands = [np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))]
    return min(cands, key=lambda v: (abs(Fraction(float(v)) - x), int(np.float32(v).view(np.int32)) & 1))


def test_fma_f32_tie_cases_by_hand():
    # a*b = 2^16 - 2^-30, c = 2^40 + 2^17: the exact sum lies just below the
    # fp32 midpoint 2^40 + 3*2^16, which fp64 rounds onto; ties-to-even of the
    # fp64 value would go up to 2^40 + 2^18, the correct result is 2^40 + 2^17
    a = np.float32(2 ** 8 * (1 + 2 ** -23))
    b = np.float32(2 ** 8 * (1 - 2 ** -23))
    c = np.float32(2 ** 40 + 2 ** 17)
    assert WL.fma_f32(a, b, c) == np.float32(2 ** 40 + 2 ** 17)
    assert np.float32(np.float64(a) * np.float64(b) + np.float64(c)) == np.float32(2 ** 40 + 2 ** 18)
    # mirrored: exact sum just above a midpoint that ties-to-even rounds down
    b2 = np.float32(2 ** 8 * (1 + 2 ** -23))          # a*b = 2^16 + 2^-6 + 2^-30
    c2 = np.float32(2 ** 40)
    x = Fraction(float(a)) * Fraction(float(b2)) + Fraction(float(c2))
    assert WL.fma_f32(a, b2, c2) == _round_fp32(x)


def test_fma_f32_matches_rationals():
    rng = np.random.default_rng(4)
    a = (rng.standard_normal(4000) * 2.0 ** rng.integers(-20, 20, 4000)).astype(np.float32)
    b = (rng.standard_normal(4000) * 2.0 ** rng.integers(-20, 20, 4000)).astype(np.float32)
    c = (rng.standard_normal(4000) * 2.0 ** rng.integers(-20, 20, 4000)).astype(np.float32)
    r = WL.fma_f32(a, b, c)
    for i in range(0, 4000, 7):
        x = Fraction(float(a[i])) * Fraction(float(b[i])) + Fraction(float(c[i]))
        assert r[i] == _round_fp32(x)


def test_embedding_stream_properties():
    seed, d = 11, 512
    x = WL.embed_points(seed, np.arange(64), d, 10, 0.1)
    assert x.dtype == np.float32 and x.shape == (64, d)
    assert np.all(x >= 0)                                   # ReLU
    assert 0.35 < np.mean(x == 0) < 0.65                    # about half zeros
    # any row regenerates alone, identically
    assert np.array_equal(WL.embed_points(seed, [37], d, 10, 0.1)[0], x[37])
    # points of the same centre are close (cosine), others are not
    lab = WL.embed_labels(seed, np.arange(64), 10)
    xn = x / np.linalg.norm(x, axis=1, keepdims=True)
    s = xn @ xn.T
    same = lab[:, None] == lab[None, :]
    assert s[same & ~np.eye(64, dtype=bool)].mean() > 0.95 > s[~same].mean()
    # Irwin-Hall normals: mean 0, variance 1 (sum of 4 uniforms, scaled)
    z = WL.irwin_hall(*WL.philox4x32_10(np.arange(200000), 7, 0, 0xC0, 1, 2))
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
