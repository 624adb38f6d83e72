"""The two-term BF16 split of the tensor-core SRP form, checked on the CPU
against exact arithmetic (no GPU).

x = x1 + x2 + e with x1 = bf16(x) and x2 = bf16(x - x1), both rounded to
nearest even. The form keeps x1*w1 + x1*w2 + x2*w1 and drops x2*w2 and
every term with e. Its sign margin charges the dropped part at most
3.1 * 2^-16 * |x| |w| per product, with |e| <= 2^-16 |x|. Below about
|x| = 2^-117 the second term x - x1 is subnormal, and bf16 rounding there
has an absolute floor: |e| <= 2^-16 |x| + 2^-134. The kernel's margin
carries that floor in its underflow terms. These tests check the bounds on
random fp32 inputs over a wide exponent range, on values one unit either
side of bf16 rounding ties, and on subnormals.
Products of bf16 values and of fp32 values are exact in fp64 (16 and 48
significant bits), so the comparison is exact.
"""
import numpy as np
import pytest


def bf16_rne(x):
    """fp32 -> bf16 (kept in an fp32 container), round to nearest even."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split(x):
    x = np.asarray(x, np.float32)
    x1 = bf16_rne(x)
    r = (x - x1).astype(np.float32)             # exact: x1 is within a factor 2 of x
    x2 = bf16_rne(r)
    e = x.astype(np.float64) - x1.astype(np.float64) - x2.astype(np.float64)
    return x1, x2, e


def inputs(seed, n):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(1.0, 2.0, size=n)
    expo = rng.integers(-120, 120, size=n)
    sign = rng.choice([-1.0, 1.0], size=n)
    x = (sign * mant * np.exp2(expo.astype(np.float64))).astype(np.float32)
    # one unit either side of a bf16 tie, and exact ties
    u = rng.integers(0x00800000, 0x7F000000, size=n // 4, dtype=np.uint64).astype(np.uint32)
    tie = (u & 0xFFFF0000) | 0x8000
    near = np.concatenate([tie, tie + 1, tie - 1]).astype(np.uint32).view(np.float32)
    sub = (rng.integers(1, 1 << 23, size=n // 8, dtype=np.uint64).astype(np.uint32)).view(np.float32)
    return np.concatenate([x, near, sub, -near])


@pytest.mark.parametrize("seed", range(4))
def test_split_residual_bound(seed):
    x = inputs(seed, 40000)
    x1, x2, e = split(x)
    assert np.all(np.isfinite(x1)) and np.all(np.isfinite(x2))
    ax = np.abs(x.astype(np.float64))
    assert np.all(np.abs(e) <= 2.0 ** -16 * ax + 2.0 ** -134)
    # the relative bound alone holds where x - x1 stays a normal number
    normal = ax >= 2.0 ** -116
    assert np.all(np.abs(e[normal]) <= 2.0 ** -16 * ax[normal])
    assert np.any(np.abs(e[~normal]) > 2.0 ** -16 * ax[~normal])    # and the floor is needed below
    # the first term alone is within bf16's unit roundoff (8 significant bits):
    # |x - x1| <= 2^-8 |x|, so the residual's bound is 2^-8 * 2^-8 = 2^-16
    d1 = np.abs(x.astype(np.float64) - x1.astype(np.float64))
    assert np.all(d1 <= 2.0 ** -8 * ax + 2.0 ** -134)
    assert d1[normal].max() > 2.0 ** -9 * ax[normal][np.argmax(d1[normal] / ax[normal])]


@pytest.mark.parametrize("seed", range(4))
def test_dropped_terms_bound(seed):
    x = inputs(100 + seed, 30000)
    w = np.random.default_rng(200 + seed).permutation(inputs(300 + seed, 30000))[: x.size]
    # keep the products in range: both operands within 2^+-60
    keep = (np.abs(x) > 2.0 ** -60) & (np.abs(x) < 2.0 ** 60) & (np.abs(w) > 2.0 ** -60) & (np.abs(w) < 2.0 ** 60)
    x, w = x[keep], w[keep]
    x1, x2, _ = split(x)
    w1, w2, _ = split(w)
    exact = x.astype(np.float64) * w.astype(np.float64)
    kept = (x1.astype(np.float64) * w1 + x1.astype(np.float64) * w2 + x2.astype(np.float64) * w1)
    dropped = np.abs(exact - kept)
    assert np.all(dropped <= 3.1 * 2.0 ** -16 * np.abs(x.astype(np.float64)) * np.abs(w.astype(np.float64)))
    # and the bound is not loose by orders of magnitude: the worst case uses a fair part of it
    ratio = dropped / np.maximum(np.abs(x.astype(np.float64) * w.astype(np.float64)), 1e-300)
    assert ratio.max() > 2.0 ** -20


def test_bf16_rne_by_hand():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa (1) wins
    assert bf16_rne(np.float32(1 + 2 ** -8)) == np.float32(1.0)
    # 1 + 3 * 2^-8 is a tie between 1 + 2^-7 and 1 + 2^-6: even mantissa wins
    assert bf16_rne(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)
    # just above the first tie rounds up
    assert bf16_rne(np.float32(1 + 2 ** -8 + 2 ** -20)) == np.float32(1 + 2 ** -7)
