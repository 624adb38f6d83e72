"""Seeded synthetic workloads and random draws for FLINNG.

This module only draws random numbers and shapes synthetic data. It holds none
of FLINNG's arithmetic (no hashing of points into tables, no group assignment,
no decoding): the CUDA library and the CPU oracle both receive what is made here
as plain arrays.

Random quantities the method itself draws (Alg. 1's permutations, the LSH
functions' parameters) are produced here once from a seed and passed to both
sides as data.

Workload shapes follow the paper's datasets (Section 6, Table 1), which are not
available here; the stand-ins are:

* ``gaussian_mixture``: dense fp32 vectors (cosine / SRP workloads).
* ``genomic_reads``: reads sampled with substitutions from a random ACGT
  reference, turned into sets of hashed k-mers (RefSeq / PromethION-shaped).
* ``url_strings``: token strings from a Zipf vocabulary turned into sets of
  character 3-grams (URL-shaped).
"""
from __future__ import annotations

import numpy as np

U32 = np.uint32
U64 = np.uint64

CONFIG_SEED_BASE = 0xF11A6


def config_seed(config_number: int) -> int:
    """Seed used for workload ``C<config_number>``."""
    return CONFIG_SEED_BASE + int(config_number)


# --------------------------------------------------------------------------
# random draws of the method (passed to both sides as data)
# --------------------------------------------------------------------------

def srp_projections(seed: int, n_proj: int, dim: int) -> np.ndarray:
    """Gaussian projection rows for sign random projections, (n_proj, dim) fp32."""
    rng = np.random.default_rng([seed, 1])
    return rng.standard_normal((n_proj, dim)).astype(np.float32)


def doph_params(seed: int, L: int, K: int) -> dict:
    """Random keys for densified one-permutation MinHash and bucket combining.

    ``doph_a`` is odd, so the 32-bit affine map it defines is a bijection;
    ``bucket_a`` entries are odd 64-bit multipliers, ``bucket_c`` 64-bit offsets.
    """
    rng = np.random.default_rng([seed, 2])
    a = int(rng.integers(0, 1 << 32, dtype=np.uint64)) | 1
    b = int(rng.integers(0, 1 << 32, dtype=np.uint64))
    s = int(rng.integers(0, 1 << 63, dtype=np.uint64)) * 2 + int(rng.integers(0, 2))
    ba = rng.integers(0, 1 << 63, size=(L, K), dtype=np.uint64) * U64(2) + U64(1)
    bc = rng.integers(0, 1 << 63, size=(L,), dtype=np.uint64) * U64(2) + \
        rng.integers(0, 2, size=(L,), dtype=np.uint64)
    return {"doph_a": a, "doph_b": b, "doph_seed": s & ((1 << 64) - 1),
            "bucket_a": np.ascontiguousarray(ba, dtype=U64),
            "bucket_c": np.ascontiguousarray(bc, dtype=U64)}


def group_permutations(seed: int, R: int, n: int, batch: int = 0) -> np.ndarray:
    """R independent uniform permutations of [0, n), shape (R, n) uint32.

    ``batch`` distinguishes the permutations of successive insert batches.
    """
    rng = np.random.default_rng([seed, 3, batch])
    out = np.empty((R, n), dtype=U32)
    for r in range(R):
        out[r] = rng.permutation(n).astype(U32)
    return out


def random_design(seed: int, R: int, n: int, B: int, batch: int = 0) -> np.ndarray:
    """A non-adaptive design other than Alg. 1's doubly regular one: each
    point joins one group per repetition, drawn uniformly and independently
    (groups of Binomial(n, 1/B) size, some possibly empty). Shape (R, n)
    uint16: row r holds the points' groups in repetition r."""
    rng = np.random.default_rng([seed, 5, batch])
    return rng.integers(0, B, size=(R, n)).astype(np.uint16)


# --------------------------------------------------------------------------
# dense vectors
# --------------------------------------------------------------------------

def gaussian_mixture(seed: int, n: int, dim: int, n_centers: int,
                     sigma: float) -> tuple[np.ndarray, np.ndarray]:
    """Points = center + N(0, sigma^2 I) with centers ~ N(0, I); fp32 (n, dim)."""
    rng = np.random.default_rng([seed, 10])
    centers = rng.standard_normal((n_centers, dim))
    labels = rng.integers(0, n_centers, size=n)
    pts = centers[labels] + sigma * rng.standard_normal((n, dim))
    return pts.astype(np.float32), labels


def noisy_queries(seed: int, points: np.ndarray, nq: int,
                  sigma: float) -> tuple[np.ndarray, np.ndarray]:
    """Queries = a random data point + N(0, sigma^2 I); returns (queries, source ids)."""
    rng = np.random.default_rng([seed, 11])
    src = rng.integers(0, points.shape[0], size=nq)
    q = points[src].astype(np.float64) + sigma * rng.standard_normal((nq, points.shape[1]))
    return q.astype(np.float32), src


# --------------------------------------------------------------------------
# sets (CSR: uint64 offsets n+1, uint32 elements)
# --------------------------------------------------------------------------

def csr_from_rows(rows: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    off = np.zeros(len(rows) + 1, dtype=U64)
    if rows:
        off[1:] = np.cumsum([len(r) for r in rows], dtype=U64)
    elems = np.concatenate(rows).astype(U32) if rows else np.zeros(0, U32)
    return off, np.ascontiguousarray(elems)


def random_sets(seed: int, n: int, universe: int, min_size: int,
                max_size: int) -> tuple[np.ndarray, np.ndarray]:
    """n sets of distinct uint32 elements drawn from [0, universe)."""
    rng = np.random.default_rng([seed, 20])
    rows = []
    for _ in range(n):
        s = int(rng.integers(min_size, max_size + 1))
        s = min(s, universe)
        rows.append(np.sort(rng.choice(universe, size=s, replace=False)).astype(U32))
    return csr_from_rows(rows)


def _dedup_sorted_rows(sorted_rows: np.ndarray) -> list[np.ndarray]:
    keep = np.ones(sorted_rows.shape, dtype=bool)
    keep[:, 1:] = sorted_rows[:, 1:] != sorted_rows[:, :-1]
    return [sorted_rows[i][keep[i]] for i in range(sorted_rows.shape[0])]


def genomic_reads(seed: int, ref_len: int, n_reads: int, read_len: int,
                  n_queries: int, kmer: int = 18, sub_lo: float = 0.01,
                  sub_hi: float = 0.10) -> dict:
    """Reads sampled from a uniform random ACGT reference with substitutions.

    Each read is the set of its k-mers: a k-mer is packed 2 bits per base
    (A=0, C=1, G=2, T=3, first base most significant, forward strand only)
    and mapped to uint32 by a seeded multiply-shift; each set is deduplicated.
    Returns CSR sets for the ``n_reads`` indexed reads and the ``n_queries``
    held-out reads drawn from the same process.
    """
    if kmer > 32:
        raise ValueError("kmer must be <= 32")
    rng = np.random.default_rng([seed, 30])
    ref = rng.integers(0, 4, size=ref_len, dtype=np.uint8)
    key = U64(int(rng.integers(0, 1 << 63, dtype=np.uint64)) * 2 + 1)
    total = n_reads + n_queries
    starts = rng.integers(0, ref_len - read_len + 1, size=total)
    rates = rng.uniform(sub_lo, sub_hi, size=total)
    nk = read_len - kmer + 1
    rows: list[np.ndarray] = []
    chunk = 8192
    for c0 in range(0, total, chunk):
        c1 = min(total, c0 + chunk)
        idx = starts[c0:c1, None] + np.arange(read_len)[None, :]
        reads = ref[idx].copy()
        sub = rng.random(reads.shape) < rates[c0:c1, None]
        shift = rng.integers(1, 4, size=reads.shape, dtype=np.uint8)
        reads[sub] = (reads[sub] + shift[sub]) & 3
        codes = np.zeros((c1 - c0, nk), dtype=U64)
        r64 = reads.astype(U64)
        for j in range(kmer):
            codes = (codes << U64(2)) | r64[:, j:j + nk]
        with np.errstate(over="ignore"):
            h = ((codes * key) >> U64(32)).astype(U32)
        h.sort(axis=1)
        rows.extend(_dedup_sorted_rows(h))
    off, el = csr_from_rows(rows[:n_reads])
    qoff, qel = csr_from_rows(rows[n_reads:])
    return {"off": off, "elems": el, "q_off": qoff, "q_elems": qel,
            "starts": starts, "rates": rates}


_ALPHABET = np.frombuffer(b"abcdefghijklmnopqrstuvwxyz0123456789", dtype=np.uint8)


def _gram_csr(buf: np.ndarray, off: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Sets of character 3-grams of the strings buf[off[i]:off[i+1]]; a gram
    is its 3 bytes packed into 24 bits (exact); each set sorted, deduplicated."""
    n = off.size - 1
    lens = np.diff(off)
    total = int(off[-1])
    if total < 3:
        return np.zeros(n + 1, U64), np.zeros(0, U32)
    b = buf[:total].astype(np.uint32)
    g = (b[:-2] << np.uint32(16)) | (b[1:-1] << np.uint32(8)) | b[2:]
    owner = np.repeat(np.arange(n, dtype=np.int64), lens)[:-2]
    pos = np.arange(total - 2, dtype=np.int64)
    ok = pos + 2 < off[owner + 1]
    key = (owner[ok].astype(U64) << U64(24)) | g[ok].astype(U64)
    key.sort()
    keep = np.ones(key.size, bool)
    keep[1:] = key[1:] != key[:-1]
    key = key[keep]
    sid = (key >> U64(24)).astype(np.int64)
    cnt = np.bincount(sid, minlength=n)
    csr = np.zeros(n + 1, U64)
    csr[1:] = np.cumsum(cnt)
    return csr, (key & U64(0xFFFFFF)).astype(U32)


def url_strings(seed: int, n: int, n_queries: int, vocab: int = 50_000,
                zipf_s: float = 1.1, median_len: float = 60.0, sigma: float = 0.5,
                edit_rate: float = 0.05) -> dict:
    """URL-shaped strings turned into sets of character 3-grams.

    A vocabulary of ``vocab`` random [a-z0-9] tokens of length 2..12 is drawn;
    a long stream of tokens is sampled by a Zipf(``zipf_s``) law over the
    vocabulary ranks and joined with '/'. String i is the next slice of the
    stream whose length is drawn lognormal (median ``median_len``, log-sd
    ``sigma``, at least 3). Queries are copies of random strings with
    ``edit_rate`` x length character edits (substitution, insertion or
    deletion with equal probability, at least one).
    """
    rng = np.random.default_rng([seed, 40])
    tok_len = rng.integers(2, 13, size=vocab).astype(np.int64)
    tok_chars = _ALPHABET[rng.integers(0, len(_ALPHABET), size=(vocab, 12))]
    w = 1.0 / np.arange(1, vocab + 1, dtype=np.float64) ** zipf_s
    w /= w.sum()
    cdf = np.cumsum(w)
    target = np.maximum(3, np.round(rng.lognormal(np.log(median_len), sigma, size=n))).astype(np.int64)
    total = int(target.sum())
    mean_tok = float((tok_len + 1) @ w)
    n_tok = int(total / mean_tok * 1.1) + 1024
    while True:
        toks = np.minimum(np.searchsorted(cdf, rng.random(n_tok)), vocab - 1)
        tl = tok_len[toks]
        if int((tl + 1).sum()) >= total:
            break
        n_tok = int(n_tok * 1.2)
    starts = np.cumsum(tl + 1) - (tl + 1)
    stream = np.full(int((tl + 1).sum()), ord("/"), np.uint8)
    within = np.arange(int(tl.sum()), dtype=np.int64) - np.repeat(np.cumsum(tl) - tl, tl)
    stream[np.repeat(starts, tl) + within] = tok_chars[np.repeat(toks, tl), within]
    del within
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(target)
    src = rng.integers(0, n, size=n_queries)
    qrows = []
    for i in src:
        s = bytearray(stream[off[i]:off[i + 1]].tobytes())
        n_ed = max(1, int(round(edit_rate * len(s))))
        for _ in range(n_ed):
            op = int(rng.integers(0, 3))
            pos = int(rng.integers(0, max(1, len(s))))
            ch = int(_ALPHABET[rng.integers(0, len(_ALPHABET))])
            if op == 0 and len(s) > 0:
                s[pos] = ch
            elif op == 1:
                s.insert(pos, ch)
            elif len(s) > 1:
                del s[pos]
        qrows.append(np.frombuffer(bytes(s), np.uint8))
    qoff = np.zeros(n_queries + 1, np.int64)
    qoff[1:] = np.cumsum([len(r) for r in qrows])
    qbuf = np.concatenate(qrows) if qrows else np.zeros(0, np.uint8)
    soff, sel = _gram_csr(stream, off)
    qsoff, qsel = _gram_csr(qbuf, qoff)
    return {"off": soff, "elems": sel, "q_off": qsoff, "q_elems": qsel, "src": src,
            "str_len": target}


# --------------------------------------------------------------------------
# embeddings streamed from a seed (YFCC100M-shaped): counter-based, so any
# point can be regenerated alone, on the host here and on the device by the
# library's generator (same definitions, implemented separately)
# --------------------------------------------------------------------------

PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
EMBED_STREAM = 0xC0
_M32 = U64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11),
    vectorised over numpy arrays of counters; returns 4 uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(x).astype(U64) for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0).astype(U64)
    k1 = np.asarray(k1).astype(U64)
    for r in range(10):
        if r:
            k0 = (k0 + U64(PHILOX_W0)) & _M32
            k1 = (k1 + U64(PHILOX_W1)) & _M32
        p0 = U64(PHILOX_M0) * c0
        p1 = U64(PHILOX_M1) * c2
        c0, c1, c2, c3 = (p1 >> U64(32)) ^ c1 ^ k0, p1 & _M32, (p0 >> U64(32)) ^ c3 ^ k1, p0 & _M32
    return tuple(x.astype(U32) for x in (c0, c1, c2, c3))


IH_SCALE = np.float32(np.sqrt(3.0) * 2.0 ** -22)


def irwin_hall(u0, u1, u2, u3) -> np.ndarray:
    """Approximate N(0, 1): the sum of four 22-bit uniforms (exact integer),
    centred, times sqrt(3) * 2^-22 (one fp32 multiply)."""
    s = sum((np.asarray(u).astype(np.int64) >> 10) for u in (u0, u1, u2, u3)) - (1 << 23)
    return s.astype(np.float32) * IH_SCALE


def fma_f32(a, b, c) -> np.ndarray:
    """Correctly rounded fp32 fused multiply-add a*b + c (one rounding).

    a*b is exact in fp64. s = fl64(a*b + c) and its error e (two-sum) give the
    exact value s + e. Rounding s to fp32 is already correct unless s sits
    exactly on a midpoint between two fp32 numbers; then the sign of e picks
    the neighbour (e = 0: ties to even)."""
    a = np.asarray(a, np.float32).astype(np.float64)
    b = np.asarray(b, np.float32).astype(np.float64)
    c = np.asarray(c, np.float32).astype(np.float64)
    p = a * b
    s = p + c
    bb = s - p
    e = (p - (s - bb)) + (c - bb)
    r0 = s.astype(np.float32)
    d = s - r0.astype(np.float64)
    other = np.where(d > 0, np.nextafter(r0, np.float32(np.inf)), np.nextafter(r0, np.float32(-np.inf)))
    tie = (d != 0) & (2 * np.abs(d) == np.abs(other.astype(np.float64) - r0.astype(np.float64)))
    upper = np.where(d > 0, other, r0)
    lower = np.where(d > 0, r0, other)
    r = np.where(tie & (e > 0), upper, np.where(tie & (e < 0), lower, r0))
    return r.astype(np.float32)


def _key(seed: int):
    return U64(seed & 0xFFFFFFFF), U64((seed >> 32) & 0xFFFFFFFF)


def embed_centers(seed: int, centers: np.ndarray, dim: int) -> np.ndarray:
    """Rows ``centers`` of the centre matrix, (len, dim) fp32 ~ N(0, 1)."""
    k0, k1 = _key(seed)
    c = np.asarray(centers, U64)[:, None]
    t = np.arange(dim, dtype=U64)[None, :]
    u = philox4x32_10(c + t * 0, t + c * 0, 0, EMBED_STREAM, k0, k1)
    return irwin_hall(*u)


def embed_labels(seed: int, idx: np.ndarray, n_centers: int) -> np.ndarray:
    k0, k1 = _key(seed)
    i = np.asarray(idx, U64)
    return (philox4x32_10(i, 0, 1, EMBED_STREAM, k0, k1)[0] % U32(n_centers)).astype(np.int64)


def embed_points(seed: int, idx, dim: int, n_centers: int, sigma: float,
                 pre_relu: bool = False) -> np.ndarray:
    """Points ``idx`` of the stream: ReLU(centre[label] + sigma * z), fp32."""
    k0, k1 = _key(seed)
    i = np.asarray(idx, U64)[:, None]
    t = np.arange(dim, dtype=U64)[None, :]
    lab = embed_labels(seed, idx, n_centers)
    cen = embed_centers(seed, lab, dim)
    z = irwin_hall(*philox4x32_10(i + t * 0, t + i * 0, 2, EMBED_STREAM, k0, k1))
    pre = fma_f32(np.float32(sigma), z, cen)
    return pre if pre_relu else np.where(pre > 0, pre, np.float32(0)).astype(np.float32)


def embed_query_sources(seed: int, jdx, n_points: int) -> np.ndarray:
    k0, k1 = _key(seed)
    j = np.asarray(jdx, U64)
    return (philox4x32_10(j, 0, 3, EMBED_STREAM, k0, k1)[0] % U32(n_points)).astype(np.int64)


def embed_queries(seed: int, jdx, n_points: int, dim: int, n_centers: int, sigma: float,
                  q_sigma: float) -> np.ndarray:
    """Queries ``jdx``: ReLU(pre-ReLU value of a random point + q_sigma * z), fp32."""
    k0, k1 = _key(seed)
    src = embed_query_sources(seed, jdx, n_points)
    pre = embed_points(seed, src, dim, n_centers, sigma, pre_relu=True)
    j = np.asarray(jdx, U64)[:, None]
    t = np.arange(dim, dtype=U64)[None, :]
    z = irwin_hall(*philox4x32_10(j + t * 0, t + j * 0, 4, EMBED_STREAM, k0, k1))
    q = fma_f32(np.float32(q_sigma), z, pre)
    return np.where(q > 0, q, np.float32(0)).astype(np.float32)
