"""Python front end of the FLINNG CPU oracle (``flinng_oracle.c``).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline / reference leg use it to produce expected values; the
library under ``paper_2106_11565_gb300`` never imports it.

Everything here is marshalling: each function hands numpy arrays to the C
function of the same name and returns numpy arrays. The arithmetic, each step
cited to the paper, lives in the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flinng_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` with gcc."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                               "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _P(t):
    return np.ctypeslib.ndpointer(dtype=t, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        u8, u16, u32, u64, f32, f64 = (_P(np.uint8), _P(np.uint16), _P(np.uint32),
                                        _P(np.uint64), _P(np.float32), _P(np.float64))
        L.oracle_exact_dot_sign.argtypes = [f32, f32, C.c_uint32]
        L.oracle_exact_dot_sign.restype = C.c_int
        L.oracle_srp_codes.argtypes = [f32, C.c_uint64, C.c_uint32, C.c_uint64, f32,
                                       C.c_uint32, C.c_uint32, u32, C.c_void_p]
        L.oracle_srp_codes.restype = C.c_uint64
        L.oracle_splitmix64.argtypes = [C.c_uint64]
        L.oracle_splitmix64.restype = C.c_uint64
        L.oracle_doph.argtypes = [u64, u32, C.c_uint64, C.c_uint32, C.c_uint32,
                                  C.c_uint32, C.c_uint64, u32]
        L.oracle_doph.restype = None
        L.oracle_minhash_buckets.argtypes = [u32, C.c_uint64, C.c_uint32, C.c_uint32,
                                             u64, u64, C.c_uint32, u32]
        L.oracle_minhash_buckets.restype = None
        L.oracle_groups.argtypes = [u32, C.c_uint32, C.c_uint64, C.c_uint64,
                                    C.c_uint32, u16]
        L.oracle_groups.restype = C.c_int
        L.oracle_members.argtypes = [u16, C.c_uint64, C.c_uint32, C.c_uint32, u64, u32]
        L.oracle_members.restype = None
        L.oracle_build_csr.argtypes = [u32, u16, C.c_uint64, C.c_uint32, C.c_uint32,
                                       C.c_uint32, C.c_uint32, u32, u16, C.c_uint64]
        L.oracle_build_csr.restype = C.c_int64
        L.oracle_counts.argtypes = [u32, u16, C.c_uint32, C.c_uint32, u32,
                                    C.c_uint32, u16]
        L.oracle_counts.restype = None
        L.oracle_query.argtypes = [u32, u16, C.c_uint32, C.c_uint32, u64, u32,
                                   C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                   u32, C.c_uint64, C.c_void_p, C.c_uint32, u32, u16]
        L.oracle_query.restype = C.c_int
        L.oracle_counts_direct.argtypes = [u32, u16, C.c_uint64, C.c_uint32, C.c_uint32,
                                           C.c_uint32, u32, u16]
        L.oracle_counts_direct.restype = None
        L.oracle_counts_multiprobe.argtypes = [u32, u16, C.c_uint64, C.c_uint32, C.c_uint32,
                                               C.c_uint32, u32, C.c_uint32, u16]
        L.oracle_counts_multiprobe.restype = None
        L.oracle_alg3.argtypes = [u16, u64, u32, C.c_uint64, C.c_uint32, C.c_uint32,
                                  C.c_uint32, C.c_uint32, u32, u16, C.c_uint32]
        L.oracle_alg3.restype = C.c_uint32
        _lib = L
    return _lib


def _c(a, t):
    return np.ascontiguousarray(a, dtype=t)


# ---------------------------------------------------------------- hashing

def exact_dot_sign(a, b) -> int:
    a = _c(a, np.float32)
    b = _c(b, np.float32)
    return int(lib().oracle_exact_dot_sign(a, b, a.size))


def srp_codes(x, w, L: int, K: int, want_proj: bool = False):
    """SRP codes (n, L) uint32; with ``want_proj`` also the fp64 projections
    (n, L*K) and the count of exact-accumulator fallbacks."""
    x = _c(x, np.float32)
    w = _c(w, np.float32)
    n, d = x.shape
    assert w.shape == (L * K, d)
    codes = np.zeros((n, L), np.uint32)
    proj = np.zeros((n, L * K), np.float64) if want_proj else None
    n_exact = lib().oracle_srp_codes(x, n, d, d, w, L, K, codes,
                                     proj.ctypes.data if want_proj else None)
    return (codes, proj, int(n_exact)) if want_proj else codes


def splitmix64(z: int) -> int:
    return int(lib().oracle_splitmix64(z & ((1 << 64) - 1)))


def doph(off, elems, nb: int, a: int, b: int, seed: int):
    """Densified one-permutation MinHash values, (n, nb) uint32."""
    off = _c(off, np.uint64)
    elems = _c(elems, np.uint32) if len(elems) else np.zeros(1, np.uint32)
    n = off.size - 1
    out = np.zeros((n, nb), np.uint32)
    lib().oracle_doph(off, elems, n, nb, a, b, seed, out)
    return out


def minhash_buckets(v, L: int, K: int, bucket_a, bucket_c, W: int):
    v = _c(v, np.uint32)
    n = v.shape[0]
    out = np.zeros((n, L), np.uint32)
    lib().oracle_minhash_buckets(v, n, L, K, _c(bucket_a, np.uint64),
                                 _c(bucket_c, np.uint64), W, out)
    return out


# ---------------------------------------------------------------- index

def groups(perm, B: int, n_old: int = 0, gid=None):
    """Cell of every point per repetition (Alg. 1); gid (N, R) uint16."""
    perm = _c(perm, np.uint32)
    R, n = perm.shape
    if gid is None:
        gid = np.zeros((n_old + n, R), np.uint16)
    assert gid.shape == (n_old + n, R) and gid.flags.c_contiguous
    if lib().oracle_groups(perm, R, n, n_old, B, gid) != 0:
        raise ValueError("perm rows must be permutations of [0, n)")
    return gid


def design_groups(groups, B: int):
    """Cells of a non-adaptive design given outright, one test per point and
    repetition (Sec. 3.1: the framework takes any non-adaptive design, the
    doubly regular one of Alg. 1 being one case). Row r of ``groups`` (R, n)
    holds each point's group in repetition r; returned point-major (n, R)
    uint16 like groups()."""
    g = np.asarray(groups)
    if g.ndim != 2:
        raise ValueError("groups must be R x n")
    if g.size and (int(g.min()) < 0 or int(g.max()) >= B):
        raise ValueError("a group id is outside [0, B)")
    return np.ascontiguousarray(g.T.astype(np.uint16))


def members(gid, B: int):
    gid = _c(gid, np.uint16)
    N, R = gid.shape
    moff = np.zeros((R, B + 1), np.uint64)
    mem = np.zeros((R, max(N, 1)), np.uint32)
    lib().oracle_members(gid, N, R, B, moff, mem)
    return moff, mem


def build_csr(buckets, gid, B: int, W: int):
    buckets = _c(buckets, np.uint32)
    gid = _c(gid, np.uint16)
    N, L = buckets.shape
    R = gid.shape[1]
    off = np.zeros((L << W) + 1, np.uint32)
    cap = max(N * L * R, 1)
    cells = np.zeros(cap, np.uint16)
    nc = lib().oracle_build_csr(buckets, gid, N, L, R, B, W, off, cells, cap)
    assert nc >= 0
    return off, cells[:nc].copy()


def counts(off, cells, L: int, W: int, qbucket, BR: int):
    cnt = np.zeros(BR, np.uint16)
    cells = _c(cells, np.uint16) if len(cells) else np.zeros(1, np.uint16)
    lib().oracle_counts(_c(off, np.uint32), cells, L, W, _c(qbucket, np.uint32), BR, cnt)
    return cnt


def counts_direct(buckets, gid, B: int, qbucket):
    """Per-cell counts from the definition (no reverse index)."""
    buckets = _c(buckets, np.uint32)
    gid = _c(gid, np.uint16)
    N, L = buckets.shape
    R = gid.shape[1]
    cnt = np.zeros(B * R, np.uint16)
    lib().oracle_counts_direct(buckets, gid, N, L, R, B, _c(qbucket, np.uint32), cnt)
    return cnt


def counts_multiprobe(buckets, gid, B: int, qbucket, P: int):
    """Per-cell counts with P probes per table (the query's bucket and its
    one-bit neighbours in bits 0 .. P-2), from the definition."""
    buckets = _c(buckets, np.uint32)
    gid = _c(gid, np.uint16)
    N, L = buckets.shape
    R = gid.shape[1]
    cnt = np.zeros(B * R, np.uint16)
    lib().oracle_counts_multiprobe(buckets, gid, N, L, R, B, _c(qbucket, np.uint32), P, cnt)
    return cnt


def alg3(cnt, moff, mem, N: int, R: int, B: int, k: int, t_min: int = 1, k_max=None):
    k_max = k if k_max is None else k_max
    ids = np.zeros(max(k_max, 1), np.uint32)
    sc = np.zeros(max(k_max, 1), np.uint16)
    n = lib().oracle_alg3(_c(cnt, np.uint16), _c(moff, np.uint64), _c(mem, np.uint32),
                          N, R, B, k, t_min, ids, sc, k_max)
    return ids[:k_max], sc[:k_max], int(n)


class OracleIndex:
    """The whole FLINNG index on the CPU: hash, group, reverse index, query."""

    def __init__(self, metric: str, R: int, B: int, L: int, K: int, W: int,
                 t_min: int = 1, srp_w=None, doph=None):
        self.metric, self.R, self.B, self.L, self.K, self.W = metric, R, B, L, K, W
        self.t_min = t_min
        self.srp_w = srp_w
        self.dp = doph
        self.N = 0
        self.buckets = np.zeros((0, L), np.uint32)
        self.gid = np.zeros((0, R), np.uint16)

    def hash(self, pts):
        if self.metric == "cosine":
            return srp_codes(pts, self.srp_w, self.L, self.K)
        off, el = pts
        v = doph(off, el, self.L * self.K, self.dp["doph_a"], self.dp["doph_b"],
                 self.dp["doph_seed"])
        return minhash_buckets(v, self.L, self.K, self.dp["bucket_a"],
                               self.dp["bucket_c"], self.W)

    def insert(self, pts, perm):
        bk = self.hash(pts)
        n = bk.shape[0]
        gid = np.zeros((self.N + n, self.R), np.uint16)
        gid[: self.N] = self.gid
        groups(perm, self.B, self.N, gid)
        self.gid = gid
        self.buckets = np.concatenate([self.buckets, bk])
        self.N += n
        self.off, self.cells = build_csr(self.buckets, self.gid, self.B, self.W)
        self.moff, self.mem = members(self.gid, self.B)

    build = insert

    def insert_groups(self, pts, groups):
        """Insert with the points' groups given (an arbitrary non-adaptive
        design, one test per repetition) instead of Alg. 1's permutations."""
        g = design_groups(groups, self.B)
        if g.shape[1] != self.R:
            raise ValueError("groups must have R rows")
        bk = self.hash(pts)
        if bk.shape[0] != g.shape[0]:
            raise ValueError("groups must have one column per point")
        self.gid = np.concatenate([self.gid, g]) if self.N else g
        self.buckets = np.concatenate([self.buckets, bk])
        self.N += bk.shape[0]
        self.off, self.cells = build_csr(self.buckets, self.gid, self.B, self.W)
        self.moff, self.mem = members(self.gid, self.B)

    def build_groups(self, pts, groups):
        """A fresh index over pts with the given design."""
        self.N = 0
        self.buckets = np.zeros((0, self.L), np.uint32)
        self.gid = np.zeros((0, self.R), np.uint16)
        self.insert_groups(pts, groups)

    def query_buckets(self, qb, k_max: int, k=None):
        qb = _c(qb, np.uint32)
        nq = qb.shape[0]
        ids = np.zeros((nq, max(k_max, 1)), np.uint32)
        sc = np.zeros((nq, max(k_max, 1)), np.uint16)
        kk = _c(k, np.uint32) if k is not None else None
        cells = self.cells if len(self.cells) else np.zeros(1, np.uint16)
        rc = lib().oracle_query(self.off, cells, self.L, self.W, self.moff, self.mem,
                                self.N, self.R, self.B, self.t_min, qb, nq,
                                kk.ctypes.data if kk is not None else None,
                                k_max, ids, sc)
        if rc != 0:
            raise ValueError("k exceeds k_max")
        return ids[:, :k_max], sc[:, :k_max]

    def query(self, q, k_max: int, k=None):
        return self.query_buckets(self.hash(q), k_max, k)
