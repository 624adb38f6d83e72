"""Python binding of libflinng.so (C ABI in ``include/flinng.h``).

Argument marshalling only: every step of hashing, index construction and
querying runs in the library's CUDA kernels. The ``flinng_*`` functions here
carry the C names; ``Index`` wraps them for numpy arrays (host memory) and
torch CUDA tensors (device memory, on the index's stream).

There is no fallback: if the compiled library is missing or no CUDA device
is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT = range(6)
COSINE_SRP, JACCARD_DOPH = 0, 1
PREC_FP32, PREC_BF16X2, PREC_BF16, PREC_FP8 = 0, 1, 2, 3
QUERY_PLAIN, QUERY_FUSED, QUERY_GRAPH = 0, 1, 2


class flinng_config(C.Structure):
    _fields_ = [("metric", C.c_uint32), ("dim", C.c_uint32), ("R", C.c_uint32),
                ("B", C.c_uint32), ("L", C.c_uint32), ("K", C.c_uint32),
                ("range_bits", C.c_uint32), ("min_threshold", C.c_uint32),
                ("precision", C.c_uint32), ("reserved", C.c_uint32),
                ("capacity", C.c_uint64)]


class flinng_params(C.Structure):
    _fields_ = [("srp_w", C.c_void_p), ("doph_a", C.c_uint32), ("doph_b", C.c_uint32),
                ("doph_seed", C.c_uint64), ("bucket_a", C.c_void_p), ("bucket_c", C.c_void_p)]


class flinng_embed_spec(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("dim", C.c_uint32), ("n_centers", C.c_uint32),
                ("sigma", C.c_float), ("q_sigma", C.c_float), ("n_points", C.c_uint64)]


class flinng_server_config(C.Structure):
    _fields_ = [("hbm_budget", C.c_uint64), ("n_slots", C.c_uint32), ("max_batch", C.c_uint32),
                ("k_max", C.c_uint32), ("max_batch_elems", C.c_uint32)]


class flinng_request(C.Structure):
    _fields_ = [("arrival_s", C.c_double), ("kind", C.c_uint32), ("index", C.c_uint32), ("k", C.c_uint32),
                ("on_device", C.c_uint32), ("n", C.c_uint64), ("data", C.c_void_p), ("perm", C.c_void_p)]


class flinng_request_result(C.Structure):
    _fields_ = [("t_admit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("status", C.c_uint32), ("version", C.c_uint32), ("batch", C.c_uint32), ("slot", C.c_uint32),
                ("d_start", C.c_double), ("d_done", C.c_double)]


REQ_QUERY, REQ_INSERT = 0, 1

# numpy mirror of flinng_request, for building long traces without ctypes loops
REQ_DTYPE = np.dtype([("arrival_s", "<f8"), ("kind", "<u4"), ("index", "<u4"), ("k", "<u4"),
                      ("on_device", "<u4"), ("n", "<u8"), ("data", "<u8"), ("perm", "<u8")], align=True)
assert REQ_DTYPE.itemsize == C.sizeof(flinng_request)
RES_DTYPE = np.dtype([("t_admit", "<f8"), ("t_start", "<f8"), ("t_done", "<f8"), ("status", "<u4"),
                      ("version", "<u4"), ("batch", "<u4"), ("slot", "<u4"), ("d_start", "<f8"),
                      ("d_done", "<f8")], align=True)
assert RES_DTYPE.itemsize == C.sizeof(flinng_request_result)


class flinng_points(C.Structure):
    _fields_ = [("x", C.c_void_p), ("ld", C.c_uint64), ("off", C.c_void_p),
                ("elems", C.c_void_p)]


# Every symbol the header declares, with its C signature.
_SIGS = {
    "flinng_create": (C.c_int, [C.POINTER(flinng_config), C.POINTER(flinng_params), C.c_void_p,
                                C.POINTER(C.c_void_p)]),
    "flinng_build": (C.c_int, [C.c_void_p, C.POINTER(flinng_points), C.c_uint64, C.c_void_p, C.c_int]),
    "flinng_insert": (C.c_int, [C.c_void_p, C.POINTER(flinng_points), C.c_uint64, C.c_void_p, C.c_int]),
    "flinng_query": (C.c_int, [C.c_void_p, C.POINTER(flinng_points), C.c_uint32, C.c_void_p,
                               C.c_uint32, C.c_void_p, C.c_void_p, C.c_int]),
    "flinng_destroy": (C.c_int, [C.c_void_p]),
    "flinng_last_error": (C.c_char_p, []),
    "flinng_size": (C.c_uint64, [C.c_void_p]),
    "flinng_device_bytes": (C.c_uint64, [C.c_void_p]),
    "flinng_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "flinng_hash": (C.c_int, [C.c_void_p, C.POINTER(flinng_points), C.c_uint64, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_int]),
    "flinng_query_buckets": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32,
                                       C.c_void_p, C.c_void_p, C.c_int]),
    "flinng_counts": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_int]),
    "flinng_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64,
                                C.POINTER(C.c_uint64), C.c_void_p]),
    "flinng_hash_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "flinng_hash_counters": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "flinng_server_staging": (C.c_int, [C.c_void_p]),
    "flinng_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "flinng_load": (C.c_int, [C.c_char_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "flinng_get_config": (C.c_int, [C.c_void_p, C.c_void_p]),
    "flinng_query_counts": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p, C.c_uint32,
                                      C.c_void_p, C.c_void_p, C.c_int]),
    "flinng_kernel_launches": (C.c_uint64, []),
    "flinng_set_query_mode": (C.c_int, [C.c_void_p, C.c_uint32]),
    "flinng_build_groups": (C.c_int, [C.c_void_p, C.POINTER(flinng_points), C.c_uint64, C.c_void_p, C.c_int]),
    "flinng_insert_groups": (C.c_int, [C.c_void_p, C.POINTER(flinng_points), C.c_uint64, C.c_void_p, C.c_int]),
    "flinng_set_tuning": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]),
    "flinng_tune_query": (C.c_int, [C.c_void_p, C.POINTER(flinng_points), C.c_uint32, C.c_uint32,
                                    C.c_int, C.c_void_p]),
    "flinng_server_create": (C.c_int, [C.POINTER(flinng_server_config), C.POINTER(C.c_void_p)]),
    "flinng_server_add_index": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_uint32)]),
    "flinng_server_device_bytes": (C.c_uint64, [C.c_void_p]),
    "flinng_server_replay": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "flinng_server_destroy": (C.c_int, [C.c_void_p]),
    "flinng_build_buckets": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_int]),
    "flinng_generate_embeddings": (C.c_int, [C.POINTER(flinng_embed_spec), C.c_int, C.c_uint64, C.c_uint64,
                                             C.c_void_p, C.c_uint64, C.c_void_p]),
    "flinng_query_noalloc": (C.c_int, [C.c_void_p, C.POINTER(flinng_points), C.c_uint32, C.c_void_p,
                                       C.c_uint32, C.c_void_p, C.c_void_p]),
    "flinng_set_tc_wait": (C.c_int, [C.c_void_p, C.c_uint64]),
    "flinng_set_probes": (C.c_int, [C.c_void_p, C.c_uint32]),
}

_lib = None


def load(path: str | None = None):
    """Load libflinng.so (built by ``_build.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libflinng.so not found at {path}: build it with "
                           "paper_2106_11565_gb300._build.build() (nvcc, sm_103a)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FlinngError(RuntimeError):
    """A failed library call: ``code`` is the FLINNG_ERR_* status, the
    message the library's own."""

    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _check(rc: int):
    if rc != OK:
        raise FlinngError(rc, load().flinng_last_error().decode())


def __getattr__(name):
    # flinng_* functions resolve to the loaded library's symbols
    if name.startswith("flinng_") and name in _SIGS:
        return getattr(load(), name)
    raise AttributeError(name)


# --------------------------------------------------------------------------
# buffer helpers: numpy -> host pointers, torch CUDA tensors -> device pointers
# --------------------------------------------------------------------------

def _is_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def kernel_launches() -> int:
    """Kernels launched by libflinng.so in this process so far."""
    return int(load().flinng_kernel_launches())


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):          # torch tensor: CUDA (device) or CPU/pinned (host)
        assert a.is_contiguous()
        return a.data_ptr()
    assert isinstance(a, np.ndarray) and a.flags.c_contiguous
    return a.ctypes.data


def _np(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Index:
    """A FLINNG index on the current CUDA device.

    ``metric``: "cosine" (dense fp32 vectors, SRP) or "jaccard" (sets, DOPH).
    ``params``: from ``workloads.srp_projections`` (cosine: the (L*K, dim)
    matrix) or ``workloads.doph_params`` (jaccard: dict).
    """

    def __init__(self, metric: str, R: int, B: int, L: int, K: int, capacity: int,
                 params, dim: int = 0, W: int | None = None, t_min: int = 1, stream=None,
                 precision: int = PREC_FP32):
        self.lib = load()
        self.metric = metric
        self.cfg = flinng_config()
        self.cfg.metric = COSINE_SRP if metric == "cosine" else JACCARD_DOPH
        self.cfg.dim = dim
        self.cfg.R, self.cfg.B, self.cfg.L, self.cfg.K = R, B, L, K
        self.cfg.range_bits = K if W is None else W
        self.cfg.min_threshold = t_min
        self.cfg.precision = precision
        self.cfg.capacity = capacity
        self.R, self.B, self.L, self.K, self.W = R, B, L, K, self.cfg.range_bits
        p = flinng_params()
        keep = []
        if metric == "cosine":
            w = _np(params, np.float32)
            keep.append(w)
            p.srp_w = w.ctypes.data
        else:
            ba = _np(params["bucket_a"], np.uint64)
            bc = _np(params["bucket_c"], np.uint64)
            keep += [ba, bc]
            p.doph_a, p.doph_b, p.doph_seed = params["doph_a"], params["doph_b"], params["doph_seed"]
            p.bucket_a, p.bucket_c = ba.ctypes.data, bc.ctypes.data
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = C.c_void_p()
        _check(self.lib.flinng_create(C.byref(self.cfg), C.byref(p), C.c_void_p(stream), C.byref(h)))
        self.h = h

    # ---- persistence
    def save(self, path: str):
        """Write the built index to a file (flinng_save)."""
        _check(self.lib.flinng_save(self.h, str(path).encode()))

    @classmethod
    def load(cls, path: str, stream=None) -> "Index":
        """An index read back from a file written by save (flinng_load)."""
        obj = cls.__new__(cls)
        obj.lib = load()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        obj.stream = stream
        h = C.c_void_p()
        _check(obj.lib.flinng_load(str(path).encode(), C.c_void_p(stream), C.byref(h)))
        obj.h = h
        obj.cfg = flinng_config()
        _check(obj.lib.flinng_get_config(h, C.byref(obj.cfg)))
        c = obj.cfg
        obj.metric = "cosine" if c.metric == COSINE_SRP else "jaccard"
        obj.R, obj.B, obj.L, obj.K, obj.W = c.R, c.B, c.L, c.K, c.range_bits
        return obj

    # ---- lifecycle
    def close(self):
        """Destroy the index and free its device memory (idempotent)."""
        if getattr(self, "h", None):
            self.lib.flinng_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def size(self) -> int:
        """Points in the index."""
        return int(self.lib.flinng_size(self.h))

    @property
    def device_bytes(self) -> int:
        """Device memory the index holds."""
        return int(self.lib.flinng_device_bytes(self.h))

    # ---- points
    def _points(self, pts):
        fp = flinng_points()
        if pts is None:
            return fp, 0, 1, []
        if self.metric == "cosine":
            x = pts if _is_cuda(pts) else _np(pts, np.float32)
            fp.x = _ptr(x)
            fp.ld = x.shape[1]
            return fp, x.shape[0], int(_is_cuda(x)), [x]
        off, el = pts
        if _is_cuda(off):
            fp.off, fp.elems = _ptr(off), _ptr(el)
            return fp, off.shape[0] - 1, 1, [off, el]
        off = _np(off, np.uint64)
        el = _np(el, np.uint32) if len(el) else np.zeros(1, np.uint32)
        fp.off, fp.elems = off.ctypes.data, el.ctypes.data
        return fp, off.shape[0] - 1, 0, [off, el]

    def _rows(self, a, n: int, dt, name: str, dev: int):
        """An R x n array of dt (host) or a contiguous R x n tensor of the same
        element size (device), on the same side as the call's other buffers:
        the library reads exactly R * n entries there."""
        if bool(_is_cuda(a)) != bool(dev):
            raise ValueError(f"{name} must live where the points do (host or device)")
        if _is_cuda(a):
            import torch
            want = {np.uint32: (torch.int32,), np.uint16: (torch.int16,) + ((torch.uint16,) if hasattr(torch, "uint16")
                                                                           else ())}[dt]
            if a.dtype not in want or not a.is_contiguous() or tuple(a.shape) != (self.R, n):
                raise ValueError(f"{name} must be a contiguous {self.R} x {n} tensor of {want[0]}")
            return a
        a = _np(a, dt)
        if a.shape != (self.R, n):
            raise ValueError(f"{name} must be {self.R} x {n}")
        return a

    def build(self, pts, perm):
        """Build from scratch over pts with Alg. 1's permutations (R x n)."""
        fp, n, dev, keep = self._points(pts)
        perm = self._rows(perm, n, np.uint32, "perm", dev)
        _check(self.lib.flinng_build(self.h, C.byref(fp), n, _ptr(perm), dev))

    def build_buckets(self, buckets, perm):
        """Build from precomputed buckets (n x L)."""
        dev = int(_is_cuda(buckets))
        b = buckets if dev else _np(buckets, np.uint32)
        perm = self._rows(perm, b.shape[0], np.uint32, "perm", dev)
        _check(self.lib.flinng_build_buckets(self.h, _ptr(b), b.shape[0], _ptr(perm), dev))

    def insert(self, pts, perm):
        """Add pts; perm (R x n) places them after the current points."""
        fp, n, dev, keep = self._points(pts)
        perm = self._rows(perm, n, np.uint32, "perm", dev)
        _check(self.lib.flinng_insert(self.h, C.byref(fp), n, _ptr(perm), dev))

    def build_groups(self, pts, groups):
        """Build with the design given outright: groups (R x n uint16), row r
        holding each point's group in repetition r."""
        fp, n, dev, keep = self._points(pts)
        g = self._rows(groups, n, np.uint16, "groups", dev)
        _check(self.lib.flinng_build_groups(self.h, C.byref(fp), n, _ptr(g), dev))

    def insert_groups(self, pts, groups):
        """Insert with the new points' groups given (R x n uint16)."""
        fp, n, dev, keep = self._points(pts)
        g = self._rows(groups, n, np.uint16, "groups", dev)
        _check(self.lib.flinng_insert_groups(self.h, C.byref(fp), n, _ptr(g), dev))

    def _out(self, dev, shape, dt):
        if dev:
            import torch
            tdt = {np.uint32: torch.int32, np.uint16: torch.int16, np.uint8: torch.uint8,
                   np.float32: torch.float32}[dt]
            return torch.empty(shape, dtype=tdt, device="cuda")
        return np.zeros(shape, dt)

    def hash(self, pts, values: bool = False, proj: bool = False):
        """Buckets (n x L), and optionally MinHash values or projections
        (n x L*K), of pts under the index's hash functions."""
        fp, n, dev, keep = self._points(pts)
        P = self.L * self.K
        b = self._out(dev, (n, self.L), np.uint32)
        v = self._out(dev, (n, P), np.uint32) if values and self.metric != "cosine" else None
        pr = self._out(dev, (n, P), np.float32) if proj and self.metric == "cosine" else None
        _check(self.lib.flinng_hash(self.h, C.byref(fp), n, _ptr(b), _ptr(v), _ptr(pr), dev))
        return b, v, pr

    def query(self, q, k_max: int, k=None, out=None):
        """Top-k_max of each query. out: optional (ids, scores) buffers of the
        queries' kind (nq x k_max uint32 and uint16 arrays for host queries,
        int32 and int16 CUDA tensors for device queries), filled and returned;
        page-locked host buffers are written in place by the kernel."""
        fp, nq, dev, keep = self._points(q)
        if out is None:
            ids = self._out(dev, (nq, k_max), np.uint32)
            sc = self._out(dev, (nq, k_max), np.uint16)
        else:
            ids, sc = out
            if tuple(ids.shape) != (nq, k_max) or tuple(sc.shape) != (nq, k_max):
                raise ValueError("out buffers must be nq x k_max")
            if bool(_is_cuda(ids)) != bool(dev) or bool(_is_cuda(sc)) != bool(dev):
                raise ValueError("out buffers must live where the queries do")
            if not dev and (ids.dtype != np.uint32 or sc.dtype != np.uint16 or not ids.flags.c_contiguous
                            or not sc.flags.c_contiguous):
                raise ValueError("host out buffers must be C-contiguous uint32 and uint16 arrays")
            if dev:
                import torch
                if (ids.dtype != torch.int32 or sc.dtype != torch.int16 or not ids.is_contiguous()
                        or not sc.is_contiguous()):
                    raise ValueError("device out buffers must be contiguous int32 and int16 tensors")
        kk = None if k is None else (k if _is_cuda(k) else _np(k, np.uint32))
        _check(self.lib.flinng_query(self.h, C.byref(fp), nq, _ptr(kk), k_max, _ptr(ids), _ptr(sc), dev))
        return ids, sc

    def _table_rows(self, a, cols: int, dt, name: str):
        """A 2-D array (host) or tensor (device) with cols columns: the
        library reads exactly rows * cols entries."""
        dev = int(_is_cuda(a))
        a = a if dev else _np(a, dt)
        if a.ndim != 2 or a.shape[1] != cols or (dev and not a.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous n x {cols} array")
        if dev and a.element_size() != np.dtype(dt).itemsize:
            raise ValueError(f"{name} must have {np.dtype(dt).itemsize}-byte elements")
        return a, dev

    def query_buckets(self, qb, k_max: int, k=None):
        """Top-k_max from query buckets (nq x L) instead of queries."""
        qb, dev = self._table_rows(qb, self.L, np.uint32, "qbuckets")
        nq = qb.shape[0]
        ids = self._out(dev, (nq, k_max), np.uint32)
        sc = self._out(dev, (nq, k_max), np.uint16)
        kk = None if k is None else (k if _is_cuda(k) else _np(k, np.uint32))
        _check(self.lib.flinng_query_buckets(self.h, _ptr(qb), nq, _ptr(kk), k_max, _ptr(ids),
                                             _ptr(sc), dev))
        return ids, sc

    def query_counts(self, counts, k_max: int, max_count: int, k=None):
        """Decode from per-cell counts (nq x B*R, e.g. summed over table
        shards); max_count is the total table count."""
        counts, dev = self._table_rows(counts, self.B * self.R, np.uint16, "counts")
        nq = counts.shape[0]
        ids = self._out(dev, (nq, k_max), np.uint32)
        sc = self._out(dev, (nq, k_max), np.uint16)
        kk = None if k is None else (k if _is_cuda(k) else _np(k, np.uint32))
        _check(self.lib.flinng_query_counts(self.h, _ptr(counts), nq, max_count, _ptr(kk), k_max, _ptr(ids),
                                            _ptr(sc), dev))
        return ids, sc

    def counts(self, qb):
        """Per-cell collision counts (nq x B*R) of query buckets (nq x L)."""
        qb, dev = self._table_rows(qb, self.L, np.uint32, "qbuckets")
        out = self._out(dev, (qb.shape[0], self.B * self.R), np.uint16)
        _check(self.lib.flinng_counts(self.h, _ptr(qb), qb.shape[0], _ptr(out), dev))
        return out

    def export(self, cells: bool = True) -> dict:
        """The index's CSR offsets, cell lists and group ids, on the host."""
        nc = C.c_uint64()
        _check(self.lib.flinng_export(self.h, None, None, 0, C.byref(nc), None))
        off = np.zeros((self.L << self.W) + 1, np.uint32)
        cl = np.zeros(max(int(nc.value), 1), np.uint16) if cells else None
        gid = np.zeros((max(self.size, 1), self.R), np.uint16)
        _check(self.lib.flinng_export(self.h, off.ctypes.data, cl.ctypes.data if cells else None,
                                      cl.size if cells else 0, C.byref(nc), gid.ctypes.data))
        return {"off": off, "cells": cl[: nc.value] if cells else None, "gid": gid[: self.size]}

    def set_query_mode(self, mode: int):
        """QUERY_PLAIN, QUERY_FUSED or QUERY_GRAPH for flinng_query."""
        _check(self.lib.flinng_set_query_mode(self.h, mode))

    def tune(self, q, k_max: int) -> dict:
        """Autotune the fused query for batches of this size class."""
        fp, nq, dev, keep = self._points(q)
        ch = np.zeros(3, np.uint32)
        _check(self.lib.flinng_tune_query(self.h, C.byref(fp), nq, k_max, dev, ch.ctypes.data))
        return {"threads": int(ch[0]), "ctas_per_sm": int(ch[1]), "cap": int(ch[2])}

    def set_tc_wait(self, limit_ns: int):
        """Limit of each tensor-core pipeline wait (flinng_set_tc_wait)."""
        _check(self.lib.flinng_set_tc_wait(self.h, limit_ns))

    def set_probes(self, probes: int):
        """Buckets probed per table (flinng_set_probes; 1 = single probe)."""
        _check(self.lib.flinng_set_probes(self.h, probes))

    def set_tuning(self, nq: int, threads: int, ctas_per_sm: int = 0, cap: int = 0):
        """Pin the fused query's launch shape for batches of nq's size class."""
        _check(self.lib.flinng_set_tuning(self.h, nq, threads, ctas_per_sm, cap))

    def hash_stats(self):
        """(undecided, exact) projection counts of the last cosine hash."""
        a, b = C.c_uint64(), C.c_uint64()
        _check(self.lib.flinng_hash_stats(self.h, C.byref(a), C.byref(b)))
        return int(a.value), int(b.value)

    def hash_counters(self) -> dict:
        """Counters of the last cosine hash or query: undecided after the
        first pass, exact, fp64 and compensated re-checks, sign flips."""
        out = (C.c_uint64 * 5)()
        _check(self.lib.flinng_hash_counters(self.h, out))
        return dict(zip(("undecided", "exact", "fp64", "compensated", "flips"), (int(v) for v in out)))


def generate_embeddings(seed: int, dim: int, n_centers: int, sigma: float, first: int, n: int,
                        queries: bool = False, q_sigma: float = 0.05, n_points: int = 0, out=None,
                        stream=None):
    """Rows [first, first+n) of the seeded embedding stream, as a CUDA tensor."""
    import torch
    sp = flinng_embed_spec(seed=seed, dim=dim, n_centers=n_centers, sigma=sigma,
                           q_sigma=q_sigma, n_points=n_points)
    if out is None:
        out = torch.empty((n, dim), dtype=torch.float32, device="cuda")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(load().flinng_generate_embeddings(C.byref(sp), int(queries), first, n, out.data_ptr(),
                                             out.stride(0), C.c_void_p(stream)))
    return out


class Server:
    """Continuous-batching server over several resident indices (C runtime)."""

    def __init__(self, hbm_budget: int, n_slots: int = 4, max_batch: int = 1024, k_max: int = 100,
                 max_batch_elems: int = 4 << 20):
        self.lib = load()
        cfg = flinng_server_config(hbm_budget=hbm_budget, n_slots=n_slots, max_batch=max_batch,
                                   k_max=k_max, max_batch_elems=max_batch_elems)
        h = C.c_void_p()
        _check(self.lib.flinng_server_create(C.byref(cfg), C.byref(h)))
        self.h, self.k_max, self.indices = h, k_max, []

    def add_index(self, index: "Index") -> int:
        """Make an index servable (admitted within the HBM budget); returns
        its id for requests."""
        i = C.c_uint32()
        _check(self.lib.flinng_server_add_index(self.h, index.h, C.byref(i)))
        self.indices.append(index)
        return int(i.value)

    @property
    def device_bytes(self) -> int:
        """Device memory the server's slots hold."""
        return int(self.lib.flinng_server_device_bytes(self.h))

    @property
    def staging(self) -> str:
        """'device gather' (a kernel reads the requests' host buffers) or
        'host copy' (inputs copied into pinned staging first)."""
        return "device gather" if self.lib.flinng_server_staging(self.h) == 1 else "host copy"

    def replay(self, reqs, out=None):
        """reqs: a ctypes array of flinng_request or a numpy array of
        REQ_DTYPE (kept alive by the caller, with every buffer it points to).
        out: optional (ids, scores) host arrays of at least len(reqs) rows of
        k_max (uint32, uint16, C-contiguous), reused across replays; by
        default fresh arrays, written once here so that the replay does not
        pay the first touch of their pages.
        Returns (ids, scores, results); results is a ctypes array for ctypes
        input, a numpy array of RES_DTYPE for numpy input."""
        n = len(reqs)
        if out is None:
            ids = np.empty((max(n, 1), self.k_max), np.uint32)
            sc = np.empty((max(n, 1), self.k_max), np.uint16)
            ids.fill(0)
            sc.fill(0)
        else:
            ids, sc = out
            assert (ids.dtype == np.uint32 and sc.dtype == np.uint16 and ids.flags.c_contiguous and
                    sc.flags.c_contiguous and ids.shape[0] >= n and sc.shape[0] >= n and
                    ids.shape[1] == self.k_max and sc.shape[1] == self.k_max)
        if isinstance(reqs, np.ndarray):
            assert reqs.dtype == REQ_DTYPE and reqs.flags.c_contiguous
            res = np.zeros(max(n, 1), RES_DTYPE)
            _check(self.lib.flinng_server_replay(self.h, reqs.ctypes.data, n, ids.ctypes.data,
                                                 sc.ctypes.data, res.ctypes.data))
            return ids[:n], sc[:n], res[:n]
        res = (flinng_request_result * max(n, 1))()
        _check(self.lib.flinng_server_replay(self.h, C.cast(reqs, C.c_void_p), n, ids.ctypes.data,
                                             sc.ctypes.data, C.cast(res, C.c_void_p)))
        return ids[:n], sc[:n], res

    def close(self):
        """Destroy the server (its indices stay the caller's)."""
        if getattr(self, "h", None):
            self.lib.flinng_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
