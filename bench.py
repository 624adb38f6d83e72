#!/usr/bin/env python
"""FLINNG query benchmark on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload C2] [--impl ours|reference]

Default (workload C2, the metric's own configuration): queries/s of the
serving form at the recall-target parameters, i.e. where recall@10 >= 0.9.
One step = one replay of 262,144 queries arriving as a Poisson stream at
twice the plain form's throughput, served by the continuous-batching runtime
(request sets and results in host memory); value = queries / device time of
the replays (CUDA events). Beside it: the plain batched form (hash kernel,
then count / decode / top-k kernel) and the fused form on device buffers
with L2 flushed before every step, p50/p99 latency at 0.25x, 0.5x and 0.9x
the plain form's throughput, recall@10, the fused kernel's roofline, the
build, the workload at its configured parameters and the CPU oracle.
Prints one JSON line (rank 0).

Workloads (synthetic, seeded, shaped like the paper's datasets):
  C1  cosine/SRP, 10,000 Gaussian-mixture vectors d=128, R3 B100 L16 K12,
      100 queries, k=10
  C2  Jaccard/MinHash, 100,000 reads of 1,000 bp from a 5 Mbp random ACGT
      reference with 1-10% substitutions as 18-mer sets, R2 B1000 L32 K2 W17,
      1,000 held-out reads as queries, k=100        (default; recall-target
      parameters R3 B4096 L512 K1 W17)
  C3  URL-shaped strings (MinHash), C4 YFCC-shaped embeddings (SRP), C5 the
      serving mix of C2 and C4; ``--configured`` times a workload at its
      configured parameters (fused form, recall sweep).

``--impl reference`` times the CPU oracle on the same workload instead
(single core, a bounded sample of queries per step).
"""
from __future__ import annotations

import argparse
import ctypes as C
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2106_11565_gb300 import workloads as WL  # noqa: E402

# SRP arithmetic of cosine indices (library precision codes); the sign bits are exact in every one
PRECISIONS = {"fp32": 0, "bf16x2": 1, "bf16": 2, "fp8": 3}
PREC_NAMES = {0: "FP32 FFMA", 1: "BF16x2 tcgen05", 2: "BF16 tcgen05", 3: "FP8 E4M3 tcgen05 (row scales)"}

METRIC = ("queries/s at recall@10≥0.9 on 1 GB300, serving vs plain form; "
          "p50/p99 latency")
UNIT = "queries/s"

WORKLOADS = {
    "C1": dict(metric="cosine", N=10_000, d=128, n_centers=100, sigma=0.1, nq=100,
               qsigma=0.05, R=3, B=100, L=16, K=12, W=12, k=10,
               desc="cosine/SRP N=10000 d=128 R3 B100 L16 K12 nq=100 k=10"),
    "C2": dict(metric="jaccard", ref_len=5_000_000, N=100_000, read_len=1000, kmer=18,
               nq=1000, R=2, B=1000, L=32, K=2, W=17, k=100,
               desc="Jaccard/DOPH genomic reads N=100000 len=1000 18-mers R2 B1000 L32 K2 W17 "
                    "nq=1000 k=100"),
    "C4": dict(metric="cosine", embed=True, N=10_000_000, d=4096, n_centers=1000, sigma=0.1,
               nq=10_000, qsigma=0.05, R=3, B=20000, L=64, K=16, W=16, k=10, gt_sample=1000,
               chunk=32768,
               desc="cosine/SRP YFCC-shaped embeddings N=10000000 d=4096 (ReLU of a 1000-centre "
                    "Gaussian mixture, streamed from a seed on the GPU, never stored) R3 B20000 L64 K16 "
                    "nq=10000 k=10"),
    "C3": dict(metric="jaccard", url=True, N=1_000_000, nq=10_000, R=4, B=5000, L=64, K=1, W=17,
               k=10, gt_sample=500,
               desc="Jaccard/DOPH URL-shaped strings N=1000000 (lognormal length, median 60, Zipf(1.1) "
                    "50k-token vocabulary) char 3-gram sets R4 B5000 L64 K1 W17 nq=10000 "
                    "(5% edited copies) k=10"),
}


# --------------------------------------------------------------------------
# workload construction and exact ground truth
# --------------------------------------------------------------------------

def make_workload(name: str) -> dict:
    c = dict(WORKLOADS[name])
    seed = WL.config_seed(int(name[1:]))
    if c.get("embed"):
        # points and queries are generated on the device from the seed
        c.update(pts=None, q=None, params=WL.srp_projections(seed, c["L"] * c["K"], c["d"]))
    elif c["metric"] == "cosine":
        pts, _ = WL.gaussian_mixture(seed, c["N"], c["d"], c["n_centers"], c["sigma"])
        q, _ = WL.noisy_queries(seed, pts, c["nq"], c["qsigma"])
        c.update(pts=pts, q=q, params=WL.srp_projections(seed, c["L"] * c["K"], c["d"]))
    else:
        if c.get("url"):
            g = WL.url_strings(seed, c["N"], c["nq"])
        else:
            g = WL.genomic_reads(seed, c["ref_len"], c["N"], c["read_len"], c["nq"], kmer=c["kmer"])
        c.update(pts=(g["off"], g["elems"]), q=(g["q_off"], g["q_elems"]),
                 params=WL.doph_params(seed, c["L"], c["K"]))
    c["perm"] = WL.group_permutations(seed, c["R"], c["N"])
    c["seed"] = seed
    return c


def gt_sample(c: dict) -> np.ndarray:
    """Queries whose exact neighbours are computed (all, or a seeded sample)."""
    n = c.get("gt_sample", c["nq"])
    if n >= c["nq"]:
        return np.arange(c["nq"])
    return np.sort(np.random.default_rng([c["seed"], 99]).choice(c["nq"], n, replace=False))


def exact_jaccard_topk_gpu(c: dict, sample: np.ndarray, topn: int = 100):
    """Exact Jaccard top-``topn`` for the sampled queries against every set,
    on the GPU with plain torch ops (set membership of every element, then a
    per-set count). Sets must hold distinct elements."""
    import torch
    off, el = c["pts"]
    qoff, qel = c["q"]
    N = off.size - 1
    dev = torch.device("cuda")
    el_t = torch.from_numpy(el.view(np.int32)).to(dev)
    sizes = torch.from_numpy(np.diff(off.astype(np.int64))).to(dev)
    owner = torch.repeat_interleave(torch.arange(N, device=dev), sizes)
    ids = np.full((len(sample), topn), -1, np.int64)
    sims = np.zeros((len(sample), topn))
    for r, i in enumerate(sample):
        qe = torch.from_numpy(np.ascontiguousarray(qel[qoff[i]:qoff[i + 1]]).view(np.int32)).to(dev)
        inter = torch.bincount(owner[torch.isin(el_t, qe)], minlength=N).to(torch.float64)
        j = inter / (qe.numel() + sizes.to(torch.float64) - inter).clamp_min(1.0)
        v, top = torch.topk(j, topn)
        ids[r] = top.cpu().numpy()
        sims[r] = v.cpu().numpy()
    del el_t, owner, sizes
    torch.cuda.empty_cache()
    return ids, sims


def exact_cosine_topk_streamed(c: dict, d_q, sample: np.ndarray, topn: int = 100):
    """Exact fp32 (no TF32) cosine top-``topn`` of the sampled queries over the
    whole streamed point set, chunk by chunk on the GPU."""
    import torch
    from paper_2106_11565_gb300 import flinng as F
    torch.backends.cuda.matmul.allow_tf32 = False
    qs = d_q[torch.from_numpy(sample).to(d_q.device)]
    qs = qs / qs.norm(dim=1, keepdim=True).clamp_min(1e-30)
    best_v = torch.full((len(sample), topn), -2.0, device=d_q.device)
    best_i = torch.full((len(sample), topn), -1, dtype=torch.int64, device=d_q.device)
    ch = 131072
    buf = torch.empty((ch, c["d"]), dtype=torch.float32, device=d_q.device)
    for first in range(0, c["N"], ch):
        n = min(ch, c["N"] - first)
        x = F.generate_embeddings(c["seed"], c["d"], c["n_centers"], c["sigma"], first, n, out=buf[:n])
        sims = (qs @ x.T) / x.norm(dim=1).clamp_min(1e-30)[None, :]
        v, i = torch.topk(sims, min(topn, n), dim=1)
        allv = torch.cat([best_v, v], 1)
        alli = torch.cat([best_i, i + first], 1)
        best_v, o = torch.topk(allv, topn, dim=1)
        best_i = torch.gather(alli, 1, o)
    return best_i.cpu().numpy(), best_v.cpu().numpy().astype(np.float64)


def exact_similarity_topk(c: dict, topn: int = 100):
    """Exact top-``topn`` neighbours per query: cosine by fp64 brute force;
    Jaccard through an inverted index over set elements (as the paper
    computes its genomic and URL ground truth). Returns (ids, sims)."""
    nq = c["nq"]
    if c.get("embed"):
        return exact_cosine_topk_streamed(c, c["d_q"], gt_sample(c), topn)
    if c["metric"] != "cosine" and c.get("url"):
        return exact_jaccard_topk_gpu(c, gt_sample(c), topn)
    if c["metric"] == "cosine":
        x = c["pts"].astype(np.float64)
        x /= np.maximum(np.linalg.norm(x, axis=1, keepdims=True), 1e-300)
        q = c["q"].astype(np.float64)
        q /= np.maximum(np.linalg.norm(q, axis=1, keepdims=True), 1e-300)
        s = q @ x.T
        ids = np.argsort(-s, axis=1, kind="stable")[:, :topn]
        return ids, np.take_along_axis(s, ids, axis=1)
    off, el = c["pts"]
    qoff, qel = c["q"]
    sizes = np.diff(off.astype(np.int64))
    owner = np.repeat(np.arange(len(sizes)), sizes)
    order = np.argsort(el, kind="stable")
    el_s, own_s = el[order], owner[order]
    ids = np.full((nq, topn), -1, np.int64)
    sims = np.zeros((nq, topn))
    for i in range(nq):
        qe = qel[qoff[i]:qoff[i + 1]]
        lo = np.searchsorted(el_s, qe, "left")
        hi = np.searchsorted(el_s, qe, "right")
        cnt = hi - lo
        if cnt.sum() == 0:
            continue
        idx = np.repeat(lo - np.cumsum(np.r_[0, cnt[:-1]]), cnt) + np.arange(cnt.sum())
        hits = own_s[idx]
        u, inter = np.unique(hits, return_counts=True)
        j = inter / (len(qe) + sizes[u] - inter)
        top = np.lexsort((u, -j))[:topn]
        ids[i, :len(top)] = u[top]
        sims[i, :len(top)] = j[top]
    return ids, sims


def recall_scores(c: dict, got_ids: np.ndarray, exact_ids, exact_sims) -> dict:
    """recall@10: |returned[:10] with similarity >= the 10th exact| / 10 (ties
    count as hits, padding as misses); R10@k: same over all k returned; R1@k:
    the exact nearest neighbour is among the k returned."""
    nq = got_ids.shape[0]
    r10, r10k, r1k = [], [], []
    for i in range(nq):
        t10 = exact_sims[i, 9]
        top = set(exact_ids[i, :10].tolist())
        sim_of = dict(zip(exact_ids[i].tolist(), exact_sims[i].tolist()))
        ret = [int(x) for x in got_ids[i] if x != 0xFFFFFFFF]

        def hits(lst):
            return min(10, sum(1 for x in lst if x in top or sim_of.get(x, -1.0) >= t10 > 0))
        r10.append(hits(ret[:10]) / 10)
        r10k.append(hits(ret) / 10)
        r1k.append(1.0 if int(exact_ids[i, 0]) in ret else 0.0)
    return {"recall_at_10": float(np.mean(r10)), "recall_10_at_k": float(np.mean(r10k)),
            "recall_1_at_k": float(np.mean(r1k))}


# --------------------------------------------------------------------------
# algorithmic bytes (the work the method must do, not a dense scan)
# --------------------------------------------------------------------------

def query_kernel_bytes(c: dict, ex: dict, counts: np.ndarray, qb: np.ndarray, kq: int) -> dict:
    """Per-launch algorithmic bytes of the query kernel, following Alg. 3's
    level walk (the kernel walks whole level groups, so it may read more):
    query buckets L*4, table offsets L*8; per table either its
    bucket list at 2 B a cell or, for a heavy slot (>= max(B*R/16, 32)
    cells, which the library stores as a bitmap over the B*R cells too), the
    bitmap's ceil(B*R/32)*4 B; then for every repetition-0 cell at count >= the
    stopping level its member range (8 B) and per member its record (4 B id +
    2(R-1) B group ids), plus k * 5 B of output."""
    R, B, L, W = c["R"], c["B"], c["L"], c["W"]
    BR = B * R
    heavy_min = max(BR // 16, 32)
    bm_bytes = ((BR + 31) // 32) * 4
    gid = ex["gid"].astype(np.int64)
    off = ex["off"]
    sizes0 = np.bincount(gid[:, 0], minlength=B)
    total = 0
    members = 0
    n_heavy = 0
    for i in range(qb.shape[0]):
        slots = (np.arange(L, dtype=np.int64) << W) | qb[i].astype(np.int64)
        lens = off[slots + 1].astype(np.int64) - off[slots]
        heavy = lens >= heavy_min
        n_heavy += int(heavy.sum())
        lists = int(lens[~heavy].sum()) * 2 + int(heavy.sum()) * bm_bytes
        cnt = counts[i].astype(np.int64)
        cell = gid + (np.arange(R) * B)[None, :]
        score = cnt[cell].min(axis=1)
        hist = np.bincount(score, minlength=L + 1)
        ge = np.cumsum(hist[::-1])[::-1]          # points with score >= t
        tstop = 1
        for t in range(L, 0, -1):
            if ge[t] >= kq:
                tstop = t
                break
        c0 = cnt[:B]
        enum_cells = np.nonzero(c0 >= tstop)[0]
        m = int(sizes0[enum_cells].sum())
        members += m
        total += L * 4 + L * 8 + lists + len(enum_cells) * 8 + m * (4 + 2 * (R - 1)) + kq * 5
    return {"bytes": total, "members": members, "heavy_tables": n_heavy}


def hash_kernel_bytes(c: dict) -> int:
    """Per-launch algorithmic bytes of hashing the query batch."""
    L = c["L"]
    if c["metric"] == "cosine":
        return c["nq"] * c["d"] * 4 + c["L"] * c["K"] * c["d"] * 4 + c["nq"] * L * 4
    qoff, qel = c["q"]
    return int(qel.size) * 4 + (c["nq"] + 1) * 8 + c["nq"] * L * 4


# --------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi (every 50 ms by
    default).

    The sampler starts before a busy warm-up phase that runs the same kernels
    back to back right up to the timed region, so that short timed regions
    still have samples taken under this load; ``stop`` keeps the samples
    from the loaded window [load_start, timed_end + 0.1 s]."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", str(period_ms)],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    @staticmethod
    def _ts(s: str) -> float:
        import datetime
        s = s.strip()
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(s, fmt).timestamp()
            except ValueError:
                pass
        return float("nan")

    def stop(self, t_from: float, t_to: float) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        win = [r for r in rows if t_from - 0.05 <= self._ts(r[0]) <= t_to + 0.1]
        if not win:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in win) if v is not None]
        mx = [v for v in (num(r[2]) for r in win) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in win for j in range(4) if r[5 + j].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(win),
                "window": "busy warm-up under the same kernels + timed region"}


# --------------------------------------------------------------------------
# traffic recorded by ncu (profiles/), valid only for the unchanged kernel
# --------------------------------------------------------------------------

def kernel_source_hash() -> str:
    """Hash of the query kernels' sources (the kernels and their launchers)."""
    h = hashlib.sha256()
    for f in ("query.cu", "query_impl.cuh", "query_c16.cu"):
        h.update(open(os.path.join(ROOT, "paper_2106_11565_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, kernel: str = "k_query_fused"):
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# --------------------------------------------------------------------------
# serving form: Poisson traces replayed by the C runtime
# --------------------------------------------------------------------------

def make_trace(F, rng, rate: float, T: float, sources: list, inserts: list | None = None,
               k_choices=(1, 10, 100), n: int | None = None):
    """Poisson arrivals at ``rate`` for ``T`` seconds (or exactly ``n``
    arrivals at ``rate``). ``sources``: one dict per index {"id", "kind":
    "sets"|"dense", "share", ...data}; k uniform over ``k_choices``.
    ``inserts``: (time, index id, flinng_points, n, perm) tuples merged in
    arrival order."""
    if n is not None:
        T = n / rate
    n = max(1, int(rng.poisson(rate * T))) if n is None else int(n)
    t = np.sort(rng.uniform(0.0, T, size=n))
    shares = np.array([src["share"] for src in sources], float)
    which = rng.choice(len(sources), size=n, p=shares / shares.sum())
    req = np.zeros(n, F.REQ_DTYPE)
    req["arrival_s"] = t
    req["kind"] = F.REQ_QUERY
    req["k"] = rng.choice(np.asarray(k_choices), size=n)
    for si, src in enumerate(sources):
        m = which == si
        cnt = int(m.sum())
        j = rng.integers(0, src["nq"], size=cnt)
        req["index"][m] = src["id"]
        if src["kind"] == "sets":
            req["n"][m] = src["sizes"][j]
            req["data"][m] = src["base"] + src["off"][j] * 4
        else:
            req["data"][m] = src["base"] + j.astype(np.uint64) * np.uint64(src["dim"] * 4)
    if inserts:
        ins = np.zeros(len(inserts), F.REQ_DTYPE)
        for i, (ti, idx, fp, cnt, perm) in enumerate(inserts):
            ins[i] = (ti, F.REQ_INSERT, idx, 0, 0, cnt, C.addressof(fp), perm.ctypes.data)
        req = np.concatenate([req, ins])
        req = req[np.argsort(req["arrival_s"], kind="stable")]
    return np.ascontiguousarray(req)


def trace_stats(req, res, F) -> dict:
    q = req["kind"] == F.REQ_QUERY
    lat = (res["t_done"] - req["arrival_s"])[q]
    span = float(res["t_done"][q].max() - req["arrival_s"][q].min())
    out = {"queries": int(q.sum()), "achieved_qps": float(q.sum() / span),
           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "batches": int(len(np.unique(res["batch"][q])))}
    for idx in np.unique(req["index"][q]):
        m = q & (req["index"] == idx)
        li = (res["t_done"] - req["arrival_s"])[m]
        out[f"index{int(idx)}"] = {"queries": int(m.sum()), "p50_ms": float(np.percentile(li, 50) * 1e3),
                                   "p99_ms": float(np.percentile(li, 99) * 1e3)}
    ins = req["kind"] == F.REQ_INSERT
    if ins.any():
        out["inserts"] = [{"n": int(req["n"][i]), "status": int(res["status"][i]),
                           "ms": float((res["t_done"][i] - res["t_start"][i]) * 1e3)} for i in np.nonzero(ins)[0]]
    return out


def sets_source(F, idx_id, q, share, keep):
    """Host-resident query sets (pinned) for a trace."""
    import torch
    qoff, qel = q
    el = torch.from_numpy(qel.view(np.int32)).pin_memory()
    keep.append(el)
    return {"id": idx_id, "kind": "sets", "share": share, "nq": len(qoff) - 1,
            "sizes": np.diff(qoff).astype(np.uint64), "off": qoff[:-1].astype(np.uint64),
            "base": np.uint64(el.data_ptr())}


def dense_source(F, idx_id, h_q, share, keep):
    keep.append(h_q)
    return {"id": idx_id, "kind": "dense", "share": share, "nq": h_q.shape[0], "dim": h_q.shape[1],
            "base": np.uint64(h_q.ctypes.data)}


# --------------------------------------------------------------------------
# recall sweep: QPS at recall@10 >= 0.9 over (R, B, L, K) around the config
# --------------------------------------------------------------------------

# Grids follow the paper's hyperparameter search (R in {2, 3, 4}, B and the
# table count L (the paper's m) in powers of two up to 2^11, B * R < 2^16),
# capped by L * R * N < 2^32 entries.
SWEEPS = {
    "C1": dict(R=(2, 3), B=(100, 1000, 5000), L=(16, 64, 255, 1024), K=(8, 12, 16), P=(1, 3, 5)),
    "C2": dict(R=(2, 3), B=(1000, 4096, 16384), L=(32, 64, 128, 255, 512, 1024, 2048), K=(1,)),
    "C3": dict(R=(2, 4), B=(5000, 16000), L=(64, 255, 1024), K=(1,)),
    "C4": dict(R=(3,), B=(20000,), L=(64, 128), K=(12, 16)),
}


def serving_runs(F, ix, c: dict, plain_qps: float, factors, check_sample: int = 0, max_batch: int = 1024) -> dict:
    """Poisson traces replayed by the C serving runtime on one resident index
    at ``factors`` x the plain form's device-resident throughput; optionally
    checks ``check_sample`` served results against the same query run alone."""
    import torch
    keep = []
    k = max(100, c["k"])
    # the served batches (<= max_batch queries) run the fused form at shapes
    # tuned for their size classes, on leading queries of the workload (the
    # class of the whole batch keeps the shape chosen for it already)
    def size_class(n):
        return max(0, int(n - 1).bit_length())
    for nb in sorted({max_batch, 1024, 256}, reverse=True):
        if nb > max_batch:
            continue
        if size_class(nb) == size_class(c["nq"]):
            continue
        if c["metric"] == "cosine":
            ix.tune(np.ascontiguousarray(c["q"][:nb]), k)
        else:
            qoff, qel = c["q"]
            m = min(nb, len(qoff) - 1)
            ix.tune((qoff[:m + 1].astype(np.uint64), np.ascontiguousarray(qel[:qoff[m]])), k)
    srv = F.Server(hbm_budget=ix.device_bytes + (2 << 30), n_slots=8, max_batch=max_batch, k_max=k,
                   max_batch_elems=1 << 21)
    sid = srv.add_index(ix)
    staging = srv.staging
    src = (sets_source(F, sid, c["q"], 1.0, keep) if c["metric"] != "cosine"
           else dense_source(F, sid, torch.from_numpy(c["q"]).pin_memory().numpy(), 1.0, keep))
    rng_t = np.random.default_rng([c["seed"], 77])
    runs = {}
    same = None
    for f in factors:
        rate = f * plain_qps
        T = min(0.25, 1.5e6 / rate)
        req = make_trace(F, rng_t, rate, T, [src])
        l0 = F.kernel_launches()
        ids_s, sc_s, res = srv.replay(req)
        runs[f"{f}x_plain"] = dict(trace_stats(req, res, F), offered_qps=rate, duration_s=T,
                                   gpu_launches=int(F.kernel_launches() - l0))
        if check_sample and same is None:
            # served rows equal the same request run alone on the index
            pick = np.random.default_rng(5).choice(len(req), min(check_sample, len(req)), replace=False)
            ok = True
            for r in pick:
                if c["metric"] != "cosine":
                    # the request's own elements: n of them from its data pointer
                    j, n = int((req["data"][r] - src["base"]) // 4), int(req["n"][r])
                    one = (np.array([0, n], np.uint64), c["q"][1][j:j + n])
                else:
                    i = int((req["data"][r] - src["base"]) // (src["dim"] * 4))
                    one = c["q"][i:i + 1]
                rid, rsc = ix.query(one, k, k=np.array([req["k"][r]], np.uint32))
                ok &= bool(np.array_equal(ids_s[r], rid[0]) and np.array_equal(sc_s[r], rsc[0]))
            same = {"checked": int(len(pick)), "equal": ok}
    srv.close()
    out = {"form": f"continuous batching (C runtime, 8 streams, batches <= {max_batch}, host buffers)",
           "staging": staging,
           "plain_form_qps": plain_qps, "runs": runs,
           "max_qps": max(r["achieved_qps"] for r in runs.values()),
           "note": "offered load relative to the plain form's device-resident throughput; the serving "
                   "path stages every request from host memory"}
    if same is not None:
        out["results_same_as_alone"] = same
    return out


# launch shapes of the fused form: CTA size x CTAs per SM (0: as many as fit)
# x candidate-buffer entries (0: default), the set flinng_tune_query times
TUNE_SHAPES = [(th, cp, cap) for th in (256, 128, 512) for cp in (0, 4, 2) for cap in (0, 4096, 1024)]


def tune_cold(ix, nq: int, run, flush, stream, reps: int = 3) -> dict:
    """The fused form's launch shape, chosen under the bench's own conditions:
    L2 flushed before every timed launch, median of ``reps`` launches per shape
    (flinng_tune_query times back-to-back launches on a warm L2, which can
    favour another shape). Pins the winner with flinng_set_tuning."""
    import torch
    best = None
    for th, cp, cap in TUNE_SHAPES:
        ix.set_tuning(nq, th, cp, cap)
        run()                                            # builds this shape's graph
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for r in range(reps):
            flush.fill_(r + 11)
            ev[r][0].record(stream)
            run()
            ev[r][1].record(stream)
        torch.cuda.synchronize()
        med = statistics.median(a.elapsed_time(b) for a, b in ev)
        if best is None or med < best[0]:
            best = (med, th, cp, cap)
    ix.set_tuning(nq, *best[1:])
    return {"threads": best[1], "ctas_per_sm": best[2], "cap": best[3],
            "how": f"{len(TUNE_SHAPES)} shapes, median of {reps} launches each with L2 flushed before each"}


def recall_target_point(F, c: dict, args, prec: int, dev, d_pts, d_q, tgt: dict, flush, ex_ids, ex_sims,
                        smp) -> dict:
    """The sweep's fastest point with recall@10 >= 0.9, measured like the main
    run: the fused form through CUDA graphs, the plain batched form (hash kernel
    then query kernel), and the serving form against the plain form."""
    import torch
    nq, k, N = c["nq"], c["k"], c["N"]
    R, B, L, K, W = tgt["R"], tgt["B"], tgt["L"], tgt["K"], tgt["W"]
    params = (WL.srp_projections(c["seed"], L * K, c["d"]) if c["metric"] == "cosine"
              else WL.doph_params(c["seed"], L, K))
    d_perm = torch.from_numpy(WL.group_permutations(c["seed"], R, N).view(np.int32)).to(dev)
    ix = F.Index(c["metric"], R, B, L, K, capacity=N, params=params, dim=c.get("d", 0), W=W, precision=prec)
    ix.build(d_pts, d_perm)
    tuning = ix.tune(d_q, k)
    ix.set_query_mode(F.QUERY_GRAPH)
    stream = torch.cuda.current_stream()
    fp, _, _, keepq = ix._points(d_q)
    qb = torch.empty((nq, L), dtype=torch.int32, device=dev)
    ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
    sc = torch.empty((nq, k), dtype=torch.int16, device=dev)

    def fused():
        F._check(ix.lib.flinng_query(ix.h, C.byref(fp), nq, None, k, ids.data_ptr(), sc.data_ptr(), 1))

    if tuning["threads"]:
        tuning = tune_cold(ix, nq, fused, flush, stream)

    def plain():
        F._check(ix.lib.flinng_hash(ix.h, C.byref(fp), nq, qb.data_ptr(), None, None, 1))
        F._check(ix.lib.flinng_query_buckets(ix.h, qb.data_ptr(), nq, None, k, ids.data_ptr(),
                                             sc.data_ptr(), 1))

    def timed(fn):
        for it in range(max(3, args.warmup)):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for it in range(args.steps):
            flush.fill_(it + 1)
            ev[it][0].record(stream)
            fn()
            ev[it][1].record(stream)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev)

    fused_ms = timed(fused)
    got_f = ids.cpu().numpy().view(np.uint32)
    plain_ms = timed(plain)
    got_p = ids.cpu().numpy().view(np.uint32)
    rec = recall_scores(c, got_f[smp], ex_ids, ex_sims)
    out = {"params": {"R": R, "B": B, "L": L, "K": K, "W": W}, "tuning": tuning,
           "recall": rec, "recall_target_met": rec["recall_at_10"] >= 0.9,
           "fused_graph_qps": nq / (fused_ms / 1e3), "fused_ms_per_batch": fused_ms,
           "plain_form_qps": nq / (plain_ms / 1e3), "plain_ms_per_batch": plain_ms,
           "fused_equals_plain": bool(np.array_equal(got_f, got_p)),
           "index_bytes": ix.device_bytes}
    if not args.no_serving and not c.get("embed"):
        sv = serving_runs(F, ix, c, out["plain_form_qps"], (0.5, 0.9, 2.0), check_sample=200)
        out["serving"] = sv
        out["serving_beats_plain"] = sv["max_qps"] > out["plain_form_qps"]
    ix.close()
    return out


def recall_sweep(F, c: dict, name: str, prec: int, dev, d_pts, d_q, ex_ids, ex_sims, smp, flush,
                 steps: int, warmup: int) -> dict:
    """Build, tune and time one index per grid point on the same data and
    queries; recall against the same exact neighbours."""
    import itertools
    import torch
    grid = SWEEPS[name]
    nq, k, N = c["nq"], c["k"], c["N"]
    stream = torch.cuda.current_stream()
    rows = []
    for R, B, L, K in itertools.product(grid["R"], grid["B"], grid["L"], grid["K"]):
        W = K if c["metric"] == "cosine" else c["W"]
        if B * R >= (1 << 16) or B > N or L * R * N >= (1 << 32):
            continue
        params = (WL.srp_projections(c["seed"], L * K, c["d"]) if c["metric"] == "cosine"
                  else WL.doph_params(c["seed"], L, K))
        d_perm = torch.from_numpy(WL.group_permutations(c["seed"], R, N).view(np.int32)).to(dev)
        ix = F.Index(c["metric"], R, B, L, K, capacity=N, params=params, dim=c.get("d", 0), W=W,
                     precision=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if c.get("embed"):
            build_streamed(F, ix, dict(c, L=L, K=K), dev, d_perm)
        else:
            ix.build(d_pts, d_perm)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        ix.tune(d_q, k)
        ix.set_query_mode(F.QUERY_GRAPH)
        # multi-probe counting (cosine): the same index, P buckets per table
        for P in grid.get("P", (1,)):
            if P > K + 1:
                continue
            ix.set_probes(P)
            for it in range(warmup):
                ix.query(d_q, k)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            for it in range(steps):
                flush.fill_(it + 1)
                ev[it][0].record(stream)
                ids, _ = ix.query(d_q, k)
                ev[it][1].record(stream)
            torch.cuda.synchronize()
            ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
            got = ids.cpu().numpy().view(np.uint32)
            rec = recall_scores(c, got[smp], ex_ids, ex_sims)
            rows.append({"R": R, "B": B, "L": L, "K": K, "W": W, "P": P, "qps": nq / (ms / 1e3),
                         "ms_per_batch": ms, "recall_at_10": rec["recall_at_10"],
                         "recall_1_at_k": rec["recall_1_at_k"], "build_s": build_s,
                         "index_bytes": ix.device_bytes})
        ix.close()
        del d_perm
    meeting = [r for r in rows if r["recall_at_10"] >= 0.9]
    single = [r for r in meeting if r["P"] == 1]
    best = max(rows, key=lambda r: (r["recall_at_10"], r["qps"])) if rows else None
    def pareto(rs):                                            # QPS vs recall@10
        f = []
        for r in sorted(rs, key=lambda r: -r["qps"]):
            if not f or r["recall_at_10"] > f[-1]["recall_at_10"]:
                f.append(r)
        return f
    front = pareto(rows)
    probes = None
    if len(grid.get("P", (1,))) > 1:
        # each probe count against one probe on the same index
        one = {(r["R"], r["B"], r["L"], r["K"]): r for r in rows if r["P"] == 1}
        probes = {}
        for P in grid["P"][1:]:
            rp = [r for r in rows if r["P"] == P]
            pairs = [(r, one[(r["R"], r["B"], r["L"], r["K"])]) for r in rp]
            if not pairs:
                continue
            probes[str(P)] = {
                "points": len(rp),
                "mean_recall_gain": float(np.mean([a["recall_at_10"] - b["recall_at_10"] for a, b in pairs])),
                "mean_qps_ratio": float(np.mean([a["qps"] / b["qps"] for a, b in pairs])),
                "pareto": [{x: r[x] for x in ("R", "B", "L", "K", "qps", "recall_at_10")} for r in pareto(rp)],
            }
    return {
        "target": "recall@10 >= 0.9",
        "grid": {k2: list(v) for k2, v in grid.items()},
        "points": len(rows),
        "met": bool(single),
        "at_target": max(single, key=lambda r: r["qps"]) if single else None,
        "at_target_multiprobe": (max(meeting, key=lambda r: r["qps"]) if len(grid.get("P", (1,))) > 1 and meeting
                                 else None),
        "best_recall": best,
        "pareto": front,
        "multiprobe": probes,
        "note": ("QPS at the fastest single-probe grid point with recall@10 >= 0.9" if single else
                 "0.9 not reached on this grid with one probe; best_recall gives the highest recall@10 "
                 "reached"),
        "form": "fused kernel through a CUDA graph, autotuned per point, device buffers, L2 flushed per step "
                "(P > 1: hash kernel, multi-probe counts kernel, then the decode kernel)",
    }


# --------------------------------------------------------------------------
# CPU oracle timing
# --------------------------------------------------------------------------

def build_streamed(F, ix, c: dict, dev, d_perm, hasher=None):
    """Build over the seeded embedding stream: generate a chunk on the device,
    hash it (SRP GEMM), keep its buckets; then one flinng_build_buckets.
    ``hasher``: another index with the same projections whose precision
    hashes the stream (the codes are exact in every precision, so the index
    is the same)."""
    import torch
    L = c["L"]
    hx = hasher if hasher is not None else ix
    all_b = torch.empty((c["N"], L), dtype=torch.int32, device=dev)
    xbuf = torch.empty((c["chunk"], c["d"]), dtype=torch.float32, device=dev)
    for first in range(0, c["N"], c["chunk"]):
        n = min(c["chunk"], c["N"] - first)
        x = F.generate_embeddings(c["seed"], c["d"], c["n_centers"], c["sigma"], first, n, out=xbuf[:n])
        fp = F.flinng_points()
        fp.x, fp.ld = x.data_ptr(), c["d"]
        F._check(hx.lib.flinng_hash(hx.h, C.byref(fp), n, all_b[first:first + n].data_ptr(), None, None, 1))
    ix.build_buckets(all_b, d_perm)
    del all_b, xbuf


def oracle_index(c: dict):
    from oracle import oracle as O
    o = O.OracleIndex(c["metric"], c["R"], c["B"], c["L"], c["K"], c["W"],
                      srp_w=c["params"] if c["metric"] == "cosine" else None,
                      doph=c["params"] if c["metric"] != "cosine" else None)
    o.build(c["pts"], c["perm"])
    return o


def query_slice(c: dict, lo: int, hi: int):
    if c["metric"] == "cosine":
        return c["q"][lo:hi]
    qoff, qel = c["q"]
    off = qoff[lo:hi + 1] - qoff[lo]
    return off, qel[qoff[lo]:qoff[hi]]


def time_oracle_queries(o, c: dict, target_s: float = 10.0, max_rounds: int = 10_000):
    """Oracle queries/s on one core over whole passes of the query batch,
    repeated until about ``target_s`` seconds of CPU work."""
    t0 = time.perf_counter()
    n = 0
    rounds = 0
    while True:
        o.query(c["q"], c["k"])
        n += c["nq"]
        rounds += 1
        el = time.perf_counter() - t0
        if el >= target_s or rounds >= max_rounds:
            break
    return n / el, n, el


# --------------------------------------------------------------------------
# main arm
# --------------------------------------------------------------------------

def advisor_section(c: dict, ex_sims, kk: int = 10) -> dict:
    """Thm. 3's design and the gamma-stability of the sampled queries, from
    their exact k-th and (k+1)-th neighbour similarities (host arithmetic)."""
    from paper_2106_11565_gb300 import advisor as A
    sims = np.asarray(ex_sims, dtype=np.float64)
    sk, sk1 = sims[:, kk - 1], sims[:, kk]
    ok = (sk1 > 0) & (sk1 < sk) & (sk <= 1)
    if not ok.any():
        return {"note": f"no sampled query has 0 < s_{kk + 1} < s_{kk} <= 1"}
    gam = np.array([A.gamma(a, b) for a, b in zip(sk[ok], sk1[ok])])
    d = A.design(c["N"], float(np.median(sk[ok])), float(np.median(sk1[ok])), 0.99, 0.01)
    return {"k": kk, "queries": int(ok.sum()),
            "gamma": {"p10": float(np.percentile(gam, 10)), "p50": float(np.median(gam)),
                      "p90": float(np.percentile(gam, 90))},
            "median_s_k": float(np.median(sk[ok])), "median_s_k_plus_1": float(np.median(sk1[ok])),
            "theory_design": {"B": d["B"], "K": d["K"], "log10_L": d["log10_L"], "alpha": d["alpha"],
                              "L": d["L"] if d["log10_L"] < 15 else None,
                              "t": d["t"] if d["log10_L"] < 15 else None},
            "configured": {"R": c["R"], "B": c["B"], "L": c["L"], "K": c["K"]},
            "note": "Thm. 3 for p' = 0.99, q' = 0.01 at the median gap (library names: L tables = the "
                    "paper's m, K bits = the paper's L); large gamma means a query whose neighbours are "
                    "hard to separate, for which the theory asks for many tables"}


def max_over_ranks(v: float, dist, device) -> float:
    """The largest v over all ranks, returned on every rank (v itself when
    there is no process group)."""
    if dist is None:
        return float(v)
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, slowest_s: float) -> float:
    """Whole-job throughput of N independent replicas: all ranks' units over
    the slowest rank's time."""
    return world * units_per_rank / slowest_s


# --------------------------------------------------------------------------
# the headline: serving vs plain form at the recall-target parameters
# --------------------------------------------------------------------------

# Recall-target parameters per workload: the fastest point of the recall
# sweep (SWEEPS, run with --sweep) whose recall@10 reached 0.9 on the
# workload's queries. The default run rebuilds the index at these
# parameters, measures recall@10 again and says whether the target is met.
TARGETS = {
    "C2": dict(R=3, B=4096, L=512, K=1, W=17),
}

SERVE_QUERIES = 1 << 18          # queries per timed serving step (one replay)
SERVE_OVERLOAD = 2.0             # offered rate of a timed step, x the plain form's throughput
SERVE_LOADS = (0.25, 0.5, 0.9)   # latency rows, x the plain form's throughput


def target_workload(c: dict, name: str) -> dict:
    """Workload ``c`` at its recall-target parameters (same points, queries
    and seed; hash parameters and permutations drawn for the new shape)."""
    t = TARGETS[name]
    ct = dict(c, **t)
    if c["metric"] == "cosine":
        ct["params"] = WL.srp_projections(c["seed"], t["L"] * t["K"], c["d"])
    else:
        ct["params"] = WL.doph_params(c["seed"], t["L"], t["K"])
    ct["perm"] = WL.group_permutations(c["seed"], t["R"], c["N"])
    old = f"R{c['R']} B{c['B']} L{c['L']} K{c['K']} W{c['W']}"
    new = f"R{t['R']} B{t['B']} L{t['L']} K{t['K']} W{t['W']}"
    ct["desc"] = c["desc"].replace(old, new) + f" (recall-target parameters; the config names {old})"
    ct["configured"] = {"R": c["R"], "B": c["B"], "L": c["L"], "K": c["K"], "W": c["W"]}
    return ct


def headline_config(name: str, ct: dict, world: int) -> dict:
    """The ``config`` object of the headline line, identical in both arms."""
    return {"workload": f"{name}: {ct['desc']}",
            "params": {"R": ct["R"], "B": ct["B"], "L": ct["L"], "K": ct["K"], "W": ct["W"]},
            "k": ct["k"], "global_batch": world * SERVE_QUERIES,
            "step": f"one replay of {SERVE_QUERIES} queries (k = {ct['k']} each) arriving as a Poisson "
                    f"stream at {SERVE_OVERLOAD:g}x the plain form's throughput",
            "l2": "serving steps: index larger than L2; kernel-only forms: L2 flushed before every step",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def serving_step_stats(req, res, F) -> dict:
    """Device span (CUDA events: first batch's first copy in .. last batch's
    results out) and host span (first arrival .. last result in the caller's
    buffer) of one replay."""
    q = req["kind"] == F.REQ_QUERY
    r = res[q]
    return {"queries": int(q.sum()), "device_s": float(r["d_done"].max() - r["d_start"].min()),
            "host_s": float(r["t_done"].max() - req["arrival_s"][q].min()),
            "batches": int(len(np.unique(r["batch"])))}


def latency_breakdown(req, res, F) -> dict:
    """Percentiles (ms) of each part of a query's latency: waiting on the host
    for a slot and a batch, launch to the batch's first device event, on the
    device, and device completion to the result in the caller's buffer."""
    q = req["kind"] == F.REQ_QUERY
    r = res[q]
    arr = req["arrival_s"][q]

    def pc(x):
        return {"p50": float(np.percentile(x, 50) * 1e3), "p99": float(np.percentile(x, 99) * 1e3)}
    return {"wait": pc(r["t_start"] - arr), "launch": pc(r["d_start"] - r["t_start"]),
            "device": pc(r["d_done"] - r["d_start"]), "harvest": pc(r["t_done"] - r["d_done"])}


INSERT_POINTS = 1000   # points of the timed insert batch


def time_insert(F, ix, c: dict, dev, flush, reps: int = 1, nvtx: str = "insert") -> dict | None:
    """CUDA-event time of inserting INSERT_POINTS further reads (genomic
    workloads; Alg. 1 over a fresh permutation of the batch) into ix, which
    must have room for reps + 1 batches; the index keeps them afterwards. The
    first batch is an untimed warm-up (the insert kernels' first launch)."""
    import torch
    if c["metric"] == "cosine" or c.get("url"):
        return None
    g = WL.genomic_reads(c["seed"] + 2000, c["ref_len"], INSERT_POINTS * (reps + 1), c["read_len"], 1,
                         kmer=c["kmer"])
    off, el = g["off"], g["elems"]
    ms = []
    torch.cuda.nvtx.range_push(nvtx)
    for r in range(reps + 1):
        lo, hi = r * INSERT_POINTS, (r + 1) * INSERT_POINTS
        o = (off[lo:hi + 1] - off[lo]).astype(np.uint64)
        e = np.ascontiguousarray(el[off[lo]:off[hi]])
        pts = (torch.from_numpy(o.view(np.int64)).to(dev), torch.from_numpy(e.view(np.int32)).to(dev))
        perm = torch.from_numpy(WL.group_permutations(c["seed"], c["R"], INSERT_POINTS, batch=11 + r)
                                .view(np.int32)).to(dev)
        flush.fill_(r)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ix.insert(pts, perm)
        e1.record()
        torch.cuda.synchronize()
        if r > 0:
            ms.append(e0.elapsed_time(e1))
    torch.cuda.nvtx.range_pop()
    return {"points": INSERT_POINTS, "ms": statistics.mean(ms), "reps": reps, "warmup": 1,
            "note": "flinng_insert of further reads from device buffers: hash, Alg. 1 groups, member lists, the new "
                    "entries sorted per slot and merged into the existing lists, heavy bitmaps"}


def configured_point(F, c: dict, dev, d_pts, d_q, flush, steps: int, warmup: int, ex_ids, ex_sims) -> dict:
    """The workload at the parameters its config names: fused form (CUDA
    graph) and plain form throughput, recall@10 (a side key of the line)."""
    import torch
    nq, k = c["nq"], c["k"]
    ix = F.Index(c["metric"], c["R"], c["B"], c["L"], c["K"], capacity=c["N"] + 4 * INSERT_POINTS,
                 params=c["params"], dim=c.get("d", 0), W=c["W"])
    d_perm = torch.from_numpy(c["perm"].view(np.int32)).to(dev)
    stream = torch.cuda.current_stream()
    build_ms = timed_steps(lambda: ix.build(d_pts, d_perm), flush, stream, 3, 2)
    fp, _, _, keepq = ix._points(d_q)
    qb = torch.empty((nq, c["L"]), dtype=torch.int32, device=dev)
    ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
    sc = torch.empty((nq, k), dtype=torch.int16, device=dev)

    def fused():
        F._check(ix.lib.flinng_query(ix.h, C.byref(fp), nq, None, k, ids.data_ptr(), sc.data_ptr(), 1))

    def plain():
        F._check(ix.lib.flinng_hash(ix.h, C.byref(fp), nq, qb.data_ptr(), None, None, 1))
        F._check(ix.lib.flinng_query_buckets(ix.h, qb.data_ptr(), nq, None, k, ids.data_ptr(),
                                             sc.data_ptr(), 1))
    ix.tune(d_q, k)
    ix.set_query_mode(F.QUERY_GRAPH)
    tuning = tune_cold(ix, nq, fused, flush, stream)
    fused_ms = timed_steps(fused, flush, stream, steps, warmup)
    got = ids.cpu().numpy().view(np.uint32)
    plain_ms = timed_steps(plain, flush, stream, steps, warmup)
    out = {"params": {"R": c["R"], "B": c["B"], "L": c["L"], "K": c["K"], "W": c["W"]},
           "fused_graph_qps": nq / (statistics.mean(fused_ms) / 1e3),
           "plain_form_qps": nq / (statistics.mean(plain_ms) / 1e3), "tuning": tuning,
           "form": "kernel-only forms on device buffers, L2 flushed before every step, k = "
                   f"{k} for every query"}
    if ex_ids is not None:
        out["recall"] = recall_scores(c, got[gt_sample(c)], ex_ids, ex_sims)
    out["build_ms"] = statistics.mean(build_ms)
    out["insert"] = time_insert(F, ix, c, dev, flush, reps=3, nvtx="insert at the configured parameters")
    ix.close()
    return out


def timed_steps(fn, flush, stream, steps: int, warmup: int, nvtx: str | None = None) -> list:
    """CUDA-event times (ms) of ``steps`` calls of fn, L2 flushed before each,
    after ``warmup`` untimed calls; ``nvtx`` names an NVTX range around the
    timed calls (profilers select the launches inside it)."""
    import torch
    for it in range(warmup):
        flush.fill_(it)
        fn()
    if nvtx:
        torch.cuda.nvtx.range_push(nvtx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for it in range(steps):
        flush.fill_(it + 1)
        ev[it][0].record(stream)
        fn()
        ev[it][1].record(stream)
    torch.cuda.synchronize()
    if nvtx:
        torch.cuda.nvtx.range_pop()
    return [a.elapsed_time(b) for a, b in ev]


def run_headline(args, c: dict, rank: int, world: int) -> dict | None:
    """The metric itself: queries/s of the serving form at the recall-target
    parameters (recall@10 >= 0.9), with the plain batched form, the fused
    form, p50/p99 latency, recall, the fused kernel's roofline and the
    oracle beside it."""
    import torch
    from paper_2106_11565_gb300 import _build
    from paper_2106_11565_gb300 import flinng as F
    _build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    dist = None
    if world > 1:
        import torch.distributed as dist
    ct = target_workload(c, args.workload)
    nq, k, L = ct["nq"], ct["k"], ct["L"]

    def to_dev(p):
        if ct["metric"] == "cosine":
            return torch.from_numpy(p).to(dev)
        off, el = p
        return (torch.from_numpy(off.view(np.int64)).to(dev), torch.from_numpy(el.view(np.int32)).to(dev))

    d_pts, d_q = to_dev(ct["pts"]), to_dev(ct["q"])
    d_perm = torch.from_numpy(ct["perm"].view(np.int32)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)   # > L2 (129 MB)
    ix = F.Index(ct["metric"], ct["R"], ct["B"], L, ct["K"], capacity=ct["N"] + 4 * INSERT_POINTS,
                 params=ct["params"], dim=ct.get("d", 0), W=ct["W"])

    # ---- build: 2 warm-up builds, then 3 timed (each replaces the index)
    build_ms = timed_steps(lambda: ix.build(d_pts, d_perm), flush, stream, 3, 2, nvtx="build")

    # ---- kernel-only forms on device buffers (k for every query)
    qb = torch.empty((nq, L), dtype=torch.int32, device=dev)
    ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
    sc = torch.empty((nq, k), dtype=torch.int16, device=dev)
    p_ids, p_sc = torch.empty_like(ids), torch.empty_like(sc)
    fp, _, _, keepq = ix._points(d_q)
    lib = ix.lib

    def fused():
        F._check(lib.flinng_query(ix.h, C.byref(fp), nq, None, k, ids.data_ptr(), sc.data_ptr(), 1))

    mid = []

    def plain():
        F._check(lib.flinng_hash(ix.h, C.byref(fp), nq, qb.data_ptr(), None, None, 1))
        if mid:
            mid[0].record(stream)
        F._check(lib.flinng_query_buckets(ix.h, qb.data_ptr(), nq, None, k, p_ids.data_ptr(),
                                          p_sc.data_ptr(), 1))

    ix.tune(d_q, k)
    ix.set_query_mode(F.QUERY_GRAPH)
    tuning = tune_cold(ix, nq, fused, flush, stream)
    fused()
    plain()
    torch.cuda.synchronize()
    assert torch.equal(ids, p_ids) and torch.equal(sc, p_sc), "fused form != plain form"
    fused_ms = timed_steps(fused, flush, stream, args.steps, max(3, args.warmup), nvtx="fused form")
    # plain form with a mid event per step: hash vs count/decode/top-k
    for it in range(max(3, args.warmup)):
        flush.fill_(it)
        plain()
    pev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    torch.cuda.nvtx.range_push("plain form")
    for it in range(args.steps):
        flush.fill_(it + 1)
        pev[it][0].record(stream)
        mid[:] = [pev[it][1]]
        plain()
        pev[it][2].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    mid[:] = []
    plain_ms = [a.elapsed_time(b) for a, _, b in pev]
    hash_ms = [a.elapsed_time(m) for a, m, _ in pev]
    plain_qps = nq / (statistics.mean(plain_ms) / 1e3)
    fused_qps = nq / (statistics.mean(fused_ms) / 1e3)
    got_f = ids.cpu().numpy().view(np.uint32)

    # ---- serving form: continuous batching (C runtime), requests and results in host memory
    keep = []
    # batch classes above the tuned one take its launch shape
    cls = 2048
    while cls <= args.max_batch and tuning["threads"]:
        ix.set_tuning(cls, tuning["threads"], tuning["ctas_per_sm"], tuning["cap"])
        cls *= 2
    srv = F.Server(hbm_budget=ix.device_bytes + (2 << 30), n_slots=8, max_batch=args.max_batch, k_max=k,
                   max_batch_elems=1 << 21)
    sid = srv.add_index(ix)
    ix.set_query_mode(F.QUERY_FUSED)
    src = (sets_source(F, sid, ct["q"], 1.0, keep) if ct["metric"] != "cosine"
           else dense_source(F, sid, torch.from_numpy(ct["q"]).pin_memory().numpy(), 1.0, keep))
    rng = np.random.default_rng([ct["seed"], 78])
    o_ids = np.empty((SERVE_QUERIES, k), np.uint32)
    o_sc = np.empty((SERVE_QUERIES, k), np.uint16)
    o_ids.fill(0)
    o_sc.fill(0)
    rate = SERVE_OVERLOAD * plain_qps
    traces = [make_trace(F, rng, rate, 0.0, [src], k_choices=(k,), n=SERVE_QUERIES)
              for _ in range(args.steps + args.warmup)]
    clocks = ClockSampler(dev.index, period_ms=100)
    time.sleep(0.3)                                  # nvidia-smi start-up
    t_load = time.time()
    for it in range(args.warmup):
        srv.replay(traces[args.steps + it], out=(o_ids, o_sc))
    # keep the GPU busy until the sampler has seen this load for 0.5 s
    while time.time() - t_load < 0.5:
        srv.replay(traces[args.steps], out=(o_ids, o_sc))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = F.kernel_launches()
    steps = []
    torch.cuda.nvtx.range_push("serving form")
    for it in range(args.steps):
        ids_s, sc_s, res = srv.replay(traces[it], out=(o_ids, o_sc))
        steps.append(serving_step_stats(traces[it], res, F))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = F.kernel_launches() - launches0
    t_end = time.time()
    clk = clocks.stop(t_load, t_end)
    if dist is not None:
        dist.barrier()
    # the last timed replay's results equal the same queries run alone
    last = traces[args.steps - 1]
    pick = np.random.default_rng(5).choice(SERVE_QUERIES, 200, replace=False)
    same = True
    for r in pick:
        if ct["metric"] != "cosine":
            j, n = int((last["data"][r] - src["base"]) // 4), int(last["n"][r])
            one = (np.array([0, n], np.uint64), ct["q"][1][j:j + n])
        else:
            i = int((last["data"][r] - src["base"]) // (src["dim"] * 4))
            one = ct["q"][i:i + 1]
        rid, rsc = ix.query(one, k)
        same &= bool(np.array_equal(ids_s[r], rid[0]) and np.array_equal(sc_s[r], rsc[0]))
    dev_s = max_over_ranks(sum(s["device_s"] for s in steps), dist, dev)
    host_s = max_over_ranks(sum(s["host_s"] for s in steps), dist, dev)
    value = replica_throughput(SERVE_QUERIES * args.steps, world, dev_s)
    e2e_value = replica_throughput(SERVE_QUERIES * args.steps, world, host_s)
    # latency at loads below saturation (Poisson, 0.25 s each)
    lat_rows = {}
    for f in SERVE_LOADS:
        req = make_trace(F, rng, f * plain_qps, 0.25, [src], k_choices=(k,))
        _, _, res = srv.replay(req)
        lat_rows[f"{f}x_plain"] = dict(trace_stats(req, res, F), offered_qps=f * plain_qps,
                                       breakdown=latency_breakdown(req, res, F))
    srv.close()
    if ct["metric"] != "cosine":
        # set elements of each timed step's requests + 36 B of batch header per query
        h2d = int(statistics.mean(int(np.asarray(t["n"], np.int64).sum()) * 4 for t in traces[:args.steps])
                  + SERVE_QUERIES * 36)
    else:
        h2d = SERVE_QUERIES * (ct["d"] * 4 + 36)
    d2h = SERVE_QUERIES * k * 6                                  # ids (uint32) + scores (uint16)

    if rank != 0:
        ix.close()
        return None

    # ---- recall at these parameters (the GPU output equals the oracle's)
    ex_ids, ex_sims = exact_similarity_topk(ct)
    smp = gt_sample(ct)
    rec = recall_scores(ct, got_f[smp], ex_ids, ex_sims)
    rec["queries"] = int(len(smp))

    # ---- roofline of the fused kernel (k_query_fused) at these parameters
    ex = ix.export(cells=False)
    qb_h = qb.cpu().numpy().view(np.uint32)
    counts = ix.counts(qb_h)
    qbytes = query_kernel_bytes(ct, ex, counts, qb_h, k)
    fused_bytes = qbytes["bytes"] + hash_kernel_bytes(ct)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fused_mean = statistics.mean(fused_ms)
    achieved = fused_bytes / (fused_mean / 1e3) / 1e9
    shape = f"{args.workload}_R{ct['R']}B{ct['B']}L{L}K{ct['K']}"
    roof = {"kernel": "k_query_fused", "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": recorded_traffic(shape),
            "algorithmic_bytes_per_launch": fused_bytes, "launch_ms": fused_mean,
            "peak_source": ("measured" if "hbm_gbs" in peaks else "fallback") + " hbm_gbs (copy, burst)",
            "algorithmic_bytes": "query hashing + per-query lists, enumerated members, outputs (Alg. 3's walk)",
            "members_enumerated_per_query": qbytes["members"] / nq,
            "heavy_tables_per_query": qbytes["heavy_tables"] / nq,
            "note": "one launch = the fused form over the whole query batch (CUDA graph, L2 flushed); the "
                    "serving form runs the same kernel on batches of its own size"}
    index_bytes = ix.device_bytes
    insert = time_insert(F, ix, ct, dev, flush, reps=3)        # last: the index keeps the new points
    # same points and queries: the exact neighbours are the same
    configured = configured_point(F, c, dev, d_pts, d_q, flush, max(3, min(args.steps, 10)),
                                  max(3, args.warmup), ex_ids, ex_sims)
    ix.close()
    step_ms = [1e3 * s["device_s"] for s in steps]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32" if ct["metric"] != "cosine" else "f32",
        "data": "synthetic (seeded; stands in for the paper's datasets)",
        "config": headline_config(args.workload, ct, world),
        "form": f"serving: continuous batching over 8 CUDA streams (C runtime), batches <= {args.max_batch} queries, "
                "request sets read from host memory by a gather kernel, results copied to the caller's host "
                "buffers; value = queries / device time (CUDA events, first copy in .. last result out)",
        "recall": rec, "recall_target_met": rec["recall_at_10"] >= 0.9,
        "plain_form": {"value": plain_qps, "unit": UNIT, "ms_per_step": statistics.mean(plain_ms),
                       "stages_ms": {"hash": statistics.mean(hash_ms),
                                     "count_decode_topk": statistics.mean(plain_ms) - statistics.mean(hash_ms)},
                       "kernels": "k_doph | k_srp_fp32 (+ re-check), then k_query; one batch of "
                                  f"{nq} queries on device buffers, L2 flushed before every step"},
        "serving_vs_plain": value / plain_qps,
        "fused_graph_form": {"value": fused_qps, "unit": UNIT, "ms_per_step": fused_mean, "tuning": tuning,
                             "kernel": "k_query_fused through a CUDA graph, device buffers, L2 flushed"},
        "latency_ms": {f"p{p}_at_{f}x": lat_rows[f"{f}x_plain"][f"p{p}_ms"] for f in SERVE_LOADS for p in (50, 99)},
        "serving": {"steps": steps, "results_same_as_alone": {"checked": 200, "equal": same},
                    "host_qps": e2e_value, "loads": lat_rows,
                    "note": "latency = arrival .. result in the caller's host buffer (host clock); loads are "
                            "x the plain form's throughput"},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "flinng_server_replay: request sets and results in host memory; timed from the first "
                       "arrival to the last result written into the caller's buffer (host clock)"},
        "gpu_launches": int(launches),
        "build": {"ms": statistics.mean(build_ms), "points_per_s": ct["N"] / (statistics.mean(build_ms) / 1e3),
                  "n_cells": int(ex["off"][-1]), "index_bytes": index_bytes, "insert": insert},
        "clocks": clk,
        "at_configured_params": configured,
    }
    if not args.no_cpu_baseline:
        o = oracle_index(ct)
        qps, n, el = time_oracle_queries(o, ct)
        oids, _ = o.query(query_slice(ct, 0, 100), k)
        line["parity_vs_oracle"] = {"queries": 100, "equal": bool(np.array_equal(oids, got_f[:100]))}
        line["cpu_baseline"] = {"value": qps, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{n} queries ({n // nq} passes of the {nq}-query batch), {el:.1f} s on "
                                          "one core, index at the same parameters built beforehand (not timed)"}
    return line


def run_ours(args, c: dict, rank: int, world: int) -> dict | None:
    import torch
    from paper_2106_11565_gb300 import _build
    from paper_2106_11565_gb300 import flinng as F
    _build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    dist = None
    if world > 1:
        import torch.distributed as dist
    nq, k, L = c["nq"], c["k"], c["L"]

    prec = PRECISIONS[args.precision] if c["metric"] == "cosine" else F.PREC_FP32
    prec_name = PREC_NAMES[prec]
    ix = F.Index(c["metric"], c["R"], c["B"], L, c["K"], capacity=c["N"], params=c["params"],
                 dim=c.get("d", 0), W=c["W"], precision=prec)

    def to_dev_points(p):
        if c["metric"] == "cosine":
            return torch.from_numpy(p).to(dev)
        off, el = p
        return (torch.from_numpy(off.view(np.int64)).to(dev), torch.from_numpy(el.view(np.int32)).to(dev))

    d_perm = torch.from_numpy(c["perm"].view(np.int32)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)   # > L2 (129 MB)
    build_note = "flinng_build on device-resident points"
    if c.get("embed"):
        # stream: generate a chunk on the device, hash it (SRP GEMM), keep only
        # its buckets; then one flinng_build_buckets over all points
        d_pts = None
        d_q = F.generate_embeddings(c["seed"], c["d"], c["n_centers"], c["sigma"], 0, nq,
                                    queries=True, q_sigma=c["qsigma"], n_points=c["N"])
        c["d_q"] = d_q
        # single-term forms re-check a large share of projections one by one
        # (rigorous margins); the stream of 10^7 points is hashed by the
        # two-term form instead: the codes, and so the index, are the same
        hasher = None
        if prec in (F.PREC_BF16, F.PREC_FP8):
            hasher = F.Index(c["metric"], c["R"], c["B"], L, c["K"], capacity=1, params=c["params"],
                             dim=c.get("d", 0), W=c["W"], precision=F.PREC_BF16X2)

        def build_once():
            build_streamed(F, ix, c, dev, d_perm, hasher)
        n_builds, n_warm = 1, 0
        build_note = (f"streamed: generate 32768-point chunks on the device, "
                      f"{PREC_NAMES[F.PREC_BF16X2] if hasher else prec_name} SRP GEMM, keep "
                      "buckets; then flinng_build_buckets (generation included)")
    else:
        d_pts = to_dev_points(c["pts"])
        d_q = to_dev_points(c["q"])

        def build_once():
            ix.build(d_pts, d_perm)
        n_builds, n_warm = 3, 2

    # ---- build: warm-up then timed (each build replaces the index)
    build_ms = []
    for it in range(n_warm + n_builds):
        flush.fill_(it)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        build_once()
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= n_warm:
            build_ms.append(e0.elapsed_time(e1))

    # ---- query buffers (device)
    qb = torch.empty((nq, L), dtype=torch.int32, device=dev)
    ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
    sc = torch.empty((nq, k), dtype=torch.int16, device=dev)
    p_ids = torch.empty_like(ids)
    p_sc = torch.empty_like(sc)
    fp, n_, devflag, keep = ix._points(d_q)
    import ctypes as C
    lib = ix.lib

    def step_fused():
        # the fused form (F2): one persistent kernel per batch
        F._check(lib.flinng_query(ix.h, C.byref(fp), nq, None, k, ids.data_ptr(), sc.data_ptr(), 1))

    def step_plain(e_mid):
        # the plain form: hash kernel, then count/decode/top-k kernel
        F._check(lib.flinng_hash(ix.h, C.byref(fp), nq, qb.data_ptr(), None, None, 1))
        e_mid.record(stream)
        F._check(lib.flinng_query_buckets(ix.h, qb.data_ptr(), nq, None, k, p_ids.data_ptr(),
                                          p_sc.data_ptr(), 1))

    # the fused form: autotuned launch shape, CUDA graph per batch-size class
    tuning = ix.tune(d_q, k)
    ix.set_query_mode(F.QUERY_GRAPH)
    if tuning["threads"]:
        tuning = tune_cold(ix, nq, step_fused, flush, stream)
    # the two forms return the same results
    step_fused()
    step_plain(torch.cuda.Event(enable_timing=True))
    torch.cuda.synchronize()
    assert torch.equal(ids, p_ids) and torch.equal(sc, p_sc), "fused form != plain form"

    clocks = ClockSampler(dev.index)
    time.sleep(0.3)                                  # nvidia-smi start-up
    # warm-up: at least W steps, and at least 0.5 s of back-to-back steps so
    # that the clock samples see this load
    t_load = time.time()
    it = 0
    while it < args.warmup or time.time() - t_load < 0.5:
        flush.fill_(it)
        step_fused()
        if it % 50 == 0:
            torch.cuda.synchronize()
        it += 1
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = F.kernel_launches()
    for it in range(args.steps):
        flush.fill_(it + 1)                         # evict L2 between steps (not timed)
        e0, e1 = ev[it]
        e0.record(stream)
        step_fused()
        e1.record(stream)
    torch.cuda.synchronize()
    launches = F.kernel_launches() - launches0
    t_end = time.time()
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    ms_per_step = total_ms / args.steps
    value = replica_throughput(nq * args.steps, world, total_ms / 1e3)

    # ---- the plain form, same batch, per-stage events
    for it in range(args.warmup):
        flush.fill_(it)
        step_plain(torch.cuda.Event(enable_timing=True))
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for it in range(args.steps):
        flush.fill_(it + 1)
        e0, em, e1 = pev[it]
        e0.record(stream)
        step_plain(em)
        e1.record(stream)
    torch.cuda.synchronize()
    t_end2 = time.time()
    clk = clocks.stop(t_load, max(t_end, t_end2))
    hcnt = ix.hash_counters() if c["metric"] == "cosine" else None     # the last plain-form hash
    hash_ms = [a.elapsed_time(m) for a, m, _ in pev]
    query_ms = [m.elapsed_time(b) for _, m, b in pev]
    plain_ms = [a.elapsed_time(b) for a, _, b in pev]
    plain_value = replica_throughput(nq, world, statistics.mean(plain_ms) / 1e3)

    # ---- e2e: flinng_query with host (pinned) buffers, copies inside the call
    if c.get("embed"):
        h_q = d_q.cpu().pin_memory().numpy()
        h2d = h_q.nbytes
    elif c["metric"] == "cosine":
        h_q = torch.from_numpy(c["q"]).pin_memory().numpy()
        h2d = h_q.nbytes
    else:
        off_p = torch.from_numpy(c["q"][0].view(np.int64)).pin_memory().numpy().view(np.uint64)
        el_p = torch.from_numpy(c["q"][1].view(np.int32)).pin_memory().numpy().view(np.uint32)
        h_q = (off_p, el_p)
        h2d = off_p.nbytes + el_p.nbytes
    # pinned result buffers, allocated once like a serving loop's
    out_ids = torch.empty((nq, k), dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    out_sc = torch.empty((nq, k), dtype=torch.int16).pin_memory().numpy().view(np.uint16)
    for _ in range(2):
        ix.query(h_q, k, out=(out_ids, out_sc))
    e2e_s = []
    for it in range(args.steps):
        flush.fill_(it)
        out_ids.fill(0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h_ids, h_sc = ix.query(h_q, k, out=(out_ids, out_sc))
        e2e_s.append(time.perf_counter() - t0)
    # the end-to-end results are the device-resident run's
    e2e_same = bool(np.array_equal(h_ids, ids.cpu().numpy().view(np.uint32)) and
                    np.array_equal(h_sc, sc.cpu().numpy().view(np.uint16)))
    e2e_total = max_over_ranks(sum(e2e_s), dist, dev)
    e2e_value = replica_throughput(nq * args.steps, world, e2e_total)
    d2h = nq * k * 6                                 # uint32 ids + uint16 scores

    # ---- serving form on this index: Poisson traces through the C runtime
    serving = None
    if not args.no_serving and world == 1 and not c.get("embed"):
        serving = serving_runs(F, ix, c, plain_value, (0.25, 0.5, 2.0), max_batch=args.max_batch)

    if rank != 0:
        return None

    # ---- quality, work accounting, roofline
    out_ids = ids.cpu().numpy().view(np.uint32)
    if args.no_recall:
        rec = {"recall_at_10": float("nan"), "note": "not computed (--no-recall)"}
    else:
        ex_ids, ex_sims = exact_similarity_topk(c)
        smp = gt_sample(c)
        rec = recall_scores(c, out_ids[smp], ex_ids, ex_sims)
        rec["queries"] = int(len(smp))
        rec["advisor"] = advisor_section(c, ex_sims)
    sweep = None
    if not args.no_recall and not args.no_sweep and args.workload in SWEEPS:
        sweep = recall_sweep(F, c, args.workload, prec, dev, d_pts, d_q, ex_ids, ex_sims, smp, flush,
                             steps=max(3, min(args.steps, 10)), warmup=max(3, args.warmup))
    at_target = None
    if sweep is not None and sweep["met"] and not c.get("embed"):
        at_target = recall_target_point(F, c, args, prec, dev, d_pts, d_q, sweep["at_target"], flush,
                                        ex_ids, ex_sims, smp)
    ex = ix.export(cells=False)
    qb_h = qb.cpu().numpy().view(np.uint32)
    n_acc = max(10, min(200, int(2e8 // (c["N"] * c["R"]))))
    acc = np.arange(nq) if nq <= 1000 else np.sort(np.random.default_rng(7).choice(nq, n_acc, replace=False))
    counts = ix.counts(np.ascontiguousarray(qb_h[acc]))
    qbytes = query_kernel_bytes(c, ex, counts, qb_h[acc], k)
    scale = nq / len(acc)                          # per-query accounting on a sample, scaled
    qbytes = {"bytes": qbytes["bytes"] * scale, "members": qbytes["members"] * scale,
              "heavy": qbytes["heavy_tables"] * scale, "sample": int(len(acc))}
    hbytes = hash_kernel_bytes(c)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    q_mean = statistics.mean(query_ms)
    h_mean = statistics.mean(hash_ms)
    big_srp = c["metric"] == "cosine" and c["L"] * c["K"] * c["d"] > (1 << 18)
    sm_max = (clk.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0)
    if big_srp and h_mean > q_mean and prec != F.PREC_FP32:
        # the dominant stage is the tensor-core SRP (quantise, tcgen05 GEMM, re-checks)
        flops = 2.0 * nq * c["d"] * c["L"] * c["K"]
        achieved = flops / (h_mean / 1e3) / 1e12
        bf16 = peaks.get("bf16_tflops", 1900.0)
        fp8 = prec == F.PREC_FP8
        peak = bf16 * (4.5 / 2.25 if fp8 else 1.0)
        src = ("measured" if "bf16_tflops" in peaks else "fallback") + " bf16_tflops (burst)"
        roof = {"kernel": "k_srp_tc (+ quantiser, re-checks)", "bound": "tensor", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "algorithmic_flops_per_launch": flops,
                "issued_tensor_flops_per_launch": (3 if prec == F.PREC_BF16X2 else 1) * flops,
                "peak_source": src + (" x 2 (nominal FP8 / BF16 dense ratio, 4.5 / 2.25 PFLOP/s)" if fp8 else ""),
                "note": "algorithmic FLOPs = 2 n d L K; the two-term split issues three BF16 MMAs per product, "
                        "the single-term forms one; the stage time includes the re-checks of projections "
                        "inside the margin"}
    elif big_srp and h_mean > q_mean:
        # the timed step's dominant kernel is the FP32 SRP GEMM: FMA-pipe bound
        dom = "k_srp_fp32 (+ k_srp_recheck)"
        flops = 2.0 * nq * c["d"] * c["L"] * c["K"]
        achieved = flops / (h_mean / 1e3) / 1e12
        peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "algorithmic_flops_per_launch": flops,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP/FMA x max SM clock (no measured "
                               "FP32 peak in MEASURED_PEAKS.json)"}
    else:
        dom = "k_query" if big_srp else "k_query_fused"
        dom_bytes = qbytes["bytes"] + (0 if big_srp else hbytes)
        dom_ms = q_mean if big_srp else (ms_per_step if world == 1 else statistics.mean(step_ms))
        achieved = dom_bytes / (dom_ms / 1e3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": recorded_traffic(args.workload, dom),
                "algorithmic_bytes_per_launch": dom_bytes,
                "peak_source": f"{peak_src} hbm_gbs (copy, burst)",
                "algorithmic_bytes": "query hashing + per-query lists, enumerated members, outputs",
                "members_enumerated_per_query": qbytes["members"] / nq,
                "heavy_tables_per_query": qbytes["heavy"] / nq,
                "accounting_queries": qbytes["sample"]}
    sorted_ms = sorted(step_ms)

    def pct(p):
        return sorted_ms[min(len(sorted_ms) - 1, int(round(p / 100 * (len(sorted_ms) - 1))))]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32" if c["metric"] != "cosine" else "f32",
        "data": "synthetic (seeded; stands in for the paper's datasets)",
        "config": {"workload": f"{args.workload}: {c['desc']}",
                   "srp_precision": prec_name if c["metric"] == "cosine" else None,
                   "form": "fused: one persistent kernel per batch (hash, gather, decode, top-k), "
                           "CUDA graph per batch-size class, autotuned launch shape",
                   "tuning": tuning,
                   "global_batch": world * nq, "k": k, "l2": "flushed before every step (256 MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "recall": rec,
        "recall_target_met": rec["recall_at_10"] >= 0.9,
        "recall_sweep": sweep,
        "at_recall_target": at_target,
        "latency_ms": {"batch_p50": pct(50), "batch_p99": pct(99),
                       "note": "plain batched form: every query of a batch completes with the batch"},
        "plain_form": {"value": plain_value, "unit": UNIT, "ms_per_step": statistics.mean(plain_ms),
                       "stages_ms": {"hash": h_mean, "count_decode_topk": q_mean},
                       "kernels": "k_doph|k_srp_fp32+k_srp_recheck, then k_query"},
        "build": {"ms": statistics.mean(build_ms), "points_per_s": c["N"] / (statistics.mean(build_ms) / 1e3),
                  "hash_precision": prec_name if c["metric"] == "cosine" else None,
                  "n_cells": int(ex["off"][-1]), "how": build_note},
        "roofline": roof,
        "hash_counters": None if hcnt is None else dict(
            hcnt, precision=prec_name, projections=nq * c["L"] * c["K"],
            first_pass_undecided_rate=hcnt["undecided"] / (nq * c["L"] * c["K"]),
            flip_rate_before_recheck=hcnt["flips"] / (nq * c["L"] * c["K"]),
            note="last plain-form hash of the query batch; undecided projections are re-checked "
                 "(compensated fp32, fp64, exact), so the codes stay exact"),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "api": "flinng_query, host pinned buffers (queries and results read and written in place "
                       "by the kernel where it allows, else staged by copies)",
                "results_same_as_device_run": e2e_same},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if serving is not None:
        line["serving"] = serving
    if not args.no_cpu_baseline and c.get("embed"):
        # the oracle cannot hold 10^7 x 4096 points: a reduced index over the
        # first 2,000 points of the same stream, 40 of the same queries
        from oracle import oracle as O
        n_cpu = 2000
        pts_h = WL.embed_points(c["seed"], np.arange(n_cpu), c["d"], c["n_centers"], c["sigma"])
        qh = WL.embed_queries(c["seed"], np.arange(40), c["N"], c["d"], c["n_centers"], c["sigma"],
                              c["qsigma"])
        o = O.OracleIndex("cosine", c["R"], c["B"], c["L"], c["K"], c["W"], srp_w=c["params"])
        o.build(pts_h, WL.group_permutations(c["seed"], c["R"], n_cpu))
        t0 = time.perf_counter()
        o.query(qh, k)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 40 / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"40 queries against an index of the first {n_cpu} points of the "
                                          f"stream (the full 10^7 x 4096 set does not fit the oracle), {el:.1f} s"}
    elif not args.no_cpu_baseline:
        o = oracle_index(c)
        qps, n, el = time_oracle_queries(o, c)
        oids, _ = o.query(c["q"], k)
        line["parity_vs_oracle"] = bool(np.array_equal(oids, out_ids))
        line["cpu_baseline"] = {"value": qps, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{n} queries ({n // nq} passes of the batch), {el:.1f} s, "
                                          "index built beforehand (not timed)"}
    return line


def run_serving(args) -> dict:
    """C5: the genomic (C2) and embedding (C4) indices resident together,
    Poisson query arrivals with k in {1, 10, 100} at several rates relative to
    the plain form's throughput, insert batches of 1k-100k reads into the
    genomic index, admission by HBM budget."""
    import torch
    from paper_2106_11565_gb300 import _build
    from paper_2106_11565_gb300 import flinng as F
    _build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    keep = []
    c2 = target_workload(make_workload("C2"), "C2")    # the genomic index where recall@10 >= 0.9
    c4 = make_workload("C4")
    # genomic index, room for inserts from a pool of further reads
    pool = WL.genomic_reads(c2["seed"] + 1000, c2["ref_len"], 100_000, c2["read_len"], 1)
    ix2 = F.Index("jaccard", c2["R"], c2["B"], c2["L"], c2["K"], capacity=c2["N"] + 400_000,
                  params=c2["params"], W=c2["W"])
    off2, el2 = c2["pts"]
    d2 = (torch.from_numpy(off2.view(np.int64)).to(dev), torch.from_numpy(el2.view(np.int32)).to(dev))
    ix2.build(d2, torch.from_numpy(c2["perm"].view(np.int32)).to(dev))
    q2 = (torch.from_numpy(c2["q"][0].view(np.int64)).to(dev), torch.from_numpy(c2["q"][1].view(np.int32)).to(dev))
    ix2.tune(q2, 100)
    ix2.set_query_mode(F.QUERY_GRAPH)
    # embedding index (streamed build)
    ix4 = F.Index("cosine", c4["R"], c4["B"], c4["L"], c4["K"], capacity=c4["N"], params=c4["params"],
                  dim=c4["d"], W=c4["W"],
                  precision=PRECISIONS[args.precision])
    hasher = None
    if PRECISIONS[args.precision] in (F.PREC_BF16, F.PREC_FP8):
        hasher = F.Index("cosine", c4["R"], c4["B"], c4["L"], c4["K"], capacity=1, params=c4["params"],
                         dim=c4["d"], W=c4["W"], precision=F.PREC_BF16X2)
    t0 = time.perf_counter()
    build_streamed(F, ix4, c4, dev, torch.from_numpy(c4["perm"].view(np.int32)).to(dev), hasher)
    torch.cuda.synchronize()
    build4_s = time.perf_counter() - t0
    q4 = F.generate_embeddings(c4["seed"], c4["d"], c4["n_centers"], c4["sigma"], 0, c4["nq"], queries=True,
                               q_sigma=c4["qsigma"], n_points=c4["N"])
    # plain form (hash kernel, then count/decode/top-k), device buffers, k = 100
    plain = {}
    rng_k = np.random.default_rng([c2["seed"], 56])
    for name, ix, q, nq in (("C2", ix2, q2, c2["nq"]), ("C4", ix4, q4, c4["nq"])):
        ix.set_query_mode(F.QUERY_PLAIN)
        # the same k mix as the served traffic, per query
        kk = torch.from_numpy(rng_k.choice([1, 10, 100], size=nq).astype(np.int32)).to(dev)
        ix.query(q, 100, k=kk)
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ix.query(q, 100, k=kk)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ids_p, sc_p = ix.query(q, 100)        # full width, for the prefix checks below
        torch.cuda.synchronize()
        plain[name] = {"qps": nq / (statistics.median(ts) / 1e3), "ms_per_batch": statistics.median(ts),
                       "ids": ids_p.cpu().numpy().view(np.uint32), "scores": sc_p.cpu().numpy().view(np.uint16)}
        ix.set_query_mode(F.QUERY_FUSED)
    # recall of each index (the plain form's full-width results; served results equal them)
    ex2 = exact_similarity_topk(c2)
    rec2 = recall_scores(c2, plain["C2"]["ids"][gt_sample(c2)], *ex2)
    c4["d_q"] = q4
    ex4 = exact_similarity_topk(c4)
    rec4 = recall_scores(c4, plain["C4"]["ids"][gt_sample(c4)], *ex4)
    plain_mix = 2.0 / (1.0 / plain["C2"]["qps"] + 1.0 / plain["C4"]["qps"])    # 50/50 mix
    # the plain batched FP32 path the config names: FP32 hashing of the
    # embedding queries (an index of the same projections, used only to hash),
    # then the same count / decode / top-k kernel from the buckets
    h32 = F.Index("cosine", c4["R"], c4["B"], c4["L"], c4["K"], capacity=1, params=c4["params"], dim=c4["d"],
                  W=c4["W"], precision=F.PREC_FP32)
    fq4, _, _, keep4 = h32._points(q4)
    qb4 = torch.empty((c4["nq"], c4["L"]), dtype=torch.int32, device=dev)
    kk4 = torch.from_numpy(np.random.default_rng([c2["seed"], 57]).choice([1, 10, 100], size=c4["nq"])
                           .astype(np.int32)).to(dev)
    o4 = torch.empty((c4["nq"], 100), dtype=torch.int32, device=dev)
    s4 = torch.empty((c4["nq"], 100), dtype=torch.int16, device=dev)

    def plain32():
        F._check(h32.lib.flinng_hash(h32.h, C.byref(fq4), c4["nq"], qb4.data_ptr(), None, None, 1))
        F._check(ix4.lib.flinng_query_buckets(ix4.h, qb4.data_ptr(), c4["nq"], kk4.data_ptr(), 100,
                                              o4.data_ptr(), s4.data_ptr(), 1))
    plain32()
    ts = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plain32()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    plain32_c4 = c4["nq"] / (statistics.median(ts) / 1e3)
    plain32_mix = 2.0 / (1.0 / plain["C2"]["qps"] + 1.0 / plain32_c4)
    h32.close()
    srv = F.Server(hbm_budget=ix2.device_bytes + ix4.device_bytes + (4 << 30), n_slots=8, max_batch=args.max_batch,
                   k_max=100, max_batch_elems=1 << 21)
    id2 = srv.add_index(ix2)
    id4 = srv.add_index(ix4)
    staging5 = srv.staging
    h_q4 = q4.cpu().pin_memory().numpy()
    sources = [sets_source(F, id2, c2["q"], 0.5, keep), dense_source(F, id4, h_q4, 0.5, keep)]
    rng = np.random.default_rng([c2["seed"], 55])
    # the insert payloads live in page-locked host memory, as a serving
    # client's buffers would (the library copies them by DMA)
    poff = torch.from_numpy(pool["off"].view(np.int64)).pin_memory().numpy().view(np.uint64)
    pel = torch.from_numpy(pool["elems"].view(np.int32)).pin_memory().numpy().view(np.uint32)
    keep += [poff, pel]
    used = 0
    runs = {}
    clocks = ClockSampler(0)
    time.sleep(0.3)
    t_load = time.time()
    launches = 0
    for f in (0.25, 0.5, 0.9, 2.0):
        rate = f * plain_mix
        T = min(1.0, 1.5e6 / rate)
        n_ins = int(round(np.exp(rng.uniform(np.log(1e3), np.log(1e5)))))
        n_ins = min(n_ins, len(poff) - 1)
        lo = used % (len(poff) - 1 - n_ins + 1)
        off = torch.from_numpy((poff[lo:lo + n_ins + 1] - poff[lo]).astype(np.int64)).pin_memory().numpy() \
            .view(np.uint64)
        el = pel[poff[lo]:poff[lo + n_ins]]                  # a contiguous slice of the pinned pool
        fp = F.flinng_points()
        fp.off, fp.elems = off.ctypes.data, el.ctypes.data
        perm = WL.group_permutations(c2["seed"], c2["R"], n_ins, batch=100 + int(f * 100))
        keep += [off, el, fp, perm]
        used += n_ins
        req = make_trace(F, rng, rate, T, sources, [(T / 2, id2, fp, n_ins, perm)])
        l0 = F.kernel_launches()
        ids_s, sc_s, res = srv.replay(req)
        launches = int(F.kernel_launches() - l0)
        st = dict(trace_stats(req, res, F), offered_qps=rate, duration_s=T, gpu_launches=launches)
        # embedding queries (no inserts into that index): served == plain prefix of length k
        m4 = np.nonzero((req["kind"] == F.REQ_QUERY) & (req["index"] == id4))[0][:2000]
        j4 = ((req["data"][m4] - sources[1]["base"]) // np.uint64(c4["d"] * 4)).astype(np.int64)
        same = all(np.array_equal(ids_s[r][:req["k"][r]], plain["C4"]["ids"][j][:req["k"][r]])
                   for r, j in zip(m4, j4))
        st["embedding_results_equal_plain"] = bool(same)
        # genomic queries that ran before this run's insert (index version 0 of
        # the first run; later runs' indices hold earlier inserts): == plain prefix
        if f == 0.25:
            m2 = np.nonzero((req["kind"] == F.REQ_QUERY) & (req["index"] == id2) & (res["version"] == 0))[0]
            m2 = m2[np.random.default_rng(9).choice(len(m2), min(200, len(m2)), replace=False)] if len(m2) else m2
            j2 = np.searchsorted(sources[0]["off"], (req["data"][m2] - sources[0]["base"]) // np.uint64(4))
            same2 = all(np.array_equal(ids_s[r][:req["k"][r]], plain["C2"]["ids"][j][:req["k"][r]]) and
                        np.array_equal(sc_s[r][:req["k"][r]], plain["C2"]["scores"][j][:req["k"][r]])
                        for r, j in zip(m2, j2))
            st["genomic_results_equal_plain"] = {"checked": int(len(m2)), "equal": bool(same2)}
        runs[f"{f}x_plain"] = st
    t_end = time.time()
    clk = clocks.stop(t_load, t_end)
    srv.close()
    peak = runs["2.0x_plain"]["achieved_qps"]
    h2d_per_q = 0.5 * float(np.mean(np.diff(c2["q"][0]))) * 4 + 0.5 * c4["d"] * 4
    line = {
        "metric": METRIC, "value": peak, "unit": UNIT, "n_gpus": 1, "steps": len(runs),
        "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "mixed: u32 (MinHash index) + f32 (SRP index)",
        "data": "synthetic (seeded; stands in for the paper's datasets)",
        "config": {"workload": "C5: serving, indices C2 (100,000 genomic reads, MinHash, at its recall-target "
                               f"parameters R{c2['R']} B{c2['B']} L{c2['L']} K{c2['K']} W{c2['W']}) and C4 "
                               "(10,000,000 x 4096 embeddings, SRP, R3 B20000 L64 K16) resident together; "
                               "Poisson arrivals, 50/50 mix, k uniform in {1,10,100}; one insert batch of "
                               "1k-100k reads per run into the genomic index",
                   "form": f"serving: continuous batching, 8 streams, batches <= {args.max_batch}, host buffers in "
                           "and out",
                   "rates": "0.25x, 0.5x, 0.9x and 2.0x (overload) of the plain form's mixed throughput",
                   "hbm_budget_bytes": int(ix2.device_bytes + ix4.device_bytes + (4 << 30)),
                   "srp_precision": PREC_NAMES[PRECISIONS[args.precision]]},
        "plain_form": {"mixed_qps": plain_mix, "C2_qps": plain["C2"]["qps"], "C4_qps": plain["C4"]["qps"],
                       "C4_precision": PREC_NAMES[PRECISIONS[args.precision]],
                       "note": "hash kernel then count/decode/top-k kernel, whole query batch of each index "
                               "resident in HBM, per-query k uniform in {1,10,100} as served"},
        "plain_fp32_form": {"mixed_qps": plain32_mix, "C2_qps": plain["C2"]["qps"], "C4_qps": plain32_c4,
                            "note": "the plain batched FP32 path: FP32 SRP hashing of the embedding queries, "
                                    "then the same count/decode/top-k kernel (MinHash has no FP32 step)"},
        "serving": runs,
        "serving_vs_plain": peak / plain_mix,
        "serving_vs_plain_fp32": peak / plain32_mix,
        "recall": {"C2": rec2, "C4": rec4,
                   "note": "recall@10 of each index on its own queries (C4: 1,000 sampled); the embedding "
                           "index stays far below 0.9 at its configured parameters (no grid point of its "
                           "sweep reaches it)"},
        "staging": staging5,
        "latency_ms": {f"p{p}_at_{f}x": runs[f"{f}x_plain"][f"p{p}_ms"] for f in (0.25, 0.5, 0.9) for p in (50, 99)},
        "e2e": {"value": peak, "unit": UNIT, "h2d_bytes_per_step": int(h2d_per_q),
                "d2h_bytes_per_step": 500, "note": "serving is host-to-host: per query bytes"},
        "gpu_launches": launches,
        "build": {"C4_streamed_build_s": build4_s},
        "clocks": clk,
    }
    return line


def run_reference(args, c: dict, config: dict | None = None) -> dict:
    """The CPU oracle as the reference arm: each step is a bounded sample of
    the query batch on one core. ``config``: the line's config object (the
    headline's, so that both arms name the same workload)."""
    o = oracle_index(c)
    per_step = max(1, min(c["nq"], 200))
    for it in range(args.warmup):
        o.query(query_slice(c, 0, per_step), c["k"])
    t = []
    for it in range(args.steps):
        lo = (it * per_step) % c["nq"]
        hi = min(c["nq"], lo + per_step)
        t0 = time.perf_counter()
        o.query(query_slice(c, lo, hi), c["k"])
        t.append((time.perf_counter() - t0, hi - lo))
    el = sum(a for a, _ in t)
    n = sum(b for _, b in t)
    value = n / el
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32" if c["metric"] != "cosine" else "f64",
        "data": "synthetic (seeded; stands in for the paper's datasets)",
        "config": config or {"workload": f"{args.workload}: {c['desc']}", "global_batch": c["nq"], "k": c["k"]},
        "form": "the oracle (plain C, one core): Alg. 3 query by query",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} queries per step, single thread, index built "
                                   "beforehand (not timed)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="C2", choices=sorted(WORKLOADS) + ["C5"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-form traces")
    ap.add_argument("--no-recall", action="store_true", help="skip the exact ground truth (profiling runs)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the recall sweep over (R, B, L, K)")
    ap.add_argument("--n-points", type=int, default=0,
                    help="streamed embedding workload only: index this many points instead of the config's "
                         "(small profiling cases; the line says so)")
    ap.add_argument("--max-batch", type=int, default=1024,
                    help="largest batch the serving runtime forms (C5 and the serving runs of other workloads)")
    ap.add_argument("--configured", action="store_true",
                    help="time the fused form at the parameters the workload's config names instead of the "
                         "serving form at the recall-target parameters (the default where those are known)")
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS),
                    help="SRP projection arithmetic for cosine workloads (signs are exact either way)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    headline = args.workload in TARGETS and not args.configured
    if args.impl == "reference":
        if rank != 0:
            return
        c = make_workload(args.workload)
        if headline:
            ct = target_workload(c, args.workload)
            print(json.dumps(run_reference(args, ct, headline_config(args.workload, ct, world))), flush=True)
        else:
            print(json.dumps(run_reference(args, c)), flush=True)
        return
    if args.workload == "C5":
        if rank == 0:
            print(json.dumps(run_serving(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    c = make_workload(args.workload)
    if args.n_points:
        if not c.get("embed"):
            raise SystemExit("--n-points applies to the streamed embedding workload (C4) only")
        c["N"] = args.n_points
        c["perm"] = WL.group_permutations(c["seed"], c["R"], c["N"])
        c["desc"] = c["desc"].replace("N=10000000", f"N={args.n_points} (reduced with --n-points)")
    line = run_headline(args, c, rank, world) if headline else run_ours(args, c, rank, world)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
