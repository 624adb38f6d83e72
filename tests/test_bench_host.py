"""Host-side pieces of bench.py, on the CPU: recall scoring, serving traces
and their statistics, the clock record's throttle check, and the traffic
record's source-hash guard (no GPU)."""
import os
import sys
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2106_11565_gb300 import flinng as F  # noqa: E402


def test_recall_scores_by_hand():
    # exact top-10 of one query: ids 0..9 with similarities 1.0 .. 0.55, then
    # id 10 ties the 10th (0.55) and id 11 is below it
    ex_ids = np.array([list(range(12))])
    ex_sims = np.array([[1.0 - 0.05 * i for i in range(10)] + [0.55, 0.5]])
    none = 0xFFFFFFFF
    # returned: 9 of the top 10, the tie (a hit), then a miss and padding
    got = np.array([[0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 11, none]], np.uint64)
    r = bench.recall_scores({}, got, ex_ids, ex_sims)
    assert r["recall_at_10"] == pytest.approx(1.0)
    assert r["recall_1_at_k"] == 1.0
    got = np.array([[11, 1, 2, 3, none, none, none, none, none, none, none, none]], np.uint64)
    r = bench.recall_scores({}, got, ex_ids, ex_sims)
    assert r["recall_at_10"] == pytest.approx(0.3) and r["recall_1_at_k"] == 0.0


def test_make_trace_and_stats():
    rng = np.random.default_rng(7)
    qoff = np.array([0, 3, 3, 10, 12], np.uint64)       # 4 query sets, one empty
    src = {"id": 2, "kind": "sets", "share": 1.0, "nq": 4, "sizes": np.diff(qoff), "off": qoff[:-1],
           "base": np.uint64(1 << 20)}
    dsrc = {"id": 5, "kind": "dense", "share": 3.0, "nq": 6, "dim": 8, "base": np.uint64(1 << 30)}
    req = bench.make_trace(F, rng, rate=20000.0, T=0.5, sources=[src, dsrc])
    n = len(req)
    assert abs(n - 10000) < 5 * np.sqrt(10000)                  # Poisson(rate * T)
    assert np.all(np.diff(req["arrival_s"]) >= 0) and req["arrival_s"].max() <= 0.5
    assert set(np.unique(req["k"]).tolist()) <= {1, 10, 100}
    s = req["index"] == 2
    d = req["index"] == 5
    assert s.sum() + d.sum() == n and abs(d.mean() - 0.75) < 0.02
    # every set request points at one of the 4 sets, with its own size
    pos = (req["data"][s] - (1 << 20)) // 4
    sets = set(zip(qoff[:-1].tolist(), np.diff(qoff).tolist()))
    assert set(zip(pos.tolist(), req["n"][s].tolist())) <= sets
    # every dense request points at a row start
    rows = (req["data"][d] - (1 << 30)) / 32
    assert np.all(rows == np.floor(rows)) and rows.max() < 6
    # statistics of a fake replay: each query done 1 ms after it arrived
    res = np.zeros(n, F.RES_DTYPE)
    res["t_done"] = req["arrival_s"] + 1e-3
    res["batch"] = np.arange(n) // 7
    st = bench.trace_stats(req, res, F)
    assert st["queries"] == n and st["p50_ms"] == pytest.approx(1.0) and st["p99_ms"] == pytest.approx(1.0)
    assert st["batches"] == len(np.unique(res["batch"]))
    assert st["index2"]["queries"] == int(s.sum())


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler_with(rows):
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    cs.f.write("\n".join(rows) + "\n")
    cs.f.flush()
    cs.p = _Done()
    return cs


def test_clock_record_reasons_and_window():
    def row(t, sm, reasons=("Not Active",) * 4):
        return f"2026/12/03 10:00:{t:06.3f}, {sm}, 2070, 900.0, 0x0, " + ", ".join(reasons)
    import datetime
    t0 = datetime.datetime.strptime("2026/12/03 10:00:00.000", "%Y/%m/%d %H:%M:%S.%f").timestamp()
    ok = [row(1.0 + 0.05 * i, 2070 if i % 5 else 2055) for i in range(20)]
    cap = [row(1.5, 1900, ("Not Active", "Not Active", "Not Active", "Active"))]
    hot = [row(9.0, 1500, ("Active", "Not Active", "Not Active", "Not Active"))]   # outside the window
    r = _sampler_with(ok + cap + hot).stop(t0 + 1.0, t0 + 2.0)
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 21
    r = _sampler_with(ok + hot).stop(t0 + 8.95, t0 + 9.1)
    assert r["reasons"] == ["hw_slowdown"]
    r = _sampler_with(ok).stop(t0 + 50.0, t0 + 51.0)
    assert r["sm_mhz"] is None and r["samples"] == 0


def test_recorded_traffic_needs_the_same_kernel_source(monkeypatch):
    path = os.path.join(ROOT, "profiles", "k_query_fused_C2_R3B4096L512K1_traffic.txt")
    rec = dict(line.split(":", 1) for line in open(path) if ":" in line and not line.startswith("#"))
    h = rec["source_sha256_16"].strip()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.recorded_traffic("C2_R3B4096L512K1") == float(rec["dram_bytes_per_launch"])
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic("C2_R3B4096L512K1") is None
    assert bench.recorded_traffic("C9") is None


def test_fixed_size_trace_and_k_choice():
    rng = np.random.default_rng(3)
    qoff = np.array([0, 3, 3, 10, 12], np.uint64)
    src = {"id": 0, "kind": "sets", "share": 1.0, "nq": 4, "sizes": np.diff(qoff), "off": qoff[:-1],
           "base": np.uint64(1 << 20)}
    req = bench.make_trace(F, rng, rate=1e6, T=0.0, sources=[src], k_choices=(100,), n=5000)
    assert len(req) == 5000 and np.all(req["k"] == 100)
    assert req["arrival_s"].max() <= 5000 / 1e6 and np.all(np.diff(req["arrival_s"]) >= 0)


def test_serving_step_and_latency_breakdown():
    n = 400
    req = np.zeros(n, F.REQ_DTYPE)
    req["arrival_s"] = np.linspace(0.0, 0.01, n)
    res = np.zeros(n, F.RES_DTYPE)
    res["t_start"] = req["arrival_s"] + 1e-4         # 0.1 ms waiting for a slot
    res["d_start"] = res["t_start"] + 2e-5           # 0.02 ms to the first device event
    res["d_done"] = res["d_start"] + 3e-4            # 0.3 ms on the device
    res["t_done"] = res["d_done"] + 5e-5             # 0.05 ms to the caller's buffer
    res["batch"] = np.arange(n) // 50
    st = bench.serving_step_stats(req, res, F)
    assert st["queries"] == n and st["batches"] == 8
    assert st["device_s"] == pytest.approx(res["d_done"].max() - res["d_start"].min())
    assert st["host_s"] == pytest.approx(0.01 + 1e-4 + 2e-5 + 3e-4 + 5e-5)
    b = bench.latency_breakdown(req, res, F)
    for part, ms in (("wait", 0.1), ("launch", 0.02), ("device", 0.3), ("harvest", 0.05)):
        assert b[part]["p50"] == pytest.approx(ms, rel=1e-6) and b[part]["p99"] == pytest.approx(ms, rel=1e-6)


def test_recall_target_workload_and_shared_config():
    c = {"metric": "jaccard", "seed": 11, "N": 50, "nq": 3, "k": 100, "R": 2, "B": 10, "L": 32, "K": 2, "W": 17,
         "desc": "sets N=50 R2 B10 L32 K2 W17 nq=3 k=100"}
    bench.TARGETS["T9"] = dict(R=3, B=16, L=64, K=1, W=17)
    try:
        ct = bench.target_workload(c, "T9")
        assert (ct["R"], ct["B"], ct["L"], ct["K"], ct["W"]) == (3, 16, 64, 1, 17)
        assert ct["perm"].shape == (3, 50) and all(sorted(r) == list(range(50)) for r in ct["perm"])
        assert len(ct["params"]["bucket_a"]) == 64 * 1
        assert "R3 B16 L64 K1 W17" in ct["desc"] and ct["configured"]["L"] == 32
        # both arms print the same config object
        assert bench.headline_config("T9", ct, 1) == bench.headline_config("T9", dict(ct), 1)
        assert bench.headline_config("T9", ct, 2)["global_batch"] == 2 * bench.SERVE_QUERIES
    finally:
        del bench.TARGETS["T9"]
