#!/usr/bin/env python
"""Benchmark of the plain database search (one query against the whole
database, Sec. III.B.3 / Sec. IV of the paper) on the GPU.

A step is one complete search with the database resident in HBM: query
profile, the scan of every pair, top-k ranking and alignment replay of the
hits.  Default workload: a 256-residue query against a synthetic
SwissProt-like database (~570k sequences, ~205M residues, lognormal lengths
with median 300 and a tail to 35,000), top-100, the paper's parameters.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  `value` is database residues/s with the
query already on the device; `e2e` is the same metric through the
host-buffer C-ABI call (query copied in, hits and alignments copied out,
every step).  `--impl reference` times the CPU oracle (the plain C
implementation of the paper's algorithm) on the host cores instead.
Multi-GPU (torchrun): every rank searches its own database shard of the
same size (weak scaling); ranks exchange only the step time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DB residues/s per query (plain vs batched); p50/p99 query latency in serving mode"
UNIT = "residues/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain-large", choices=["plain-large", "plain-small"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-budget-s", type=float, default=12.0,
                    help="wall-time budget of the oracle CPU baseline sample")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain comparison")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-seconds", type=float, default=20.0,
                    help="offered seconds of traffic per serving rate (requests = rate x this, at most 10,000)")
    ap.add_argument("--no-bimodal", action="store_true",
                    help="skip the load-balance workload (both schedules)")
    ap.add_argument("--no-small", action="store_true", help="skip the plain-small workload section")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the integer issue-rate measurement (the roofline then uses the derived peak)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(name, rank):
    from paper_1508_06561_gb300 import synth
    if name == "plain-small":
        db, q, k = synth.plain_small(0)
        wl = "plain-q64-2k"
    else:
        db, q, k = synth.plain_large(seed_db=2 + rank)
        wl = "plain-q256-swissprot-like-570k"
    cfg = {"workload": wl, "n_seqs": int(db.n), "residues": int(db.residues), "qlen": int(len(q)), "k": int(k),
           "params": "PGP=0 GOP=10 GEP=5 LFactor=0.5 SFactor=1 MinFactor=0.5 Rounds=1 BLOSUM62",
           "queries_per_step": 1,
           "l2": ("no flush: the %.0f MB residue stream exceeds the 129 MB L2" % (db.residues / 1e6)
                  if db.residues > 129e6 else "database fits in L2; steps run warm")}
    return db, q, k, cfg


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = (uuid or "").lower().replace("gpu-", "")
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "hs_bench_clocks_%d.csv" % os.getpid())

    def start(self):
        self.f = open(self.path, "w")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:                     # no nvidia-smi: the line says "unsampled"
            self.proc = None
            self.f.close()
            os.remove(self.path)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons, n = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            lines = f.readlines()
        os.remove(self.path)
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0].lower():
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            n += 1
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": n}


# --------------------------------------------------------------------------
# ncu traffic recorded in profiles/ (valid only for the same kernel source)
# --------------------------------------------------------------------------
def kernel_source_hash():
    h = hashlib.sha256()
    for f in ["hs_device.cuh", "hs_scan.cu", "hs_internal.h"]:
        with open(os.path.join(ROOT, "paper_1508_06561_gb300", "csrc", f), "rb") as src:
            h.update(src.read())
    return h.hexdigest()[:16]


def measured_hbm_gbs():
    """The measured copy bandwidth (MEASURED_PEAKS.json), else the documented fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def recorded_traffic(workload_name):
    path = os.path.join(ROOT, "profiles", "scan_kernel_%s.md" % workload_name)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        text = f.read()
    m = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


# --------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline field)
# --------------------------------------------------------------------------
def oracle_rate(db, q, seed, budget_s, rng_seed=0, first=2000):
    """Oracle residues/s on a growing random sample of the database, stopping
    once `budget_s` of wall time is spent (or the database is exhausted)."""
    import oracle as O
    O.build()
    M, p = O.blosum62(), O.paper_params()
    order = np.random.default_rng(rng_seed).permutation(db.n)
    lens = db.lengths()
    done, res, t_used, chunk = 0, 0, 0.0, first
    threads = os.cpu_count() or 1
    while done < db.n and t_used < budget_s:
        idx = np.sort(order[done:done + chunk])
        t0 = time.perf_counter()
        _, _, used = O.search_scores(db.codes, db.offsets, q, M, p, seed, idx=idx, nthreads=threads, want_cells=False)
        dt = time.perf_counter() - t0
        t_used += dt
        res += int(lens[idx].sum())
        done += len(idx)
        rate = res / max(t_used, 1e-9)
        chunk = int(min(max(chunk, rate * min(2.0, budget_s - t_used) / max(lens.mean(), 1)), db.n - done)) or 1
        threads = used
    return res / t_used, threads, done, res, t_used


def run_reference(args, world, rank):
    if rank != 0:
        return
    db, q, k, cfg = workload(args.workload, 0)
    import oracle as O
    O.build()
    M, p = O.blosum62(), O.paper_params()
    lens = db.lengths()
    threads = os.cpu_count() or 1
    # per-step sample sized so the whole run takes about two minutes
    rate, threads, _, _, _ = oracle_rate(db, q, args.seed, 1.0, rng_seed=99, first=2000)
    per_step_s = max(0.02, 120.0 / max(1, args.steps + args.warmup))
    n_per_step = int(max(50, min(db.n, per_step_s * rate / max(lens.mean(), 1))))
    rng = np.random.default_rng(12345)
    total_res, total_t = 0, 0.0
    for step in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(db.n, n_per_step, replace=False))
        t0 = time.perf_counter()
        _, _, used = O.search_scores(db.codes, db.offsets, q, M, p, args.seed, idx=idx, nthreads=threads,
                                     want_cells=False)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            total_t += dt
            total_res += int(lens[idx].sum())
    value = total_res / total_t
    sample = ("each step: %d random sequences (%.1f%% of the %d-sequence database), scores only, "
              "%d host threads" % (n_per_step, 100.0 * n_per_step / db.n, db.n, used))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# batched vs plain on the same queries (64 queries, lengths uniform in
# [30, 1000], top-100: the shape of the batched workload)
# --------------------------------------------------------------------------
def batched_section(P, D, db, params, seed, reps=3):
    import torch

    from paper_1508_06561_gb300 import autotune, synth
    rng = np.random.default_rng(3)
    qs = [synth.residues(rng, int(L)) for L in rng.integers(30, 1001, 64)]
    k = 100
    best, tune_s = autotune.tune(D, qs, k, params)
    cat = torch.from_numpy(np.concatenate(qs)).cuda()
    off = np.zeros(len(qs) + 1, np.int64)
    np.cumsum([len(q) for q in qs], out=off[1:])
    offd = torch.from_numpy(off).cuda()
    seeds = torch.full((len(qs),), seed, dtype=torch.int64, device="cuda")
    mq = int(max(len(q) for q in qs))
    st = torch.cuda.Stream()

    def timed_batch(tuning):
        with torch.cuda.stream(st):
            out = P.search_batch_device(D, cat, offd, seeds, mq, k, params, tuning, st)     # warm-up
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(reps):
                P.search_batch_device(D, cat, offd, seeds, mq, k, params, tuning, st, out["workspace"], out)
            b.record(st)
        st.synchronize()
        assert int(out["status"].item()) == 0
        used = int(out["ops_used"].item())
        return a.elapsed_time(b) / 1000.0 / reps, out["hits"].cpu().numpy().copy(), out["ops"][:used].cpu().numpy().copy()

    t_default, h_def, o_def = timed_batch(autotune.DEFAULT)
    t_batch, h_tuned, o_tuned = timed_batch(best)
    same = bool(np.array_equal(h_def, h_tuned) and np.array_equal(o_def, o_tuned))
    # the same queries, one plain device search each
    qd = [torch.from_numpy(q).cuda() for q in qs]
    longest = int(np.argmax([len(q) for q in qs]))
    with torch.cuda.stream(st):
        o1 = P.search_device(D, qd[longest], k, params, seed=seed, stream=st)
        ws = o1["workspace"]
        for q in qd:
            P.search_device(D, q, k, params, seed=seed, stream=st, workspace=ws, out=o1)
        a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a2.record(st)
        for _ in range(reps):
            for q in qd:
                P.search_device(D, q, k, params, seed=seed, stream=st, workspace=ws, out=o1)
        b2.record(st)
    st.synchronize()
    t_plain = a2.elapsed_time(b2) / 1000.0 / reps
    res = db.residues * len(qs)
    small = batched_small_db(P, qs, params, seed)
    return {"workload": "batched-64q-u30-1000-swissprot-like-570k", "queries": len(qs), "k": k,
            "value": res / t_batch, "unit": UNIT, "ms_per_batch": t_batch * 1000.0,
            "plain_same_queries": res / t_plain, "plain_ms": t_plain * 1000.0,
            "speedup_vs_plain": t_plain / t_batch, "tuning": best,
            "default_tuning": autotune.DEFAULT, "default_ms_per_batch": t_default * 1000.0,
            "tuned_speedup_vs_default": t_default / t_batch, "tuned_output_identical": same,
            "tuning_evaluated": len(tune_s),
            "tuning_candidates_ms": {kk: v * 1000.0 for kk, v in tune_s.items()},
            "small_db": small}


def batched_small_db(P, qs, params, seed, k=10, reps=20):
    """The same 64 queries against the 2,000-target database, where one
    query cannot fill the GPU: one batched call vs one plain search each."""
    import torch

    from paper_1508_06561_gb300 import synth
    db, _, _ = synth.plain_small(0)
    D = P.Database(db.codes, db.offsets)
    cat = torch.from_numpy(np.concatenate(qs)).cuda()
    off = np.zeros(len(qs) + 1, np.int64)
    np.cumsum([len(q) for q in qs], out=off[1:])
    offd = torch.from_numpy(off).cuda()
    seeds = torch.full((len(qs),), seed, dtype=torch.int64, device="cuda")
    mq = int(max(len(q) for q in qs))
    qd = [torch.from_numpy(q).cuda() for q in qs]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        out = P.search_batch_device(D, cat, offd, seeds, mq, k, params, None, st)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            P.search_batch_device(D, cat, offd, seeds, mq, k, params, None, st, out["workspace"], out)
        b.record(st)
        o1 = P.search_device(D, qd[int(np.argmax([len(q) for q in qs]))], k, params, seed=seed, stream=st)
        for q in qd:
            P.search_device(D, q, k, params, seed=seed, stream=st, workspace=o1["workspace"], out=o1)
        a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a2.record(st)
        for _ in range(reps):
            for q in qd:
                P.search_device(D, q, k, params, seed=seed, stream=st, workspace=o1["workspace"], out=o1)
        b2.record(st)
    st.synchronize()
    assert int(out["status"].item()) == 0 and int(o1["status"].item()) == 0
    t_batch = a.elapsed_time(b) / 1000.0 / reps
    t_plain = a2.elapsed_time(b2) / 1000.0 / reps
    D.close()
    res = db.residues * len(qs)
    return {"workload": "batched-64q-u30-1000-plain-small-2k", "k": k, "value": res / t_batch, "unit": UNIT,
            "ms_per_batch": t_batch * 1000.0, "plain_ms": t_plain * 1000.0, "speedup_vs_plain": t_plain / t_batch}


# --------------------------------------------------------------------------
# serving: Poisson arrivals of single-query requests (lengths lognormal,
# median 250, clamped to [20, 2000], one seed each) against the resident
# database, continuous batching; p50/p99 latency beside throughput
# --------------------------------------------------------------------------
def serving_section(P, D, db, params, seconds, rates=(50.0, 200.0, 1000.0)):
    from paper_1508_06561_gb300 import serve, synth
    out = {"workload": "serving-swissprot-like-570k", "k": 100, "rates": [],
           "requests_note": "rate x %.0f s of offered traffic per rate, at most the stream's 10,000" % seconds}
    for rate in rates:
        n = int(min(10_000, max(50, rate * seconds)))
        t_arr, qs, seeds = synth.serving_stream(5, n, rate)
        srv = serve.Server(D, k=100, params=params, max_batch=64, slots=3, max_total_qlen=65536)
        futs = []
        t0 = time.perf_counter()
        for ta, q, sd in zip(t_arr, qs, seeds):
            delay = t0 + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            futs.append(srv.submit(q, int(sd)))
        res = [f.result(timeout=600) for f in futs]
        t_end = time.perf_counter()
        srv.close()
        # the same request alone must give the same answer as in the mix
        same = True
        for i in np.linspace(0, n - 1, 5).astype(int):
            h0, o0 = P.search(D, qs[i], 100, params, int(seeds[i]))
            same &= bool(np.array_equal(res[i][0], h0) and np.array_equal(res[i][1], o0))
        lat = serve.latency_stats(srv.latencies)
        ov = serve.overlap_stats(srv.intervals)
        nb = [b for b, _ in srv.batches]
        out["rates"].append({"offered_req_s": rate, "requests": n, "p50_ms": lat["p50_ms"], "p99_ms": lat["p99_ms"],
                             "mean_ms": lat["mean_ms"], "served_req_s": n / (t_end - t0),
                             "residues_per_s": n * db.residues / (t_end - t0), "batches": len(nb),
                             "mean_batch": float(np.mean(nb)), "max_batch": int(np.max(nb)),
                             "device_busy_frac": ov["device_busy_ms"] / 1000.0 / (t_end - t0),
                             "batches_overlapping_frac": ov["overlap_frac"], "max_batches_in_flight": ov["max_in_flight"],
                             "alone_equals_mix": same})
    return out


# --------------------------------------------------------------------------
# load balance: 16 queries (6x50, 5x500, 5x2000) against 100k targets, 90%
# of 50-150 letters and 10% of 5,000-35,000, top-50, under the length-binned
# schedule and in database order (same results, different balance)
# --------------------------------------------------------------------------
def bimodal_section(P):
    import torch

    from paper_1508_06561_gb300 import synth
    db, queries, k = synth.bimodal(4)
    D = P.Database(db.codes, db.offsets)
    out = {"workload": "bimodal-100k-16q", "residues": int(db.residues), "n_seqs": int(db.n), "k": k}
    st = torch.cuda.Stream()
    qd = [torch.from_numpy(q).cuda() for q in queries]
    longest = int(np.argmax([len(q) for q in queries]))
    for name, sched in (("length_binned", P.Database.SCHEDULE_LENGTH), ("input_order", P.Database.SCHEDULE_INPUT)):
        D.set_schedule(sched)
        with torch.cuda.stream(st):
            o1 = P.search_device(D, qd[longest], k, stream=st)
            ws = o1["workspace"]
            for q in qd:
                P.search_device(D, q, k, stream=st, workspace=ws, out=o1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            per = []
            for q in qd:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                P.search_device(D, q, k, stream=st, workspace=ws, out=o1)
                e1.record(st)
                per.append((len(q), e0, e1))
            b.record(st)
        st.synchronize()
        t = a.elapsed_time(b) / 1000.0
        by_len = {}
        for L, e0, e1 in per:
            by_len.setdefault(int(L), []).append(e0.elapsed_time(e1))
        out[name] = {"value": len(qd) * db.residues / t, "unit": UNIT, "ms_total": t * 1000.0,
                     "ms_per_query_by_qlen": {str(L): float(np.mean(v)) for L, v in sorted(by_len.items())}}
    out["binned_speedup"] = out["input_order"]["ms_total"] / out["length_binned"]["ms_total"]
    D.close()
    return out


# --------------------------------------------------------------------------
# integer issue rates (libhspeak.so): the denominators of the scan's roofline
# --------------------------------------------------------------------------
def int_peaks(dev, uuid):
    import ctypes as C

    from paper_1508_06561_gb300 import build
    L = C.CDLL(build.PEAK_LIB)
    L.hsp_measure.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double),
                              C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    out = {"how": "libhspeak.so: 8 interleaved dependency chains per thread, 1024-thread blocks on every SM, "
                  "best of 5 launches by CUDA events"}
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)
    for name, op, iters in (("iadd", 0, 20000), ("dpx_vimax3", 1, 8000), ("dpx_viaddmax", 2, 8000)):
        rate, ms, ops = C.c_double(), C.c_double(), C.c_int64()
        rc = L.hsp_measure(op, iters, 5, None, C.byref(rate), C.byref(ms), C.byref(ops))
        if rc != 0:
            raise RuntimeError("hsp_measure(%s) failed: %d" % (name, rc))
        out[name] = {"tops": rate.value / 1e12, "ms": ms.value, "ops_per_launch": int(ops.value)}
    out["clocks"] = clocks.stop()
    return out


# --------------------------------------------------------------------------
# plain single query on the small database (64-residue query, 2,000 targets,
# top-10): the whole database sits in L2, so steps run warm
# --------------------------------------------------------------------------
def small_section(P, params, seed, steps=2000):
    import torch

    from paper_1508_06561_gb300 import synth
    db, q, k = synth.plain_small(0)
    D = P.Database(db.codes, db.offsets)
    st = torch.cuda.Stream()
    qd = torch.from_numpy(q).cuda()
    # a search here takes tens of microseconds on the device, less than one
    # Python call: the device-side rate is timed by replaying a CUDA graph of
    # `per_graph` searches (hs_search_device allocates nothing and never
    # synchronises, so it can be captured)
    per_graph = 50
    with torch.cuda.stream(st):
        out = P.search_device(D, qd, k, params, seed=seed, stream=st)
        for _ in range(20):
            P.search_device(D, qd, k, params, seed=seed, stream=st, workspace=out["workspace"], out=out)
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        for _ in range(per_graph):
            P.search_device(D, qd, k, params, seed=seed, stream=st, workspace=out["workspace"], out=out)
    reps = max(1, steps // per_graph)
    with torch.cuda.stream(st):
        for _ in range(3):
            g.replay()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            g.replay()
        b.record(st)
    st.synchronize()
    assert int(out["status"].item()) == 0
    steps = reps * per_graph
    t = a.elapsed_time(b) / 1000.0
    n_e2e = 500
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        P.search(D, q, k, params, seed=seed, stream=st)
    te = time.perf_counter() - t0
    D.close()
    return {"workload": "plain-q64-2k", "n_seqs": int(db.n), "residues": int(db.residues), "qlen": int(len(q)),
            "k": int(k), "value": steps * db.residues / t, "unit": UNIT, "ms_per_search": t * 1000.0 / steps,
            "timing": "CUDA graph of %d searches replayed %d times, CUDA events" % (per_graph, reps),
            "e2e": {"value": n_e2e * db.residues / te, "unit": UNIT, "ms_per_search": te * 1000.0 / n_e2e},
            "l2": "database fits in L2; steps run warm"}


# --------------------------------------------------------------------------
# full-slide pair-wise mode (Fig. 1 as printed, Rounds = 20 as the paper
# runs it for alignment quality) on the small database: 64-residue query,
# 2,000 targets, top-10
# --------------------------------------------------------------------------
def full_section(P, seed, steps=20):
    import torch

    from paper_1508_06561_gb300 import synth
    db, q, k = synth.plain_small(0)
    D = P.Database(db.codes, db.offsets)
    params = P.Params(mode=1, rounds=20)
    st = torch.cuda.Stream()
    qd = torch.from_numpy(q).cuda()
    with torch.cuda.stream(st):
        cnt = P.search_device(D, qd, k, params, seed=seed, stream=st, want_cells=True)
    st.synchronize()
    cells = int(cnt["cells"][: D.n].sum().item())
    with torch.cuda.stream(st):
        out = P.search_device(D, qd, k, params, seed=seed, stream=st)
        for _ in range(3):
            P.search_device(D, qd, k, params, seed=seed, stream=st, workspace=out["workspace"], out=out)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(steps):
            P.search_device(D, qd, k, params, seed=seed, stream=st, workspace=out["workspace"], out=out)
        b.record(st)
    st.synchronize()
    assert int(out["status"].item()) == 0
    t = a.elapsed_time(b) / 1000.0 / steps
    D.close()
    return {"workload": "full-slide-rounds20-q64-2k", "mode": "full slide (Fig. 1), Rounds = 20", "n_seqs": int(db.n),
            "residues": int(db.residues), "qlen": int(len(q)), "k": int(k), "value": db.residues / t, "unit": UNIT,
            "ms_per_search": t * 1000.0, "pairs_per_s": db.n / t, "cells_per_search": cells,
            "cells_per_s": cells / t}


# --------------------------------------------------------------------------
# the GPU arm
# --------------------------------------------------------------------------
def run_ours(args, world, rank, local):
    import ctypes as C

    import torch

    import paper_1508_06561_gb300 as P
    from paper_1508_06561_gb300 import _lib

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        P.build.build()                     # no-op when the library is current
    if world > 1:
        torch.distributed.barrier()         # the other ranks load what rank 0 checked
    L = _lib.lib()

    db, q, k, cfg = workload(args.workload, rank)
    D = P.Database(db.codes, db.offsets)
    params = P.Params()
    stream = torch.cuda.Stream(dev)
    qd = torch.from_numpy(q).to(dev)

    # one untimed search counts the algorithmic work: per pair, the cells
    # (one add each) and the shifts (one compare each), packed by the trace hook
    tr = _lib.hs_trace()
    tr.pack_shifts = 1
    L.hs_db_set_trace(D.handle, C.byref(tr))
    with torch.cuda.stream(stream):
        out = P.search_device(D, qd, k, params, seed=args.seed, stream=stream, want_cells=True)
    stream.synchronize()
    packed = out["cells"][: D.n]
    cells_per_search = int((packed & ((1 << 40) - 1)).sum().item())
    shifts_per_search = int((packed >> 40).sum().item())
    assert int(out["status"].item()) == 0
    tr.pack_shifts = 0
    out = P.search_device(D, qd, k, params, seed=args.seed, stream=stream)   # buffers without counters
    ws = out["workspace"]

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    peaks = int_peaks(dev, uuid) if (rank == 0 and not args.no_peaks) else None

    # trace hook: events around the scan kernel of every timed step

    def step(ev_pair=None):
        if ev_pair is not None:
            tr.scan_start = ev_pair[0].cuda_event
            tr.scan_stop = ev_pair[1].cuda_event
        else:
            tr.scan_start = tr.scan_stop = None
        P.search_device(D, qd, k, params, seed=args.seed, stream=stream, workspace=ws, out=out)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
    stream.synchronize()
    launches_per_step = int(tr.launches)

    scan_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
    for a, b in scan_events:          # torch creates events on first record
        a.record(stream)
        b.record(stream)
    stream.synchronize()
    t_begin, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(uuid) if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.4)
    with torch.cuda.stream(stream):
        t_begin.record(stream)
        for i in range(args.steps):
            step(scan_events[i])
        t_end.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    if world > 1:
        torch.distributed.barrier()
    assert int(out["status"].item()) == 0
    ms_total = t_begin.elapsed_time(t_end)
    scan_ms = [a.elapsed_time(b) for a, b in scan_events]
    L.hs_db_set_trace(D.handle, None)

    t = torch.tensor([ms_total], device=dev, dtype=torch.float64)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * db.residues * args.steps / (ms_max / 1000.0)

    # end to end: the host-buffer call a user makes (query H2D, hits+ops D2H)
    h2d, d2h = C.c_int64(), C.c_int64()
    L.hs_search_transfer_bytes(len(q), k, C.byref(h2d), C.byref(d2h))
    n_e2e = max(3, min(args.steps, 500))
    for _ in range(3):
        P.search(D, q, k, params, seed=args.seed, stream=stream)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        hits, ops = P.search(D, q, k, params, seed=args.seed, stream=stream)
    e2e_s = time.perf_counter() - t0
    te = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
    if world > 1:
        torch.distributed.all_reduce(te, op=torch.distributed.ReduceOp.MAX)
    e2e_value = world * db.residues * n_e2e / float(te.item())

    if rank != 0:
        D.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # Roofline of the scan kernel, T_roof = max(B / HBM, Ops / P_int): Ops = one
    # integer add per cell plus one compare per shift (both counted by the
    # kernel); P_int = the measured 32-bit integer add rate of this GPU
    # (libhspeak.so, above), else SMs x 128 INT32 lanes x max SM clock; B =
    # the residues, and per pair its schedule entry (4 B) and two offsets
    # (16 B) read and its score (4 B) written.
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    scan_s = float(np.mean(scan_ms)) / 1000.0
    ops_per_search = cells_per_search + shifts_per_search
    achieved = ops_per_search / scan_s / 1e12
    derived = sms * 128 * 2070e6 / 1e12
    if peaks is not None:
        peak = peaks["iadd"]["tops"]
        basis = ("measured: 32-bit integer add issue rate %.2f T/s (libhspeak.so, SM clock %s MHz during it; "
                 "derived %d SMs x 128 lanes x 2070 MHz = %.2f T/s)" %
                 (peak, (peaks["clocks"] or {}).get("sm_mhz"), sms, derived))
    else:
        peak = derived
        basis = "%d SMs x 128 INT32 lanes x 2070 MHz (derived)" % sms
    alg_bytes = db.residues + 24 * db.n
    hbm_gbs = measured_hbm_gbs()
    t_alu_us = ops_per_search / (peak * 1e12) * 1e6
    t_hbm_us = alg_bytes / (hbm_gbs * 1e9) * 1e6
    traffic = recorded_traffic(cfg["workload"])

    batched = serving = None
    if world == 1 and not args.no_batched and args.workload == "plain-large":
        batched = batched_section(P, D, db, params, args.seed)
    if world == 1 and not args.no_serving and args.workload == "plain-large":
        serving = serving_section(P, D, db, params, args.serve_seconds)
    bimodal = bimodal_section(P) if (world == 1 and not args.no_bimodal and args.workload == "plain-large") else None
    small = small_section(P, params, args.seed) if (world == 1 and not args.no_small
                                                     and args.workload == "plain-large") else None
    full = full_section(P, args.seed) if (world == 1 and not args.no_small and args.workload == "plain-large") else None
    cpu_rate, cpu_threads, ns, nres, tcpu = oracle_rate(db, q, args.seed, args.cpu_budget_s) \
        if world == 1 else (None, None, 0, 0, 0.0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": cfg,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d.value),
                "d2h_bytes_per_step": int(d2h.value), "steps": n_e2e},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": {"bound": "alu" if t_alu_us >= t_hbm_us else "hbm", "achieved": achieved, "peak": peak,
                     "unit": "Tops/s", "frac": achieved / peak, "traffic": traffic, "kernel": "scan_wide_kernel",
                     "scan_ms": scan_s * 1000.0, "ops_per_launch": ops_per_search,
                     "cells_per_launch": cells_per_search, "shifts_per_launch": shifts_per_search,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "t_roof_us": max(t_alu_us, t_hbm_us), "t_alu_us": t_alu_us, "t_hbm_us": t_hbm_us,
                     "peak_basis": basis,
                     "byte_lane_peak": 4 * peak,
                     "byte_lane_frac": cells_per_search / scan_s / 1e12 / (4 * peak)},
        "clocks": clk,
    }
    if peaks is not None:
        line["int_peaks"] = peaks
    if batched is not None:
        line["batched"] = batched
    if serving is not None:
        line["serving"] = serving
    if bimodal is not None:
        line["bimodal"] = bimodal
    if small is not None:
        line["plain_small"] = small
    if full is not None:
        line["full_slide"] = full
    if cpu_rate is not None:
        line["cpu_baseline"] = {"value": cpu_rate, "unit": UNIT, "cores": cpu_threads, "kind": "oracle",
                                "sample": "%d random sequences (%d residues) of the same database, scores only, "
                                          "%.1f s" % (ns, nres, tcpu)}
    D.close()
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
