"""Benchmark: exact HAC dendrograms of 10^6 points (5-D Gaussian mixture) on GB300.

One step = the n = 10^6 workload's whole hot path: a full hac_run (initial
layout + every NN-chain round until one cluster remains) under Ward AND under
average linkage, on device-resident points, in the FP32-bulk + FP64-re-score
mode (the Section 5 cache on for average).  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--linkages ward,average]
                  [--precision f32|f64] [--workload gmm5d_1m_f32] [--impl ours|reference]

--impl reference times the CPU baseline, a plain multithreaded FP64 NN-chain
(oracle/hac_parchain_cpu.c), on the same workload on every host core, each
linkage stopped at --cpu-cap seconds.  Multi-GPU runs are
independent replicas (a dendrogram computation does not shard): each rank
clusters its own copy and value = all ranks' points / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HAC wall time & distance evals/s vs HBM roofline at n=1M; serving p50/p99 ms"
UNIT = "points/s"

# Per-launch DRAM traffic of the kernels other than the sweep is not scaled
# from small captures (their launches differ too much in size): null.
TRAFFIC = {}
# DRAM bytes (read + write) per point pair of the dense sweep, from a
# small-case ncu capture of the current kernel (profiles/
# k_dense_sweep32_gmm5d_100k.md: 385.1 MB for 4.995e9 pairs); the bench
# scales it by the pairs of a full launch
SWEEP_DRAM_PER_PAIR = 385.1e6 / 4.995e9


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def fp32_peak(local: int):
    """FP32 multiply-add throughput measured on this GPU (the library's FMA
    probe: scalar and packed f32x2 loops, CUDA events), with the SM clock
    sampled during it.  Returns (TFLOP/s, description)."""
    import ctypes

    from paper_2106_04727_gb300 import build as libbuild

    lib = ctypes.CDLL(libbuild.build_probe())
    lib.hac_probe_fma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_float)]
    best = {}
    with Clocks(local) as clk:
        for packed in (0, 1):
            tf, ms = ctypes.c_double(), ctypes.c_float()
            rc = lib.hac_probe_fma(packed, 5, ctypes.byref(tf), ctypes.byref(ms))
            if rc != 0:
                raise RuntimeError(f"FMA probe failed ({rc})")
            best["f32x2" if packed else "scalar"] = tf.value
    c = clk.summary() or {}
    peak = max(best.values())
    return peak, (f"measured: FMA-loop probe, {best['scalar']:.1f} TFLOP/s scalar, "
                  f"{best['f32x2']:.1f} TFLOP/s packed f32x2, median SM clock "
                  f"{c.get('sm_mhz')} MHz during the probe")


def same_tree(a, b, rtol):
    """Two dendrograms (dicts of arrays a, b, h, size) have the same merges
    (cid_a, cid_b, size) and heights within rtol; returns (same, largest
    relative height difference)."""
    import numpy as np

    ka = np.lexsort((a["b"], a["a"]))
    kb = np.lexsort((b["b"], b["a"]))
    same = len(ka) == len(kb) and all(np.array_equal(np.asarray(a[f])[ka], np.asarray(b[f])[kb])
                                      for f in ("a", "b", "size"))
    if not same:
        return False, float("inf")
    ha, hb = np.asarray(a["h"])[ka], np.asarray(b["h"])[kb]
    err = float(np.max(np.abs(ha - hb) / np.maximum(np.abs(hb), 1e-300))) if len(ha) else 0.0
    return err <= rtol, err


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return None
        try:
            sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
            mx = max(float(r[2]) for r in self.rows)
        except Exception:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, dist, device) -> float:
    """The largest value over all ranks: a replicated job takes as long as its
    slowest rank.  `dist` is torch.distributed (initialised) or None."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(workload: str, linkages, cap_s: float, n=None):
    """The plain multithreaded CPU NN-chain (oracle/hac_parchain_cpu.c:
    Algorithm 1 on every host core, FP64, linear memory, the range queries of
    Section 4) on the workload, each linkage stopped at cap_s seconds between
    rounds.  A capped linkage counts cap_s, so the rate is an upper bound."""
    import numpy as np

    import oracle
    from paper_2106_04727_gb300 import inputs

    X = inputs.workload(workload, n=n).astype(np.float64)
    cores = os.cpu_count() or 1
    per, tot, capped = {}, 0.0, []
    for lk in linkages:
        r = oracle.parchain_cpu(X, lk, threads=cores, timeout_s=cap_s)
        per[lk] = {"seconds": round(r["seconds"], 3), "complete": r["complete"],
                   "merges": int(len(r["a"])), "rounds": r["n_rounds"],
                   "point_pairs": r["point_pairs"]}
        tot += r["seconds"] if r["complete"] else max(r["seconds"], cap_s)
        if not r["complete"]:
            capped.append(lk)
    where = "" if not capped else (f"; {', '.join(capped)} stopped at the {cap_s:g} s cap "
                                   f"(> cap: the rate is an upper bound)")
    return {"value": len(X) / tot, "unit": UNIT, "cores": cores, "kind": "oracle",
            "implementation": "multithreaded CPU NN-chain (oracle/hac_parchain_cpu.c), FP64",
            "n": len(X), "capped": bool(capped), "per_linkage": per,
            "sample": f"all {len(X)} points of {workload} ({'+'.join(linkages)}), one step "
                      f"(both linkages) on {cores} host threads{where}"}, tot


def run_reference(args):
    """The CPU baseline as the reference arm: K steps of the whole workload
    on the host cores (warm-up steps on a 20,000-point sample of it)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n_ref = getattr(args, "ref_n", None)
    for _ in range(args.warmup):
        cpu_baseline(args.workload, args.linkages, args.cpu_cap, n=min(20000, n_ref or 20000))
    ts = []
    cb = None
    for _ in range(args.steps):
        cb, dt = cpu_baseline(args.workload, args.linkages, args.cpu_cap, n=n_ref)
        ts.append(dt)
    tot = sum(ts)
    n = cb["n"]
    v = n * len(ts) / tot
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(ts), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "linkages": "+".join(args.linkages),
                       "n": n, "cap_s_per_linkage": args.cpu_cap,
                       "note": "the whole workload on the host cores; warm-up steps on a "
                               "20,000-point sample"},
            "cpu_baseline": dict(cb, value=v),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SERVING_METRIC = "serving p50/p99 ms and jobs/s (4,096-request stream)"


def _pct(v, q):
    import numpy as np
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


def _serve(hac, srv, reqs, pts, arrivals=None):
    """Submit a request stream (all at t=0, or at the given arrival times) and
    wait for every result; latency = completion - arrival."""
    t0 = time.perf_counter()
    tickets, t_sub = [], []
    for i, (r, X) in enumerate(zip(reqs, pts)):
        if arrivals is not None:
            dt = t0 + arrivals[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
        t_sub.append(time.perf_counter() - t0)
        tickets.append(hac.hac_submit(srv, X, r["linkage"]))
    lat, res = [], []
    for i, (t, r) in enumerate(zip(tickets, reqs)):
        rc = hac.hac_server_wait(srv, t, 3600.0)
        rc, m, ms = hac.hac_poll(srv, t, r["n"])
        if rc != hac.HAC_OK:
            raise hac.HacError(rc, "serving request")
        late = t_sub[i] - (arrivals[i] if arrivals is not None else 0.0)
        lat.append(ms + 1e3 * late)
        res.append(m)
    span = time.perf_counter() - t0
    return {"jobs": len(reqs), "makespan_s": span, "jobs_per_s": len(reqs) / span,
            "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99), "max_ms": max(lat)}, res


def _per_instance(hac, reqs, pts, prec, slots):
    """The plain per-instance GPU path: hac_create + hac_run + hac_dendrogram,
    one request after the other; all requests arrive at t=0."""
    t0 = time.perf_counter()
    lat, res = [], []
    for r, X in zip(reqs, pts):
        res.append(hac.cluster(X, r["linkage"], precision=prec, cache_slots=slots,
                               with_rounds=False))
        lat.append(1e3 * (time.perf_counter() - t0))
    span = time.perf_counter() - t0
    return {"jobs": len(reqs), "makespan_s": span, "jobs_per_s": len(reqs) / span,
            "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99), "max_ms": max(lat)}, res


def serving_measure(args, steps, warmup, local):
    """The serving stream: requests of uneven n, d and linkage, continuous
    batching in the library's server (FP32 bulk + FP64 re-score): saturated
    (every request at t = 0) jobs/s and latencies, Poisson arrivals at 0.7 x
    that rate, and on a sample of the stream the batched server against the
    plain per-instance FP64 GPU path (hac_create + hac_run + hac_dendrogram
    per request), the same requests one after the other in FP32 + re-score,
    and a batched FP64 server, with the trees compared to the FP64 ones."""
    import numpy as np
    import torch

    from paper_2106_04727_gb300 import hac, inputs

    slots = args.serving_cache_slots
    reqs = inputs.serving_requests(args.requests, seed=4)
    pts = [inputs.request_points(r) for r in reqs]
    cap = args.engine_points
    srv = hac.hac_server_create(cap, precision=hac.PREC_F32_RECHECK, cache_slots=slots)
    srv64 = None
    try:
        # warm-up: engines of every kind allocated, then W short streams
        warm = inputs.serving_requests(96, seed=5, n_hi=4096)
        wpts = [inputs.request_points(r) for r in warm]
        for lk in range(3):
            for d in (2, 3, 5, 10):
                t = hac.hac_submit(srv, inputs.gaussian_mixture(100, d, 4, seed=d), lk)
                hac.hac_server_wait(srv, t, 600.0)
                hac.hac_poll(srv, t, 100)
        for _ in range(warmup):
            _serve(hac, srv, warm, wpts)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        st0 = hac.hac_server_stats(srv)
        sat = []
        with Clocks(local) as clk:
            for i in range(steps):
                flush.fill_(float(i))
                torch.cuda.synchronize()
                sat.append(_serve(hac, srv, reqs, pts)[0])
        st1 = hac.hac_server_stats(srv)
        best = max(sat, key=lambda x: x["jobs_per_s"])
        # Poisson arrivals at 0.7 x the saturated rate
        rate = 0.7 * best["jobs_per_s"]
        gaps = -np.log(1.0 - inputs.uniform(4, 77, len(reqs))) / rate
        poisson, _ = _serve(hac, srv, reqs, pts, arrivals=np.cumsum(gaps))
        poisson["rate_jobs_per_s"] = rate
        # the per-instance paths on a sample of the same stream
        k = min(args.sample, len(reqs))
        sreq, spts = reqs[:k], pts[:k]
        batched_s, res_b = _serve(hac, srv, sreq, spts)
        per64, res_64 = _per_instance(hac, sreq, spts, hac.PREC_F64, slots)
        seq32, _ = _per_instance(hac, sreq, spts, hac.PREC_F32_RECHECK, slots)
        same, err = 0, 0.0
        for a, b in zip(res_b, res_64):
            ok, e = same_tree(hac.result_dict(a), b, 1e-5)
            same += int(ok)
            err = max(err, e)
        srv64 = hac.hac_server_create(cap, precision=hac.PREC_F64, cache_slots=slots)
        for lk in range(3):
            for d in (2, 3, 5, 10):
                t = hac.hac_submit(srv64, inputs.gaussian_mixture(100, d, 4, seed=d), lk)
                hac.hac_server_wait(srv64, t, 600.0)
                hac.hac_poll(srv64, t, 100)
        batched64_s, _ = _serve(hac, srv64, sreq, spts)
    finally:
        hac.hac_server_destroy(srv)
        hac.hac_server_destroy(srv64)
    out = {"saturated": sat, "poisson": poisson,
           "sample": {"requests": k, "batched_f32_recheck": batched_s,
                      "batched_f64": batched64_s,
                      "per_instance_f64": per64, "sequential_f32_recheck": seq32,
                      "speedup_batched_vs_per_instance_f64":
                          batched_s["jobs_per_s"] / per64["jobs_per_s"],
                      "same_trees_as_f64": f"{same}/{k}",
                      "max_rel_height_err_vs_f64": err}}
    return out, reqs, pts, st0, st1, clk.summary()


def run_serving(args):
    """The serving stream as its own benchmark line."""
    import numpy as np
    import torch

    import oracle
    from paper_2106_04727_gb300 import hac  # noqa: F401

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if rank != 0:
        return
    res, reqs, pts, st0, st1, clocks = serving_measure(args, args.steps, args.warmup, local)
    sat = res["saturated"]
    best = max(sat, key=lambda x: x["jobs_per_s"])
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle on the stream's requests of n <= 4096 (O(n^2) memory), first 24
        small = [(r, X) for r, X in zip(reqs, pts) if r["n"] <= 4096][:24]
        t0 = time.perf_counter()
        for r, X in small:
            oracle.nnchain(X.astype(np.float64), r["linkage"])
        dt = time.perf_counter() - t0
        cpu = {"value": len(small) / dt, "unit": "jobs/s", "cores": 1, "kind": "oracle",
               "sample": f"first {len(small)} requests of the stream with n <= 4096 "
                         f"(sum n = {sum(r['n'] for r, _ in small)}), serial FP64 "
                         f"Lance-Williams NN-chain, {dt:.2f} s"}
    pts_bytes = sum(int(X.nbytes) for X in pts)
    rec_bytes = sum(32 * (r["n"] - 1) for r in reqs)
    ms_step = 1e3 * sum(x["makespan_s"] for x in sat) / len(sat)
    line = {
        "metric": SERVING_METRIC, "value": best["jobs_per_s"], "unit": "jobs/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "serving_4096", "requests": len(reqs),
                   "points": int(sum(r["n"] for r in reqs)),
                   "n": "log-uniform [64, 65536]", "d": "{2,3,5,10}",
                   "linkages": "complete+average+ward", "precision": "f32",
                   "cache_slots": args.serving_cache_slots, "engine_points": args.engine_points,
                   "step": "the whole stream submitted at t=0, every result read back",
                   "l2": "flushed before each timed step (256 MB write); inputs are new "
                         "host data each step"},
        "serving": res,
        "server": {k2: st1[k2] - st0.get(k2, 0) if isinstance(st1[k2], (int, float)) and
                   k2 not in ("engines", "max_resident", "device_bytes", "status") else st1[k2]
                   for k2 in st1},
        "roofline": None,
        "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
        "clocks": clocks,
        "e2e": {"value": best["jobs_per_s"], "unit": "jobs/s",
                "h2d_bytes_per_step": pts_bytes, "d2h_bytes_per_step": rec_bytes,
                "note": "the server API takes host points and returns host records: "
                        "value is already end to end"},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


ABLATION_METRIC = "range-query ablation: time and distance evaluations, pruning on vs off"


def run_ablation(args):
    """The range query's effect (the paper's pruning-off comparison and its
    D / naive-work statistics): each linkage clustered with the range query
    and with every cluster as a candidate (HAC_FLAG_NO_PRUNE), on the paper's
    GaussianDisc and UniformFill shapes at growing n."""
    import numpy as np
    import torch

    from paper_2106_04727_gb300 import hac, inputs

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if rank != 0:
        return
    # the ablation measures the range query itself: average linkage stays on
    # it (no dense matrix) in both runs
    os.environ["HAC_DENSE_K"] = "0"
    prec = hac.PREC_F64 if args.precision == "f64" else hac.PREC_F32_RECHECK
    rows = []
    sizes = [int(x) for x in args.ablation_sizes.split(",")]
    for shape in ("gaussiandisc2d_1m_f32", "uniformfill2d_1m_f32"):
        for n in sizes:
            X = inputs.workload(shape, n=n)
            for lk in args.linkages:
                slots = args.cache_slots if lk in ("complete", "average") else 0
                r = {}
                for mode, flag in (("pruned", False), ("all_pairs", True)):
                    for _ in range(args.warmup if mode == "pruned" else 1):
                        hac.cluster(X, lk, precision=prec, cache_slots=slots, no_prune=flag,
                                    with_rounds=False)
                    res = hac.cluster(X, lk, precision=prec, cache_slots=slots, no_prune=flag,
                                      with_rounds=False)
                    st = res["stats"]
                    r[mode] = {"ms": st["ms_total"], "cluster_pairs": st["cluster_pairs"],
                               "point_pairs": st["point_pairs"], "leaf_tests": st["leaf_tests"],
                               "nodes": st["nodes_visited"]}
                    r["naive_pairs"] = st["naive_pairs"]
                    r["rounds"] = st["rounds"]
                    r["_h"] = r.get("_h", []) + [res]
                a, b = r.pop("_h")
                same = bool(np.array_equal(a["a"], b["a"]) and np.array_equal(a["b"], b["b"]))
                rows.append({"shape": shape.split("_")[0], "n": n, "linkage": lk, **r,
                             "same_tree": same,
                             "speedup": r["all_pairs"]["ms"] / r["pruned"]["ms"],
                             "cluster_pair_fraction": r["pruned"]["cluster_pairs"] / r["naive_pairs"]})
    top = [x["speedup"] for x in rows if x["n"] == max(sizes)]
    line = {"metric": ABLATION_METRIC, "value": float(np.exp(np.mean(np.log(top)))),
            "unit": "x (geometric-mean speedup of the range query at the largest n)",
            "n_gpus": 1, "steps": 1, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == hac.PREC_F64 else "f32+f64", "data": "synthetic",
            "config": {"workload": "ablation", "shapes": "GaussianDisc, UniformFill (2-D)",
                       "sizes": sizes, "linkages": "+".join(args.linkages)},
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_ablation_reference(args):
    """The oracle on the ablation's smallest samples (host core): its NN-chain
    over the full distance matrix is the no-range-query baseline of the CPU."""
    import numpy as np

    import oracle
    from paper_2106_04727_gb300 import inputs

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n = int(args.ablation_sizes.split(",")[0])
    rows, tot = [], 0.0
    for shape in ("gaussiandisc2d_1m_f32", "uniformfill2d_1m_f32"):
        X = inputs.workload(shape, n=n).astype(np.float64)
        for lk in args.linkages:
            t0 = time.perf_counter()
            oracle.nnchain(X, lk)
            dt = time.perf_counter() - t0
            tot += dt
            rows.append({"shape": shape.split("_")[0], "n": n, "linkage": lk, "ms": 1e3 * dt})
    v = len(rows) / tot
    print(json.dumps({
        "metric": ABLATION_METRIC, "value": v, "unit": "clusterings/s", "n_gpus": args.gpus,
        "steps": 1, "warmup": 0, "ms_per_step": 1e3 * tot, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference", "config": {"workload": "ablation", "sizes": [n]}, "rows": rows,
        "cpu_baseline": {"kind": "oracle", "cores": 1, "value": v, "unit": "clusterings/s",
                         "sample": f"{len(rows)} clusterings of {n} points"},
        "e2e": {"value": v, "unit": "clusterings/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def run_serving_reference(args):
    """The oracle on the serving stream's small requests (host core)."""
    import numpy as np

    import oracle
    from paper_2106_04727_gb300 import inputs

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    reqs = inputs.serving_requests(args.requests, seed=4)
    small = [r for r in reqs if r["n"] <= 4096][:24]
    ts = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for r in small:
            oracle.nnchain(inputs.request_points(r).astype(np.float64), r["linkage"])
        if i >= args.warmup:
            ts.append(time.perf_counter() - t0)
    v = len(small) * len(ts) / sum(ts)
    sample = (f"first {len(small)} requests of the stream with n <= 4096 per step, serial FP64 "
              f"Lance-Williams NN-chain")
    print(json.dumps({
        "metric": SERVING_METRIC, "value": v, "unit": "jobs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / len(ts),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": "serving_4096", "note": "bounded sample; host core"},
        "cpu_baseline": {"kind": "oracle", "cores": 1, "value": v, "unit": "jobs/s",
                         "sample": sample},
        "e2e": {"value": v, "unit": "jobs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gmm5d_1m_f32")
    ap.add_argument("--linkages", default="ward,average")
    ap.add_argument("--precision", default="f32", choices=["f64", "f32"])
    ap.add_argument("--cache-slots", type=int, default=128,
                    help="Section 5 cache slots per cluster for complete/average")
    ap.add_argument("--cpu-cap", type=float, default=30.0,
                    help="CPU baseline: seconds per linkage before it stops between rounds")
    ap.add_argument("--ref-n", type=int, default=None,
                    help="reference arm: points of the workload (default: all of it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-f64", action="store_true",
                    help="skip the all-FP64 run of the workload after the timed steps")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving-stream summary of the default line")
    ap.add_argument("--requests", type=int, default=4096, help="serving: stream length")
    ap.add_argument("--sample", type=int, default=256,
                    help="serving: requests timed on the per-instance paths")
    ap.add_argument("--ablation-sizes", default="5000,10000,20000,50000",
                    help="ablation: point counts")
    ap.add_argument("--serving-cache-slots", type=int, default=64,
                    help="serving: cache slots per cluster (complete/average engines)")
    ap.add_argument("--engine-points", type=int, default=1 << 21,
                    help="serving: points per engine (one engine per linkage and d)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.linkages = [x for x in args.linkages.split(",") if x]
    if args.workload == "ablation":
        if args.impl == "reference":
            return run_ablation_reference(args)
        return run_ablation(args)
    if args.workload == "serving":
        if args.impl == "reference":
            return run_serving_reference(args)
        return run_serving(args)
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_2106_04727_gb300 import hac, inputs

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    prec = hac.PREC_F64 if args.precision == "f64" else hac.PREC_F32_RECHECK
    X = inputs.workload(args.workload)
    n, d = X.shape
    stream = torch.cuda.current_stream()
    Xd = torch.from_numpy(X).to("cuda")
    handles = {lk: hac.hac_create_device(Xd.data_ptr(), n, d, X.dtype, lk) for lk in args.linkages}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        out = {}
        for lk, h in handles.items():
            rc = hac.hac_run(h, precision=prec, cache_slots=args.cache_slots,
                             stream=stream.cuda_stream)
            if rc != 0:
                raise hac.HacError(rc, "hac_run")
            out[lk] = hac.hac_stats(h)
        return out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stats = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))              # evict L2 before each timed step (untimed)
            ev[i][0].record(stream)
            stats.append(step())
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times = [a.elapsed_time(b) for a, b in ev]
    tot_ms = max_over_ranks(sum(times), dist, "cuda")
    value = ws * n * args.steps / (tot_ms / 1e3)

    def agg(key, lk=None):
        return sum(s[l][key] for s in stats for l in s if lk is None or l == lk)

    hbm, peak_kind = _peaks()
    fp32_tflops, fp32_src = fp32_peak(local)
    # kernels, measured by the library with CUDA events on the launching stream
    q_ms, q_bytes, q_launch = agg("ms_query"), agg("query_bytes"), agg("query_launches")
    b_ms, b_pairs, b_launch = agg("ms_big"), agg("big_point_pairs"), agg("big_launches")
    s_ms, s_pairs = agg("ms_dense"), agg("dense_point_pairs")
    s_launch = sum(1 for st in stats for l in st if st[l]["dense_k"] > 0)
    flops_per_pair = 3 * d + 2   # d subtractions, d multiply-adds (2 flops), sqrt, add
    kern = {
        "k_query": {"bound": "hbm", "ms": q_ms / args.steps, "launches": q_launch // args.steps,
                    "achieved": q_bytes / (q_ms / 1e3) / 1e9 if q_ms else 0.0, "peak": hbm,
                    "unit": "GB/s", "traffic": TRAFFIC.get(("k_query", args.workload))},
        "k_big_eval32": {"bound": "alu", "ms": b_ms / args.steps,
                         "launches": b_launch // args.steps,
                         "achieved": b_pairs * flops_per_pair / (b_ms / 1e3) / 1e12 if b_ms else 0.0,
                         "peak": fp32_tflops, "unit": "TFLOP/s",
                         "traffic": TRAFFIC.get(("k_big_eval32", args.workload))},
        "k_dense_sweep32": {"bound": "alu", "ms": s_ms / args.steps,
                            "launches": s_launch // args.steps,
                            "achieved": s_pairs * flops_per_pair / (s_ms / 1e3) / 1e12
                            if s_ms else 0.0,
                            "peak": fp32_tflops, "unit": "TFLOP/s",
                            "traffic": SWEEP_DRAM_PER_PAIR * s_pairs / max(s_launch, 1)
                            if s_launch else None,
                            "traffic_note": "DRAM bytes per point pair of a small-case ncu "
                                            "capture, times the pairs of a launch"},
    }
    for k in kern.values():
        k["frac"] = k["achieved"] / k["peak"] if k["peak"] else 0.0
    dom = max(kern, key=lambda k: kern[k]["ms"])
    roof = dict(kern[dom])
    roof["kernel"] = dom
    roof["peak_source"] = fp32_src if roof["bound"] == "alu" else peak_kind + " (HBM copy)"
    per_lk = {}
    for lk in args.linkages:
        ms = agg("ms_total", lk) / args.steps
        s0 = stats[-1][lk]
        per_lk[lk] = {"ms_per_run": ms, "rounds": s0["rounds"], "nn_searches": s0["nn_searches"],
                      "cluster_pairs": s0["cluster_pairs"], "point_pairs": s0["point_pairs"],
                      "cluster_pair_evals_per_s": s0["cluster_pairs"] / (ms / 1e3),
                      "point_pair_evals_per_s": s0["point_pairs"] / (ms / 1e3),
                      "cache_hits": s0["cache_hits"], "ms_search": s0["ms_query"],
                      "ms_big_pairs": s0["ms_big"], "ms_dense_sweep": s0["ms_dense"],
                      "dense_k": s0["dense_k"], "dense_rounds": s0["dense_rounds"],
                      "point_pairs_over_minimum": s0["point_pairs"] / (n * (n - 1) / 2)}
    # the plain all-FP64 GPU path on the same workload (untimed by the steps):
    # its wall time per linkage and whether its tree is the FP32 + re-score one
    c2 = None
    if rank == 0 and not args.no_f64 and prec != hac.PREC_F64:
        c2 = {}
        for lk, h in handles.items():
            m32 = hac.hac_dendrogram(h, n)
            d32 = {"a": m32["cid_a"].copy(), "b": m32["cid_b"].copy(), "h": m32["height"].copy(),
                   "size": m32["size"].copy()}
            rc = hac.hac_run(h, precision=hac.PREC_F64, cache_slots=args.cache_slots,
                             stream=stream.cuda_stream)
            if rc != 0:
                raise hac.HacError(rc, "hac_run (FP64)")
            st64 = hac.hac_stats(h)
            m64 = hac.hac_dendrogram(h, n)
            d64 = {"a": m64["cid_a"], "b": m64["cid_b"], "h": m64["height"], "size": m64["size"]}
            ok, err = same_tree(d32, d64, 1e-5)
            c2[lk] = {"ms_f64": st64["ms_total"], "ms_f32_recheck": per_lk[lk]["ms_per_run"],
                      "speedup_f32_recheck": st64["ms_total"] / per_lk[lk]["ms_per_run"],
                      "same_tree": ok, "max_rel_height_err": err,
                      "ms_dense_sweep_f64": st64["ms_dense"]}
    e2e = None
    cpu = None
    if rank == 0 and not args.no_e2e:
        # end to end through the public API from pinned host memory
        Xp = torch.from_numpy(X).pin_memory().numpy()
        e2e_t = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for lk in args.linkages:
                res = hac.cluster(Xp, lk, precision=prec, with_rounds=False,
                                  cache_slots=args.cache_slots)
                assert len(res["a"]) == n - 1
            e2e_t.append(time.perf_counter() - t0)
        e2e = {"value": n / min(e2e_t), "unit": UNIT,
               "h2d_bytes_per_step": int(X.nbytes) * len(args.linkages),
               "d2h_bytes_per_step": int((n - 1) * 32) * len(args.linkages)}
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        cpu, _ = cpu_baseline(args.workload, args.linkages, args.cpu_cap)
    for h in handles.values():
        hac.hac_destroy(h)
    del Xd, flush
    torch.cuda.empty_cache()
    serving = None
    if rank == 0 and not args.no_serving:
        res, _, _, _, _, sclk = serving_measure(args, 1, 1, local)
        sat = res["saturated"][0]
        smp = res["sample"]
        serving = {"metric": SERVING_METRIC, "requests": args.requests,
                   "saturated_jobs_per_s": sat["jobs_per_s"],
                   "saturated_p50_ms": sat["p50_ms"], "saturated_p99_ms": sat["p99_ms"],
                   "poisson_rate_jobs_per_s": res["poisson"]["rate_jobs_per_s"],
                   "poisson_p50_ms": res["poisson"]["p50_ms"],
                   "poisson_p99_ms": res["poisson"]["p99_ms"],
                   "sample_requests": smp["requests"],
                   "batched_f32_recheck_jobs_per_s": smp["batched_f32_recheck"]["jobs_per_s"],
                   "per_instance_f64_jobs_per_s": smp["per_instance_f64"]["jobs_per_s"],
                   "speedup_batched_vs_per_instance_f64":
                       smp["speedup_batched_vs_per_instance_f64"],
                   "same_trees_as_f64": smp["same_trees_as_f64"],
                   "max_rel_height_err_vs_f64": smp["max_rel_height_err_vs_f64"],
                   "clocks": sclk}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == hac.PREC_F64 else "f32+f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "d": d,
                       "linkages": "+".join(args.linkages), "precision": args.precision,
                       "cache_slots": args.cache_slots, "parallelism": f"replicas{ws}",
                       "step": "one full dendrogram per linkage",
                       "l2": "flushed before each timed step (256 MB write)"},
            "hac": per_lk,
            "roofline": roof,
            "kernels": kern,
            "gpu_launches": int(agg("kernel_launches")),
            "clocks": clk.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "c2_f64": c2,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
