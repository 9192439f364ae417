"""Benchmark: exact HAC dendrogram of 10^6 points (5-D Gaussian mixture) on GB300.

One step = one full hac_run (initial layout + every NN-chain round until one
cluster remains) on a device-resident instance, i.e. the whole hot path.
Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--linkage ward]
                  [--precision f64|f32] [--workload gmm5d_1m_f32] [--impl ours|reference]

--impl reference times the CPU oracle (FP64 Lance-Williams NN-chain) on a
bounded sample of the same workload on the host cores.  Multi-GPU runs are
independent replicas (the dendrogram computation does not shard): each rank
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

METRIC = "HAC wall time & distance evals/s vs HBM roofline at n=1M"
UNIT = "points/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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


def cpu_baseline(workload: str, linkage: str, n_sample: int):
    """The oracle, as it stands, on a bounded sample of the workload (1 core)."""
    import numpy as np

    import oracle
    from paper_2106_04727_gb300 import inputs

    X = inputs.workload(workload, n=n_sample).astype(np.float64)
    t0 = time.perf_counter()
    oracle.nnchain(X, linkage)
    dt = time.perf_counter() - t0
    return {"value": n_sample / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n_sample} points of {workload} ({linkage}), serial FP64 "
                      f"Lance-Williams NN-chain, {dt:.2f} s; O(n^2) so its points/s "
                      f"falls further at 10^6 points"}, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np  # noqa: F401

    ts = []
    for i in range(args.warmup + args.steps):
        cb, dt = cpu_baseline(args.workload, args.linkage, args.ref_sample)
        if i >= args.warmup:
            ts.append(dt)
    tot = sum(ts)
    v = args.ref_sample * len(ts) / tot
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(ts), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "linkage": args.linkage,
                       "n": args.ref_sample, "note": "bounded sample; host cores"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": v, "unit": UNIT,
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gmm5d_1m_f32")
    ap.add_argument("--linkage", default="ward", choices=["ward", "average", "complete"])
    ap.add_argument("--precision", default="f64", choices=["f64", "f32"])
    ap.add_argument("--cache-slots", type=int, default=-1,
                    help="Section 5 cache slots per cluster (default 64 for complete/average)")
    ap.add_argument("--ref-sample", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.cache_slots < 0:
        args.cache_slots = 0 if args.linkage == "ward" else 64
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
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
    h = hac.hac_create_device(Xd.data_ptr(), n, d, X.dtype, args.linkage)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        rc = hac.hac_run(h, precision=prec, cache_slots=args.cache_slots,
                         stream=stream.cuda_stream)
        if rc != 0:
            raise hac.HacError(rc, "hac_run")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, stats = [], []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with Clocks(local) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))              # evict L2 between timed steps (untimed)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            stats.append(hac.hac_stats(h))
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(times)
    if dist:
        t = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    value = ws * n * args.steps / (tot_ms / 1e3)

    # dominant kernel: the nearest-neighbour search
    q_ms = sum(s["ms_query"] for s in stats)
    q_bytes = sum(s["query_bytes"] for s in stats)
    q_launch = sum(s["query_launches"] for s in stats)
    peak, peak_kind = _peaks()
    achieved = q_bytes / (q_ms / 1e3) / 1e9 if q_ms > 0 else 0.0
    st = stats[-1]
    e2e = None
    cpu = None
    if rank == 0 and not args.no_e2e:
        # end to end through the public API from pinned host memory
        Xp = torch.from_numpy(X).pin_memory().numpy()
        e2e_t = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = hac.cluster(Xp, args.linkage, precision=prec, with_rounds=False,
                              cache_slots=args.cache_slots)
            e2e_t.append(time.perf_counter() - t0)
            assert len(res["a"]) == n - 1
        e2e = {"value": n / min(e2e_t), "unit": UNIT, "h2d_bytes_per_step": int(X.nbytes),
               "d2h_bytes_per_step": int((n - 1) * 24)}
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        cpu, _ = cpu_baseline(args.workload, args.linkage, args.ref_sample)
    hac.hac_destroy(h)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == hac.PREC_F64 else "f32+f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "d": d, "linkage": args.linkage,
                       "precision": args.precision, "cache_slots": args.cache_slots,
                       "parallelism": f"replicas{ws}",
                       "l2": "flushed between steps (256 MB write)"},
            "hac": {"wall_s_per_run": tot_ms / args.steps / 1e3, "rounds": st["rounds"],
                    "nn_searches": st["nn_searches"], "cluster_pairs": st["cluster_pairs"],
                    "point_pairs": st["point_pairs"], "nodes_visited": st["nodes_visited"],
                    "leaf_tests": st["leaf_tests"], "query_launches": st["query_launches"],
                    "cluster_pair_evals_per_s": st["cluster_pairs"] / (times[-1] / 1e3),
                    "point_pair_evals_per_s": st["point_pairs"] / (times[-1] / 1e3),
                    "ms_init": st["ms_init"], "ms_nn": st["ms_nn"], "ms_merge": st["ms_merge"],
                    "ms_update": st["ms_update"], "ms_query": st["ms_query"],
                    "device_bytes": st["device_bytes"], "host_wall_s": wall / args.steps},
            "roofline": {"kernel": "k_query64", "bound": "hbm", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": peak_kind,
                         "bytes_per_launch": q_bytes / max(q_launch, 1),
                         "ms_per_launch": q_ms / max(q_launch, 1)},
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
            "clocks": clk.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
