"""Tuner for the thresholds of the GPU-wide pair evaluation and for the
compile-time tile shapes.

The library reads three knobs when a handle is created:

  HAC_BIG_PAIRS     pairs of at least this many point pairs go to the GPU-wide
                    kernels instead of being evaluated by the searching warp
  HAC_WARP_BUDGET   point pairs a search evaluates itself before it hands
                    every further pair of at least 2^12 point pairs over
  cache_slots       Section 5 cache slots per cluster (a run option)

This script clusters one workload under every combination of the given
values (one warm-up run, then ``--runs`` timed runs each, timed as the
library reports them: hac_stats' ms_total, the wall time of the blocking
hac_run) and prints one JSON line per combination and a last line with the
fastest, as the settings to export.

    python -m paper_2106_04727_gb300.tune --workload gmm5d_1m_f32 --linkage average

With --shapes it tunes the compile-time tile and block shapes instead: every
combination of the given macro values is compiled as its own library
variant (build.build(defines=...), in _build/variants/), and each variant
clusters the workload in a child process (this script with --lib, the
thresholds at their defaults); one JSON line per variant, then the fastest.

    python -m paper_2106_04727_gb300.tune --shapes "HAC_DS_PPT8=2,4;HAC_DS_MINB=2,3"

The macros: HAC_DS_PPT8 / HAC_DS_MINB (rows per thread of the dense sweep for
d <= 8 / its resident tiles per SM), HAC_QWARPS (warps per block of the
search), HAC_QMINB / HAC_QMINB_COMPLETE (its resident blocks per SM, which
bound its registers; the second for complete linkage),
HAC_Q_OUTLINE (1: its warp-wide pair evaluations compiled out of line),
HAC_BR_T / HAC_BR_C (terminals per CTA / records per staged tile of
the exhaustive scans), HAC_CM_WARPS (warps per block of the cache update).
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import statistics


SHAPES = ("HAC_DS_PPT8", "HAC_DS_MINB", "HAC_QWARPS", "HAC_QMINB", "HAC_QMINB_COMPLETE", "HAC_Q_OUTLINE", "HAC_BR_T",
          "HAC_BR_C", "HAC_CM_WARPS")


def shape_grid(spec: str):
    """'A=1,2;B=3' -> [{'A': 1, 'B': 3}, {'A': 2, 'B': 3}] (known macros only)."""
    axes = []
    for part in [p for p in spec.split(";") if p.strip()]:
        name, vals = part.split("=")
        name = name.strip()
        if name not in SHAPES:
            raise ValueError(f"unknown shape macro {name}")
        axes.append([(name, int(v)) for v in vals.split(",")])
    return [dict(c) for c in itertools.product(*axes)]


def tune_shapes(args):
    """Build and time one library variant per combination of shape macros."""
    import subprocess
    import sys

    from paper_2106_04727_gb300 import build

    results = []
    for defines in shape_grid(args.shapes):
        lib = build.build(defines=defines)
        cmd = [sys.executable, "-m", "paper_2106_04727_gb300.tune", "--lib", lib,
               "--workload", args.workload, "--linkage", args.linkage, "--runs", str(args.runs),
               "--big", "65536", "--budget", "262144", "--slots", args.slots]
        if args.n:
            cmd += ["--n", str(args.n)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"variant {defines} failed:\n{r.stderr[-2000:]}")
        best = json.loads(r.stdout.strip().splitlines()[-1])["best"]
        row = dict(defines, ms=best["ms"], ms_search=best["ms_search"])
        results.append(row)
        print(json.dumps(row), flush=True)
    best = min(results, key=lambda r: r["ms"])
    print(json.dumps({"best": best, "workload": args.workload, "linkage": args.linkage}),
          flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="gmm5d_1m_f32")
    ap.add_argument("--n", type=int, default=None, help="draw the workload at this size")
    ap.add_argument("--linkage", default="average")
    ap.add_argument("--big", default="32768,65536,131072")
    ap.add_argument("--budget", default="131072,262144,1048576")
    ap.add_argument("--slots", default="128")
    ap.add_argument("--runs", type=int, default=2)
    ap.add_argument("--shapes", default=None,
                    help="tile-shape macros to tune, e.g. 'HAC_DS_PPT8=2,4;HAC_DS_MINB=2,3'")
    ap.add_argument("--lib", default=None, help="run with this compiled libhac.so")
    args = ap.parse_args(argv)
    if args.shapes:
        return tune_shapes(args)

    from paper_2106_04727_gb300 import build, hac, inputs

    if args.lib:
        build.LIB = args.lib  # a compiled variant: loaded as is, never rebuilt
        hac.load(build_if_missing=False)

    X = inputs.workload(args.workload, n=args.n)
    grid = list(itertools.product([int(v) for v in args.big.split(",")],
                                  [int(v) for v in args.budget.split(",")],
                                  [int(v) for v in args.slots.split(",")]))
    results = []
    for big, budget, slots in grid:
        os.environ["HAC_BIG_PAIRS"] = str(big)
        os.environ["HAC_WARP_BUDGET"] = str(budget)
        h = hac.hac_create(X, args.linkage)   # the knobs are read here
        try:
            times = []
            for i in range(1 + args.runs):
                rc = hac.hac_run(h, precision=hac.PREC_F32_RECHECK, cache_slots=slots)
                if rc != hac.HAC_OK:
                    raise hac.HacError(rc, "hac_run")
                if i:
                    times.append(hac.hac_stats(h)["ms_total"])
            st = hac.hac_stats(h)
        finally:
            hac.hac_destroy(h)
        row = {"HAC_BIG_PAIRS": big, "HAC_WARP_BUDGET": budget, "cache_slots": slots,
               "ms": statistics.median(times), "point_pairs": st["point_pairs"],
               "ms_search": st["ms_query"], "ms_big": st["ms_big"]}
        results.append(row)
        print(json.dumps(row), flush=True)
    best = min(results, key=lambda r: r["ms"])
    print(json.dumps({"best": best, "workload": args.workload, "linkage": args.linkage,
                      "n": len(X)}), flush=True)


if __name__ == "__main__":
    main()
