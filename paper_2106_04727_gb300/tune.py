"""Tuner for the thresholds of the GPU-wide pair evaluation.

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
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import statistics


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="gmm5d_1m_f32")
    ap.add_argument("--n", type=int, default=None, help="draw the workload at this size")
    ap.add_argument("--linkage", default="average")
    ap.add_argument("--big", default="32768,65536,131072")
    ap.add_argument("--budget", default="131072,262144,1048576")
    ap.add_argument("--slots", default="128")
    ap.add_argument("--runs", type=int, default=2)
    args = ap.parse_args(argv)

    from paper_2106_04727_gb300 import hac, inputs

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
