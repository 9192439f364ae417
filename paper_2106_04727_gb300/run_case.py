"""Run one clustering of a named synthetic workload and print its counters.

    python -m paper_2106_04727_gb300.run_case --workload gmm5d_1m_f32 --n 100000 \
        --linkage average --precision f32 --cache-slots 128 [--dense-k 4096] [--runs 1] \
        [--lib path/to/libhac.so]

A single process, one GPU, device-resident input: the command the profile
summaries under profiles/ run under ncu (small cases), and a quick way to time
one configuration.  Prints one JSON line per run (hac_stats of that run).
"""
from __future__ import annotations

import argparse
import json
import os


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="gmm5d_1m_f32")
    ap.add_argument("--n", type=int, default=None, help="points (default: the workload's)")
    ap.add_argument("--linkage", default="average")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--cache-slots", type=int, default=0)
    ap.add_argument("--dense-k", type=int, default=None,
                    help="average linkage: dense-matrix threshold (HAC_DENSE_K)")
    ap.add_argument("--runs", type=int, default=1)
    ap.add_argument("--lib", default=None, help="run with this compiled libhac.so")
    args = ap.parse_args()
    if args.dense_k is not None:
        os.environ["HAC_DENSE_K"] = str(args.dense_k)  # read by hac_create

    from . import build, hac, inputs

    if args.lib:
        build.LIB = args.lib  # a compiled variant: loaded as is, never rebuilt
        hac.load(build_if_missing=False)
    X = inputs.workload(args.workload, n=args.n)
    prec = hac.PREC_F64 if args.precision == "f64" else hac.PREC_F32_RECHECK
    h = hac.hac_create(X, args.linkage)
    try:
        for _ in range(args.runs):
            rc = hac.hac_run(h, precision=prec, cache_slots=args.cache_slots)
            if rc != hac.HAC_OK:
                raise hac.HacError(rc, "hac_run")
            st = hac.hac_stats(h)
            print(json.dumps({"workload": args.workload, "n": len(X), "linkage": args.linkage,
                              "precision": args.precision, **st}), flush=True)
    finally:
        hac.hac_destroy(h)


if __name__ == "__main__":
    main()
