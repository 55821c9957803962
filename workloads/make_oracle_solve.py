"""Record the FP64 oracle's own GMRES solve of a workload's plane-wave system.

The reference arm of bench.py times the oracle's product on a box subsample and
scales it to a whole solve; the number of products in that solve comes from this
file: the oracle's GMRES(50) (oracle.gmres over the brute-force oracle.operator)
run once to the stated tolerance.

Usage: python workloads/make_oracle_solve.py shell16 [--tol 1e-6] [--grouped]
Writes workloads/oracle_solve.json (merged with what is there).  --grouped uses the
displacement-grouped FP64 product (oracle.operator_grouped, pinned to the brute force
within 1e-13), which makes the 5,000-box shell32 solve take minutes per product
instead of most of an hour.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
import workloads as W  # noqa: E402

BUILDERS = {"tiny": W.tiny, "shell16": W.shell16, "shell32": W.shell32}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="+")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--grouped", action="store_true")
    args = ap.parse_args()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_solve.json")
    for name in args.names:
        p = BUILDERS[name]()
        p.alpha = W.alpha_for(name)
        kh, pol = W.plane_wave_spec(1)
        v = oracle.plane_wave_rhs(p, kh, pol)[0]
        calls = []

        def matvec(x):
            t = time.time()
            op = oracle.operator_grouped if args.grouped else oracle.operator
            y = op(p, x[None, :], "full")[0]
            calls.append(time.time() - t)
            print(name, "product", len(calls), f"{calls[-1]:.1f} s", flush=True)
            return y

        x, iters, hist = oracle.gmres(matvec, v, restart=50, tol=args.tol)
        table = json.load(open(path)) if os.path.exists(path) else {}
        table[f"{name}@{args.tol:g}"] = dict(iterations=iters, products=len(calls), history=hist,
                                             seconds_per_product=sum(calls) / max(1, len(calls)),
                                             threads=oracle.num_threads(),
                                             method=("oracle.gmres(restart 50, x0 = 0) on " +
                                                     ("oracle.operator_grouped (displacement-grouped FP64)"
                                                      if args.grouped else "oracle.operator (brute force)")))
        with open(path, "w") as f:
            json.dump(table, f, indent=1)
        print(name, "iterations", iters, "products", len(calls), flush=True)


if __name__ == "__main__":
    main()
