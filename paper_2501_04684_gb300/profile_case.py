"""A mid-size far-zone product for kernel profiling (ncu) of libie.

Builds a sphere-shell scatterer small enough that its coupling stores stay within
a few GB, runs `--reps` far-zone products in each requested precision and exits.
Example (the translation kernel of one BF16X3 product):

  python -m paper_2501_04684_gb300.profile_case --grid 10 --radius 4 --prec bf16x3

With --prec cvfcnn the plan fits the translation networks (FP64 Jacobi SVDs); --map N also
runs the mapping construction for N boxes' worth of seeded point-dipole functions.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=10)
    ap.add_argument("--radius", type=float, default=4.0)
    ap.add_argument("--prec", default="bf16x3", help="comma list of fp32,bf16x3,fp16x3,bf16x1,fp16x1,cvfcnn")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--symmetry", type=int, default=0, choices=[0, 1])
    ap.add_argument("--map", type=int, default=0,
                    help="also map this many boxes' worth of seeded point-dipole functions (ie_map_basis)")
    args = ap.parse_args()
    import numpy as np
    import torch

    import paper_2501_04684_gb300 as ie
    import workloads as W

    names = {v: k for k, v in ie.PREC_NAMES.items()}
    precs = [names[s] for s in args.prec.split(",")]
    boxes = W.sphere_shell(args.grid, args.radius)
    p = W.make_problem("profile", args.grid, boxes, 32, seed_P=61, alpha=1.0)
    mask = ie.precmask(*precs)
    with ie.Plan(ie.problem_from(p, mask, args.nrhs, symmetry=args.symmetry)) as plan:
        st = plan.stats
        c = torch.from_numpy(W.coefficients(p, args.nrhs, 62).astype(np.complex64)).cuda()
        y = torch.zeros_like(c)
        for prec in precs:
            for _ in range(args.reps):
                ie.ie_matvec(plan.handle, ie.IE_FAR, prec, c, y, args.nrhs)
        torch.cuda.synchronize()
        if args.map:
            fun_off, pos, mom = W.point_dipole_basis(p.nb[:args.map], 63, a=p.a)
            ie.ie_map_basis(p.k, p.eta, p.a, fun_off, pos, mom, tikhonov=W.MAPPED_TIKHONOV)
        print(f"profile case: {st['n_boxes']} boxes, {st['n_far_pairs']} far pairs, {st['n_far_disp']} groups "
              f"on {st['n_coupling_blocks']} stored blocks, "
              f"{st['device_bytes'] / 1e9:.2f} GB on the device; precisions {args.prec} x {args.reps}")


if __name__ == "__main__":
    main()
