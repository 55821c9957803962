"""Freeze the self-term alpha of each workload with the FP64 oracle.

alpha = alpha_rel * sigma, sigma = ||P D_off P^T||_2 estimated by power iteration
(oracle.operator_norm), alpha_rel = 1.25, rounded to 3 significant digits.  With
alpha > sigma the system matrix alpha I + P D_off P^T is nonsingular and GMRES
contracts the residual by at least sigma/alpha per step.

Usage: python workloads/make_alpha.py tiny shell16 [--iters N]
Writes workloads/alpha.json (merged with what is there).

With --check the frozen alpha is kept and a longer power iteration (from the same seed)
is recorded beside it as sigma_check / history_check, with alpha / sigma_check: how far
the frozen value's margin over sigma holds once the estimate has converged further.
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

ALPHA_REL = 1.25


def mapped(p):
    """p with P replaced by the oracle's mapping (eq. 11) of seeded point-dipole functions."""
    fun_off, pos, mom = W.point_dipole_basis(p.nb, W.SEED_MAPPED[p.name], a=p.a)
    P, _ = oracle.map_basis(p.k, p.eta, p.a, p.lattice, 128, 1.5, fun_off, pos, mom, tikhonov=W.MAPPED_TIKHONOV)
    p.P = P
    p.name = p.name + "_mapped"
    return p


BUILDERS = {
    "tiny": lambda: W.tiny(),
    "shell16": lambda: W.shell16(),
    "shell16_identity": lambda: W.shell16(identity=True),
    "shell32": lambda: W.shell32(),
    "tiny_lfb8": lambda: W.lfb(W.tiny(), "lfb8"),
    "tiny_lfb256": lambda: W.lfb(W.tiny(), "lfb256"),
    "shell16_lfb8": lambda: W.lfb(W.shell16(), "lfb8"),
    "shell16_lfb256": lambda: W.lfb(W.shell16(), "lfb256"),
    "tiny_mapped": lambda: mapped(W.tiny()),
    "shell16_mapped": lambda: mapped(W.shell16()),
}


def sig3(x: float) -> float:
    return float(f"{x:.3g}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="+")
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--check", action="store_true",
                    help="keep the frozen alpha; record a longer power iteration beside it")
    args = ap.parse_args()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "alpha.json")
    for name in args.names:
        p = BUILDERS[name]()
        t0 = time.time()
        sigma, hist = oracle.operator_norm(p, iters=args.iters, log=lambda s: print(name, s, flush=True))
        table = json.load(open(path)) if os.path.exists(path) else {}
        if args.check:
            entry = table[name]
            entry.update(sigma_check=sigma, iters_check=args.iters, history_check=hist,
                         alpha_over_sigma_check=entry["alpha"] / sigma,
                         seconds_check=round(time.time() - t0, 1))
        else:
            table[name] = dict(alpha=sig3(ALPHA_REL * sigma), sigma=sigma, alpha_rel=ALPHA_REL,
                               iters=args.iters, history=hist, seconds=round(time.time() - t0, 1),
                               method="oracle.operator_norm (FP64 power iteration on K^H K)")
        with open(path, "w") as f:
            json.dump(table, f, indent=1)
        print(name, "alpha", table[name]["alpha"], "sigma", sigma, flush=True)


if __name__ == "__main__":
    main()
