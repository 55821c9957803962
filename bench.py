#!/usr/bin/env python
"""Benchmark of the group-by-group far-zone solver on one workload.

Default (the headline line): the 32^3 sphere-shell scatterer (5,000 boxes, 160,000
basis unknowns, 24.9 M far box pairs, plane-wave excitation).  A step is one full
solve to a relative residual of 1e-5 in the mixed form: GMRES(50) on FP16X3 tensor-
core products inside an outer FP64 refinement loop.  Every GMRES iteration runs the
mapping (Alg. 1), the displacement-grouped translation (Alg. 2), the inverse mapping
(Alg. 3), the stored near product and the Arnoldi/Givens update on the GPU.  The
same solve in plain FP32 (FP32 SIMT products) and the other mixed forms are timed
on the same plan; far-zone products/s per precision, the translation kernel's
roofline, the FP64 CPU oracle on a box subsample and a bounded serving run (config
5) go into the same JSON line.  Coupling blocks are generated once per plan
(amortised, timed separately).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload shell32|shell16|batch64|serve]

N > 1 runs under torchrun: every rank solves its own replica (no collective on the
data path; scaling "weak"), timing = max over ranks.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "far-zone matvecs/s + GMRES solves/s (p50/p99) mixed vs plain FP32, same GB300, err≤1e-5"
WORKLOAD = ("shell16: 16^3 grid of a=lambda/4 boxes, sphere shell r=7 boxes (1,264 boxes, 40,448 basis unknowns, "
            "242,688 dipole unknowns, 1,575,248 far pairs in 16,540 displacement groups), nb=32, "
            "x-polarised plane wave along +z, GMRES(50)")
WORKLOAD32 = ("shell32: 32^3 grid of a=lambda/4 boxes, sphere shell r=14 boxes (5,000 boxes, 160,000 basis unknowns, "
              "960,000 dipole unknowns, 24,910,952 far pairs in 112,160 displacement groups), nb=32, "
              "x-polarised plane wave along +z, GMRES(50), rel. residual 1e-5")
HEAD32 = "mixed_fp16x3"          # the headline path of the shell32 line
CPU_SAMPLE_BOXES = 64            # target boxes of the oracle's timed sample (cpu_baseline)
REF_SAMPLE_BOXES = 8             # target boxes per step of the reference arm
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="shell32", choices=["shell32", "shell16", "batch64", "serve"],
                    help="shell32 is the headline line (with a bounded serving record); the others measure "
                         "the plain-path shell, batching and serving workloads on their own")
    ap.add_argument("--no-serve", action="store_true", help="shell32: leave out the bounded serving record")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="shell32: leave out the translation-network record (shell16, trained networks)")
    ap.add_argument("--lfb", default=None, choices=["lfb8", "lfb256"],
                    help="shell16 only: the same geometry with box edge lambda/8 or lambda/256 "
                         "(low-frequency regime)")
    ap.add_argument("--mapped", action="store_true",
                    help="shell16 only: P built on the GPU by the mapping construction (eq. 11) from seeded "
                         "point-dipole basis functions instead of random")
    ap.add_argument("--symmetry", type=int, default=None, choices=[0, 1],
                    help="1: symmetry-compressed coupling store (one block per sorted |d|); default 1 for shell32 "
                         "(the headline) and serve (one shared store for every request), 0 otherwise")
    ap.add_argument("--requests", type=int, default=12, help="serve: requests per run")
    ap.add_argument("--record-requests", type=int, default=6,
                    help="shell32: requests of the bounded serving record")
    ap.add_argument("--serve-load", type=float, nargs="+", default=[0.5, 0.9],
                    help="serve: offered loads as fractions of the plain form's capacity")
    ap.add_argument("--serve-batch", type=int, default=4, help="serve: most requests merged into one plan")
    ap.add_argument("--serve-workers", type=int, default=4, help="serve: worker threads (streams)")
    args = ap.parse_args()
    if args.symmetry is None:
        args.symmetry = 1 if args.workload in ("shell32", "serve") else 0
    return args


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ distributed
def dist_setup(args, backend: str = "nccl"):
    """One process per GPU from the launcher's environment (replicas: no data collective;
    the process group serves the barriers and the max over ranks only)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, units_per_rank: int, slowest_ms: float) -> float:
    """Whole-job throughput of `world` replicas that each processed `units_per_rank` units,
    timed by the slowest rank."""
    return world * units_per_rank / (slowest_ms / 1e3)


# ------------------------------------------------------------------ reference arm (FP64 CPU oracle)
def shell32_config(symmetry: int = 0, world: int = 1) -> dict:
    """`config` of the headline line, shared by both arms."""
    return {"workload": WORKLOAD32, "path": HEAD32,
            "path_desc": ("outer FP64 refinement (residual r = v - Z x from FP16X3 products, differences and norms "
                          "in FP64) around GMRES(50) on FP16X3 tcgen05 products (fp16 hi+lo split, FP32 "
                          "accumulate, FP32 Krylov vectors, FP64 dots and Givens) to 5e-6; stop at 1e-5"),
            "tol": 1e-5, "nrhs": 1, "symmetry": symmetry,
            "l2": ("no flush needed: each product streams >= 33 GB of coupling images (> 129 MB L2)" if not symmetry
                   else "symmetry-compressed store (2,780 blocks, 820 MB of images per 16-bit store, > 129 MB L2); "
                        "inputs (48 permuted copies) and slabs are rewritten every product"),
            "parallelism": "replicas" if world > 1 else "single"}


def shell16_config(ie, symmetry: int = 0, world: int = 1, workload: str = WORKLOAD) -> dict:
    """`config` of the shell16 line, shared by both arms."""
    hp = solve_paths(ie)[HEADLINE]
    return {"workload": workload, "path": HEADLINE, "path_desc": hp["desc"], "tol": hp["opts"]["tol"],
            "nrhs": 1, "symmetry": symmetry,
            "l2": ("no flush needed: each product streams >= 4.9 GB of coupling blocks (> 129 MB L2)"
                   if not symmetry else
                   "symmetry-compressed store (473 blocks, 139 MB); inputs and slabs are rewritten each product"),
            "parallelism": "replicas" if world > 1 else "single"}


def oracle_sample_time(p, nboxes: int, seed_c: int, seed_sub: int, reps: int = 1):
    """Wall time of the FP64 brute-force oracle product (near + far) on `nboxes` seeded
    target boxes; the median of `reps` runs."""
    import oracle
    import workloads as W
    c = W.coefficients(p, 1, seed_c)
    targets = W.subsample_boxes(p, nboxes, seed_sub)
    oracle.build()
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.operator(p, c, "full", targets=targets)
        times.append(time.perf_counter() - t0)
    return statistics.median(times), len(targets), times


def run_reference(args):
    """The FP64 CPU oracle on the headline workload: every step is the brute-force product
    on REF_SAMPLE_BOXES seeded target boxes (the work that is timed); `value` scales that
    to whole solves (full product x the products of the oracle's own GMRES)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import workloads as W
    name = args.workload if args.workload in ("shell16", "shell32") else "shell32"
    p = W.shell32() if name == "shell32" else W.shell16()
    p.alpha = W.alpha_for(name)
    tol = 1e-5 if name == "shell32" else HEADLINE_TOL
    prods = oracle_products(name, tol)
    if prods is None:
        print(json.dumps({"impl": "reference", "unavailable": f"workloads/oracle_solve.json has no {name} entry "
                                                               f"(run workloads/make_oracle_solve.py {name})"}))
        return
    oracle.build()
    c = W.coefficients(p, 1, W.SEED_C[name])
    targets = W.subsample_boxes(p, REF_SAMPLE_BOXES, W.SEED_SUBSAMPLE[name])
    for _ in range(args.warmup):
        oracle.operator(p, c, "full", targets=targets)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.operator(p, c, "full", targets=targets)
        times.append(time.perf_counter() - t0)
    t_step = statistics.median(times)
    t_solve = t_step * p.n_boxes / len(targets) * prods
    solves_per_s = 1.0 / t_solve
    sample = (f"each step: brute-force FP64 oracle product (near + far, site pair by site pair) on {len(targets)} of "
              f"{p.n_boxes} target boxes ({1e3 * t_step:.0f} ms); value extrapolated: x {p.n_boxes / len(targets):.0f} "
              f"to a full product, x {prods} products (the oracle's own GMRES(50) on this system to {tol:g})")
    if name == "shell32":
        config = shell32_config(args.symmetry, world)
    else:
        import paper_2501_04684_gb300 as ie
        config = shell16_config(ie, args.symmetry, world)
    line = {"impl": "reference", "metric": METRIC, "value": solves_per_s, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "value_basis": "extrapolated from the timed sample steps (ms_per_step is the sample's own time)",
            "extrapolated_solve_s": t_solve,
            "cpu_baseline": {"value": solves_per_s, "unit": "solves/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": solves_per_s, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
class Ctx:
    """Device, stream and bound library shared by the workload runners."""

    def __init__(self, args):
        self.args = args
        self.world, self.rank, self.local = dist_setup(args)
        import numpy as np
        import torch

        import __graft_entry__
        __graft_entry__.build()
        import paper_2501_04684_gb300 as ie
        import workloads as W
        self.np, self.torch, self.ie, self.W = np, torch, ie, W
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        self.stream = torch.cuda.Stream(device=self.dev)
        torch.cuda.set_stream(self.stream)

    def ev(self):
        return self.torch.cuda.Event(enable_timing=True)


def time_solves(ctx, plan, v, x, nrhs, opts, steps, warmup, clocks=False):
    """`steps` solves of one path, CUDA events on the solve stream around each."""
    ie, torch, np = ctx.ie, ctx.torch, ctx.np

    def once():
        s, info = ie.ie_solve(plan.handle, v, x, nrhs, opts, ctx.stream)
        if s != ie.IE_OK:
            raise RuntimeError(f"solve did not converge: {info}")
        return info

    for _ in range(warmup):
        once()
    torch.cuda.synchronize()
    ev = [(ctx.ev(), ctx.ev()) for _ in range(steps)]
    infos = []
    barrier(ctx.world)
    torch.cuda.synchronize()
    l0 = ie.ie_kernel_launches()
    clk = Clocks(ctx.local) if clocks else None
    if clk:
        clk.__enter__()
    try:
        for k in range(steps):
            ev[k][0].record(ctx.stream)
            infos.append(once())
            ev[k][1].record(ctx.stream)
        torch.cuda.synchronize()
    finally:
        if clk:
            clk.__exit__()
    barrier(ctx.world)
    lat = [a.elapsed_time(b) for a, b in ev]
    total = max_over_ranks(sum(lat), ctx.world)
    return dict(solves_per_s=aggregate_rate(ctx.world, steps, total), ms=total / steps, steps=steps,
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                iterations=infos[-1]["iterations"], matvecs=infos[-1]["matvecs"],
                refinements=infos[-1]["refinements"], relres=infos[-1]["relres"],
                launches=ie.ie_kernel_launches() - l0, clocks=clk.summary() if clk else None)


def time_far(ctx, plan, c, nrhs, precs, reps, warmup=3):
    """Far-zone products per precision: whole product (events) and translation kernel
    (events inside the library, on the launching stream)."""
    ie, torch = ctx.ie, ctx.torch
    y = torch.zeros_like(c)
    out = {}
    for prec in precs:
        for _ in range(warmup):
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, c, y, nrhs, ctx.stream)
        torch.cuda.synchronize()
        e0, e1 = ctx.ev(), ctx.ev()
        e0.record(ctx.stream)
        for _ in range(reps):
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, c, y, nrhs, ctx.stream)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        mv_ms = max_over_ranks(e0.elapsed_time(e1), ctx.world) / reps
        ie.ie_plan_profile(plan.handle, True)
        for _ in range(reps):
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, c, y, nrhs, ctx.stream)
        torch.cuda.synchronize()
        s2 = ie.ie_plan_stats_get(plan.handle)
        ie.ie_plan_profile(plan.handle, False)
        k_ms = s2["translate_ms"] / max(1, s2["translate_launches"])
        out[ie.PREC_NAMES[prec]] = dict(matvecs_per_s=aggregate_rate(ctx.world, 1, mv_ms), ms=mv_ms,
                                        translate_kernel_ms=k_ms)
    return out


def tc_roofline(pairs_x_rhs: int, kernel_ms: float, products: int, summary: str | None, kernel: str,
                sustained: bool = False) -> dict:
    """Roofline of a translation launch; sustained = the kernel runs for seconds, so the
    power-capped sustained dense peak is the bound."""
    peaks = measured_peaks()
    flops = products * pairs_x_rhs * 8 * 192 * 192
    ach = flops / (kernel_ms / 1e3) / 1e12
    peak = peaks["bf16_sustained"] if sustained else peaks["bf16"]
    source = peaks["source"].replace("burst", "sustained") if sustained else peaks["source"]
    r = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
         "traffic": profiled_traffic(summary, "translate_tc.cu") if summary else None,
         "kernel": kernel, "peak_source": source, "algorithmic_flops_per_launch": flops, "dram_gbs": None}
    if r["traffic"]:
        r["dram_gbs"] = r["traffic"] / (kernel_ms / 1e3) / 1e9
    return r


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if (args.lfb is not None or args.mapped) and args.workload != "shell16":
        raise SystemExit("--lfb and --mapped apply to the shell16 workload only")
    ctx = Ctx(args)
    runner = {"shell16": run_shell16, "shell32": run_shell32, "batch64": run_batch64, "serve": run_serve}
    result = runner[args.workload](ctx)
    if ctx.rank == 0 and result is not None:
        print(json.dumps(result), flush=True)
    if ctx.world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_shell16(ctx):
    args, ie, W, torch, np = ctx.args, ctx.ie, ctx.W, ctx.torch, ctx.np
    world, stream = ctx.world, ctx.stream
    p = W.shell16() if args.lfb is None else W.lfb(W.shell16(), args.lfb)
    workload = WORKLOAD if args.lfb is None else WORKLOAD.replace("a=lambda/4", f"a=lambda/{round(1 / p.a)}")
    mapping = None
    if args.mapped:
        p, mapping = map_shell(ctx, p)
        workload = workload.replace("basis unknowns", "basis unknowns, P mapped from point-dipole functions")
    p.alpha = W.alpha_for(p.name)
    precs = [ie.IE_PREC_FP32, ie.IE_PREC_BF16X3, ie.IE_PREC_FP16X3, ie.IE_PREC_BF16X1, ie.IE_PREC_FP16X1]
    tc_precs = [ie.IE_PREC_BF16X3, ie.IE_PREC_FP16X3, ie.IE_PREC_BF16X1, ie.IE_PREC_FP16X1]
    t0 = time.perf_counter()
    plan = ie.Plan(ie.problem_from(p, ie.precmask(*precs), symmetry=args.symmetry), stream)
    plan_s = time.perf_counter() - t0
    st = plan.stats
    kh, pol = W.plane_wave_spec(1)
    v = torch.zeros((1, p.n), dtype=torch.complex64, device=ctx.dev)
    ie.ie_rhs_plane_wave(plan.handle, kh, pol, v, stream)
    x = torch.zeros_like(v)
    paths = {name: dict(spec, opts=ie.solve_opts(**spec["opts"])) for name, spec in solve_paths(ie).items()}
    warm = max(3, args.warmup)
    # autotune the tensor-core translation (tile width, item order) once per precision
    tuned = {ie.PREC_NAMES[q]: ie.ie_plan_tune(plan.handle, q, 1, stream) for q in tc_precs}

    # ---- timed region: K solves of the headline path (CUDA events on the solve stream)
    head = time_solves(ctx, plan, v, x, 1, paths[HEADLINE]["opts"], args.steps, warm, clocks=True)
    others = {name: time_solves(ctx, plan, v, x, 1, path["opts"], args.steps, warm)
              for name, path in paths.items() if name != HEADLINE}

    # ---- far-zone products per precision and the translation kernel's own time
    c = torch.from_numpy(W.coefficients(p, 1, W.SEED_C["shell16"]).astype(np.complex64)).to(ctx.dev)
    far = time_far(ctx, plan, c, 1, precs, max(5, args.steps))

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    e2e = time_e2e(ctx, plan, v, x, paths[HEADLINE]["opts"], args.steps)

    # ---- roofline of the dominant kernel of the headline path
    pairs = st["n_far_pairs"]
    roofline = tc_roofline(pairs, far["fp16x3"]["translate_kernel_ms"], 3, None if args.symmetry else "translate_tc_fp16x3_shell16.md",
                           "translate_tc_kernel<fp16,x3>")
    if args.lfb is not None and roofline.get("traffic") is not None:
        roofline["traffic_note"] = ("captured at a=lambda/4: the box edge changes only the values, not the "
                                    "work list or the bytes moved")
    simt_ach = pairs * 8 * 192 * 192 / (far["fp32"]["translate_kernel_ms"] / 1e3) / 1e12
    roofline_fp32 = {"bound": "alu", "achieved": simt_ach, "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": simt_ach / FP32_SIMT_PEAK_TFLOPS, "kernel": "translate_simt_kernel",
                     "traffic": None,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}

    hp = paths[HEADLINE]
    result = {
        "metric": METRIC, "value": head["solves_per_s"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": hp["dtype"], "data": "synthetic",
        "config": shell16_config(ie, args.symmetry, world, workload),
        "solve": {k: head[k] for k in ("p50_ms", "p99_ms", "iterations", "matvecs", "refinements", "relres")},
        "vs_plain_fp32": head["solves_per_s"] / others["plain"]["solves_per_s"],
        "paths": {name: {k: r[k] for k in ("solves_per_s", "p50_ms", "p99_ms", "iterations", "matvecs", "refinements",
                                           "relres")} | {"desc": paths[name]["desc"]}
                  for name, r in others.items()},
        "far_matvecs": far,
        "tuned": tuned,
        "plan_seconds": plan_s,
        "gpu_launches": int(head["launches"]),
        "clocks": head["clocks"],
        "e2e": e2e,
        "roofline": roofline,
        "roofline_fp32": roofline_fp32,
    }
    plan.close()
    if not args.no_surrogate and args.lfb is None and not args.mapped:
        result["surrogate"] = surrogate_record(ctx)
    if mapping is not None:
        result["mapping"] = mapping
    if ctx.rank == 0 and world == 1:
        result["cpu_baseline"] = cpu_baseline(p, "shell16", oracle_products(p.name, HEADLINE_TOL) or head["matvecs"],
                                              "the oracle's own GMRES(50) to the same tolerance")
    return result


def map_shell(ctx, p):
    """P of the shell from seeded point-dipole functions by ie_map_basis (host in, host out,
    timed with the copies), and the map kernel's FP64 roofline."""
    import dataclasses
    ie, W, np = ctx.ie, ctx.W, ctx.np
    fun_off, pos, mom = W.point_dipole_basis(p.nb, W.SEED_MAPPED["shell16"], a=p.a)
    t = W.MAPPED_TIKHONOV
    ie.ie_map_basis(p.k, p.eta, p.a, fun_off[:9], pos, mom, tikhonov=t, stream=ctx.stream)          # warm-up
    times = []
    for _ in range(3):
        t0 = time.perf_counter()
        P, res = ie.ie_map_basis(p.k, p.eta, p.a, fun_off, pos, mom, tikhonov=t, stream=ctx.stream)
        times.append(time.perf_counter() - t0)
    n_fun = len(fun_off) - 1
    t_call = sorted(times)[1]
    # algorithmic FP64 work per function: C = A^+ B (192 x 384 complex MACs) and the
    # residual A C - B (the same), 8 real flops per complex MAC
    flops = n_fun * 2 * 192 * 384 * 8
    ach = flops / t_call / 1e12
    q = dataclasses.replace(p, P=P, name=p.name + "_mapped")
    return q, {"functions": n_fun, "dipoles": int(fun_off[-1]), "tikhonov": t, "ms": t_call * 1e3,
               "functions_per_s": n_fun / t_call,
               "residual_on_S_max": float(res.max()), "residual_on_S_median": float(np.median(res)),
               "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                            "note": "whole call: host copies of 124 MB of P and the one-off QR included"}}


def shell32_paths(ie) -> dict:
    """Solve forms of the headline line (all to a relative residual of 1e-5); HEAD32 is
    the value's step, "plain" the FP32 comparison."""
    return {
        "mixed_fp16x3": dict(opts=ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X3, refine=1,
                                                refine_prec=ie.IE_PREC_FP16X3, inner_tol=5e-6),
                             dtype="fp16x3 tensor products (fp16 hi+lo split, f32 accumulate), f32 GMRES, f64 "
                                   "refinement residual"),
        "fp16x3_gmres": dict(opts=ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X3),
                             dtype="fp16x3 tensor products, f32 GMRES (residual recomputed with fp16x3 products at "
                                   "each restart)"),
        "mixed_bf16x3": dict(opts=ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_BF16X3, refine=1,
                                                refine_prec=ie.IE_PREC_FP16X3, inner_tol=1e-3),
                             dtype="bf16x3 inner GMRES to 1e-3, f64 refinement on fp16x3 residuals"),
        "mixed_fp16x1": dict(opts=ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X1, refine=1,
                                                refine_prec=ie.IE_PREC_FP16X3, inner_tol=1e-3),
                             dtype="single fp16 products in the inner GMRES to 1e-3, f64 refinement on fp16x3 "
                                   "residuals"),
        "plain": dict(opts=ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP32),
                      dtype="f32 (FP32 SIMT products, f32 GMRES, f64 dots)"),
    }


def run_shell32(ctx):
    """Headline: the 32^3 shell (5,000 boxes) solved to 1e-5 in the mixed form and in
    plain FP32 on one plan; far products per precision; roofline; oracle sample; a
    bounded serving record."""
    args, ie, W, torch, np = ctx.args, ctx.ie, ctx.W, ctx.torch, ctx.np
    world, stream = ctx.world, ctx.stream
    p = W.shell32()
    p.alpha = W.alpha_for("shell32")
    precs = [ie.IE_PREC_FP32, ie.IE_PREC_BF16X3, ie.IE_PREC_FP16X3, ie.IE_PREC_BF16X1, ie.IE_PREC_FP16X1]
    t0 = time.perf_counter()
    plan = ie.Plan(ie.problem_from(p, ie.precmask(*precs), symmetry=args.symmetry), stream)
    plan_s = time.perf_counter() - t0
    st = plan.stats
    kh, pol = W.plane_wave_spec(1)
    v = torch.zeros((1, p.n), dtype=torch.complex64, device=ctx.dev)
    ie.ie_rhs_plane_wave(plan.handle, kh, pol, v, stream)
    x = torch.zeros_like(v)
    tuned = {ie.PREC_NAMES[q]: ie.ie_plan_tune(plan.handle, q, 1, stream) for q in precs if q != ie.IE_PREC_FP32}
    paths = shell32_paths(ie)
    warm = max(3, args.warmup)
    # ---- timed region: K solves of the headline path (CUDA events on the solve stream)
    head = time_solves(ctx, plan, v, x, 1, paths[HEAD32]["opts"], args.steps, warm, clocks=True)
    # the comparison forms: the plain path with the same K, the others with at most 5 steps
    others = {}
    for name, path in paths.items():
        if name == HEAD32:
            continue
        k = args.steps if name == "plain" else min(args.steps, 5)
        others[name] = time_solves(ctx, plan, v, x, 1, path["opts"], k, 1 if name == "plain" else 2)
    # ---- far-zone products per precision and the translation kernel's own time
    c = torch.from_numpy(W.coefficients(p, 1, W.SEED_C["shell32"]).astype(np.complex64)).to(ctx.dev)
    far = time_far(ctx, plan, c, 1, precs, max(3, min(args.steps, 10)))
    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    e2e = time_e2e(ctx, plan, v, x, paths[HEAD32]["opts"], args.steps)
    pairs = st["n_far_pairs"]
    roofline = tc_roofline(pairs, far["fp16x3"]["translate_kernel_ms"], 3,
                           "translate_tc_fp16x3_shell32_sym.md" if args.symmetry else "translate_tc_fp16x3_shell32.md",
                           "translate_tc_kernel<fp16,x3>")
    simt_ach = pairs * 8 * 192 * 192 / (far["fp32"]["translate_kernel_ms"] / 1e3) / 1e12
    roofline_fp32 = {"bound": "alu", "achieved": simt_ach, "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": simt_ach / FP32_SIMT_PEAK_TFLOPS, "kernel": "translate_simt_kernel",
                     "traffic": profiled_traffic("translate_simt_fp32_shell32_sym.md" if args.symmetry
                                                 else "translate_simt_fp32_shell32.md", "translate_simt.cu"),
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    keys = ("solves_per_s", "p50_ms", "p99_ms", "iterations", "matvecs", "refinements", "relres")
    result = {
        "metric": METRIC, "value": head["solves_per_s"], "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": warm, "ms_per_step": head["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": paths[HEAD32]["dtype"], "data": "synthetic",
        "config": shell32_config(args.symmetry, world),
        "solve": {k: head[k] for k in keys if k != "solves_per_s"},
        "vs_plain_fp32": head["solves_per_s"] / others["plain"]["solves_per_s"],
        "paths": {name: {k: r[k] for k in keys} | {"dtype": paths[name]["dtype"], "steps": r["steps"]}
                  for name, r in others.items()},
        "far_matvecs": far,
        "far_vs_plain_fp32": {q: far[q]["matvecs_per_s"] / far["fp32"]["matvecs_per_s"] for q in far},
        "tuned": tuned, "plan_seconds": plan_s, "device_bytes": st["device_bytes"],
        "gpu_launches": int(head["launches"]), "clocks": head["clocks"],
        "e2e": e2e, "roofline": roofline, "roofline_fp32": roofline_fp32,
    }
    plan.close()
    del v, x, c
    torch.cuda.empty_cache()
    if ctx.rank == 0 and world == 1:
        prods = oracle_products("shell32", 1e-5)
        basis = "the oracle's own GMRES(50) on this system to 1e-5"
        if prods is None:
            prods, basis = others["plain"]["matvecs"], "the plain FP32 GPU solve's products (no oracle record)"
        result["cpu_baseline"] = cpu_baseline(p, "shell32", prods, basis)
    if not args.no_serve:
        result["serve"] = serve_record(ctx)
    if not args.no_surrogate:
        result["surrogate"] = surrogate_record(ctx)
    return result


def surrogate_one(ctx, symmetry: int, solves_too: bool) -> dict:
    """Translation networks of §3 on shell16 in one store mode: trained on the GPU (first
    stage, e^u < 1e-3), then far products with the networks on the tensor cores and in FP32
    beside the FP16X3 block product on the same plan, their distance from it, and (solves_too)
    a refined solve to 1e-5 whose inner GMRES runs on the tensor-core networks."""
    args, ie, W, torch, np = ctx.args, ctx.ie, ctx.W, ctx.torch, ctx.np
    p = W.shell16()
    p.alpha = W.alpha_for("shell16")
    precs = [ie.IE_PREC_FP16X3, ie.IE_PREC_CVFCNN, ie.IE_PREC_CVFCNN_FP32]
    t0 = time.perf_counter()
    plan = ie.Plan(ie.problem_from(p, ie.precmask(*precs), symmetry=symmetry), ctx.stream)
    plan_s = time.perf_counter() - t0
    st = plan.stats
    info = ie.ie_cvfcnn_train(plan.handle, None, ctx.stream)
    c = torch.from_numpy(W.coefficients(p, 1, W.SEED_C["shell16"]).astype(np.complex64)).to(ctx.dev)
    far = time_far(ctx, plan, c, 1, precs, 10)
    ys = {}
    for q in precs:
        y = torch.zeros_like(c)
        ie.ie_matvec(plan.handle, ie.IE_FAR, q, c, y, 1, ctx.stream)
        ys[ie.PREC_NAMES[q]] = y
    torch.cuda.synchronize()
    rel = lambda a, b: float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))  # noqa: E731
    kh, pol = W.plane_wave_spec(1)
    v = torch.zeros((1, p.n), dtype=torch.complex64, device=ctx.dev)
    ie.ie_rhs_plane_wave(plan.handle, kh, pol, v, ctx.stream)
    x = torch.zeros_like(v)
    opts_net = ie.solve_opts(tol=1e-5, restart=50, prec=ie.IE_PREC_CVFCNN, refine=1, refine_prec=ie.IE_PREC_FP16X3,
                             inner_tol=1e-3)
    opts_blk = ie.solve_opts(tol=1e-5, restart=50, prec=ie.IE_PREC_FP16X3)
    keys = ("solves_per_s", "p50_ms", "iterations", "matvecs", "refinements", "relres")
    solves = ({"cvfcnn_refined": time_solves(ctx, plan, v, x, 1, opts_net, 3, 1),
               "fp16x3": time_solves(ctx, plan, v, x, 1, opts_blk, 3, 1)} if solves_too else {})
    H = st["cvfcnn_hidden"]
    pairs = st["n_far_pairs"]
    peaks = measured_peaks()
    # algorithmic work: 2 x 192 x H complex multiply-adds (8 real flops each) per pair
    ach = pairs * 8 * 2 * 192 * H / (far["cvfcnn"]["translate_kernel_ms"] / 1e3) / 1e12
    ach32 = pairs * 8 * 2 * 192 * H / (far["cvfcnn_fp32"]["translate_kernel_ms"] / 1e3) / 1e12
    out = {
        "workload": ("shell16 (1,264 boxes, 1,575,248 far pairs), " +
                     ("symmetry-compressed store: one network per canonical displacement"
                      if symmetry else "full store: the canonical networks turned into every displacement's frame") +
                     f" ({st['n_coupling_blocks']} stored), H = {H}"),
        "plan_seconds": plan_s,
        "training": {k: info[k] for k in ("networks", "converged", "eu_max", "eu_mean", "steps_max", "seconds")},
        "far_matvecs": far,
        "network_vs_block": {"cvfcnn": rel(ys["cvfcnn"], ys["fp16x3"]),
                             "cvfcnn_fp32": rel(ys["cvfcnn_fp32"], ys["fp16x3"]),
                             "cvfcnn_vs_cvfcnn_fp32": rel(ys["cvfcnn"], ys["cvfcnn_fp32"])},
        "kernel_vs_fp16x3_block": far["fp16x3"]["translate_kernel_ms"] / far["cvfcnn"]["translate_kernel_ms"],
        "solves": {name: {k: r[k] for k in keys} for name, r in solves.items()},
        "roofline_fp32": {"bound": "alu", "achieved": ach32, "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
                          "frac": ach32 / FP32_SIMT_PEAK_TFLOPS, "kernel": "cvfcnn_translate_kernel",
                          "traffic": None,
                          "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peaks["bf16"], "unit": "TFLOP/s",
                     "frac": ach / peaks["bf16"], "kernel": "cvfcnn_tc_kernel",
                     "traffic": None if symmetry else profiled_traffic("cvfcnn_tc_shell16.md", "cvfcnn_tc.cu"),
                     "peak_source": peaks["source"] + " (fp16 runs at the bf16 rate)",
                     "algorithmic_flops_per_launch": pairs * 8 * 2 * 192 * H},
    }
    plan.close()
    del v, x, c, ys
    torch.cuda.empty_cache()
    return out


def surrogate_record(ctx) -> dict:
    """The networks' record in both store modes (each trains its canonical networks): the
    full store, where each displacement has its own network and block, and the symmetric
    store, where items of the block product pack the groups of one stored block."""
    full = surrogate_one(ctx, 0, False)
    sym = surrogate_one(ctx, 1, True)
    return {"full_store": full, "symmetric_store": sym,
            "kernel_vs_fp16x3_block": {"full_store": full["kernel_vs_fp16x3_block"],
                                       "symmetric_store": sym["kernel_vs_fp16x3_block"]}}


def time_e2e(ctx, plan, v, x, opts, steps):
    """The headline solve through the C ABI with the right-hand side copied in from
    pinned host memory and the solution copied back, inside the timed region."""
    ie, torch = ctx.ie, ctx.torch
    vh = v.cpu().pin_memory()
    xh = torch.zeros_like(vh).pin_memory()
    e0, e1 = ctx.ev(), ctx.ev()
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    for _ in range(steps):
        v.copy_(vh, non_blocking=True)
        s, info = ie.ie_solve(plan.handle, v, x, 1, opts, ctx.stream)
        if s != ie.IE_OK:
            raise RuntimeError(f"solve did not converge: {info}")
        xh.copy_(x, non_blocking=True)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), ctx.world)
    return {"value": aggregate_rate(ctx.world, steps, ms), "unit": "solves/s",
            "h2d_bytes_per_step": int(vh.numel() * vh.element_size()),
            "d2h_bytes_per_step": int(xh.numel() * xh.element_size())}


def run_batch64(ctx):
    """Batching workload: 64 scatterers in one plan, every kernel one launch over all
    of them; far products per precision and one mixed solve of the whole batch."""
    args, ie, W, torch, np = ctx.args, ctx.ie, ctx.W, ctx.torch, ctx.np
    b = W.batch64()
    R = b.max_rhs
    def far_pairs(m):   # ordered pairs at Chebyshev distance >= 2 = all pairs minus the 27-cell stencil's
        cells = set(map(tuple, m.box_ijk.tolist()))
        near = sum((x + dx, y + dy, z + dz) in cells for (x, y, z) in cells
                   for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1))
        return m.n_boxes ** 2 - near
    pair_rhs = sum(far_pairs(m) * q for m, q in zip(b.members, b.nrhs))   # far (pair, own rhs) columns
    precs = [ie.IE_PREC_FP16X1, ie.IE_PREC_FP16X3]
    t0 = time.perf_counter()
    plan = ie.Plan(ie.problem_from_batch(b, ie.precmask(*precs), symmetry=args.symmetry, exact_rhs=True), ctx.stream)
    plan_s = time.perf_counter() - t0
    st = plan.stats
    kh, pol = b.padded_waves()
    v = torch.zeros((R, b.n), dtype=torch.complex64, device=ctx.dev)
    ie.ie_rhs_plane_wave(plan.handle, kh, pol, v, ctx.stream)
    x = torch.zeros_like(v)
    tuned = {"fp16x3": ie.ie_plan_tune(plan.handle, ie.IE_PREC_FP16X3, R, ctx.stream)}   # the solve's precision
    opts = ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X3)
    solve = time_solves(ctx, plan, v, x, R, opts, max(1, args.steps), args.warmup, clocks=True)
    c = torch.from_numpy(np.concatenate([W.coefficients(m, R, 500 + g) for g, m in enumerate(b.members)],
                                        axis=1).astype(np.complex64)).to(ctx.dev)
    far = time_far(ctx, plan, c, R, precs, 1, warmup=1)
    mixed_bytes = st["device_bytes"]
    plan.close()
    del v, x
    torch.cuda.empty_cache()
    # the plain FP32 product on its own plan (one FP32 store)
    t0 = time.perf_counter()
    plan32 = ie.Plan(ie.problem_from_batch(b, ie.precmask(ie.IE_PREC_FP32), symmetry=args.symmetry, exact_rhs=True),
                     ctx.stream)
    plan32_s = time.perf_counter() - t0
    far |= time_far(ctx, plan32, c, R, [ie.IE_PREC_FP32], 1, warmup=1)
    plan32.close()
    out = {
        "metric": METRIC, "value": solve["solves_per_s"] * b.n_groups, "unit": "scatterer solves/s",
        "n_gpus": ctx.world, "steps": max(1, args.steps), "warmup": args.warmup, "ms_per_step": solve["ms"],
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp16x3 tensor products, f32 GMRES",
        "data": "synthetic",
        "config": {"workload": (f"batch64: 64 scatterers (sphere/cube/ellipsoid shells r=3..14 on 32^3, nb 16..64, "
                                f"1..8 plane waves; seed 41): {st['n_boxes']} boxes, {b.n} basis unknowns, "
                                f"{st['n_far_pairs']} far pairs in {st['n_far_disp']} displacement groups, "
                                f"{sum(b.nrhs)} right-hand sides in {R} columns, each scatterer translating "
                                f"only its own"),
                   "tol": 1e-5},
        "solve": {k: solve[k] for k in ("ms", "iterations", "matvecs", "refinements", "relres")},
        "far_matvecs": far, "tuned": tuned, "plan_seconds": plan_s, "plan_fp32_seconds": plan32_s,
        "device_bytes": mixed_bytes,
        "far_pair_rhs": pair_rhs,
        "gpu_launches": int(solve["launches"]), "clocks": solve["clocks"],
        "roofline": tc_roofline(pair_rhs, far["fp16x3"]["translate_kernel_ms"], 3, None,
                                "translate_tc_kernel<fp16,x3>", sustained=True),
    }
    return out


def serve_setup(ctx, count: int):
    """The seeded serving requests (Poisson arrivals at 1 Hz, seed 51) and their problems."""
    W = ctx.W
    reqs = W.serve_requests(count=count, rate_hz=1.0)
    problems = []
    for r in reqs:
        nb = r["nb"]
        problems.append(W.Problem(name=f"req{len(problems)}", G=r["G"], box_ijk=r["box_ijk"], nb=nb,
                                  P=W.random_P(W.rng(r["seed_P"]), nb), alpha=W.batch_alpha(nb)))
    return reqs, problems


def serve_forms(ie) -> dict:
    return {
        "mixed": ([ie.IE_PREC_FP16X3], ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X3)),
        "plain": ([ie.IE_PREC_FP32], ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP32)),
    }


def serve_run(ctx, reqs, problems, form, rate, batch, budget, symmetry, foot):
    """One serving run: the seeded arrivals replayed at `rate` (x the 1 Hz process), every
    request solved to 1e-5 in `form`; latency from submission to completion."""
    ie, np = ctx.ie, ctx.np
    from paper_2501_04684_gb300 import serve as S
    precs, opts = serve_forms(ie)[form]
    srv = S.Server(precs, opts, budget, workers=ctx.args.serve_workers, batch=batch, symmetry=symmetry)
    srv.prepare_stores(problems)        # shared coupling-block stores: server state, made before the clock
    gaps = np.diff([0.0] + [q["t_arrival"] for q in reqs])
    todo = [S.Request(rid=i, problem=pr, khat=q["khat"], pol=q["pol"]) for i, (q, pr) in
            enumerate(zip(reqs, problems))]
    for r in todo:          # footprints are part of the request's description: taken before the clock
        key = (form, r.rid)
        if key not in foot:
            foot[key] = srv.footprint_of(r, 4)
        r.footprint = foot[key]
    try:
        t_begin = time.perf_counter()
        for i, r in enumerate(todo):
            time.sleep(max(0.0, gaps[i] / rate))
            srv.submit(r)
        done = srv.drain(len(reqs))
        wall = time.perf_counter() - t_begin
    finally:
        srv.close()
    bad = [r for r in done if r.status != ie.IE_OK]
    lat = [r.latency for r in done if r.status == ie.IE_OK]
    pc = S.percentiles(lat)
    return {"rate_hz": rate, "batch": batch, "completed": len(lat), "failed": len(bad),
            "errors": sorted({r.error or ie.lib().ie_status_str(r.status).decode() for r in bad})[:3],
            "solves_per_s": len(lat) / wall, "p50_s": pc["p50"], "p99_s": pc["p99"],
            "mean_service_s": float(np.mean([r.t_done - r.t_start for r in done])),
            "peak_device_bytes": srv.peak_used, "wall_s": wall,
            "mode": "stepped" if srv.stepped else "blocking", "max_live_solves": srv.max_live,
            "shared_store_bytes": srv.store_bytes}


def serve_record(ctx):
    """Bounded serving record of the headline line (config 5): the first
    --record-requests seeded Poisson arrivals, replayed back to back (capacity) in the mixed
    and the plain form, then at --serve-load[-1] x the plain capacity."""
    args, torch = ctx.args, ctx.torch
    reqs, problems = serve_setup(ctx, args.record_requests)
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.9)
    foot = {}
    sym = 1
    cap = {form: serve_run(ctx, reqs, problems, form, 1e9, 1, budget, sym, foot) for form in ("mixed", "plain")}
    load = args.serve_load[-1]
    rate = load * cap["plain"]["solves_per_s"] / max(1e-9, len(reqs) / max(1e-9, reqs[-1]["t_arrival"]))
    loaded = {form: serve_run(ctx, reqs, problems, form, rate, 1, budget, sym, foot) for form in ("mixed", "plain")}
    return {"workload": (f"{len(reqs)} Poisson arrivals (seed 51) of sphere-shell scatterers of 200..20,000 boxes "
                         f"(log-uniform), nb=32, 1..4 plane waves each, tol 1e-5; plans attached to one shared "
                         f"symmetry-compressed coupling store made before the clock; solves stepped one GMRES(50) "
                         f"cycle at a time on 4 streams"),
            "capacity_solves_per_s": {f: cap[f]["solves_per_s"] for f in cap},
            "load_x_plain_capacity": load,
            "p50_s": {f: loaded[f]["p50_s"] for f in loaded}, "p99_s": {f: loaded[f]["p99_s"] for f in loaded},
            "solves_per_s": {f: loaded[f]["solves_per_s"] for f in loaded},
            "runs": {"capacity": cap, "loaded": loaded}}


def run_serve(ctx):
    """Serving workload: Poisson arrivals of scattering solves (200..20,000 boxes log-
    uniform, 1..4 plane waves), admitted by device footprint; p50/p99 from arrival to
    completion for the mixed and the plain FP32 forms."""
    args, ie, torch = ctx.args, ctx.ie, ctx.torch
    reqs, problems = serve_setup(ctx, args.requests)
    free, total = torch.cuda.mem_get_info()
    budget = int(free * 0.9)
    forms = serve_forms(ie)
    foot = {}

    def run(form, rate, batch):
        return serve_run(ctx, reqs, problems, form, rate, batch, budget, args.symmetry, foot)

    # capacity: requests back to back (every arrival at once); the offered loads are
    # fractions of the plain form's capacity and both forms see the same arrivals
    cap = {form: run(form, 1e9, 1) for form in forms}
    base = cap["plain"]["solves_per_s"]
    out_forms = {form: [cap[form] | {"load": None}] for form in forms}
    for frac in args.serve_load:
        for form in forms:
            out_forms[form].append(run(form, frac * base, 1) | {"load": frac})
            if args.serve_batch > 1:
                out_forms[form].append(run(form, frac * base, args.serve_batch) | {"load": frac})
    head = [r for r in out_forms["mixed"] if r["load"] == args.serve_load[-1] and r["batch"] == 1][0]
    plain_same = [r for r in out_forms["plain"] if r["load"] == args.serve_load[-1] and r["batch"] == 1][0]
    return {
        "metric": METRIC, "value": head["solves_per_s"], "unit": "solves/s", "n_gpus": ctx.world,
        "steps": len(reqs), "warmup": 0, "ms_per_step": 1e3 / max(head["solves_per_s"], 1e-12),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp16x3 tensor products, f32 GMRES", "data": "synthetic",
        "config": {"workload": (f"serve: {len(reqs)} Poisson arrivals (seed 51), sphere shells of 200..20,000 "
                                f"boxes (log-uniform), nb=32, 1..4 plane waves, tol 1e-5; HBM budget "
                                f"{budget / 1e9:.0f} GB; offered loads x plain capacity {args.serve_load}"),
                   "symmetry": args.symmetry},
        "p50_s": head["p50_s"], "p99_s": head["p99_s"],
        "plain_p50_s": plain_same["p50_s"], "plain_p99_s": plain_same["p99_s"],
        "capacity_solves_per_s": {form: cap[form]["solves_per_s"] for form in forms},
        "forms": out_forms,
    }


def solve_paths(ie) -> dict:
    """Solve forms measured on the workload; HEADLINE is the value's step."""
    return {
        "fp16x3": dict(opts=dict(tol=1e-5, restart=50, prec=ie.IE_PREC_FP16X3),
                       dtype="fp16x3 tensor products (fp16 hi+lo split, f32 accumulate), f32 GMRES, f64 dots",
                       desc="GMRES(50) on FP16X3 tcgen05 products to 1e-5 (true residual checked against the FP64 "
                            "oracle in the tests)"),
        "mixed_refine": dict(opts=dict(tol=1e-5, restart=50, prec=ie.IE_PREC_BF16X3, refine=1,
                                       refine_prec=ie.IE_PREC_FP16X3, inner_tol=1e-3),
                             dtype="bf16x3 tensor products, f32 GMRES, f64 refinement",
                             desc="outer FP64 refinement (residual from FP16X3 products) around GMRES(50) on BF16X3 "
                                  "products to 1e-3; stop at 1e-5"),
        "mixed_fp16x1": dict(opts=dict(tol=1e-5, restart=50, prec=ie.IE_PREC_FP16X1, refine=1,
                                       refine_prec=ie.IE_PREC_FP16X3, inner_tol=1e-3),
                             dtype="fp16 tensor products, f32 GMRES, f64 refinement",
                             desc="refinement (FP16X3 residual) around GMRES(50) on single fp16 products to 1e-3"),
        "plain": dict(opts=dict(tol=1e-6, restart=50, prec=ie.IE_PREC_FP32), dtype="f32",
                      desc="plain FP32 path: GMRES(50) on FP32 SIMT products to 1e-6"),
    }


FP64_PEAK_TFLOPS = 1.25    # GB300 FP64 rate (non-tensor); far below its FP32 and tensor rates
HEADLINE = "fp16x3"
HEADLINE_TOL = 1e-5


def source_digest(*sources: str) -> str:
    """sha256 (16 hex digits) of kernel code with // comments and blank lines removed, so
    that editing comments keeps a profile valid while any code change voids it.  A source
    "file.cu:signature" stands for the one function of file.cu that starts with signature."""
    import hashlib
    import re
    lines = []
    for source in sources:
        name, _, sig = source.partition(":")
        text = open(os.path.join(ROOT, "paper_2501_04684_gb300", "csrc", name)).read()
        if sig:
            i = text.index(sig)
            text = text[i:text.index("\n}\n", i) + 3]
        lines += [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln.strip()).encode()).hexdigest()[:16]


def profiled_traffic(summary: str, *sources: str):
    """DRAM bytes per launch from a committed ncu summary, or None once the kernel code
    (its source and the work-list builder, api.cu's work_list) has changed since the
    counters were taken (the summary records the code digest)."""
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
        digest = source_digest(*sources, "api.cu:ie_status work_list(")
    except OSError:
        return None
    fields = dict(line.split(": ", 1) for line in text.splitlines() if ": " in line and not line.startswith(("|", " ")))
    if fields.get("kernel_code_sha256_16", "").strip() != digest:
        return None
    try:
        return int(fields["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def oracle_products(name: str, tol: float):
    """Products the oracle's own GMRES needs to reach `tol` on a workload's plane-wave
    system (recorded by workloads/make_oracle_solve.py); None when not recorded."""
    try:
        table = json.load(open(os.path.join(ROOT, "workloads", "oracle_solve.json")))
    except (OSError, ValueError):
        return None
    for key, e in table.items():
        if key.split("@")[0] == name and float(key.split("@")[1]) <= tol:
            hist = e["history"]
            return next((k for k, h in enumerate(hist) if h <= tol), e["products"])
    return None


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"bf16": float(d["bf16_tflops"]), "bf16_sustained": float(d["bf16_tflops_sustained"]),
                "hbm": float(d["hbm_gbs"]), "source": "of measured (MEASURED_PEAKS.json, burst bf16)"}
    except (OSError, KeyError, ValueError):
        return {"bf16": 1900.0, "bf16_sustained": 1700.0, "hbm": 6800.0, "source": "of fallback"}


def cpu_baseline(p, name: str, products: int, basis: str, boxes: int | None = None) -> dict:
    """The FP64 oracle as it stands, on a bounded sample of the same workload: the brute-
    force product on a seeded subsample of target boxes, timed, then scaled to a solve."""
    import oracle
    import workloads as W
    boxes = boxes or (CPU_SAMPLE_BOXES if name == "shell32" else 8)
    t, nt, _ = oracle_sample_time(p, boxes, W.SEED_C[name], W.SEED_SUBSAMPLE[name])
    t_matvec = t * p.n_boxes / nt
    v = 1.0 / (max(1, products) * t_matvec)
    return {"value": v, "unit": "solves/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"brute-force FP64 product (near + far) on {nt} of {p.n_boxes} target boxes ({t:.1f} s), "
                       f"extrapolated to a full product x {products} products ({basis})")}


if __name__ == "__main__":
    main()
