#!/usr/bin/env python
"""Benchmark of the group-by-group far-zone solver on one workload.

A step is one full GMRES solve of the 16^3 sphere-shell scatterer (1,264 boxes,
40,448 basis unknowns, plane-wave excitation): every GMRES iteration runs the
mapping (Alg. 1), the displacement-grouped translation (Alg. 2), the inverse
mapping (Alg. 3), the stored near product and the Arnoldi/Givens update on the
GPU.  Coupling blocks are generated once per plan (amortised, timed separately).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank solves its own replica (no collective on the
data path; scaling "weak"), timing = max over ranks.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
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
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    return ap.parse_args()


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
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
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
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ reference arm (FP64 CPU oracle)
def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import oracle
    import workloads as W
    p = W.shell16()
    p.alpha = W.alpha_for("shell16")
    c = W.coefficients(p, 1, W.SEED_C["shell16"])
    targets = W.subsample_boxes(p, 8, W.SEED_SUBSAMPLE["shell16"])
    iters = 60        # GMRES(50) iterations to 1e-6 on this workload (GPU plain path measures it)
    oracle.build()
    for _ in range(args.warmup):
        oracle.operator(p, c, "full", targets=targets[:1])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.operator(p, c, "full", targets=targets)
        times.append(time.perf_counter() - t0)
    t_sample = statistics.median(times)
    t_matvec = t_sample * p.n_boxes / len(targets)
    solves_per_s = 1.0 / (iters * t_matvec)
    sample = (f"brute-force FP64 oracle product (near + far, site pair by site pair) on {len(targets)} of "
              f"{p.n_boxes} target boxes, scaled to a full product x {iters} GMRES iterations")
    line = {"impl": "reference", "metric": METRIC, "value": solves_per_s, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / solves_per_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": solves_per_s, "unit": "solves/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": solves_per_s, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    world, rank, local = dist_setup(args)
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2501_04684_gb300 as ie
    import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    p = W.shell16()
    p.alpha = W.alpha_for("shell16")
    precs = [ie.IE_PREC_FP32, ie.IE_PREC_BF16X3, ie.IE_PREC_FP16X3, ie.IE_PREC_BF16X1]
    t0 = time.perf_counter()
    plan = ie.Plan(ie.problem_from(p, ie.precmask(*precs)), stream)
    plan_s = time.perf_counter() - t0
    st = plan.stats
    kh, pol = W.plane_wave_spec(1)
    v = torch.zeros((1, p.n), dtype=torch.complex64, device=dev)
    ie.ie_rhs_plane_wave(plan.handle, kh, pol, v, stream)
    x = torch.zeros_like(v)
    paths = {name: dict(spec, opts=ie.solve_opts(**spec["opts"])) for name, spec in solve_paths(ie).items()}

    def solve_once(path):
        s, info = ie.ie_solve(plan.handle, v, x, 1, path["opts"], stream)
        if s != ie.IE_OK:
            raise RuntimeError(f"solve did not converge: {info}")
        return info

    def time_path(path, steps, clocks=False):
        for _ in range(max(3, args.warmup)):
            solve_once(path)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        infos = []
        barrier(world)
        torch.cuda.synchronize()
        l0 = ie.ie_kernel_launches()
        clk = Clocks(local) if clocks else None
        if clk:
            clk.__enter__()
        try:
            for k in range(steps):
                ev[k][0].record(stream)
                infos.append(solve_once(path))
                ev[k][1].record(stream)
            torch.cuda.synchronize()
        finally:
            if clk:
                clk.__exit__()
        barrier(world)
        lat = [a.elapsed_time(b) for a, b in ev]
        total = max_over_ranks(sum(lat), world)
        return dict(solves_per_s=world * steps / (total / 1e3), ms=total / steps,
                    p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                    iterations=infos[-1]["iterations"], matvecs=infos[-1]["matvecs"],
                    refinements=infos[-1]["refinements"], relres=infos[-1]["relres"],
                    launches=ie.ie_kernel_launches() - l0, clocks=clk.summary() if clk else None)

    # ---- timed region: K solves of the headline path (CUDA events on the solve stream)
    head = time_path(paths[HEADLINE], args.steps, clocks=True)
    others = {name: time_path(path, args.steps) for name, path in paths.items() if name != HEADLINE}

    # ---- far-zone products per precision and the translation kernel's own time
    nfar = max(5, args.steps)
    c = torch.from_numpy(W.coefficients(p, 1, W.SEED_C["shell16"]).astype(np.complex64)).to(dev)
    y = torch.zeros_like(c)
    far = {}
    for prec in precs:
        for _ in range(3):
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, c, y, 1, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nfar):
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, c, y, 1, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        mv_ms = max_over_ranks(e0.elapsed_time(e1), world) / nfar
        ie.ie_plan_profile(plan.handle, True)
        for _ in range(nfar):
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, c, y, 1, stream)
        torch.cuda.synchronize()
        s2 = ie.ie_plan_stats_get(plan.handle)
        ie.ie_plan_profile(plan.handle, False)
        k_ms = s2["translate_ms"] / max(1, s2["translate_launches"])
        far[ie.PREC_NAMES[prec]] = dict(matvecs_per_s=world * 1e3 / mv_ms, ms=mv_ms, translate_kernel_ms=k_ms)

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    vh = v.cpu().pin_memory()
    xh = torch.zeros_like(vh).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        v.copy_(vh, non_blocking=True)
        solve_once(paths[HEADLINE])
        xh.copy_(x, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world)
    e2e = {"value": world * args.steps / (e2e_ms / 1e3), "unit": "solves/s",
           "h2d_bytes_per_step": int(vh.numel() * vh.element_size()),
           "d2h_bytes_per_step": int(xh.numel() * xh.element_size())}

    # ---- roofline of the dominant kernel of the headline path
    pairs = st["n_far_pairs"]
    peaks = measured_peaks()
    tc_flops = 3 * pairs * 8 * 192 * 192                      # three bf16 products per complex MAC term
    tc_ms = far["bf16x3"]["translate_kernel_ms"]
    tc_ach = tc_flops / (tc_ms / 1e3) / 1e12
    roofline = {"bound": "tensor", "achieved": tc_ach, "peak": peaks["bf16"], "unit": "TFLOP/s",
                "frac": tc_ach / peaks["bf16"],
                "traffic": profiled_traffic("translate_tc_bf16x3_shell16.md", "translate_tc.cu"),
                "kernel": "translate_tc_kernel<bf16,x3>", "peak_source": peaks["source"],
                "algorithmic_flops_per_launch": tc_flops,
                "dram_gbs": None}
    if roofline["traffic"]:
        roofline["dram_gbs"] = roofline["traffic"] / (tc_ms / 1e3) / 1e9
    simt_ach = pairs * 8 * 192 * 192 / (far["fp32"]["translate_kernel_ms"] / 1e3) / 1e12
    roofline_fp32 = {"bound": "alu", "achieved": simt_ach, "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": simt_ach / FP32_SIMT_PEAK_TFLOPS, "kernel": "translate_simt_kernel",
                     "traffic": profiled_traffic("translate_simt_fp32_shell16.md", "translate_simt.cu"),
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}

    hp = paths[HEADLINE]
    result = {
        "metric": METRIC, "value": head["solves_per_s"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": hp["dtype"], "data": "synthetic",
        "config": {"workload": WORKLOAD, "path": HEADLINE, "path_desc": hp["desc"], "tol": hp["opts"].tol,
                   "nrhs": 1, "l2": "no flush needed: each product streams >= 4.9 GB of coupling blocks (> 129 MB L2)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "solve": {k: head[k] for k in ("p50_ms", "p99_ms", "iterations", "matvecs", "refinements", "relres")},
        "vs_plain_fp32": head["solves_per_s"] / others["plain"]["solves_per_s"],
        "paths": {name: {k: r[k] for k in ("solves_per_s", "p50_ms", "p99_ms", "iterations", "matvecs", "refinements",
                                           "relres")} | {"desc": paths[name]["desc"]}
                  for name, r in others.items()},
        "far_matvecs": far,
        "plan_seconds": plan_s,
        "gpu_launches": int(head["launches"]),
        "clocks": head["clocks"],
        "e2e": e2e,
        "roofline": roofline,
        "roofline_fp32": roofline_fp32,
    }
    if rank == 0 and world == 1:
        result["cpu_baseline"] = cpu_baseline(p, head["matvecs"])
    plan.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def solve_paths(ie) -> dict:
    """Solve forms measured on the workload; HEADLINE is the value's step."""
    return {
        "mixed": dict(opts=dict(tol=1e-5, restart=50, prec=ie.IE_PREC_BF16X3, refine=1,
                                refine_prec=ie.IE_PREC_FP16X3, inner_tol=1e-3),
                      dtype="bf16x3 tensor products, f32 GMRES, f64 refinement",
                      desc="outer FP64 refinement (residual from FP16X3 products) around GMRES(50) on BF16X3 "
                           "products to 1e-3; stop at 1e-5"),
        "mixed_bf16x1": dict(opts=dict(tol=1e-5, restart=50, prec=ie.IE_PREC_BF16X1, refine=1,
                                       refine_prec=ie.IE_PREC_FP16X3, inner_tol=1e-2),
                             dtype="bf16 tensor products, f32 GMRES, f64 refinement",
                             desc="refinement (FP16X3 residual) around GMRES(50) on single bf16 products to 1e-2"),
        "fp16x3": dict(opts=dict(tol=1e-5, restart=50, prec=ie.IE_PREC_FP16X3), dtype="fp16x3",
                       desc="GMRES(50) on FP16X3 products to 1e-5, no refinement"),
        "plain": dict(opts=dict(tol=1e-6, restart=50, prec=ie.IE_PREC_FP32), dtype="f32",
                      desc="plain FP32 path: GMRES(50) on FP32 SIMT products to 1e-6"),
    }


HEADLINE = "mixed"


def profiled_traffic(summary: str, source: str):
    """DRAM bytes per launch from a committed ncu summary, or None once the kernel source
    has changed since the counters were taken (the summary records the source hash)."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
        src = open(os.path.join(ROOT, "paper_2501_04684_gb300", "csrc", source), "rb").read()
    except OSError:
        return None
    fields = dict(line.split(": ", 1) for line in text.splitlines() if ": " in line and not line.startswith(("|", " ")))
    if fields.get("kernel_source_sha256_16", "").strip() != hashlib.sha256(src).hexdigest()[:16]:
        return None
    try:
        return int(fields["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"bf16": float(d["bf16_tflops"]), "bf16_sustained": float(d["bf16_tflops_sustained"]),
                "hbm": float(d["hbm_gbs"]), "source": "of measured (MEASURED_PEAKS.json, burst bf16)"}
    except (OSError, KeyError, ValueError):
        return {"bf16": 1900.0, "bf16_sustained": 1700.0, "hbm": 6800.0, "source": "of fallback"}


def cpu_baseline(p, iters: int) -> dict:
    """The FP64 oracle as it stands, on a bounded sample of the same workload."""
    import oracle
    import workloads as W
    c = W.coefficients(p, 1, W.SEED_C["shell16"])
    targets = W.subsample_boxes(p, 8, W.SEED_SUBSAMPLE["shell16"])
    oracle.build()
    t0 = time.perf_counter()
    oracle.operator(p, c, "full", targets=targets)
    t = time.perf_counter() - t0
    t_matvec = t * p.n_boxes / len(targets)
    v = 1.0 / (max(1, iters) * t_matvec)
    return {"value": v, "unit": "solves/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"brute-force FP64 product (near + far) on {len(targets)} of {p.n_boxes} target boxes "
                       f"({t:.1f} s), scaled to a full product x {iters} GMRES iterations")}


if __name__ == "__main__":
    main()
