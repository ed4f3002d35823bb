#!/usr/bin/env python
"""Benchmark: time-to-1e-6 of the CSLP-preconditioned matrix-free Helmholtz solve on one GB300.

Workload (one step = one full solve, the whole hot path): the three-layer wedge model on the
unit cube, n = 128 intervals per direction (129^3 = 2,146,689 unknowns, Sommerfeld on every
face), max k h = 0.625, point source at the top-face centre, complex128 throughout:
right-preconditioned GMRES(30) with one CSLP V-cycle per step, to ||b - A x|| / ||b|| <= 1e-6.

Printed (one JSON line on rank 0): value = device time per solve (ms), the dominant kernel's
roofline from live CUDA-event timings inside the timed region, the end-to-end time through the
C ABI with host buffers, the FP64 CPU oracle timed on a bounded sample, clocks sampled during
the timed region, and variants (mixed precision; n = 256) when --variants is on.

--impl reference times the FP64 CPU oracle (the reference arm) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-6 solve & stencil HBM GB/s at 1 GB300: FP64 vs mixed vs batched"
UNIT = "ms"
# FP64 peak derived from the nominal 1.25 TFLOP/s at 2070 MHz on 152 SMs: 2 FP64 FMA per SM
# per clock, so 152 * 2 * 2 flop * 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
SAMPLE_STEPS = 30  # Arnoldi steps in the oracle sample (one GMRES(30) restart cycle)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=128, help="intervals per direction of the wedge workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", type=int, default=2,
                    help="0: headline only; 1: + precision, Krylov and cycle variants at n = 128 and 256; "
                         "2: + batched and adjoint workloads; 3: + the CSLP shift sweep (beta2 x V/F-cycle)")
    ap.add_argument("--orth", choices=["fp64", "df"], default="fp64",
                    help="Gram-Schmidt arithmetic: native FP64 or double-float FP32 pairs")
    ap.add_argument("--reorth", choices=["selective", "always"], default="selective",
                    help="second Gram-Schmidt pass on every step, or only when the first pass lost half of |w|")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="fp64: complex128 throughout (the benchmark); mixed: complex64 cycle under FP64 FGMRES(30)")
    ap.add_argument("--cycle", choices=["v", "f"], default="v", help="multigrid cycle of the preconditioner")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-kernel timed leg")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.f = open(self.path, "w")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# CPU oracle sample (runs in a child process so its OpenMP runtime stays apart from torch)
# ------------------------------------------------------------------------------------------
ORACLE_CHILD = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import oracle
from paper_2308_06085_gb300 import inputs as I
w = I.workload("wedge", {n})
o = oracle.Solver(w["n"], w["h"], oracle.SOMMERFELD, w["k2"])
b = oracle.rhs_point(o.shape, oracle.SOMMERFELD, w["h"], w["sources"])
out = {{}}
if {full}:
    t = time.perf_counter(); r = o.gmres(b, restart=30, tol=1e-6); out["full_ms"] = 1e3 * (time.perf_counter() - t)
    out["full_iters"] = r["iters"]
ts = []
for _ in range({reps}):
    t = time.perf_counter(); o.gmres(b, restart=30, tol=1e-6, max_iter={steps}); ts.append(time.perf_counter() - t)
out["sample_s"] = ts
print(json.dumps(out))
"""


def oracle_sample(n, reps, full=False, steps=SAMPLE_STEPS):
    from oracle import build_oracle

    build_oracle.build()
    cores = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS=str(cores))
    code = ORACLE_CHILD.format(root=ROOT, n=n, full=bool(full), reps=reps, steps=steps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1]), cores


# ------------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle
# ------------------------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    res, cores = oracle_sample(args.n, args.warmup + args.steps, full=True)
    per_step = res["sample_s"][args.warmup:]
    iters = res["full_iters"]
    ms = 1e3 * statistics.mean(per_step) / SAMPLE_STEPS * iters
    n = args.n
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": workload_config(n),
        "cpu_baseline": {"value": ms, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: {SAMPLE_STEPS} Arnoldi steps (one GMRES(30) cycle) of the FP64 oracle on "
                                   f"the {n}^3-interval wedge, per-step time x the oracle's #Matvec ({iters}); "
                                   f"full oracle solve once: {res['full_ms']:.0f} ms"},
        "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_full_solve_ms": res["full_ms"], "oracle_iterations": iters,
    }
    print(json.dumps(line))
    return 0


def workload_config(n, precision="fp64", cycle="v"):
    outer = "FP64 right-preconditioned GMRES(30)" if precision == "fp64" else "FP64 FGMRES(30), complex64 cycle"
    cyc = "V-cycle" if cycle == "v" else "F-cycle"
    return {"workload": f"wedge n={n} ({n + 1}^3 = {(n + 1) ** 3:,} unknowns), Sommerfeld, point source at top-face "
                        f"centre, max kh 0.625, {outer} + 1 CSLP {cyc}, tol 1e-6",
            "n": n, "unknowns": (n + 1) ** 3, "krylov": "GMRES(30)" if precision == "fp64" else "FGMRES(30)",
            "precision": "complex128" if precision == "fp64" else "complex64 cycle / complex128 outer",
            "beta": [1.0, -0.5], "omega": 0.8,
            "l2": f"working set > L2: the Krylov basis alone is 31 x {16 * (n + 1) ** 3 / 1e6:.0f} MB = "
                  f"{31 * 16 * (n + 1) ** 3 / 1e9:.2f} GB, so every step streams from HBM"}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def file_hash(rel):
    return hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()[:16]


def ncu_traffic(kernel_name):
    """DRAM traffic of one launch of `kernel_name` from the committed ncu summary
    (profiles/ncu_traffic.json), or None when a source file of that kernel changed since the
    counters were taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        k = json.load(open(path)).get("kernels", {}).get(kernel_name)
    except ValueError:
        return None
    if not k:
        return None
    try:
        if any(file_hash(f) != h for f, h in k.get("source_files", {}).items()):
            return None
    except OSError:
        return None
    return k


def max_over_ranks(value, dist, device):
    """The largest per-rank value (the job's time is its slowest replica's)."""
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_solves(torch, s, b, steps, x=None):
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x = torch.zeros_like(b) if x is None else x
    infos = []
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(steps):
        x.zero_()
        _, info = s.solve(b, x)
        infos.append(info)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, infos, x


def run_ours(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_2308_06085_gb300 import helm, inputs

    n = args.n
    w = inputs.workload("wedge", n)
    s = helm.Solver(w["n"], w["h"], w["k2"], helm.SOMMERFELD, krylov="gmres" if args.precision == "fp64" else "fgmres",
                    restart=30, tol=1e-6, orth=args.orth, reorth=args.reorth, precision=args.precision,
                    cycle=args.cycle)
    b = s.rhs_point(w["sources"])
    for _ in range(args.warmup):
        _, info = s.solve(b)
    # timed region: K full solves, device time by CUDA events on the launching stream
    clocks = ClockSampler(local)
    s.profile(False)  # resets the launch counter
    if dist:
        dist.barrier()
    ms, infos, x = time_solves(torch, s, b, args.steps)
    if dist:
        dist.barrier()
    _, launches = s.profile_read()
    clk = clocks.stop()
    if dist:
        ms = max_over_ranks(ms, dist, "cuda")
    iters = infos[-1]["iterations"]
    relres = infos[-1]["rel_residual"]
    # the same K solves again with per-kernel CUDA events (kernel roofline)
    ms_prof = None
    fams = [{"name": "none", "launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0}]
    if not args.no_profile:
        s.profile(True)
        ms_prof, _, _ = time_solves(torch, s, b, args.steps)
        fams, _ = s.profile_read()
        s.profile(False)
    fams.sort(key=lambda f: -f["ms"])
    total_ms = sum(f["ms"] for f in fams)
    top = fams[0]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fp64_kernels = ("k_mdot", "k_gs_update")
    if top["ms"] <= 0:
        roof = {"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None}
    elif top["name"] in fp64_kernels and args.orth == "fp64":
        achieved = top["flops"] / (top["ms"] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "FP64: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)"}
    else:
        achieved = top["bytes"] / (top["ms"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6800 GB/s"}
    roof["kernel"] = top["name"] + ("_df" if args.orth == "df" and top["name"] in fp64_kernels else "")
    roof["launches"] = top["launches"]
    roof["avg_launch_us"] = 1e3 * top["ms"] / max(top["launches"], 1)
    roof["share_of_kernel_time"] = top["ms"] / total_ms if total_ms else None
    roof["hbm_gbs_achieved"] = top["bytes"] / (top["ms"] * 1e-3) / 1e9 if top["ms"] > 0 else None
    tr = ncu_traffic(roof["kernel"])
    roof["traffic"] = None if tr is None else tr.get("dram_bytes_per_launch")
    if tr is not None:
        roof["traffic_algorithmic_bytes"] = tr.get("algorithmic_bytes_per_launch")
        roof["traffic_note"] = tr.get("note")
    kernels = [{"name": f["name"], "launches": f["launches"], "ms_per_step": f["ms"] / args.steps,
                "share": f["ms"] / total_ms if total_ms else None,
                "gbs": f["bytes"] / (f["ms"] * 1e-3) / 1e9 if f["ms"] else None,
                "fp64_tflops": f["flops"] / (f["ms"] * 1e-3) / 1e12 if f["ms"] else None}
               for f in fams if f["launches"]]

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(torch, s, b, args.steps)

    variants = {}
    if args.variants and rank == 0:
        variants = run_variants(torch, helm, inputs, args)

    line = {
        "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32 cycle / f64 outer",
        "data": "synthetic", "config": workload_config(n, args.precision, args.cycle),
        "iterations": iters, "rel_residual": relres, "roofline": roof, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk, "ms_per_step_profiled": ms_prof, "kernels": kernels, "variants": variants,
    }
    if rank == 0 and not args.no_cpu_baseline:
        res, cores = oracle_sample(n, 1)
        t = res["sample_s"][0]
        line["cpu_baseline"] = {
            "value": 1e3 * t / SAMPLE_STEPS * iters, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{SAMPLE_STEPS} Arnoldi steps (one GMRES(30) cycle) of the FP64 oracle on the same workload, "
                      f"{t:.2f} s; per-step time x the GPU solve's #Matvec ({iters})"}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    s.close()
    if rank == 0:
        print(json.dumps(line))
    return 0


def end_to_end(torch, s, b, steps):
    bh = b.cpu().pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    xh.zero_()
    s.solve(bh, xh)
    t0 = time.perf_counter()
    for _ in range(steps):
        xh.zero_()
        s.solve(bh, xh)
    e2e_ms = 1e3 * (time.perf_counter() - t0) / steps
    nbytes = b.numel() * 16
    return {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": nbytes,
            "note": "helm_solve with pinned host b and x: H2D of b and x0, D2H of x inside each step"}


def run_variants(torch, helm, inputs, args):
    out = {}
    for name, n, prec, krylov, orth, cycle, *extra in [
            ("wedge_n128_fp64_nographs", 128, "fp64", "gmres", args.orth, "v", {"graphs": False}),
            ("wedge_n128_fp64_gs_4fma", 128, "fp64", "gmres", args.orth, "v", {"gs_sums": False}),
            ("wedge_n128_mixed", 128, "mixed", "fgmres", args.orth, "v"),
            ("wedge_n128_mixed_orth_df", 128, "mixed", "fgmres", "df", "v"),
            ("wedge_n128_mixed_orth_df_sweeps_unfused", 128, "mixed", "fgmres", "df", "v", {"fuse_down": 0, "fuse_up": 0}),
            ("wedge_n128_mixed_orth_df_sweeps_fused", 128, "mixed", "fgmres", "df", "v", {"fuse_down": 2, "fuse_up": 1}),
            ("wedge_n128_fp64_orth_df", 128, "fp64", "gmres", "df", "v"),
            ("wedge_n128_fp64_fcycle", 128, "fp64", "gmres", args.orth, "f"),
            ("wedge_n128_mixed_orth_df_fcycle", 128, "mixed", "fgmres", "df", "f"),
            ("wedge_n128_fp64_bicgstab", 128, "fp64", "bicgstab", args.orth, "v"),
            ("wedge_n128_mixed_bicgstab", 128, "mixed", "bicgstab", args.orth, "v"),
            ("wedge_n128_fp64_idr4", 128, "fp64", "idrs", args.orth, "v"),
            ("wedge_n128_mixed_idr4", 128, "mixed", "idrs", args.orth, "v"),
            ("wedge_n128_fp64_idr4_fcycle", 128, "fp64", "idrs", args.orth, "f"),
            ("wedge_n128_mixed_idr4_fcycle", 128, "mixed", "idrs", args.orth, "f"),
            ("mixed_n256_fp64", 256, "fp64", "gmres", args.orth, "v"),
            ("mixed_n256_mixed", 256, "mixed", "fgmres", args.orth, "v"),
            ("mixed_n256_mixed_orth_df", 256, "mixed", "fgmres", "df", "v"),
            ("mixed_n256_mixed_orth_df_fcycle", 256, "mixed", "fgmres", "df", "f"),
            ("mixed_n256_mixed_idr4", 256, "mixed", "idrs", args.orth, "v")]:
        w = inputs.workload("mixed" if n == 256 else "wedge", n)
        s = helm.Solver(w["n"], w["h"], w["k2"], helm.SOMMERFELD, krylov=krylov, precision=prec, orth=orth,
                        reorth=args.reorth, cycle=cycle, max_iter=8000, **(extra[0] if extra else {}))
        b = s.rhs_point(w["sources"])
        s.solve(b)
        ms, infos, _ = time_solves(torch, s, b, 2)
        out[name] = {"ms": ms, "iterations": infos[-1]["iterations"], "rel_residual": infos[-1]["rel_residual"],
                     "unknowns": (n + 1) ** 3}
        s.close()
        del s
        torch.cuda.empty_cache()
    out.update(run_closed_off_table1(torch, helm, inputs))
    out.update(run_closed_off_weak(torch, helm, inputs))
    if args.variants >= 3:
        out.update(run_shift_sweep(torch, helm, inputs, args))
    if args.variants >= 2:
        out.update(run_batched_variant(torch, helm, inputs))
        out.update(run_batched_variant(torch, helm, inputs, orth="df"))
        out.update(run_batched_variant(torch, helm, inputs, orth="df", cycle="f"))
        out.update(run_adjoint_variant(torch, helm, inputs))
    return out


def paper_golden(name):
    rows = []
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def run_closed_off(torch, helm, inputs, n, solvers, steps):
    """Time the closed-off problem (Sec. 2.1, k = 40, Dirichlet) in the paper's configuration:
    coarsest grid by the 17-node rule (Sec. 4.2), FP64, GMRES(200) (no restart is reached),
    preconditioned from the left with the paper's stopping rule or from the right, and
    Bi-CGSTAB / IDR(4) on the true residual."""
    w = inputs.workload("closed_off", n)
    b = torch.from_numpy(w["rhs"]).cuda()
    out = {}
    for krylov, side in solvers:
        s = helm.Solver(w["n"], w["h"], w["k2"], helm.DIRICHLET, coarsest_n=w["coarsest_n"], krylov=krylov,
                        restart=200 if krylov == "gmres" else 30, max_iter=3000, side=side)
        s.solve(b)
        ms, infos, _ = time_solves(torch, s, b, steps)
        it = infos[-1]["iterations"]
        out[f"closed_off_n{n}_k40_{krylov}" + ("_left" if side == "left" else "")] = {
            "ms": ms, "iterations": it, "ms_per_iteration": ms / max(it, 1), "rel_residual": infos[-1]["rel_residual"],
            "unknowns": (n - 1) ** 3, "coarsest_nodes": w["coarsest_n"] + 1}
        s.close()
        del s
        torch.cuda.empty_cache()
    return out


def run_closed_off_table1(torch, helm, inputs):
    """Table 1 (Sec. 5.1.3): 65^3 nodes; the paper prints #Matvec 145 (GMRES), 359-407
    (Bi-CGSTAB) and 192-211 (IDR(4)) over four processor layouts."""
    paper = {r[0]: [int(v) for v in r[1:]] for r in paper_golden("table1_matvec.txt")}
    out = run_closed_off(torch, helm, inputs, 64, (("gmres", "left"), ("gmres", "right"), ("bicgstab", "right"),
                                                  ("idrs", "right")), 2)
    for key, name in (("gmres_left", "GMRES"), ("gmres", "GMRES"), ("bicgstab", "Bi-CGSTAB"), ("idrs", "IDR(4)")):
        out[f"closed_off_n64_k40_{key}"]["paper_matvec_table1"] = paper[name]
    return out


def run_closed_off_weak(torch, helm, inputs):
    """Table 2 (Sec. 5.2): 129^3, 193^3 and 257^3 nodes, GMRES (left) and IDR(4), beside the
    paper's #Matvec and wall-clock times on 8, 27 and 64 CPU cores, and Table 3's seconds per
    GMRES iteration of the paper's code at 129^3 (context: other hardware)."""
    out = {}
    rows = paper_golden("weak_scaling_matvec.txt")
    per_iter = {int(r[1]): float(r[2]) for r in rows if r[0] == "per_iter"}
    for r in rows:
        if r[0] == "per_iter":
            continue
        n = int(r[0]) - 1
        res = run_closed_off(torch, helm, inputs, n, (("gmres", "left"), ("idrs", "right")), 1)
        res[f"closed_off_n{n}_k40_gmres_left"].update(paper_matvec_table2=int(r[2]), paper_s_table2=float(r[3]),
                                                      paper_np=int(r[1]))
        res[f"closed_off_n{n}_k40_idrs"].update(paper_matvec_table2=int(r[4]), paper_s_table2=float(r[5]),
                                                paper_np=int(r[1]))
        if n == 128:
            res["closed_off_n128_k40_gmres_left"]["paper_s_per_iteration_table3"] = per_iter
        out.update(res)
    return out


def run_shift_sweep(torch, helm, inputs, args):
    """Sec. 5.1.4: the CSLP shift beta2 in [-1, -0.5] against V- and F-cycle preconditioning, on
    the wedge at n = 128 and 256 (complex64 cycle, FP64 FGMRES(30) with double-float
    Gram-Schmidt), one timed solve each after a warm-up solve."""
    out = {}
    for n in (128, 256):
        w = inputs.workload("mixed" if n == 256 else "wedge", n)
        for beta2 in (-0.5, -0.75, -1.0):
            for cycle in ("v", "f"):
                s = helm.Solver(w["n"], w["h"], w["k2"], helm.SOMMERFELD, krylov="fgmres", precision="mixed",
                                orth="df", beta2=beta2, cycle=cycle, max_iter=3000)
                b = s.rhs_point(w["sources"])
                s.solve(b)
                ms, infos, _ = time_solves(torch, s, b, 1)
                out[f"shift_n{n}_beta2_{-beta2:g}_{cycle}cycle"] = {
                    "ms": ms, "iterations": infos[-1]["iterations"], "rel_residual": infos[-1]["rel_residual"],
                    "status": infos[-1]["status"]}
                s.close()
                del s
                torch.cuda.empty_cache()
    return out


def run_batched_variant(torch, helm, inputs, orth="fp64", cycle="v"):
    """32 point sources (4 x 8 grid in the plane x3 = 0.1) on the n = 128 wedge: one batched
    solve (complex64 V-cycle, FP64 FGMRES(30)) against the same 32 sources solved one by one."""
    w = inputs.workload("batched", 128)
    s = helm.Solver(w["n"], w["h"], w["k2"], helm.SOMMERFELD, krylov="fgmres", precision="mixed", orth=orth,
                    cycle=cycle)
    B = torch.stack([s.rhs_point([p]) for p in w["sources"]])
    s.solve_batched(B)  # warm-up: allocates the 32-wide workspace, tunes its launch shapes, captures its graphs
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    X, infos = s.solve_batched(B)
    e1.record(st)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    s.solve(B[0])
    torch.cuda.synchronize()
    e0.record(st)
    seq_iters = []
    for r in range(B.shape[0]):
        _, info = s.solve(B[r])
        seq_iters.append(info["iterations"])
    e1.record(st)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    res = {"batched_n128_32src_mixed" + ("_orth_df" if orth == "df" else "") + ("_fcycle" if cycle == "f" else ""): {
        "ms": ms_b, "ms_per_source": ms_b / B.shape[0], "sequential_ms": ms_s, "speedup_vs_sequential": ms_s / ms_b,
        "iterations_max": max(i["iterations"] for i in infos), "iterations_min": min(i["iterations"] for i in infos),
        "rel_residual_max": max(i["rel_residual"] for i in infos), "sequential_iterations_max": max(seq_iters),
        "unknowns_per_source": (128 + 1) ** 3}}
    s.close()
    del s, B, X
    torch.cuda.empty_cache()
    return res


def run_adjoint_variant(torch, helm, inputs):
    """Adjoint-state gradient on the n = 192 smooth random model: 8 sources, receivers on the
    plane x3 = 0.9, complex64 V-cycle / FP64 FGMRES(30); one forward and one adjoint solve per
    source.  Observed data come from forward solves on the perturbed model (timing only)."""
    import numpy as np

    w = inputs.workload("adjoint", 192)
    shape = inputs.unknown_shape(w["n"], helm.SOMMERFELD)
    N3, N2, N1 = shape
    k = w["receiver_plane"]
    rec = np.arange(k * N2 * N1, (k + 1) * N2 * N1)
    k2_true = w["k2"] * inputs.gaussian_bump(w["n"], amp=0.05, width=0.1) ** -2
    st_ = helm.Solver(w["n"], w["h"], k2_true, helm.SOMMERFELD, krylov="fgmres", precision="mixed")
    recd = torch.from_numpy(rec).cuda()
    d = torch.stack([st_.solve(st_.rhs_point([p]))[0].reshape(-1)[recd] for p in w["sources"]]).contiguous()
    st_.close()
    res = {}
    g_ref = None
    for name, orth in (("adjoint_n192_8src_mixed", "fp64"), ("adjoint_n192_8src_mixed_orth_df", "df")):
        s = helm.Solver(w["n"], w["h"], w["k2"], helm.SOMMERFELD, krylov="fgmres", precision="mixed", orth=orth)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        loss, grad, info = s.adjoint_grad(w["sources"], rec, d)
        e1.record(st)
        torch.cuda.synchronize()
        res[name] = {"ms": e0.elapsed_time(e1), "loss": loss, "solves": 2 * len(w["sources"]),
                     "iterations_total": info["iterations"], "rel_residual_max": info["rel_residual"],
                     "grad_norm": float(grad.norm()), "unknowns": (192 + 1) ** 3}
        if g_ref is None:
            g_ref = grad.clone()
        else:  # the two Gram-Schmidt arithmetics give the same gradient to the solve accuracy
            res[name]["grad_rel_diff_vs_fp64_orth"] = float((grad - g_ref).norm() / g_ref.norm())
        s.close()
        del s, grad
        torch.cuda.empty_cache()
    return res


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
