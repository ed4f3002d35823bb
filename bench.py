#!/usr/bin/env python
"""Benchmark: time-to-1e-6 of the CSLP-preconditioned matrix-free Helmholtz solve on one GB300,
FP64 against mixed precision against batched right-hand sides.

Headline workload (one step = one full solve, the whole hot path): the three-layer wedge model
on the unit cube at n = 256 intervals per direction (257^3 = 16,974,593 unknowns, Sommerfeld on
every face), the frequency of the n = 128 wedge (max k h = 0.3125), point source at the
top-face centre; right-preconditioned GMRES(30) with one CSLP V-cycle per step in complex128
throughout, to ||b - A x|| / ||b|| <= 1e-6.  `value` is the device time per solve.

Beside it, in the same run and printed on the same line:
  - mixed: the same workload with a complex64 V-cycle under FP64 flexible GMRES(30) (FP64
    residual, orthogonalisation and coarsest solve);
  - batched: 32 point sources on the n = 128 wedge (a 4 x 8 grid at depth 0.1) solved in one
    batched launch (complex64 V-cycle, FP64 FGMRES(30) and orthogonalisation), against the same
    32 sources solved one after another;
  - the dominant kernel's roofline from live CUDA-event timings, and the finest-level complex64
    V-cycle kernel's roofline from the mixed solve;
  - the end-to-end time through the C ABI with host buffers, the FP64 CPU oracle timed on a
    bounded sample (16 threads and 1 thread), and clocks sampled during the timed region.

--impl reference times the FP64 CPU oracle (the reference arm) on the host cores.
--ncu-region / --write-traffic capture and record the DRAM traffic of chosen kernels.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import re
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
HEADLINE = "mixed"         # the wedge at n = 256 with the n = 128 frequency (inputs.workload)
HEADLINE_N = 256
BATCH_N = 128
FP64_KERNELS = ("k_mdot", "k_gs_update")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=HEADLINE_N, help="intervals per direction of the headline wedge")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the mixed and batched forms")
    ap.add_argument("--variants", type=int, default=0,
                    help="0: headline and forms only; 1: + precision, Krylov and cycle variants at n = 128 and 256 "
                         "and the paper's closed-off tables; 2: + batched and adjoint variants; 3: + the CSLP shift "
                         "sweep (beta2 x V/F-cycle)")
    ap.add_argument("--orth", choices=["fp64", "df"], default="fp64",
                    help="Gram-Schmidt arithmetic: native FP64 or double-float FP32 pairs")
    ap.add_argument("--reorth", choices=["selective", "always"], default="selective",
                    help="second Gram-Schmidt pass on every step, or only when the first pass lost half of |w|")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="fp64: complex128 throughout (the headline); mixed: complex64 cycle under FP64 FGMRES(30)")
    ap.add_argument("--cycle", choices=["v", "f"], default="v", help="multigrid cycle of the preconditioner")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-kernel timed leg")
    ap.add_argument("--ncu-region", choices=["gs", "vcycle64", "vcycle32"], default=None,
                    help="run one deterministic sequence of launches between cudaProfilerStart/Stop for an ncu "
                         "capture with --profile-from-start off (see profiles/)")
    ap.add_argument("--write-traffic", metavar="CSV", default=None,
                    help="record the DRAM bytes of an ncu --csv capture of --ncu-region into profiles/ncu_traffic.json")
    ap.add_argument("--traffic-out", default=None, help="where --write-traffic writes (default profiles/ncu_traffic.json)")
    return ap.parse_args(argv)


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
# CPU oracle samples (in a child process, so its OpenMP runtime stays apart from torch)
# ------------------------------------------------------------------------------------------
ORACLE_CHILD = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import oracle
from paper_2308_06085_gb300 import inputs as I
w = I.workload({name!r}, {n})
o = oracle.Solver(w["n"], w["h"], oracle.SOMMERFELD, w["k2"])
b = oracle.rhs_point(o.shape, oracle.SOMMERFELD, w["h"], w["sources"])
out = []
for steps in {plan!r}:
    t = time.perf_counter()
    o.gmres(b, restart=30, tol=1e-6, max_iter=steps)
    out.append([steps, time.perf_counter() - t])
print(json.dumps(out))
"""


def oracle_samples(name, n, plan, threads):
    """Wall time of each bounded oracle sample: GMRES(30) from x0 = 0 stopped after `steps`
    Arnoldi steps (initial residual, the steps, the end-of-cycle update and the explicit
    residual), for each entry of `plan`, with `threads` OpenMP threads."""
    from oracle import build_oracle

    build_oracle.build()
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    code = ORACLE_CHILD.format(root=ROOT, name=name, n=n, plan=list(plan))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3600)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_count(name, n):
    """The oracle's own #Matvec for the workload, stored by tests/golden/make_wedge_counts.py
    (which calls only the oracle), or None."""
    path = os.path.join(ROOT, "tests", "golden", "wedge_oracle_counts.txt")
    if not os.path.exists(path):
        return None
    for ln in open(path):
        f = ln.split()
        if ln.strip() and not ln.startswith("#") and f[0] == name and int(f[1]) == n:
            return int(f[2])
    return None


def step_model(samples):
    """Per-Arnoldi-step time and per-cycle overhead from samples of two sizes: the slope
    between the mean times of the smallest and the largest sample size, and the rest of the
    smallest sample.  With one size only, the whole sample time per step (no overhead)."""
    by = {}
    for steps, t in samples:
        by.setdefault(steps, []).append(t)
    sizes = sorted(by)
    lo, hi = sizes[0], sizes[-1]
    tlo, thi = statistics.mean(by[lo]), statistics.mean(by[hi])
    if hi == lo:
        return tlo / lo, 0.0
    step = (thi - tlo) / (hi - lo)
    return step, max(tlo - lo * step, 0.0)


def extrapolate(step, overhead, iters, restart=30):
    """Solve time from the step model: #Matvec steps and one cycle overhead per restart cycle.
    Gram-Schmidt of later steps works on up to 30 vectors, more than in the sampled first
    steps, so this underestimates the oracle's solve."""
    cycles = -(-iters // restart)
    return iters * step + cycles * overhead


# ------------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle
# ------------------------------------------------------------------------------------------
REF_SAMPLE = 4  # Arnoldi steps of the larger sample


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.n
    cores = os.cpu_count() or 1
    # warm-up steps: one-step samples; timed steps alternate four-step and one-step samples
    plan = [1] * args.warmup + [REF_SAMPLE if i % 2 == 0 else 1 for i in range(args.steps)]
    res = oracle_samples(HEADLINE, n, plan, cores)
    timed = res[args.warmup:]
    step, overhead = step_model(timed)
    stored = oracle_count(HEADLINE, n)
    iters = stored if stored is not None else 299
    src = "the oracle's stored count" if stored is not None else "the GPU solve's count, no stored oracle count"
    ms = 1e3 * extrapolate(step, overhead, iters)
    ms_step = 1e3 * statistics.mean(t for _, t in timed)
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(n),
        "cpu_baseline": {"value": ms, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step one bounded sample: FP64 oracle GMRES(30) stopped after {REF_SAMPLE} "
                                   f"(even steps) or 1 (odd steps) Arnoldi steps on the same workload; value = "
                                   f"#Matvec ({iters}, {src}) x the per-step slope "
                                   f"{1e3 * step:.0f} ms + per-cycle overhead {1e3 * overhead:.0f} ms "
                                   f"(extrapolated; ms_per_step is the mean sample time)"},
        "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_iterations": iters, "oracle_step_ms": 1e3 * step, "oracle_cycle_overhead_ms": 1e3 * overhead,
    }
    print(json.dumps(line))
    return 0


def workload_config(n, precision="fp64", cycle="v"):
    outer = "FP64 right-preconditioned GMRES(30)" if precision == "fp64" else "FP64 FGMRES(30), complex64 cycle"
    cyc = "V-cycle" if cycle == "v" else "F-cycle"
    return {"workload": f"wedge n={n}, {n + 1}^3 unknowns, Sommerfeld, top-centre source, omega of the n=128 wedge, "
                        f"{outer} + 1 CSLP {cyc}, tol 1e-6",
            "n": n, "unknowns": (n + 1) ** 3, "krylov": "GMRES(30)" if precision == "fp64" else "FGMRES(30)",
            "precision": "complex128" if precision == "fp64" else "complex64 cycle / complex128 outer",
            "beta2": -0.5, "omega": 0.8,
            "l2": f"working set > L2: the Krylov basis alone is 31 x {16 * (n + 1) ** 3 / 1e6:.0f} MB = "
                  f"{31 * 16 * (n + 1) ** 3 / 1e9:.2f} GB, so every step streams from HBM"}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def file_hash(rel):
    return hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()[:16]


def ncu_traffic(kernel_name):
    """The committed ncu record of `kernel_name` (profiles/ncu_traffic.json, written by
    --write-traffic from a capture), or None when any source file it lists has changed since
    the capture: a record is never carried over to an edited kernel."""
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


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def kernel_rows(fams, steps):
    total = sum(f["ms"] for f in fams)
    return [{"name": f["name"], "launches": f["launches"], "launches_per_step": f["launches"] / steps,
             "ms_per_step": f["ms"] / steps,
             "share": f["ms"] / total if total else None,
             "gbs": f["bytes"] / (f["ms"] * 1e-3) / 1e9 if f["ms"] else None,
             "fp64_tflops": f["flops"] / (f["ms"] * 1e-3) / 1e12 if f["ms"] else None}
            for f in sorted(fams, key=lambda f: -f["ms"]) if f["launches"]]


def roofline_of(fam, hbm_peak, alu, orth="fp64", record_suffix=""):
    """Roofline entry of one kernel family from its CUDA-event totals: FP64-issue bound for the
    FP64 Gram-Schmidt kernels, HBM bound otherwise; traffic from the committed ncu record,
    scaled to this family's average launch (None when stale)."""
    if fam["ms"] <= 0:
        return {"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None}
    gbs = fam["bytes"] / (fam["ms"] * 1e-3) / 1e9
    if alu:
        achieved = fam["flops"] / (fam["ms"] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "FP64: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)"}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    name = fam["name"] + ("_df" if orth == "df" and fam["name"] in FP64_KERNELS else "")
    roof.update(kernel=name, launches=fam["launches"], avg_launch_us=1e3 * fam["ms"] / max(fam["launches"], 1),
                hbm_gbs_achieved=gbs)
    tr = ncu_traffic(name + record_suffix)
    alg = fam["bytes"] / max(fam["launches"], 1)
    roof["traffic"] = None if tr is None else tr["dram_over_algorithmic"] * alg
    if tr is not None:
        roof["traffic_over_algorithmic"] = tr["dram_over_algorithmic"]
        roof["traffic_capture"] = tr.get("capture")
    return roof


def end_to_end(torch, s, b, steps):
    bh = b.cpu().pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    s.solve(bh, xh, zero_guess=True)
    t0 = time.perf_counter()
    for _ in range(steps):
        s.solve(bh, xh, zero_guess=True)
    e2e_ms = 1e3 * (time.perf_counter() - t0) / steps
    nbytes = b.numel() * 16
    return {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "steps": steps, "note": "helm_solve_zero (the solve from x = 0, as the timed solves) with pinned host b "
                                    "and x: H2D of b and D2H of x inside each step"}


def form_mixed(torch, helm, inputs, n, steps, fp64_ms, hbm_peak):
    """The headline workload with a complex64 V-cycle under FP64 FGMRES(30) (FP64 outer
    residual, orthogonalisation and coarsest solve): time per solve, and the roofline of the
    finest-level complex64 V-cycle kernels from one profiled solve."""
    w = inputs.workload(HEADLINE, n)
    s = helm.Solver(w["n"], w["h"], w["k2"], helm.SOMMERFELD, krylov="fgmres", precision="mixed", orth="fp64",
                    restart=30, tol=1e-6)
    b = s.rhs_point(w["sources"])
    s.solve(b)
    ms, infos, _ = time_solves(torch, s, b, steps)
    s.profile(True)
    time_solves(torch, s, b, 1)
    fams, _ = s.profile_read()
    s.profile(False)
    s.close()
    finest = [f for f in fams if f["name"].endswith("(finest)") and f["launches"]]
    top = max(finest, key=lambda f: f["ms"]) if finest else None
    out = {"ms": ms, "iterations": infos[-1]["iterations"], "rel_residual": infos[-1]["rel_residual"],
           "speedup_vs_fp64": fp64_ms / ms, "steps": steps,
           "finest_vcycle_kernels": [{"name": f["name"], "gbs": f["bytes"] / (f["ms"] * 1e-3) / 1e9,
                                      "frac": f["bytes"] / (f["ms"] * 1e-3) / 1e9 / hbm_peak,
                                      "us_per_launch": 1e3 * f["ms"] / f["launches"]} for f in finest]}
    return out, (roofline_of(top, hbm_peak, alu=False, record_suffix=" c64") if top else None)


def form_batched(torch, helm, inputs, fp64_single_ms=None):
    """32 point sources on the n = 128 wedge in one batched launch (complex64 V-cycle, FP64
    FGMRES(30) and orthogonalisation) against the same 32 sources solved one after another
    with the same context."""
    w = inputs.workload("batched", BATCH_N)
    s = helm.Solver(w["n"], w["h"], w["k2"], helm.SOMMERFELD, krylov="fgmres", precision="mixed", orth="fp64")
    B = torch.stack([s.rhs_point([p]) for p in w["sources"]])
    s.solve_batched(B)  # warm-up: the 32-wide workspace, its launch shapes and graphs
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
    seq = []
    for r in range(B.shape[0]):
        _, info = s.solve(B[r])
        seq.append(info["iterations"])
    e1.record(st)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    nb = B.shape[0]
    s.close()
    del B, X
    torch.cuda.empty_cache()
    return {"sources": nb, "ms": ms_b, "ms_per_source": ms_b / nb, "sequential_ms": ms_s,
            "sequential_ms_per_source": ms_s / nb, "speedup_vs_sequential": ms_s / ms_b,
            "iterations_max": max(i["iterations"] for i in infos), "iterations_min": min(i["iterations"] for i in infos),
            "iterations_mean": sum(i["iterations"] for i in infos) / nb,
            "rel_residual_max": max(i["rel_residual"] for i in infos), "sequential_iterations_max": max(seq),
            "sequential_iterations_mean": sum(seq) / nb, "unknowns_per_source": (BATCH_N + 1) ** 3}


def cpu_baseline(iters_gpu, n):
    """The FP64 oracle on the host cores, on bounded samples of the headline workload: 1- and
    4-step samples with every core give the per-step slope and per-cycle overhead, scaled to the
    oracle's #Matvec; a 1-step sample on one thread is scaled by the same model."""
    cores = os.cpu_count() or 1
    stored = oracle_count(HEADLINE, n)
    iters = stored if stored is not None else iters_gpu
    res = oracle_samples(HEADLINE, n, [1, REF_SAMPLE, 1, REF_SAMPLE], cores)
    step, overhead = step_model(res)
    ms = 1e3 * extrapolate(step, overhead, iters)
    t1 = statistics.mean(t for s_, t in res if s_ == 1)
    one = oracle_samples(HEADLINE, n, [1], 1)[0][1]
    ms1 = ms * one / t1
    return {"value": ms, "unit": UNIT, "cores": cores, "kind": "oracle",
            "value_1_thread": ms1, "cores_1_thread": 1,
            "sample": f"FP64 oracle GMRES(30) on the same workload stopped after 1 and {REF_SAMPLE} Arnoldi steps "
                      f"({', '.join(f'{t:.1f}' for _, t in res)} s at {cores} threads; one 1-step sample at 1 thread, "
                      f"{one:.1f} s): value = #Matvec ({iters}, " + ("the oracle's stored count" if stored else
                      "the GPU solve's") + f") x per-step slope {1e3 * step:.0f} ms + per-cycle overhead "
                      f"{1e3 * overhead:.0f} ms, extrapolated; value_1_thread scales it by the 1-step times",
            "iterations": iters}


def run_ours(args):
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

    if args.ncu_region:
        return ncu_region(torch, helm, inputs, args.ncu_region)
    n = args.n
    w = inputs.workload(HEADLINE, n)
    mixed = args.precision == "mixed"
    s = helm.Solver(w["n"], w["h"], w["k2"], helm.SOMMERFELD, krylov="fgmres" if mixed else "gmres",
                    restart=30, tol=1e-6, orth=args.orth, reorth=args.reorth, precision=args.precision,
                    cycle=args.cycle)
    b = s.rhs_point(w["sources"])
    for _ in range(args.warmup):
        s.solve(b)
    # timed region: K full solves, device time by CUDA events on the launching stream
    clocks = ClockSampler(local)
    s.profile(False)  # resets the launch counter
    if dist:
        dist.barrier()
    ms, infos, _ = time_solves(torch, s, b, args.steps)
    if dist:
        dist.barrier()
    _, launches = s.profile_read()
    clk = clocks.stop()
    if dist:
        ms = max_over_ranks(ms, dist, "cuda")
    iters = infos[-1]["iterations"]
    relres = infos[-1]["rel_residual"]
    hbm_peak = peaks().get("hbm_gbs", 6800.0)
    # per-kernel CUDA events over a few more solves (kernel roofline)
    psteps = min(args.steps, 2)
    fams = []
    ms_prof = None
    if not args.no_profile:
        s.profile(True)
        ms_prof, _, _ = time_solves(torch, s, b, psteps)
        fams, _ = s.profile_read()
        s.profile(False)
    fams = [f for f in fams if f["launches"]]
    if fams:
        top = max(fams, key=lambda f: f["ms"])
        roof = roofline_of(top, hbm_peak, alu=top["name"] in FP64_KERNELS and args.orth == "fp64", orth=args.orth)
        roof["share_of_kernel_time"] = top["ms"] / sum(f["ms"] for f in fams)
    else:
        roof = {"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None}
    kernels = kernel_rows(fams, psteps)

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None if args.no_e2e else end_to_end(torch, s, b, min(args.steps, 3))
    s.close()
    del s
    torch.cuda.empty_cache()

    cfg = workload_config(n, args.precision, args.cycle)
    forms = {}
    if rank == 0 and not args.no_forms:
        forms["mixed"], c64roof = form_mixed(torch, helm, inputs, n, min(args.steps, 3), ms, hbm_peak)
        forms["batched"] = form_batched(torch, helm, inputs)
        fm, fb = forms["mixed"], forms["batched"]
        cfg.update(mixed_form="same workload, complex64 V-cycle under FP64 FGMRES(30) with FP64 orthogonalisation",
                   mixed_ms=fm["ms"], mixed_iterations=fm["iterations"], mixed_speedup_vs_fp64=fm["speedup_vs_fp64"],
                   batched_form=f"32 sources on the n={BATCH_N} wedge, one batched launch, complex64 V-cycle, FP64 "
                                f"FGMRES(30) and orthogonalisation",
                   batched_ms=fb["ms"], batched_ms_per_source=fb["ms_per_source"],
                   batched_sequential_ms_per_source=fb["sequential_ms_per_source"],
                   batched_speedup_vs_sequential=fb["speedup_vs_sequential"],
                   batched_iterations_max=fb["iterations_max"])
        if c64roof:
            roof.update(c64_kernel=c64roof["kernel"] + " (mixed solve)", c64_achieved=c64roof["achieved"],
                        c64_unit="GB/s", c64_peak=c64roof["peak"], c64_frac=c64roof["frac"],
                        c64_traffic=c64roof["traffic"], c64_avg_launch_us=c64roof["avg_launch_us"])
    variants = {}
    if args.variants and rank == 0:
        variants = run_variants(torch, helm, inputs, args)

    line = {
        "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if not mixed else "f32 cycle / f64 outer", "data": "synthetic", "config": cfg,
        "iterations": iters, "rel_residual": relres, "roofline": roof, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk, "ms_per_step_profiled": ms_prof, "forms": forms, "kernels": kernels[:10],
    }
    if variants:
        line["variants"] = variants
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(iters, n)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------------------
# ncu traffic records: a deterministic region of launches, then the counters written beside
# the algorithmic bytes the library's profiler counted for the same launches
# ------------------------------------------------------------------------------------------
REGION_OUT = os.path.join(ROOT, "_build", "ncu_regions")  # scratch, not tracked
REGION_KERNELS = {  # ncu -k filter for each region
    "gs": "regex:k_mdot|k_gs_update",
    "vcycle64": "regex:k_smooth0|k_stencil|k_restrict|k_prolong|k_rr|k_up|k_down",
    "vcycle32": "regex:k_smooth0|k_stencil|k_restrict|k_prolong|k_rr|k_up|k_down",
}


def ncu_region(torch, helm, inputs, kind):
    """One deterministic sequence of launches between cudaProfilerStart and cudaProfilerStop
    (for `ncu --profile-from-start off`), on the headline workload at n = 256 with a small
    Krylov basis so that the device holds a few GB:
      gs       : 8 Arnoldi steps of FP64 GMRES with a second Gram-Schmidt pass on every step
                 and plain launches (k_mdot / k_gs_update with 1..8 basis vectors);
      vcycle64 : one FP64 V-cycle (cslp_vcycle, complex128), then one product with A;
      vcycle32 : one Arnoldi step of the mixed solve (its complex64 V-cycle; the FP32 kernels are
                 told apart from the FP64 outer ones by their template arguments).
    The library's profiler runs over the same launches; its per-family launch counts and
    algorithmic bytes go to _build/ncu_regions/ncu_region_<kind>.json for --write-traffic."""
    w = inputs.workload(HEADLINE, HEADLINE_N)
    if kind == "gs":
        s = helm.Solver(w["n"], w["h"], w["k2"], helm.SOMMERFELD, restart=8, max_iter=8, reorth="always",
                        graphs=False)
        b = s.rhs_point(w["sources"])
        run = lambda: s.solve(b)  # noqa: E731
    elif kind == "vcycle64":  # one FP64 V-cycle, then one product with A
        s = helm.Solver(w["n"], w["h"], w["k2"], helm.SOMMERFELD, restart=2, max_iter=1)
        r = torch.from_numpy(inputs.random_vector(s.shape, 7)).cuda()
        z = torch.empty_like(r)
        v = torch.empty_like(r)

        def run():
            s.vcycle(r, out=z)
            s.apply(z, out=v)
    else:  # one Arnoldi step of the mixed solve: its complex64 V-cycle reads the complex128 v_j
        s = helm.Solver(w["n"], w["h"], w["k2"], helm.SOMMERFELD, krylov="fgmres", precision="mixed", restart=2,
                        max_iter=1, graphs=False)
        b = s.rhs_point(w["sources"])
        run = lambda: s.solve(b)  # noqa: E731
    try:
        run()  # warm-up (and, for gs, the solve's graphs and tuning are already done at create)
    except helm.HelmError:
        pass  # ENOCONV: the gs region stops after max_iter steps on purpose
    torch.cuda.synchronize()
    s.profile(True)
    cudart = torch.cuda.cudart()
    cudart.cudaProfilerStart()
    try:
        run()
    except helm.HelmError:
        pass
    torch.cuda.synchronize()
    cudart.cudaProfilerStop()
    fams, launches = s.profile_read()
    s.profile(False)
    s.close()
    os.makedirs(REGION_OUT, exist_ok=True)
    rec = {"region": kind, "unknowns": (HEADLINE_N + 1) ** 3, "workload": f"{HEADLINE} n={HEADLINE_N}",
           "kernel_filter": REGION_KERNELS[kind],
           "families": {f["name"]: {"launches": f["launches"], "bytes": f["bytes"]} for f in fams if f["launches"]}}
    with open(os.path.join(REGION_OUT, f"ncu_region_{kind}.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps({"ncu_region": kind, "launches": launches}))
    return 0


def _family_of(kernel):
    """Profiler family of an ncu kernel name (demangled, with template arguments), or None."""
    m = re.search(r"\b(k_[a-z0-9_]+)\s*(?:<([^>]*)>)?", kernel)
    if not m:
        return None
    base, targs = m.group(1), m.group(2) or ""
    if base == "k_stencil":
        args = [a.strip() for a in targs.split(",")]
        return {"0": "k_stencil(apply)", "1": "k_stencil(resid)", "2": "k_stencil(jacobi)"}.get(
            args[1] if len(args) > 1 else "")
    alias = {"k_gs_update_sums": "k_gs_update", "k_smooth0_resid32": "k_smooth0", "k_restrict2": "k_restrict",
             "k_prolong2": "k_prolong_add"}
    if base in ("k_mdot", "k_gs_update", "k_smooth0", "k_restrict", "k_prolong_add", "k_down32", "k_up", "k_rr") or \
            base in alias:
        return alias.get(base, base)
    return None


def _template_real(kernel):
    """First template argument of an ncu kernel name ("double", "float") or ""."""
    m = re.search(r"\bk_[a-z0-9_]+\s*<\s*([a-z]+)", kernel)
    return m.group(1) if m else ""


DOWN_FAMILIES = ("k_smooth0", "k_stencil(resid)", "k_restrict", "k_down32", "k_rr")


def read_ncu_csv(path):
    """(kernel name, DRAM bytes, duration ns) per captured launch of an `ncu --csv` log (one row
    per launch and metric), in launch order."""
    rows = {}
    order = []
    with open(path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        key = r["ID"]
        if key not in rows:
            rows[key] = {"kernel": r["Kernel Name"], "dram": 0.0, "ns": None}
            order.append(key)
        name, unit = r["Metric Name"], r.get("Metric Unit", "")
        v = float(r["Metric Value"].replace(",", ""))
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9,
                 "nsecond": 1, "usecond": 1e3, "msecond": 1e6, "ns": 1, "us": 1e3, "ms": 1e6}.get(unit, 1)
        if name.startswith("dram__bytes_"):
            rows[key]["dram"] += v * scale
        elif name == "gpu__time_duration.sum":
            rows[key]["ns"] = v * scale
    return [rows[k] for k in order]


SOURCES = {"gs": ["paper_2308_06085_gb300/csrc/krylov.cu", "paper_2308_06085_gb300/csrc/common.cuh",
                  "paper_2308_06085_gb300/csrc/vecred.cuh"],
           "vcycle64": ["paper_2308_06085_gb300/csrc/stencil.cu", "paper_2308_06085_gb300/csrc/common.cuh"],
           "vcycle32": ["paper_2308_06085_gb300/csrc/stencil.cu", "paper_2308_06085_gb300/csrc/common.cuh"]}


NCU_TRAFFIC_CMD = ("ncu --profile-from-start off --metrics dram__bytes_read.sum,dram__bytes_write.sum,"
                   "gpu__time_duration.sum --clock-control none -k '{k}' --csv --log-file traffic_{kind}.csv "
                   "python bench.py --ncu-region {kind}")


def write_traffic(csv_path, kind, out_path=None):
    """Record, per kernel family of the region, the DRAM bytes ncu measured over the captured
    launches against the algorithmic bytes the library counted for them, with hashes of the
    sources as they were when captured (run in the same call as the capture)."""
    region = json.load(open(os.path.join(REGION_OUT, f"ncu_region_{kind}.json")))
    launches = read_ncu_csv(csv_path)
    fams = region["families"]
    out_path = out_path or os.path.join(ROOT, "profiles", "ncu_traffic.json")
    rec = json.load(open(out_path)) if os.path.exists(out_path) else {}
    rec["note"] = ("per kernel family: DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of ncu-captured "
                   "launches over the algorithmic bytes the library's profiler counted for the same launches; an "
                   "entry reads as stale (null) once a listed source file changes")
    kernels = rec.setdefault("kernels", {})
    groups = {}
    for ln in launches:
        fam = _family_of(ln["kernel"])
        if kind == "vcycle32" and _template_real(ln["kernel"]) == "double":
            fam = None  # the outer FP64 residual and A-product of the mixed step
        if fam:
            groups.setdefault(fam, []).append(ln)
    hashes = {f: file_hash(f) for f in SOURCES[kind]}
    suffix = "" if kind != "vcycle32" else " c64"
    for fam, lst in groups.items():
        if kind == "gs":
            name, alg = fam, fams.get(fam, {}).get("bytes")
            use = lst
            if not alg or fams[fam]["launches"] != len(lst):
                continue
        elif fam + " (finest)" in fams:  # finest level: first launch of a down-sweep kernel, last of an up-sweep one
            use = [lst[0] if fam in DOWN_FAMILIES else lst[-1]]
            f = fams[fam + " (finest)"]
            if f["launches"] != 1:
                continue
            name, alg = fam + " (finest)" + suffix, f["bytes"]
        else:  # a kernel launched once in the region (the product with A)
            f = fams.get(fam)
            if not f or f["launches"] != len(lst):
                continue
            use, name, alg = lst, fam + suffix, f["bytes"]
        dram = sum(u["dram"] for u in use)
        kernels[name] = {"dram_over_algorithmic": dram / alg, "dram_bytes": dram, "algorithmic_bytes": alg,
                         "launches": len(use), "duration_us": sum(u["ns"] or 0 for u in use) / 1e3,
                         "source_files": hashes,
                         "capture": f"region {kind} on {region['workload']}: {len(use)} launch(es) of "
                                    f"{use[0]['kernel'][:80]}",
                         "command": NCU_TRAFFIC_CMD.format(k=REGION_KERNELS[kind], kind=kind)}
        print(f"{name}: dram/algorithmic = {dram / alg:.3f} over {len(use)} launch(es)")
    rec.pop("command", None)
    with open(out_path, "w") as f:
        json.dump(rec, f, indent=1)
    return 0


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


def run_closed_off(torch, helm, inputs, n, solvers, steps, coarse_tol=0.0):
    """Time the closed-off problem (Sec. 2.1, k = 40, Dirichlet) in the paper's configuration:
    coarsest grid by the 17-node rule (Sec. 4.2), FP64, GMRES(200) (no restart is reached),
    preconditioned from the left with the paper's stopping rule or from the right, and
    Bi-CGSTAB / IDR(4) on the true residual.  coarse_tol > 0: the coarsest grid solved by GMRES
    to that tolerance, as the paper does (Sec. 5), instead of by the dense inverse."""
    w = inputs.workload("closed_off", n)
    b = torch.from_numpy(w["rhs"]).cuda()
    out = {}
    for krylov, side in solvers:
        s = helm.Solver(w["n"], w["h"], w["k2"], helm.DIRICHLET, coarsest_n=w["coarsest_n"], krylov=krylov,
                        restart=200 if krylov == "gmres" else 30, max_iter=3000, side=side, coarse_tol=coarse_tol)
        s.solve(b)
        ms, infos, _ = time_solves(torch, s, b, steps)
        it = infos[-1]["iterations"]
        out[f"closed_off_n{n}_k40_{krylov}" + ("_left" if side == "left" else "") +
            ("_coarse_gmres" if coarse_tol > 0 else "")] = {
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
    # the same with the paper's own coarsest-grid solve, GMRES to 1e-11
    out.update(run_closed_off(torch, helm, inputs, 64, (("gmres", "left"), ("bicgstab", "right"), ("idrs", "right")), 2,
                              coarse_tol=1e-11))
    for key, name in (("gmres_left", "GMRES"), ("gmres", "GMRES"), ("bicgstab", "Bi-CGSTAB"), ("idrs", "IDR(4)"),
                      ("gmres_left_coarse_gmres", "GMRES"), ("bicgstab_coarse_gmres", "Bi-CGSTAB"),
                      ("idrs_coarse_gmres", "IDR(4)")):
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


def main(argv=None):
    args = parse(argv)
    if args.write_traffic:
        return write_traffic(args.write_traffic, args.ncu_region, args.traffic_out)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
