#!/usr/bin/env python
"""Benchmark of the matrix-free PA elasticity operator on GB300.

Default workload (one "step"): one FP64 operator apply for every degree of
the operator sweep p in {1, 2, 4, 6, 8} on an n^3 cube with ~3M vector dofs
per degree (n = 99, 50, 25, 16, 12), every element its own random affine
map (scales in [0.5, 2], shear up to 0.3), lambda and mu from E = 1,
nu = 0.3, x ~ U[-1, 1].  value = total dofs of the step / device time of the
step (GDoF/s, higher is better).

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
independent copy of the workload (weak scaling, no collective on the data
path); the timed region is bracketed by a barrier and synchronisation and
the slowest rank's time is used.

--impl reference times the plain CPU oracle (test infrastructure) on the
host cores instead, on a bounded sample of the same workload.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as syn  # noqa: E402

METRIC = "Op GDoF/s vs p (FP64 vs FP32-refined); GMG-PCG solves/s, p50/p99 latency"
SWEEP = (1, 2, 4, 6, 8)
# FP64: 2 FMA / clk / SM (4 flop); FP32: 128 FMA / clk / SM (256 flop)
FLOP_PER_CLK_SM = {"f64": 4.0, "f32": 256.0}
SM_MAX_MHZ_NOMINAL = 2070.0  # used only when no clock sample was taken


def derived_peak_tflops(dtype_name: str, sms: int, mhz: float) -> float:
    """FMA-unit peak from unit counts and a clock: SMs x flop/clk/SM x MHz."""
    return sms * FLOP_PER_CLK_SM[dtype_name] * mhz * 1e6 / 1e12


def peak_clock_mhz(clocks: dict) -> float:
    """The SM clock of the derived peak: the median sampled during the timed
    region (nominal maximum when nvidia-smi gave no sample)."""
    v = clocks.get("sm_mhz") if clocks else None
    return float(v) if v else SM_MAX_MHZ_NOMINAL


def flops_per_element(p: int) -> int:
    """Algorithmic FLOPs per element of the fused sum-factorised apply
    (Table 6 of the paper): 30 D^3 Q + 36 D^2 Q^2 + 36 D Q^3 + 113 Q^3 + 12 D^3."""
    D, Q = p + 1, p + 2
    return 30 * D ** 3 * Q + 36 * D ** 2 * Q ** 2 + 36 * D * Q ** 3 + 113 * Q ** 3 + 12 * D ** 3


def algorithmic_bytes(p: int, n: int, elem: int) -> int:
    """Minimum HBM traffic of one apply: x read + y written once (L-vector)
    and the 12-value geometry record per element."""
    ndofs = 3 * (n * p + 1) ** 3
    return 2 * ndofs * elem + n ** 3 * 12 * elem


def sweep_workload_name(precision: str, ps) -> str:
    """The operator sweep's description (the same for both arms)."""
    ns = [syn.sweep_n(p) for p in ps]
    dofs = sum(3 * (n * p + 1) ** 3 for n, p in zip(ns, ps))
    return (f"{precision.upper()} op_apply sweep p in {{{','.join(map(str, ps))}}}, n^3 unit cube "
            f"(n = {', '.join(map(str, ns))}; {dofs / 1e6:.2f}M dofs per step), "
            "per-element random affine maps (scales U[0.5,2], shear U[-0.3,0.3]), "
            "E=1 nu=0.3, x ~ U[-1,1], unconstrained")


def workload(p: int, scale: float = 1.0):
    n = max(1, int(round(syn.sweep_n(p) * scale)))
    mesh = syn.random_affine_cube(n, seed=1000 + p)
    x = syn.uniform_vector(mesh.n_dofs(p), seed=2000 + p)
    return n, mesh, x


# Sources of each precision's element kernels (default launch shapes)
KERNEL_SOURCES = {"f64": ("pa_apply.cuh", "pa_apply_f64.cu"),
                  "f32": ("pa_apply_line.cuh", "pa_apply_plane.cuh", "pa_apply_f32.cu")}


def kernel_source_hash(dtype_name: str) -> str:
    """Hash of one precision's element-kernel sources and of its rows of the
    default launch table (the shapes the sweep runs), so stored ncu traffic
    goes stale with them."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2601_08374_gb300", "csrc")
    for f in KERNEL_SOURCES[dtype_name]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "pa_api.cu"), "rb") as fh:
        api = fh.read().decode()
    i = api.index("ApplyLaunch default_apply_launch(")
    tag = dtype_name[1:]  # "64" / "32"
    for line in api[i:api.index("\n}\n", i)].splitlines():
        if line.strip().startswith("static const int") and f"{tag}[" in line:
            h.update(line.strip().encode())
    return h.hexdigest()[:16]


# ncu DRAM bytes (read + write) per launch of the element kernel, keyed by
# (precision, p): one-kernel captures of the sweep's element launches,
# valid only while that precision's kernel sources and launch-table rows
# hash to the stored value.  The E-vector writes mostly stay in L2 and reach
# DRAM during the assembly kernel, so for p >= 4 the figure is essentially
# the reads of x and of the geometry records.
TRAFFIC_HASH = {"f64": "2d363831e8cf3acf", "f32": "fea991816cb21415"}
ELEMENT_KERNEL_NAMES = {0: "pa_apply_flat_kernel", 1: "pa_apply_line_kernel<FUSE=0>", 2: "pa_apply_line_kernel<FUSE=1>",
                        3: "pa_apply_line_kernel<FUSE=1,SPLIT=1>", 4: "pa_apply_tc_kernel (tcgen05 kind::tf32)",
                        5: "pa_apply_plane_kernel<SPLIT=0>", 6: "pa_apply_plane_kernel<SPLIT=1>",
                        7: "pa_apply_line_kernel<FUSE=1,TWO=1>"}
TRAFFIC_BYTES: dict = {
    ("f64", 1): 252023552, ("f64", 2): 61121280, ("f64", 4): 27019008, ("f64", 6): 22349824, ("f64", 8): 22127360,
    ("f32", 1): 96720128, ("f32", 2): 18404608, ("f32", 4): 13148672, ("f32", 6): 11208960, ("f32", 8): 11102720,
}


# Coarse-level solve of the V-cycle: inexact, relative tolerance 1e-2 and at
# most 10 iterations (the paper's coarse-solve setting, Sec. 3.2).
COARSE_RTOL, COARSE_MAXIT = 1e-2, 10
# Chebyshev-Jacobi smoother of the solve rows: degree 4 on [0.05, 1.2] of the
# estimated lambda_max (the library's default interval), the fastest setting
# of the degree / interval sweep (--gmg-sweep); the paper's setting, degree 2
# (Sec. 5.2) on the interval [0.3, 1.2], is kept as one extra beam row
CHEB_ORDER = 4
PAPER_SMOOTHER = (2, 0.3, 1.2)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, out_dir: str = ""):
        self.dev = device_index
        self.proc = None
        # the raw samples: a directory given on the command line, else a
        # temporary file (the JSON line carries their summary either way)
        d = out_dir or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_rank{device_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [t.strip() for t in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, ws: int, device) -> float:
    """The largest x over all ranks (a timing: the job is as slow as its
    slowest rank); the identity for a single process."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gdofs(ws: int, dofs_per_rank_step: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: the dofs every rank applied over the slowest
    rank's time (replicas: each rank runs the same per-GPU workload)."""
    return ws * dofs_per_rank_step * steps / seconds / 1e9


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2601_08374_gb300 as pa

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = pa.PA_FP64 if args.precision == "fp64" else pa.PA_FP32
    dt = torch.float64 if prec == pa.PA_FP64 else torch.float32
    elem = 8 if prec == pa.PA_FP64 else 4
    dtype_name = "f64" if prec == pa.PA_FP64 else "f32"
    lam, mu = syn.lame(1.0, 0.3)
    ps = [int(s) for s in args.ps.split(",")]
    stream = torch.cuda.current_stream()

    cases = []
    for p in ps:
        n, mesh, x = workload(p)
        op = pa.Operator(n, n, n, mesh.affine, p, lam, mu, precision=prec)
        if args.launch:
            v, e, t = (int(a) for a in args.launch.split(","))
            pa.pa_op_set_launch(op.h, v, e, t)
        elif not args.no_autotune:
            pa.pa_op_autotune(op.h, stream)
        xt = torch.tensor(x, dtype=dt, device="cuda")
        yt = torch.empty_like(xt)
        cases.append(dict(p=p, n=n, op=op, x=xt, y=yt, ndofs=op.ndofs, ne=op.nelem, launch=pa.pa_op_get_launch(op.h)))
    total_dofs = sum(c["ndofs"] for c in cases)

    def step():
        for c in cases:
            pa.pa_op_apply(c["op"].h, c["x"], c["y"], stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for c in cases:
        pa.pa_op_profile(c["op"].h, True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device(), args.clocks_dir) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    per_case = []
    for c in cases:
        te, ta, na = pa.pa_op_profile_read(c["op"].h)
        pa.pa_op_profile(c["op"].h, False)
        c["elem_ms"], c["asm_ms"], c["napplies"] = te, ta, na
    ms = max_over_ranks(ms, ws, "cuda")

    # ---- single pair: each operator applied back to back to one x / y
    # (its vectors stay in L2 where they fit), beside the rotating figure;
    # the median over 20 timed repeats of 10 back-to-back applies
    for c in cases:
        pa.pa_op_apply(c["op"].h, c["x"], c["y"], stream)
        reps = []
        for _ in range(20):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(10):
                pa.pa_op_apply(c["op"].h, c["x"], c["y"], stream)
            e1.record(stream)
            e1.synchronize()
            reps.append(e0.elapsed_time(e1) / 10)
        c["single_pair_ms"] = statistics.median(reps)

    # ---- measured FMA rate of the CUDA cores (the ceiling beside the derived one)
    fma_measured = pa.pa_measure_fma_rate(prec, stream)
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    # ---- end to end through the host-buffer C ABI call (pinned buffers)
    hosts = []
    for c in cases:
        xh = c["x"].cpu().pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        hosts.append((xh, yh))
    handles = [c["op"].h for c in cases]
    xs_host = [h[0] for h in hosts]
    ys_host = [h[1] for h in hosts]
    pa.pa_op_apply_host_batch(handles, xs_host, ys_host, stream)
    e2e_steps = max(3, args.steps // 4)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # each step timed on the host clock (the call returns when y is on the
    # host); the median step is the estimate, robust to a stalled host
    step_s = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        pa.pa_op_apply_host_batch(handles, xs_host, ys_host, stream)
        step_s.append(time.perf_counter() - t0)
    e2e_s = statistics.median(step_s) * e2e_steps
    e2e_mean_s = sum(step_s)
    e2e_s = max_over_ranks(e2e_s, ws, "cuda")
    bytes_step = sum(c["ndofs"] * elem for c in cases)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return None

    value = job_gdofs(ws, total_dofs, args.steps, ms * 1e-3)
    # roofline of the dominant kernel (the fused element kernel), aggregated
    # over the sweep: algorithmic flops of all its launches / their event
    # time, against the FMA-unit peak at the clock sampled during the run
    clocks = clk.summary()
    mhz = peak_clock_mhz(clocks)
    peak = derived_peak_tflops(dtype_name, sms, mhz)
    fl_total = sum(flops_per_element(c["p"]) * c["ne"] * c["napplies"] for c in cases)
    el_ms = sum(c["elem_ms"] for c in cases)
    achieved = fl_total / (el_ms * 1e-3) / 1e12
    traffic = None
    if TRAFFIC_HASH.get(dtype_name) == kernel_source_hash(dtype_name):
        tb = [TRAFFIC_BYTES.get((dtype_name, c["p"])) for c in cases]
        if all(t is not None for t in tb):
            traffic = int(sum(tb) / len(tb))
    for c in cases:
        fl = flops_per_element(c["p"]) * c["ne"]
        t_el = c["elem_ms"] / max(c["napplies"], 1)
        t_all = (c["elem_ms"] + c["asm_ms"]) / max(c["napplies"], 1)
        per_case.append({"p": c["p"], "n": c["n"], "ndofs": c["ndofs"],
                         "gdofs": round(c["ndofs"] / (t_all * 1e-3) / 1e9, 4),
                         "element_ms": round(t_el, 4), "assemble_ms": round((c["asm_ms"]) / max(c["napplies"], 1), 4),
                         "tflops_alg": round(fl / (t_el * 1e-3) / 1e12, 4),
                         "frac_alu": round(fl / (t_el * 1e-3) / 1e12 / peak, 4),
                         "hbm_gbs_alg": round(algorithmic_bytes(c["p"], c["n"], elem) / (t_all * 1e-3) / 1e9, 1),
                         "single_pair_gdofs": round(c["ndofs"] / (c["single_pair_ms"] * 1e-3) / 1e9, 4),
                         "single_pair_timing": "median of 20 repeats of 10 back-to-back applies",
                         "launch": list(c["launch"])})
    out = {
        "metric": METRIC,
        "value": round(value, 4),
        "unit": "GDoF/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": dtype_name,
        "data": "synthetic",
        "config": {
            "workload": sweep_workload_name(args.precision, ps),
            "l2": ("inputs larger than L2: each step applies 5 operators in turn; one step touches "
                   f"{sum(c['ndofs'] * elem * 2 + c['ne'] * 12 * elem + c['ne'] * 3 * (c['p'] + 1) ** 3 * elem for c in cases) / 1e9:.2f} GB"),
            "parallelism": f"replicas x{ws}",
        },
        "per_p": per_case,
        "roofline": {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": " + ".join(ELEMENT_KERNEL_NAMES[v] for v in sorted({c["launch"][0] for c in cases})),
                     "peak_source": (f"derived: {sms} SMs x {FLOP_PER_CLK_SM[dtype_name]:.0f} {dtype_name} flop/clk/SM "
                                     f"x {mhz:.0f} MHz (median SM clock sampled during the timed region)"),
                     "measured_fma_peak": round(fma_measured, 4),
                     "frac_of_measured_fma_peak": round(achieved / fma_measured, 4),
                     "measured_peak_source": "pa_measure_fma_rate: independent FMA chains on every SM, best of 5"},
        "e2e": {"value": round(job_gdofs(ws, total_dofs, e2e_steps, e2e_s), 4), "unit": "GDoF/s",
                "h2d_bytes_per_step": bytes_step, "d2h_bytes_per_step": bytes_step,
                "api": "pa_op_apply_host_batch (the step's operators from pinned host buffers, copies "
                       "overlapped with the applies)", "steps": e2e_steps,
                "estimate": "median step time (host clock)",
                "mean_steps_value": round(ws * total_dofs * e2e_steps / e2e_mean_s / 1e9, 4)},
        "gpu_launches": 2 * len(cases) * args.steps,
        "clocks": clocks,
    }
    if not args.no_solve:
        out["solve"] = run_solves(args, pa, torch)
    if args.batch_ops > 0:
        out["batched_apply"] = run_batched_apply(args, pa, torch)
    if args.serve_requests > 0:
        out["serving"] = run_serving(args, pa, torch)
    if args.precision == "fp64" and not args.no_fp32:
        out["fp32_sweep"] = run_fp32_sweep(args, pa, torch, sms, mhz)
    if args.ablation_ps:
        out["ablation"] = run_ablation(args, pa, torch)
    if not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(ps, args)
    print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    for c in cases:
        c["op"].close()
    return out


def run_solves(args, pa, torch):
    """GMG-PCG solves/s: the cantilever beam (32x4x4 elements, p = 4 -> 2 -> 1,
    FP64 and mixed; also with two h-levels under the p-levels), the beam
    refined once more (64x8x8) with and without three h-levels, and the
    near-incompressible random-affine cubes (~8M dofs, p = 6 and 8, FP64
    and mixed).  Setup (operators, diagonals,
    eigenvalue estimates, graph capture on the first solve) is untimed."""
    out = []
    beam = syn.box_mesh(32, 4, 4, hi=(8.0, 1.0, 1.0))
    cases = [dict(key="beam", name="beam 32x4x4 p=4 (4->2->1) E=1 nu=0.3 f=(0,0,-1), x=0 clamped", mesh=beam,
                  p=4, levels=[4, 2, 1], nu=0.3, modes=None, f0=(0.0, 0.0, -1.0), reps=args.solve_reps),
             dict(key="beam2mat", name="two-material beam 32x4x4 p=4 (4->2->1): lambda=mu=50 for x<4, lambda=mu=1 beyond; "
                       "traction (0,0,-1e-2) on x=8, x=0 clamped (the paper's benchmark physics)", mesh=beam,
                  p=4, levels=[4, 2, 1], nu=None, mat=syn.two_material(beam, 4.0), modes=None, f0=(0.0, 0.0, 0.0),
                  traction=(1, (0.0, 0.0, -1e-2)), reps=args.solve_reps),
             dict(key="beamh", name="beam 32x4x4 p=4 (4->2->1, then h-levels 16x2x2 and 8x1x1 at p=1) E=1 nu=0.3 f=(0,0,-1), "
                       "x=0 clamped", mesh=beam, p=4, levels=[4, 2, 1], h=2, nu=0.3, modes=None,
                  f0=(0.0, 0.0, -1.0), reps=args.solve_reps)]
    cases.append(dict(key="beam_paper", name="beam 32x4x4 p=4 (4->2->1) as above, with the paper's smoother setting: "
                           "Chebyshev degree 2 on [0.3, 1.2] lambda_max", mesh=beam, p=4, levels=[4, 2, 1], nu=0.3,
                      modes=None, f0=(0.0, 0.0, -1.0), reps=args.solve_reps, smoother=PAPER_SMOOTHER))
    cases.append(dict(key="beam_c1", name="beam 32x4x4 p=4 (4->2->1) as above, coarse solve capped at one PCG "
                           "iteration (instead of the paper's 1e-2 / at most 10)", mesh=beam, p=4, levels=[4, 2, 1],
                      nu=0.3, modes=None, f0=(0.0, 0.0, -1.0), reps=args.solve_reps, coarse=(COARSE_RTOL, 1),
                      solve_modes=("fp64", "mixed_fcg")))
    beam2 = syn.box_mesh(64, 8, 8, hi=(8.0, 1.0, 1.0))
    for h in (0, 3):
        cases.append(dict(key="beam64h" if h else "beam64",
                          name=f"beam 64x8x8 p=4 (4->2->1{', then 3 h-levels to 8x1x1' if h else ''}) E=1 nu=0.3 "
                               "f=(0,0,-1), x=0 clamped", mesh=beam2, p=4, levels=[4, 2, 1], h=h, nu=0.3, modes=None,
                          f0=(0.0, 0.0, -1.0), reps=args.solve_reps, solve_modes=("fp64", "mixed_fcg")))
    if not args.quick_solves:
        for p, n in ((6, syn.mixed_n(6)), (8, syn.mixed_n(8))):
            lv = [p, p // 2, 1] if p == 6 else [8, 4, 2, 1]
            cases.append(dict(key=f"cube{p}", name=f"cube {n}^3 p={p} random affine maps nu=0.45 smooth force, x=0 clamped",
                              mesh=syn.random_affine_cube(n, seed=3000 + p), p=p, levels=lv, nu=0.45,
                              modes=syn.smooth_force_modes(seed=3100 + p), f0=(0.0, 0.0, 0.0), reps=max(1, args.solve_reps // 2)))
        cases.append(dict(key="cube6_c1", name=f"cube {syn.mixed_n(6)}^3 p=6 as above, coarse solve capped at one PCG "
                               "iteration", mesh=syn.random_affine_cube(syn.mixed_n(6), seed=3006), p=6, levels=[6, 3, 1],
                          nu=0.45, modes=syn.smooth_force_modes(seed=3106), f0=(0.0, 0.0, 0.0),
                          reps=max(1, args.solve_reps // 2), coarse=(COARSE_RTOL, 1), solve_modes=("mixed_ir",)))
    if args.solve_cases:
        keep = set(args.solve_cases.split(","))
        cases = [c for c in cases if c["key"] in keep]
    eager = args.solve_eager_maxit > 0
    cap = args.solve_eager_maxit if eager else 1000
    for c in cases:
        m, p = c["mesh"], c["p"]
        lam, mu = syn.lame(1.0, c["nu"]) if c["nu"] is not None else (0.0, 0.0)
        ess = syn.clamp_mask(m, p)
        op = pa.Operator(m.nx, m.ny, m.nz, m.affine, p, lam, mu, ess_mask=ess, mat=c.get("mat"))
        b = op.rhs(f0=c["f0"], modes=c["modes"], traction=c.get("traction"))
        h = c.get("h", 0)
        row = {"case": c["name"], "ndofs": op.ndofs, "levels": c["levels"], "h_levels": h, "rtol": 1e-10,
               "smoother": list(c.get("smoother", (CHEB_ORDER, 0.05, 1.2))),
               "coarse_rtol_maxit": list(c.get("coarse", (COARSE_RTOL, COARSE_MAXIT)))}
        sols = {}
        for mode, key in ((pa.PA_SOLVE_FP64, "fp64"), (pa.PA_SOLVE_MIXED, "mixed_ir"), (pa.PA_SOLVE_MIXED_FCG, "mixed_fcg")):
            if key not in c.get("solve_modes", ("fp64", "mixed_ir", "mixed_fcg")):
                continue
            if args.solve_modes and key not in args.solve_modes.split(","):
                continue
            crtol, cmax = c.get("coarse", (COARSE_RTOL, COARSE_MAXIT))
            k, lo, hi = c.get("smoother", (CHEB_ORDER, 0.05, 1.2))
            s = pa.pa_solver_create_hp(op.h, c["levels"], h, k, crtol, cmax, mode)
            pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_CHEB_LOWER, lo)
            pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_CHEB_UPPER, hi)
            if eager:
                pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_GRAPHS, 0)
            x = torch.zeros_like(b)
            code, info = pa.pa_gmg_pcg_solve(s, b, x, 1e-10, cap)  # warm-up (captures the graphs)
            times = []
            for _ in range(c["reps"]):
                x.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                code, info = pa.pa_gmg_pcg_solve(s, b, x, 1e-10, cap)
                times.append(time.perf_counter() - t0)
            sols[key] = x.clone()
            row[key] = {"status": int(code), "solves_per_s": round(1.0 / statistics.median(times), 3),
                        "median_s": round(statistics.median(times), 5), "iterations": info.iterations,
                        "coarse_iterations": info.coarse_iterations,
                        "true_rel_residual": float(f"{info.rel_residual:.3e}"),
                        "tolerance_met": int(info.tolerance_met)}
            if mode == pa.PA_SOLVE_MIXED:
                row[key]["refinements"] = info.refinements
            pa.pa_solver_destroy(s)
        for key in ("mixed_ir", "mixed_fcg"):
            if key not in sols or "fp64" not in sols:
                continue
            d = (sols[key] - sols["fp64"]).norm() / sols["fp64"].norm()
            row[key]["rel_diff_vs_fp64"] = float(f"{float(d):.3e}")
            row[key]["speedup_over_fp64"] = round(row[key]["solves_per_s"] / row["fp64"]["solves_per_s"], 3)
        out.append(row)
        op.close()
    return out


def run_batched_apply(args, pa, torch):
    """Many small operators (the sizes of the served requests' fine levels,
    p in {2,4,6,8}, n^3 with n in 4..8, FP32) applied one launch pair each
    versus one batched launch pair per degree."""
    rng = np.random.default_rng(77)
    ops, xs, ys = [], [], []
    for k in range(args.batch_ops):
        p = int(rng.choice([2, 4, 6, 8]))
        n = int(rng.integers(4, 9))
        m = syn.random_affine_cube(n, seed=5000 + k)
        op = pa.Operator(n, n, n, m.affine, p, 1.0, 0.5, precision=pa.PA_FP32)
        x = torch.tensor(syn.uniform_vector(op.ndofs, seed=k), dtype=torch.float32, device="cuda")
        ops.append(op)
        xs.append(x)
        ys.append(torch.empty_like(x))
    stream = torch.cuda.current_stream()
    handles = [o.h for o in ops]
    dofs = sum(o.ndofs for o in ops)

    def one_by_one():
        for o, x, y in zip(ops, xs, ys):
            pa.pa_op_apply(o.h, x, y, stream)

    def batched():
        pa.pa_op_apply_batch(handles, xs, ys, stream)

    res = {}
    for name, fn in (("individual", one_by_one), ("batched", batched)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.batch_reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.batch_reps
        res[name] = {"ms": round(ms, 4), "gdofs": round(dofs / (ms * 1e-3) / 1e9, 3)}
    for o in ops:
        o.close()
    res["operators"] = args.batch_ops
    res["total_dofs"] = dofs
    res["speedup"] = round(res["individual"]["ms"] / res["batched"]["ms"], 3)
    return res


def serving_requests(pa, count, seed):
    """The served stream: p uniform in {2,4,6,8}; a cube n^3 (n ~ U{8..32}) or
    an 8:1:1 beam (8k x k x k, k ~ U{4..16}); E log-uniform in [0.1, 10];
    nu ~ U[0.2, 0.45]; 3 seeded sine modes of body force per component;
    clamped at x = 0; mixed-precision solve (FP64 flexible CG, FP32 V-cycle)
    to 1e-10."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        p = int(rng.choice([2, 4, 6, 8]))
        if rng.random() < 0.5:
            n = int(rng.integers(8, 33))
            dims, box = (n, n, n), (0, 0, 0, 1.0, 1.0, 1.0)
        else:
            kk = int(rng.integers(4, 17))
            dims, box = (8 * kk, kk, kk), (0, 0, 0, 8.0, 1.0, 1.0)
        E = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
        nu = float(rng.uniform(0.2, 0.45))
        modes = syn.smooth_force_modes(seed=int(rng.integers(1 << 30)))
        out.append(pa.make_request(*dims, box, p, E, nu, modes=modes, rtol=1e-10, maxit=1000,
                                   mode=pa.PA_SOLVE_MIXED_FCG, keep_solution=False))
    return out


def ua_geometry_timing(pa, torch, c, stream, reps=20):
    """Element-kernel time of one FP32 plane-kernel operator with the stored
    geometry records and with UA geometry (J only, J^-1 and detJ recomputed
    in the kernel), measured the same way: warm-up, then `reps` back-to-back
    applies of the same x / y with per-launch CUDA events."""
    op = c["op"]
    out = {"p": c["p"], "launch": list(pa.pa_op_get_launch(op.h)),
           "geometry_bytes_stored": int(c["ne"] * 12 * 4), "geometry_bytes_ua": int(c["ne"] * 9 * 4)}
    for mode, key in ((pa.PA_GEOMETRY_STORED, "element_ms_stored"), (pa.PA_GEOMETRY_UA, "element_ms_ua")):
        pa.pa_op_set_geometry_mode(op.h, mode)
        for _ in range(3):
            pa.pa_op_apply(op.h, c["x"], c["y"], stream)
        pa.pa_op_profile(op.h, True)
        for _ in range(reps):
            pa.pa_op_apply(op.h, c["x"], c["y"], stream)
        te, _, na = pa.pa_op_profile_read(op.h)
        pa.pa_op_profile(op.h, False)
        out[key] = round(te / max(na, 1), 5)
    pa.pa_op_set_geometry_mode(op.h, pa.PA_GEOMETRY_STORED)
    out["ua_over_stored"] = round(out["element_ms_ua"] / out["element_ms_stored"], 4)
    return out


def run_fp32_sweep(args, pa, torch, sms, mhz):
    """The same operator sweep in FP32 (the apply of the mixed-precision
    solves): GDoF/s per p and over the sweep, with the element kernel's
    algorithmic FP32 rate against the derived FP32 peak.  Same workloads,
    timing and L2 rule as the FP64 line."""
    lam, mu = syn.lame(1.0, 0.3)
    stream = torch.cuda.current_stream()
    cases = []
    for p in [int(v) for v in args.ps.split(",")]:
        n, mesh, x = workload(p)
        op = pa.Operator(n, n, n, mesh.affine, p, lam, mu, precision=pa.PA_FP32)
        if not args.no_autotune:
            pa.pa_op_autotune(op.h, stream)
        xt = torch.tensor(x, dtype=torch.float32, device="cuda")
        cases.append(dict(p=p, op=op, x=xt, y=torch.empty_like(xt), ndofs=op.ndofs, ne=op.nelem,
                          launch=pa.pa_op_get_launch(op.h)))
    for _ in range(args.warmup):
        for c in cases:
            pa.pa_op_apply(c["op"].h, c["x"], c["y"], stream)
    for c in cases:
        pa.pa_op_profile(c["op"].h, True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(3, args.steps)
    e0.record(stream)
    for _ in range(steps):
        for c in cases:
            pa.pa_op_apply(c["op"].h, c["x"], c["y"], stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    peak = derived_peak_tflops("f32", sms, mhz)
    fma_measured = pa.pa_measure_fma_rate(pa.PA_FP32, stream)
    fma2_measured = pa.pa_measure_fma_rate(pa.PA_FMA_FP32X2, stream)
    per_p, fl_tot, el_tot = [], 0.0, 0.0
    ua = []
    for c in cases:
        te, ta, na = pa.pa_op_profile_read(c["op"].h)
        pa.pa_op_profile(c["op"].h, False)
        if c["p"] <= 2 and c["launch"][0] == 5:
            ua.append(ua_geometry_timing(pa, torch, c, stream))
        fl = flops_per_element(c["p"]) * c["ne"]
        fl_tot += fl * na
        el_tot += te
        per_p.append({"p": c["p"], "gdofs": round(c["ndofs"] / ((te + ta) / na * 1e-3) / 1e9, 3),
                      "frac_alu": round(fl / (te / na * 1e-3) / 1e12 / peak, 4), "launch": list(c["launch"])})
        c["op"].close()
    return {"value": round(sum(c["ndofs"] for c in cases) * steps / (ms * 1e-3) / 1e9, 4), "unit": "GDoF/s",
            "dtype": "f32", "element_kernel_tflops_alg": round(fl_tot / (el_tot * 1e-3) / 1e12, 3),
            "frac_of_derived_fp32_peak": round(fl_tot / (el_tot * 1e-3) / 1e12 / peak, 4),
            "derived_fp32_peak_tflops": round(peak, 3), "measured_fp32_fma_peak_tflops": round(fma_measured, 3),
            "measured_fp32_paired_fma_peak_tflops": round(fma2_measured, 3),
            "frac_of_measured_fp32_peak": round(fl_tot / (el_tot * 1e-3) / 1e12 / fma_measured, 4), "per_p": per_p,
            "ua_geometry": ua}


def run_ablation(args, pa, torch):
    """The paper's optimisation stack (Table 8) stage by stage on the GPU, FP64,
    on the sweep's workloads: baseline (two kernels, Q values through HBM,
    dense O(p^6) contractions, 81-term stress), + sum factorisation, + Voigt,
    + fusion (the production kernel).  Median of CUDA-event-timed applies
    (element kernels and assembly) per stage."""
    out = []
    for p in [int(v) for v in args.ablation_ps.split(",")]:
        n, mesh, x = workload(p)
        lam, mu = syn.lame(1.0, 0.3)
        op = pa.Operator(n, n, n, mesh.affine, p, lam, mu)
        xt = torch.tensor(x, dtype=torch.float64, device="cuda")
        y = torch.empty_like(xt)
        st = torch.cuda.current_stream()
        row = {"p": p, "n": n, "ndofs": op.ndofs}
        ms = {}
        for stage in range(4):
            pa.pa_op_apply_stage(op.h, stage, xt, y)  # first use allocates the stage's buffers
            times = []
            for _ in range(args.ablation_reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                pa.pa_op_apply_stage(op.h, stage, xt, y)
                e1.record(st)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            ms[stage] = statistics.median(times)
        names = ["baseline", "+sumfact", "+voigt", "+fusion"]
        for stage in range(4):
            row[names[stage]] = {"ms": round(ms[stage], 4), "gdofs": round(op.ndofs / (ms[stage] * 1e-3) / 1e9, 4),
                                 "speedup_vs_baseline": round(ms[0] / ms[stage], 2)}
        out.append(row)
        op.close()
    return {"dtype": "f64", "recipe": "sweep workloads (n^3 unit cube, random affine elements, E=1 nu=0.3), "
            "unconstrained; each stage's time includes its element kernels and the assembly", "per_p": out}


def small_requests(pa, count, seed):
    """A burst of small solves (the batch lane's workload): p uniform in
    {2,4,6,8}, cube n^3 with n ~ U{3..8}, otherwise the served stream's
    recipe."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        p = int(rng.choice([2, 4, 6, 8]))
        n = int(rng.integers(3, 9))
        E = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
        nu = float(rng.uniform(0.2, 0.45))
        modes = syn.smooth_force_modes(seed=int(rng.integers(1 << 30)))
        out.append(pa.make_request(n, n, n, (0, 0, 0, 1.0, 1.0, 1.0), p, E, nu, modes=modes, rtol=1e-10, maxit=1000,
                                   mode=pa.PA_SOLVE_MIXED_FCG, keep_solution=False))
    return out


def run_serving(args, pa, torch):
    """Continuous-admission serving of a Poisson stream.  A calibration burst
    of the first requests is solved twice, all submitted at once: in plain
    FP64 with one slot and no batching (the FP64-alone capacity) and in the
    served form (mixed precision, several slots, small solves in the lockstep
    batch lane).  The Poisson arrival rate is a fraction of the served
    capacity.  Reports p50/p99 latency (submit to completion) and completed
    solves/s, the calibration burst again with h-levels off (p-levels
    only), and a burst of small solves served with and without the batch
    lane."""
    import threading
    reqs = serving_requests(pa, args.serve_requests, seed=4242)
    budget = int(args.serve_budget_gb * (1 << 30))
    ncal = min(len(reqs), args.serve_calibration)

    def burst(rs, slots, batch=1, h_levels=1):
        srv = pa.pa_server_create(budget, slots)
        pa.pa_server_set_option(srv, pa.PA_SERVER_OPT_BATCH, batch)
        pa.pa_server_set_option(srv, pa.PA_SERVER_OPT_H_LEVELS, h_levels)
        t0 = time.perf_counter()
        ts = [pa.pa_server_submit(srv, r) for r in rs]
        res = [pa.pa_server_wait(srv, t) for t in ts]
        dt = time.perf_counter() - t0
        st = pa.pa_server_stats(srv)
        pa.pa_server_destroy(srv)
        st.mean_setup_s = float(np.mean([r[2].setup_s for r in res]))
        st.mean_solve_s = float(np.mean([r[2].solve_s for r in res]))
        return len(rs) / dt, sum(1 for r in res if r[0] == pa.PA_OK), st

    fp64_reqs = []
    for r in reqs[:ncal]:
        r2 = pa.pa_request.from_buffer_copy(r)
        r2.mode = pa.PA_SOLVE_FP64
        fp64_reqs.append(r2)
    fp64_cap, fp64_ok, _ = burst(fp64_reqs, 1, batch=0)
    cap, cal_ok, _ = burst(reqs[:ncal], args.serve_slots)
    cap_noh, noh_ok, _ = burst(reqs[:ncal], args.serve_slots, h_levels=0)
    small = small_requests(pa, args.serve_small, seed=99)
    small_off, small_off_ok, st_off = burst(small, args.serve_slots, batch=0)
    small_on, small_on_ok, st_small = burst(small, args.serve_slots, batch=1)
    small_off_noh, _, _ = burst(small, args.serve_slots, batch=0, h_levels=0)
    small_on_noh, _, st_small_noh = burst(small, args.serve_slots, batch=1, h_levels=0)
    rate = args.serve_load * cap
    arrivals = np.cumsum(np.random.default_rng(7).exponential(1.0 / rate, size=len(reqs)))

    def stream(batch):
        """The Poisson stream through a fresh server (lane on or off)."""
        srv = pa.pa_server_create(budget, args.serve_slots)
        pa.pa_server_set_option(srv, pa.PA_SERVER_OPT_BATCH, batch)
        tickets = [None] * len(reqs)
        start = time.perf_counter()

        def submitter():
            for i, r in enumerate(reqs):
                delay = arrivals[i] - (time.perf_counter() - start)
                if delay > 0:
                    time.sleep(delay)
                tickets[i] = pa.pa_server_submit(srv, r)

        th = threading.Thread(target=submitter)
        th.start()
        res = {"lat": [], "status": [], "iters": [], "solve_s": [], "hlev": []}
        for i in range(len(reqs)):
            while tickets[i] is None:
                time.sleep(0.001)
            code, info, tm, _ = pa.pa_server_wait(srv, tickets[i])
            res["status"].append(code)
            res["lat"].append(tm.latency_s)
            res["iters"].append(info.iterations)
            res["solve_s"].append(tm.solve_s)
            res["hlev"].append(tm.h_levels)
        th.join()
        res["wall"] = time.perf_counter() - start
        res["stats"] = pa.pa_server_stats(srv)
        pa.pa_server_destroy(srv)
        return res

    off = stream(0) if args.serve_lane_off else None
    on = stream(1)
    lat, statuses, iters, solve_s, hlev = on["lat"], on["status"], on["iters"], on["solve_s"], on["hlev"]
    wall, st = on["wall"], on["stats"]
    lat = np.array(lat)
    return {"requests": len(reqs), "slots": args.serve_slots, "budget_gb": args.serve_budget_gb,
            "calibration_requests": ncal,
            "fp64_alone_solves_per_s": round(fp64_cap, 3),
            "served_burst_solves_per_s": round(cap, 3),
            "served_over_fp64_alone": round(cap / fp64_cap, 3),
            "served_burst_solves_per_s_h_levels_off": round(cap_noh, 3),
            "h_levels_speedup": round(cap / cap_noh, 3),
            "arrival_rate_per_s": round(rate, 3), "load_fraction": args.serve_load,
            "solves_per_s": round(len(reqs) / wall, 3),
            "p50_latency_s": round(float(np.percentile(lat, 50)), 4),
            "p99_latency_s": round(float(np.percentile(lat, 99)), 4),
            "mean_solve_s": round(float(np.mean(solve_s)), 4), "mean_iterations": round(float(np.mean(iters)), 1),
            "requests_with_h_levels": int(sum(1 for h in hlev if h > 0)),
            "ok": int(sum(1 for c in statuses if c == pa.PA_OK)),
            "calibration_ok": [fp64_ok, cal_ok, noh_ok],
            "p99_over_p50": round(float(np.percentile(lat, 99) / np.percentile(lat, 50)), 3),
            "batch_lane": {"batched": int(st.batched), "ticks": int(st.batch_ticks),
                           "mean_members_per_tick": round(st.batch_member_ticks / max(st.batch_ticks, 1), 2),
                           "max_members": int(st.batch_max_members)},
            "lane_off": None if off is None else {
                "solves_per_s": round(len(reqs) / off["wall"], 3),
                "p50_latency_s": round(float(np.percentile(off["lat"], 50)), 4),
                "p99_latency_s": round(float(np.percentile(off["lat"], 99)), 4),
                "p99_over_p50": round(float(np.percentile(off["lat"], 99) / np.percentile(off["lat"], 50)), 3),
                "ok": int(sum(1 for c in off["status"] if c == pa.PA_OK))},
            "small_burst": {"requests": len(small), "recipe": "p U{2,4,6,8}; cube n^3, n ~ U{3..8}; mixed precision",
                            "solves_per_s_lane_off": round(small_off, 3), "solves_per_s_lane_on": round(small_on, 3),
                            "lane_speedup": round(small_on / small_off, 3), "ok": [small_off_ok, small_on_ok],
                            "h_levels_off": {"solves_per_s_lane_off": round(small_off_noh, 3),
                                             "solves_per_s_lane_on": round(small_on_noh, 3),
                                             "lane_speedup": round(small_on_noh / small_off_noh, 3),
                                             "mean_members_per_tick": round(st_small_noh.batch_member_ticks
                                                                            / max(st_small_noh.batch_ticks, 1), 2)},
                            "mean_setup_s_off_on": [round(st_off.mean_setup_s, 4), round(st_small.mean_setup_s, 4)],
                            "mean_solve_s_off_on": [round(st_off.mean_solve_s, 4), round(st_small.mean_solve_s, 4)],
                            "mean_members_per_tick": round(st_small.batch_member_ticks / max(st_small.batch_ticks, 1), 2),
                            "max_members": int(st_small.batch_max_members)},
            "peak_used_gb": round(st.peak_used_bytes / (1 << 30), 2),
            "recipe": "Poisson arrivals; p U{2,4,6,8}; cube n^3 n~U{8..32} or beam 8k x k x k k~U{4..16}; "
                      "E log-U[0.1,10]; nu U[0.2,0.45]; 3 sine modes/component; x=0 clamped; FP64 flexible CG with an "
                      "FP32 V-cycle (mixed precision), rtol 1e-10"}


def _lanczos_extremes(pa, torch, op, ess, steps=80):
    """Extreme eigenvalues of D^-1 A (through the symmetric D^-1/2 A D^-1/2)
    from `steps` Lanczos steps with full reorthogonalisation, using the
    operator's apply and diagonal (a check of the smoother's power-iteration
    estimate; not part of any solve)."""
    dis = op.diag().rsqrt()
    g = torch.Generator(device="cuda").manual_seed(0)
    v = torch.rand(op.ndofs, dtype=torch.float64, device="cuda", generator=g) - 0.5
    if ess is not None:
        v[torch.tensor(ess, device="cuda").bool()] = 0.0
    v /= v.norm()
    basis, alpha, beta = [v], [], []
    vprev, b = torch.zeros_like(v), 0.0
    for _ in range(steps):
        w = dis * op.apply(dis * v)
        a = float(torch.dot(w, v))
        alpha.append(a)
        w = w - a * v - b * vprev
        for u in basis:
            w -= torch.dot(w, u) * u
        b = float(w.norm())
        if b < 1e-14:
            break
        beta.append(b)
        vprev, v = v, w / b
        basis.append(v)
    n = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:n - 1], 1) + np.diag(beta[:n - 1], -1)
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])


def run_gmg_sweep(args):
    """Diagnosis of the GMG-PCG iteration counts (--gmg-sweep): for the beam
    (32x4x4, p = 4, nu = 0.3) and the nu = 0.45 random-affine cubes (p = 6
    and 8), the power-iteration lambda_max of every smoothed level beside an
    80-step Lanczos estimate of the extreme eigenvalues of D^-1 A, and the
    iterations and solve time for Chebyshev degrees k and target intervals
    [lo, hi] * lambda_max, for the first-kind Chebyshev smoother and the
    fourth-kind one (upper end only)."""
    import torch

    import paper_2601_08374_gb300 as pa
    torch.cuda.set_device(0)
    out = {"cases": []}
    beam = syn.box_mesh(32, 4, 4, hi=(8.0, 1.0, 1.0))
    cases = [("beam 32x4x4 p=4 nu=0.3", beam, 4, [4, 2, 1], 0.3, None, (0.0, 0.0, -1.0),
              [pa.PA_SOLVE_FP64, pa.PA_SOLVE_MIXED_FCG])]
    for p in (6, 8):
        n = syn.mixed_n(p)
        cases.append((f"cube {n}^3 p={p} nu=0.45 random affine", syn.random_affine_cube(n, seed=3000 + p), p,
                      [6, 3, 1] if p == 6 else [8, 4, 2, 1], 0.45, syn.smooth_force_modes(seed=3100 + p),
                      (0.0, 0.0, 0.0), [pa.PA_SOLVE_MIXED_FCG]))
    ks = [int(v) for v in args.gmg_sweep_k.split(",")]
    intervals = [tuple(float(t) for t in iv.split(":")) for iv in args.gmg_sweep_intervals.split(",")]
    kinds = [int(v) for v in args.gmg_sweep_kinds.split(",")]
    lo_min = min(lo for lo, _ in intervals)
    for name, m, p, lv, nu, modes, f0, solve_modes in cases:
        lam, mu = syn.lame(1.0, nu)
        ess = syn.clamp_mask(m, p)
        op = pa.Operator(m.nx, m.ny, m.nz, m.affine, p, lam, mu, ess_mask=ess)
        b = op.rhs(f0=f0, modes=modes)
        row = {"case": name, "levels": lv, "lambda": [], "sweep": []}
        s = pa.pa_solver_create(op.h, lv, 2, COARSE_RTOL, COARSE_MAXIT, pa.PA_SOLVE_FP64)
        x = torch.zeros_like(b)
        _, info = pa.pa_gmg_pcg_solve(s, b, x, 1e-10, 2000)
        pa.pa_solver_destroy(s)
        for li, pl in enumerate(lv[:-1]):
            el = syn.clamp_mask(m, pl)
            o2 = pa.Operator(m.nx, m.ny, m.nz, m.affine, pl, lam, mu, ess_mask=el)
            lmin, lmax = _lanczos_extremes(pa, torch, o2, el)
            o2.close()
            row["lambda"].append({"p": pl, "power10": round(info.lambda_max[li], 4), "lanczos_max": round(lmax, 4),
                                  "lanczos_min": float(f"{lmin:.4e}")})
        for mode in solve_modes:
            for k in ks:
                s = pa.pa_solver_create(op.h, lv, k, COARSE_RTOL, COARSE_MAXIT, mode)
                for kind in kinds:
                    pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_CHEB_KIND, kind)
                    # the fourth kind has no lower end: one row per upper end
                    ivs = intervals if kind == 1 else [(lo_min, hi) for hi in sorted({hi for _, hi in intervals})]
                    for lo, hi in ivs:
                        pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_CHEB_LOWER, lo)
                        pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_CHEB_UPPER, hi)
                        pa.pa_gmg_pcg_solve(s, b, x.zero_(), 1e-10, 2000)  # captures the graphs
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        code, info = pa.pa_gmg_pcg_solve(s, b, x.zero_(), 1e-10, 2000)
                        dt = time.perf_counter() - t0
                        row["sweep"].append({"mode": {0: "fp64", 2: "mixed_fcg"}[mode], "kind": kind, "k": k,
                                             "lo": lo if kind == 1 else 0.0, "hi": hi,
                                             "iterations": info.iterations, "status": int(code), "s": round(dt, 4),
                                             "rho": round(info.rel_residual ** (1.0 / max(info.iterations, 1)), 4)})
                pa.pa_solver_destroy(s)
        out["cases"].append(row)
        op.close()
    print(json.dumps(out), flush=True)
    return out


def _oracle_sweep(ps, scale, per_p=None):
    import oracle
    lam, mu = syn.lame(1.0, 0.3)
    dofs, secs = 0, 0.0
    for p in ps:
        n, mesh, x = workload(p, scale)
        oracle.ref(p)  # reference blocks built outside the timing
        t0 = time.perf_counter()
        oracle.apply(p, n, n, n, mesh.affine, lam, mu, x)
        dt = time.perf_counter() - t0
        secs += dt
        dofs += mesh.n_dofs(p)
        if per_p is not None:
            per_p.append({"p": p, "n": n, "ndofs": mesh.n_dofs(p), "s": round(dt, 4),
                          "gdofs": round(mesh.n_dofs(p) / dt / 1e9, 6)})
    return dofs, secs


def cpu_baseline(ps, args):
    """The plain FP64 oracle timed on the host cores: the operator sweep at
    full size (one step, per degree as well), the 4^3 p = 2 clamped cube of
    the small apply configuration, and the direct solve of the cantilever
    beam (32x4x4, p = 4: sparse LU of the assembled matrix plus one
    refinement step) that the GPU solves are gated against."""
    import oracle
    per_p = []
    dofs, secs = _oracle_sweep(ps, 1.0, per_p)
    out = {"value": round(dofs / secs / 1e9, 6), "unit": "GDoF/s", "cores": oracle.max_threads(), "kind": "oracle",
           "sample": "one full step: the oracle's element-matrix apply for every p of the sweep at full size, "
                     "FP64, OpenMP over elements", "per_p": per_p}
    # the small apply configuration (4^3 unit cube, p = 2, x = 0 clamped)
    m = syn.box_mesh(4, 4, 4)
    lam, mu = syn.lame(1.0, 0.3)
    ess = syn.clamp_mask(m, 2)
    x = syn.uniform_vector(m.n_dofs(2), seed=0)
    oracle.apply(2, 4, 4, 4, m.affine, lam, mu, x, ess=ess)
    reps, t0 = 0, time.perf_counter()
    while reps < 10 or time.perf_counter() - t0 < 0.5:
        oracle.apply(2, 4, 4, 4, m.affine, lam, mu, x, ess=ess)
        reps += 1
    dt = (time.perf_counter() - t0) / reps
    out["config_small_cube_apply"] = {"ndofs": m.n_dofs(2), "s_per_apply": round(dt, 6),
                                      "gdofs": round(m.n_dofs(2) / dt / 1e9, 6), "reps": reps}
    if not args.no_oracle_solve:
        beam = syn.box_mesh(32, 4, 4, hi=(8.0, 1.0, 1.0))
        ess = syn.clamp_mask(beam, 4)
        b = oracle.load(4, 32, 4, 4, beam.affine, f0=(0.0, 0.0, -1.0), ess=ess)
        t0 = time.perf_counter()
        _, res = oracle.solve_sparse(4, 32, 4, 4, beam.affine, lam, mu, b, ess)
        dt = time.perf_counter() - t0
        out["beam_solve"] = {"ndofs": len(b), "s": round(dt, 3), "solves_per_s": round(1.0 / dt, 5),
                             "rel_residual": float(f"{res:.3e}"),
                             "method": "assembly of the element matrices, sparse LU (scipy SuperLU, one thread), "
                                       "one refinement step with the element-by-element apply"}
    return out


def run_reference(args):
    ws, rank, local = dist_setup()
    if rank != 0:
        return None
    import oracle
    ps = [int(s) for s in args.ps.split(",")]
    for _ in range(args.warmup):
        _oracle_sweep(ps, 1.0)
    dofs, secs = 0, 0.0
    for _ in range(args.steps):
        d, s = _oracle_sweep(ps, 1.0)
        dofs += d
        secs += s
    v = dofs / secs / 1e9
    sample = ("each step: the oracle's element-matrix apply for every p of the sweep at full size (the GPU "
              "arm's step), FP64, OpenMP over elements")
    out = {"metric": METRIC, "value": round(v, 6), "unit": "GDoF/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": sweep_workload_name("fp64", ps),
                      "parallelism": "host cores"},
           "cpu_baseline": {"value": round(v, 6), "unit": "GDoF/s", "cores": oracle.max_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(v, 6), "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--ps", default=",".join(map(str, SWEEP)))
    ap.add_argument("--gmg-sweep", action="store_true",
                    help="diagnose the GMG-PCG iteration counts (eigenvalue estimates, Chebyshev degree/interval sweep) "
                         "instead of the benchmark")
    ap.add_argument("--gmg-sweep-k", default="1,2,3,4,5,6")
    ap.add_argument("--gmg-sweep-kinds", default="1,4", help="Chebyshev kinds of the sweep (1: first kind on "
                    "[lo, hi] * lambda_max, 4: fourth kind on [0, hi * lambda_max])")
    ap.add_argument("--gmg-sweep-intervals", default="0.3:1.2,0.1:1.2,0.05:1.2,0.02:1.2,0.01:1.2,0.05:1.1,0.3:1.5")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-solve", action="store_true", help="skip the oracle's beam solve in cpu_baseline")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip the GMG-PCG solve measurements")
    ap.add_argument("--quick-solves", action="store_true", help="only the beam solve")
    ap.add_argument("--solve-reps", type=int, default=4)
    ap.add_argument("--clocks-dir", default="", help="directory for the raw nvidia-smi clock samples "
                    "(default: a temporary directory)")
    ap.add_argument("--solve-cases", default="", help="comma list of solve-case keys to run (default: all): "
                    "beam, beam2mat, beamh, beam_paper, beam_c1, beam64, beam64h, cube6, cube8, cube6_c1")
    ap.add_argument("--solve-modes", default="", help="comma list of fp64, mixed_ir, mixed_fcg (default: each case's)")
    ap.add_argument("--solve-eager-maxit", type=int, default=0,
                    help="profiling aid: graphs off and this iteration cap for every solve (0: graphs, cap 1000)")
    ap.add_argument("--batch-ops", type=int, default=96, help="0 skips the batched-apply measurement")
    ap.add_argument("--batch-reps", type=int, default=20)
    ap.add_argument("--serve-requests", type=int, default=256, help="0 skips the serving measurement")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=160.0)
    ap.add_argument("--serve-load", type=float, default=0.8, help="arrival rate / measured capacity")
    ap.add_argument("--serve-calibration", type=int, default=16)
    ap.add_argument("--serve-small", type=int, default=64, help="small-solve burst served with and without batching")
    ap.add_argument("--serve-lane-off", type=int, default=1, help="also serve the stream with the batch lane off")
    ap.add_argument("--ablation-ps", default="2,4,8", help="degrees of the Table 8 stage ladder ('' skips it)")
    ap.add_argument("--ablation-reps", type=int, default=5)
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32 operator sweep of the FP64 line")
    ap.add_argument("--launch", default="", help="fixed element-kernel shape 'variant,elems_per_cta,threads' "
                                                 "(skips the autotuner)")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    if args.gmg_sweep:
        return run_gmg_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    main()
