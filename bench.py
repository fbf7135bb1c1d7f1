#!/usr/bin/env python
"""Throughput of the conservative dG-Arakawa Navier-Stokes time step on GB300 GPUs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--precision fp64|mixed] [--impl native|reference] [--no-cpu-baseline]

A step is one time step of the whole hot path: the Arakawa bracket + viscous term + AB3
update (one fused kernel) and the CG Poisson solve (one persistent cooperative kernel), on
synthetic fields shaped like the paper's runs.  Default workload (the largest single run):
1024 x 1024 periodic cells on [0, 2pi]^2, n = 5 nodes per dimension (26.2M dof), random-phase
vorticity with E(k) ~ k^4 exp(-(k/6)^2), D = 0, dt = 2e-4, CG tolerance 1e-10; float64 is the
headline, the mixed-precision modes are timed in the same run with their one-step error.

Prints ONE JSON line on rank 0.  value = dof * steps / device seconds, summed over ranks
(each rank advances its own replica: the simulations are independent units, no collective is
in the data path).  --impl reference times the FP64 NumPy oracle on the host cores instead.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: cells per side, n, viscosity, dt, CG tol, initial field
    "shear512_n4": dict(N=512, n=4, D=1e-4, dt=5e-4, tol=1e-10, field="shear_layer"),
    "sinsin32_n3": dict(N=32, n=3, D=0.0, dt=1e-3, tol=1e-12, field="sin_sin_noise"),
    "random1024_n5": dict(N=1024, n=5, D=0.0, dt=2e-4, tol=1e-10, field="random_phase"),
    # not single runs: handled by run_batch / run_serve
    "batch64": dict(N=0, n=0, D=0.0, dt=0.0, tol=1e-10, field="random_phase"),
    "serve": dict(N=0, n=0, D=0.0, dt=0.0, tol=1e-10, field="mixed"),
    # one bracket evaluation, N = 100, P = 1..4 (Table 1): handled by run_bracket
    "bracket_table1": dict(N=100, n=4, D=0.0, dt=0.0, tol=0.0, field="random_phase"),
}
# Table 1: milliseconds per bracket evaluation at N = 100 on a GeForce GTX 570 and on a Xeon
# E3-1225 V2 with 4 threads, FP64
TABLE1_MS = {1: (0.05, 0.08), 2: (0.26, 0.52), 3: (0.71, 3.85), 4: (1.47, 9.08)}
DEFAULT_WORKLOAD = "random1024_n5"
L2_BYTES = 129 * 1024 * 1024
# FP64 and FP32 FMA peaks of a GB300 from the unit counts and the maximum SM clock: 152 SMs x
# 2 DFMA / 128 FFMA per clock x 2 flop x 2.070 GHz.  profiles/fma_peak_gb300.json holds the
# measured figures (an FMA-chain microbenchmark with its sampled clocks), used when present.
FP64_PEAK_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_PEAK_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def fma_peaks():
    """(fp64 TFLOP/s, fp32 TFLOP/s, source) of the FMA pipes."""
    try:
        with open(os.path.join(ROOT, "profiles", "fma_peak_gb300.json")) as f:
            d = json.load(f)
        return d["fp64_fma_tflops"], d["fp32_fma_tflops"], "measured (profiles/fma_peak_gb300.json)"
    except (OSError, KeyError, ValueError):
        return FP64_PEAK_NOMINAL_TFLOPS, FP32_PEAK_NOMINAL_TFLOPS, "nominal: unit counts x 2.070 GHz"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def measured_traffic(kernel, workload, precision, iters_per_launch=None, precond=None):
    """DRAM bytes (read + write) per launch of `kernel` on this workload, precision and
    preconditioner from the ncu capture recorded in profiles/<kernel>_traffic.json, scaled from
    the capture's CG iterations per launch to iters_per_launch (the traffic of a solve grows
    with its iteration count; None if there is no record)."""
    path = os.path.join(ROOT, "profiles", "%s_traffic.json" % kernel)
    try:
        rows = json.load(open(path))["captures"]
    except (OSError, KeyError, ValueError):
        return None
    for r in rows:
        if (r.get("workload") == workload and r.get("precision") == precision
                and (precond is None or r.get("precond") == precond)):
            b = float(r["dram_bytes_per_launch"])
            k = r.get("iters_per_launch")
            if iters_per_launch and k:
                b *= (iters_per_launch + 1.0) / (k + 1.0)   # setup ~ one iteration's traffic
            return b
    return None


def make_field(name, X, Y):
    from paper_1311_7477_gb300 import fields
    if name == "shear_layer":
        return fields.shear_layer(X, Y)
    if name == "sin_sin_noise":
        return fields.sin_sin_noise(X, Y, amp=1e-3, seed=0)
    if name == "random_phase":
        return fields.random_phase(X, Y, seed=1)
    raise ValueError(name)


# ----------------------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = str(gpu_index)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu, "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[3], parts[4], parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[4]) if v.lower() == "active"})
        try:
            pw = max(float(r[2]) for r in rows)
        except ValueError:
            pw = None
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": rows[0][1], "reasons": reasons, "samples": len(rows),
                "power_w_max": pw}


def _gpu_index_for_smi(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return local_rank


# ----------------------------------------------------------------------------------------
# oracle sample (CPU baseline and the reference arm)
# ----------------------------------------------------------------------------------------
SAMPLE_CELLS = 128          # reference arm: one full oracle step per timed step
BASELINE_CELLS = 256        # cpu_baseline: full oracle steps, repeated to about 10 s
BASELINE_SECONDS = 10.0


def oracle_sample(wl, cg_sample_iters=4, precond="twolevel", cells=SAMPLE_CELLS, min_seconds=0.0):
    """Times the FP64 oracle on a cells^2 periodic grid of the same n, field and parameters:
    one right-hand side (bracket + viscous term + AB3 update), the Poisson setup and
    cg_sample_iters CG iterations with the given preconditioner -- repeated until min_seconds
    of CPU time have been spent (at least once).  Returns seconds per dof for each part (the
    oracle's cost is linear in the dof count, up to the log of its FFT)."""
    import numpy as np
    from oracle.operators import Operators
    from oracle.solver import TwoLevel, pcg, poisson_rhs
    from oracle.tables import Grid
    g = Grid(cells, cells, wl["n"])
    ops = Operators(g)
    M = TwoLevel(ops) if oracle_precond(precond) == "twolevel" else None
    X, Y = g.mesh()
    w = make_field(wl["field"], X, Y)
    psi = 0.01 * np.sin(X) * np.cos(Y)
    R1 = np.zeros_like(w)
    dof = w.size
    t_rhs = t_setup = t_cg = 0.0
    reps = 0
    while reps == 0 or t_rhs + t_setup + t_cg < min_seconds:
        t0 = time.perf_counter()
        R = -ops.bracket(psi, w)
        if wl["D"] != 0.0:
            R = R + wl["D"] * ops.laplacian(w)
        w1 = w + wl["dt"] * (23.0 * R - 16.0 * R1 + 5.0 * R1) / 12.0
        t1 = time.perf_counter()
        b = poisson_rhs(ops, w1)
        t2 = time.perf_counter()
        pcg(ops, b, psi, 1e-30, cg_sample_iters, fixed_iters=cg_sample_iters, precond=M)
        t3 = time.perf_counter()
        t_rhs, t_setup, t_cg = t_rhs + (t1 - t0), t_setup + (t2 - t1), t_cg + (t3 - t2)
        reps += 1
    # pcg includes one setup apply (r0 = b - A x0) besides the iterations
    return {"rhs_s_per_dof": t_rhs / reps / dof, "setup_s_per_dof": t_setup / reps / dof,
            "cg_s_per_dof_iter": t_cg / reps / dof / (cg_sample_iters + 1), "sample_dof": dof,
            "cells": cells, "reps": reps, "cg_iters": cg_sample_iters,
            "cpu_s": t_rhs + t_setup + t_cg}


def oracle_precond(precond):
    """The preconditioner the oracle legs time: the oracle's spectral one stores an n^2 x n^2
    block inverse per wave vector (about 10 GB at 1024^2 cells, n = 5), so those legs time the
    two-level one in its place."""
    return "twolevel" if precond == "spectral" else precond


def oracle_iters_per_step(name, precond="twolevel"):
    precond = oracle_precond(precond)
    path = os.path.join(ROOT, "tests", "golden", "cg_iterations_%s_%s.json" % (name, precond))
    if os.path.exists(path):
        d = json.load(open(path))
        if d.get("ab3_iters_mean"):
            return float(d["ab3_iters_mean"]), "the oracle's own CG iterations per AB3 step on this workload"
    return None, None


def cpu_baseline(name, wl, native_iters, precond="twolevel", threads=1):
    """Runs the oracle sample (full steps on a BASELINE_CELLS^2 grid, about BASELINE_SECONDS
    of CPU time) in a child process with the given number of BLAS/OpenMP threads; returns the
    cpu_baseline object of the JSON line."""
    k, ksrc = oracle_iters_per_step(name, precond)
    if k is None:
        k, ksrc = native_iters, "CG iterations per step measured on the GPU in this run"
    kint = max(1, int(round(k)))
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    code = ("import json,sys; sys.path.insert(0,%r); import bench; "
            "print(json.dumps(bench.oracle_sample(bench.WORKLOADS[%r], %d, %r, %d, %r)))"
            % (ROOT, name, kint, precond, BASELINE_CELLS, BASELINE_SECONDS))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        return {"value": None, "unit": "Mdof·steps/s", "cores": threads, "kind": "oracle",
                "sample": "failed: " + out.stderr.strip()[-200:]}
    s = json.loads(out.stdout.strip().splitlines()[-1])
    sec_per_dof_step = s["rhs_s_per_dof"] + s["setup_s_per_dof"] + (kint + 1) * s["cg_s_per_dof_iter"]
    return {"value": 1e-6 / sec_per_dof_step, "unit": "Mdof·steps/s", "cores": threads, "kind": "oracle",
            "sample": ("FP64 NumPy oracle, %d thread(s): %d full AB3 steps (bracket + viscous term + update, "
                       "Poisson setup, %d CG iterations with the %s preconditioner; %s) on a %dx%d-cell "
                       "grid of the same n=%d, field and parameters (%d dof), rate per dof; %.1f s of CPU"
                       % (threads, s["reps"], kint, oracle_precond(precond), ksrc, s["cells"], s["cells"], wl["n"],
                          s["sample_dof"], s["cpu_s"])),
            "parts_s_per_dof": s}


def oracle_bracket_ms(n, N=100, calls=3):
    """Milliseconds per oracle bracket evaluation on the N x N grid (host cores)."""
    import numpy as np
    from oracle.operators import Operators
    from oracle.tables import Grid
    from paper_1311_7477_gb300 import fields
    g = Grid(N, N, n)
    ops = Operators(g)
    X, Y = g.mesh()
    f, w = fields.random_phase(X, Y, seed=2), fields.random_phase(X, Y, seed=3)
    ops.bracket(f, w)
    t0 = time.perf_counter()
    for _ in range(calls):
        ops.bracket(f, w)
    return (time.perf_counter() - t0) / calls * 1e3


def run_reference(args, wl, name):
    """--impl reference: the oracle on the host cores, each step one bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if name == "bracket_table1":
        for _ in range(args.warmup):
            oracle_bracket_ms(4, calls=1)
        t0 = time.perf_counter()
        ms = sum(oracle_bracket_ms(4, calls=1) for _ in range(args.steps)) / args.steps
        value = 100 * 100 * 16 / (ms / 1e3) / 1e6
        cores = int(os.environ.get("OMP_NUM_THREADS", "0") or 0) or 1
        print(json.dumps({
            "impl": "reference", "metric": "Mdof/s (one bracket evaluation)", "value": value, "unit": "Mdof/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "bracket_table1", "cells": "100x100", "n": 4, "dof": 160000},
            "cpu_baseline": {"value": value, "unit": "Mdof/s", "cores": cores, "kind": "oracle",
                             "sample": "FP64 NumPy oracle bracket on the 100x100-cell n=4 grid, %d calls, %.1f s"
                                       % (args.steps, time.perf_counter() - t0)},
            "e2e": {"value": value, "unit": "Mdof/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    k, ksrc = oracle_iters_per_step(name, args.precond)
    if k is None:
        k, ksrc = 30.0, "assumed 30 CG iterations per step (no measured count for this workload)"
    kint = max(1, int(round(k)))
    for _ in range(args.warmup):
        oracle_sample(wl, kint, args.precond)
    t0 = time.perf_counter()
    secs = []
    for _ in range(args.steps):
        s = oracle_sample(wl, kint, args.precond)
        secs.append(s["rhs_s_per_dof"] + s["setup_s_per_dof"] + (kint + 1) * s["cg_s_per_dof_iter"])
    wall = time.perf_counter() - t0
    dof = wl["N"] * wl["N"] * wl["n"] ** 2
    sec_per_step = sum(secs) / len(secs) * dof
    value = dof / sec_per_step / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", "0") or 0) or 1
    line = {"impl": "reference", "metric": "Mdof·steps/s", "value": value, "unit": "Mdof·steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(name, wl, "fp64"),
            "cpu_baseline": {"value": value, "unit": "Mdof·steps/s", "cores": cores, "kind": "oracle",
                             "sample": "each step: one full oracle AB3 step (RHS, Poisson setup, %d CG iterations; "
                                       "%s) on a %dx%d-cell grid of the same n, field and parameters, "
                                       "rate per dof applied to %dx%d cells; %.1f s wall"
                                       % (kint, ksrc, SAMPLE_CELLS, SAMPLE_CELLS, wl["N"], wl["N"], wall)},
            "e2e": {"value": value, "unit": "Mdof·steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _config(name, wl, precision):
    dof = wl["N"] * wl["N"] * wl["n"] ** 2
    return {"workload": name, "cells": "%dx%d" % (wl["N"], wl["N"]), "n": wl["n"], "dof": dof,
            "domain": "[0,2pi]^2 periodic", "field": wl["field"], "D": wl["D"], "dt": wl["dt"],
            "cg_tol": wl["tol"], "precision": precision, "parallelism": "replicas (one simulation per GPU)"}


# ----------------------------------------------------------------------------------------
# multi-GPU bookkeeping: one independent simulation (replica) per rank, no collective in the
# data path; the elapsed time is the maximum over ranks and the rate counts every rank's dof
# ----------------------------------------------------------------------------------------
def max_over_ranks(x, dist, device):
    """The maximum of a per-rank float over all ranks (x itself with one process)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(dof_per_rank, steps, world, seconds):
    """Mdof.steps/s of the whole job: every rank advances its own dof_per_rank replica."""
    return dof_per_rank * steps * world / seconds / 1e6


# ----------------------------------------------------------------------------------------
# native arm
# ----------------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed", "mixed64", "fp64pc32"],
                    help="default: fp64 for the single runs, mixed for batch64 and serve")
    ap.add_argument("--precond", default="spectral", choices=["jacobi", "twolevel", "spectral"])
    ap.add_argument("--no-mixed-compare", action="store_true")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-steps-scale", type=float, default=0.25)
    ap.add_argument("--serve-max-cells", type=int, default=1024)
    ap.add_argument("--serve-groups", type=int, default=0, help="block groups of the batch (0: automatic)")
    ap.add_argument("--batch-compare-fp64", action="store_true",
                    help="batch64: also run the ensemble in float64 and compare each member")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "mixed" if args.workload in ("batch64", "serve") else "fp64"
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl, args.workload)
        return
    if args.workload == "batch64":
        run_batch(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    if args.workload == "bracket_table1":
        run_bracket(args)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3 (the first two steps are RK4 start-up steps)")

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    from paper_1311_7477_gb300 import build as _build
    _build.build()
    from paper_1311_7477_gb300 import dg, fields

    precision = _prec(dg, args.precision)
    N, n = wl["N"], wl["n"]
    g = dg.Grid(N, N, n)
    g.set_precond(args.precond)
    dof = g.dof
    xn, yn, _ = g.nodes()
    X, Y = fields.mesh_from_nodes(xn, yn)
    w0 = make_field(wl["field"], X, Y)
    stream = torch.cuda.current_stream()
    w0_dev = torch.from_numpy(w0).cuda()
    sim = dg.Sim(g, w0_dev, D=wl["D"], dt=wl["dt"], precision=precision, cg_tol=wl["tol"], cg_maxit=200000)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (includes the two RK4 start-up steps)
    sim.step(args.warmup)
    info0 = sim.status()
    sim.set_timing(True)
    sampler = ClockSampler(_gpu_index_for_smi(local_rank)) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    barrier()
    clocks = sampler.stop() if sampler else None
    ms = ev0.elapsed_time(ev1)
    info1 = sim.status()
    cnt = sim.counters()
    ms = max_over_ranks(ms, dist, "cuda")
    iters = (info1.cg_iters_total - info0.cg_iters_total) / max(args.steps, 1)

    # --- end to end through the host-buffer entry points: resume a checkpoint from pinned
    # host memory, step with the invariants read back every step, download omega and psi.
    ke = args.e2e_steps or max(3, min(args.steps, 10))
    shape = g.shape
    dstate = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(5)]
    step_k = sim.get_state(*dstate)
    hstate = [torch.empty(shape, dtype=torch.float64).pin_memory() for _ in range(5)]
    for h, d in zip(hstate, dstate):
        h.copy_(d)
    hout = [torch.empty(shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    barrier()
    t0 = time.perf_counter()
    sim.upload(step_k, *hstate)
    for _ in range(ke):
        sim.step(1)
        sim.invariants()
    sim.download(hout[0], hout[1])
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")

    # --- the precision modes on the same workload: each timed like the headline, with its
    # one-step error from the identical state against the float64 path (which the full-size
    # parity tests pin to the FP64 oracle at 1e-12 per step on this configuration)
    modes = None
    fp64_peak, fp32_peak, fma_src = fma_peaks()
    peaks, peak_src = measured_peaks()
    if not args.no_mixed_compare:
        modes = {}
        st = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(5)]
        kk = sim.get_state(*st)
        ref_w, ref_p = torch.empty_like(st[0]), torch.empty_like(st[0])
        ref = dg.Sim(g, st[0], D=wl["D"], dt=wl["dt"], precision=dg.DG_FP64, cg_tol=wl["tol"], cg_maxit=200000)
        ref.set_state(kk, *st)
        ref.step(1)
        ref.get(ref_w, ref_p)
        ref.close()
        what = {"fp64": "float64 throughout (the headline path)",
                "fp64pc32": "float64 throughout except the CG preconditioner, applied in float32",
                "mixed64": "float64 bracket/viscous term/update, float32 inner PCG, float64 refinement residual",
                "mixed": "bracket and viscous term in double-float on the float32 pipe, float32 inner PCG, "
                         "float64 update and refinement residual"}
        for mname, mprec in (("fp64", dg.DG_FP64), ("fp64pc32", dg.DG_FP64_PC32), ("mixed64", dg.DG_MIXED64),
                             ("mixed", dg.DG_MIXED)):
            if mname == args.precision:
                continue
            ms_ = dg.Sim(g, st[0], D=wl["D"], dt=wl["dt"], precision=mprec, cg_tol=wl["tol"], cg_maxit=200000)
            ms_.set_state(kk, *st)
            ms_.step(1)
            w1, p1 = torch.empty_like(st[0]), torch.empty_like(st[0])
            ms_.get(w1, p1)
            torch.cuda.synchronize()
            err = {"omega_rel_l2": float(torch.linalg.norm(w1 - ref_w) / torch.linalg.norm(ref_w)),
                   "psi_rel_l2": float(torch.linalg.norm(p1 - ref_p) / torch.linalg.norm(ref_p)),
                   "psi_relres": float(ms_.status().cg_relres_last)}
            del w1, p1
            ms_.step(max(args.warmup - 1, 1))
            i0 = ms_.status().cg_iters_total
            ms_.set_timing(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            ms_.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            mms = e0.elapsed_time(e1)
            info = ms_.status()
            c = ms_.counters()
            k_in = (info.cg_iters_total - i0) / args.steps
            sol_ms = c.cg_ms / max(c.cg_launches, 1)
            entry = {"value": whole_job_rate(dof, args.steps, world, mms / 1e3), "unit": "Mdof·steps/s",
                     "ms_per_step": mms / args.steps, "rhs_ms": c.rhs_ms / max(c.rhs_launches, 1),
                     "solve_ms": sol_ms, "cg_iters_per_step": k_in,
                     "refine_sweeps_last": int(info.refine_sweeps_last),
                     "error_vs_fp64_one_step": err, "what": what[mname]}
            if mprec in (dg.DG_MIXED, dg.DG_MIXED64):
                # the refinement solve's algorithmic bytes per dof: extrapolation setup 16, each
                # float64 residual sweep 32 (y, omega in; residual out), each float32 inner
                # iteration 32 (e, r, p read and written, q written and read: 8 x 4 B)
                sweeps = max(int(info.refine_sweeps_last), 1)
                byts = dof * (16 + 32 * (sweeps + 1) + 32 * k_in)
                gbs = byts / (sol_ms / 1e3) / 1e9
                entry["roofline"] = {"kernel": "mixed_cg_kernel", "bound": "hbm", "achieved": gbs,
                                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                                     "peak_source": peak_src,
                                     "traffic": measured_traffic("cg_kernel", args.workload, mname,
                                                                 precond=args.precond),
                                     "bytes_per_dof": "16 + 32 (sweeps + 1) + 32 x inner iterations",
                                     "note": "HBM fraction by the refinement's algorithmic bytes; with one "
                                             "inner iteration per solve the kernel is bound by its float64 "
                                             "residual applications, not by HBM"}
            modes[mname] = entry
            ms_.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    value = whole_job_rate(dof, args.steps, world, ms / 1e3)
    # roofline of the dominant kernel (the persistent CG solve), from its live event timing
    cg_ms_per_launch = cnt.cg_ms / max(cnt.cg_launches, 1)
    rhs_ms_per_launch = cnt.rhs_ms / max(cnt.rhs_launches, 1)
    it_per_launch = (info1.cg_iters_total - info0.cg_iters_total) / max(cnt.cg_launches, 1)
    # the method's count per dof: a CG iteration is one operator apply (8(n+4)+4 flop with the
    # derivatives applied as matrix-free 1D operators) and the vector work (10 flop), and moves
    # x, r, p (read and written) and q (written and read): 64 B in float64; the setup is one
    # apply and 4 flop, 48 B (three vectors read, three written)
    import math
    s8 = 8
    flops_iter_m = 8 * (n + 4) + 14
    flops_setup_m = 8 * (n + 4) + 4
    bytes_iter_m, bytes_setup_m = 8 * s8, 6 * s8
    # this implementation's count: the assembled 1D operator (2 directions x (n + 4) FMA), the
    # vector updates and dot products, and the two-level preconditioner (cell block solve n^2
    # FMA, restriction and prolongation, the coarse DFT: 4 passes of 5 log2(N) flop per cell)
    flops_iter_i = 4 * (n + 4) + 10
    bytes_iter_i = 8 * 8
    if args.precond == "twolevel":
        flops_iter_i += 2 * n * n + 4 + 2 + 4 * 5 * math.log2(N) / (n * n)
        bytes_iter_i += 2 * 8            # z written and read
    elif args.precond == "spectral":
        # real 2D DFT forward and inverse (5 log2(N^2) flop per dof), four n x n complex
        # transforms of the half spectrum (16 n flop per dof); r read, the spectrum written and
        # read three times, z written: 8 + 6 * 8 + 8 B per dof (float64 complex, half spectrum)
        flops_iter_i += 5 * math.log2(N * N) + 16 * n
        bytes_iter_i += 8 + 6 * 8 + 8
    # the setup's initial residual b - Ahat(2 psi^k - psi^{k-1}) comes from the operator products
    # the previous solves kept (no operator application in the timed AB3 steps): 8 flop
    flops_setup_i = 8
    sec = cg_ms_per_launch / 1e3
    fp64 = args.precision in ("fp64", "fp64pc32")
    pk = fp64_peak if fp64 else fp32_peak
    ach_m = dof * (flops_iter_m * it_per_launch + flops_setup_m) / sec / 1e12
    ach_i = dof * (flops_iter_i * it_per_launch + flops_setup_i) / sec / 1e12
    gbs_m = dof * (bytes_iter_m * it_per_launch + bytes_setup_m) / sec / 1e9
    traffic = measured_traffic("cg_kernel", args.workload, args.precision, it_per_launch, args.precond)
    roof = {"kernel": "cg_kernel (persistent CG Poisson solve)", "bound": "alu",
            "achieved": ach_m, "peak": pk, "unit": "TFLOP/s", "frac": ach_m / pk, "traffic": traffic,
            "peak_source": ("FP64" if fp64 else "FP32") + " FMA pipe, " + fma_src,
            "count": "method: per dof and CG iteration 8(n+4)+14 flop, 64 B; setup 8(n+4)+4 flop, 48 B",
            "implementation_count": {"achieved": ach_i, "frac": ach_i / pk,
                                     "flops_per_dof_iter": flops_iter_i, "flops_per_dof_setup": flops_setup_i,
                                     "bytes_per_dof_iter": bytes_iter_i,
                                     "what": "assembled 1D operators + %s preconditioner work" % args.precond},
            "hbm": {"achieved": gbs_m, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": gbs_m / peaks["hbm_gbs"], "peak_source": peak_src},
            "launch_ms": cg_ms_per_launch, "iters_per_launch": it_per_launch,
            "traffic_vs_method_bytes": (traffic / (dof * (bytes_iter_m * it_per_launch + bytes_setup_m))
                                        if traffic else None)}
    line = {"metric": "Mdof·steps/s", "value": value, "unit": "Mdof·steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": dict(_config(args.workload, wl, args.precision), cg_preconditioner=args.precond,
                           l2=("no flush: the per-step working set (%.0f MB of state and CG vectors) exceeds "
                               "the 129 MB L2" % (12 * dof * 8 / 1e6))),
            "cg_iters_per_step": iters, "rhs_ms": rhs_ms_per_launch, "roofline": roof,
            "precision_modes": modes,
            "gpu_launches": int(cnt.launches), "clocks": clocks,
            "e2e": {"value": dof * ke * world / e2e_s / 1e6, "unit": "Mdof·steps/s",
                    "h2d_bytes_per_step": int(5 * dof * 8 / ke), "d2h_bytes_per_step": int(2 * dof * 8 / ke) + 24,
                    "steps": ke,
                    "what": "upload of the full stepper state from pinned host memory, %d steps each followed "
                            "by a host read of (V, E, Omega), download of omega and psi" % ke}}
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload, wl, iters, args.precond)
    else:
        line["cpu_baseline"] = None
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def run_bracket(args):
    """Table 1: one evaluation of the bracket of Eq. J (dg_bracket, float64) at N = 100 for
    P = 1..4, timed per call with CUDA events around the call alone; a 512 MB buffer is
    written between calls so each call reads its inputs from HBM, not from L2.  Also one
    large grid (1000 x 1000 cells, n = 4) for the kernel's bandwidth roofline.  value = the
    P = 4 rate in Mdof/s; vs_baseline = value / the GTX 570's P = 4 rate."""
    import numpy as np
    import torch
    from paper_1311_7477_gb300 import build as _build
    _build.build()
    from paper_1311_7477_gb300 import dg, fields
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    peaks, peak_src = measured_peaks()
    fp64_peak, _, fma_src = fma_peaks()
    cpu_ms = {}
    if not args.no_cpu_baseline:
        for n in (1, 2, 3, 4):
            cpu_ms[n] = oracle_bracket_ms(n)

    def time_bracket(g, f, w, J, calls, fn=None):
        fn = fn or dg.dg_bracket
        times = []
        for i in range(args.warmup + calls):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(g, f, w, J, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if i >= args.warmup:
                times.append(e0.elapsed_time(e1))
        return float(np.median(times)), times

    rows = []
    launches = 0
    sampler = ClockSampler(_gpu_index_for_smi(0))
    sampler.start()
    time.sleep(0.3)
    for N, n in ((100, 1), (100, 2), (100, 3), (100, 4), (1000, 4)):
        g = dg.Grid(N, N, n)
        xn, yn, _ = g.nodes()
        X, Y = fields.mesh_from_nodes(xn, yn)
        f = torch.from_numpy(fields.random_phase(X, Y, seed=2)).cuda()
        w = torch.from_numpy(fields.random_phase(X, Y, seed=3)).cuda()
        J = torch.empty_like(w)
        med, times = time_bracket(g, f, w, J, args.steps)
        med_x, _ = time_bracket(g, f, w, J, args.steps, dg.dg_bracket_mixed)
        launches += 2 * args.steps
        dof = g.dof
        row = {"P": n, "N": N, "dof": dof, "ms": med, "ms_min": min(times), "mdof_per_s": dof / med / 1e3,
               "hbm_gbs_algorithmic": 24 * dof / (med / 1e3) / 1e9,
               "double_float_ms": med_x, "double_float_mdof_per_s": dof / med_x / 1e3}
        if N == 100:
            gpu_p, cpu_p = TABLE1_MS[n]
            row.update({"paper_gtx570_ms": gpu_p, "paper_xeon4_ms": cpu_p, "speedup_vs_gtx570": gpu_p / med,
                        "oracle_ms": cpu_ms.get(n)})
        rows.append(row)
        g.close()
    # end to end: inputs from pinned host memory, J back to pinned host memory
    g = dg.Grid(100, 100, 4)
    xn, yn, _ = g.nodes()
    X, Y = fields.mesh_from_nodes(xn, yn)
    hf = torch.from_numpy(fields.random_phase(X, Y, seed=2)).pin_memory()
    hw = torch.from_numpy(fields.random_phase(X, Y, seed=3)).pin_memory()
    hJ = torch.empty_like(hw).pin_memory()
    df, dw, dJ = torch.empty_like(hf, device="cuda"), torch.empty_like(hw, device="cuda"), torch.empty_like(hw,
                                                                                                          device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        df.copy_(hf, non_blocking=True)
        dw.copy_(hw, non_blocking=True)
        dg.dg_bracket(g, df, dw, dJ, stream=stream)
        hJ.copy_(dJ, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    launches += args.steps
    clocks = sampler.stop()
    p4, big = rows[3], rows[4]
    big_s = big["ms"] / 1e3
    big_tf = (12 * (4 + 4) + 12) * big["dof"] / big_s / 1e12
    line = {"metric": "Mdof/s (one bracket evaluation, Table 1)", "value": p4["mdof_per_s"], "unit": "Mdof/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": p4["ms"],
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": p4["mdof_per_s"] / (160000 / 1.47e-3 / 1e6), "dtype": "f64", "data": "synthetic",
            "config": {"workload": "bracket_table1", "cells": "100x100", "n": 4, "dof": 160000,
                       "field": "random phase psi and omega", "precision": "fp64",
                       "l2": "flushed between calls (512 MB written)"},
            "rows": rows,
            "roofline": {"kernel": "rhs_kernel in bracket-only mode, 1000x1000 cells, n=4", "bound": "alu",
                         "achieved": big_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": big_tf / fp64_peak,
                         "traffic": measured_traffic("rhs_kernel", "bracket1000_n4", "fp64"),
                         "peak_source": "FP64 FMA pipe, " + fma_src,
                         "algorithmic_per_dof": {"flops": 12 * (4 + 4) + 12, "bytes": 24},
                         "hbm": {"achieved": big["hbm_gbs_algorithmic"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                 "frac": big["hbm_gbs_algorithmic"] / peaks["hbm_gbs"],
                                 "peak_source": peak_src}},
            "gpu_launches": launches, "clocks": clocks,
            "e2e": {"value": 160000 / e2e_s / 1e6, "unit": "Mdof/s", "h2d_bytes_per_step": 2 * 160000 * 8,
                    "d2h_bytes_per_step": 160000 * 8,
                    "what": "psi and omega copied from pinned host memory, dg_bracket, J copied back, per call"},
            "cpu_baseline": ({"value": 160000 / (cpu_ms[4] / 1e3) / 1e6, "unit": "Mdof/s", "cores": 1,
                              "kind": "oracle", "sample": "NumPy oracle bracket, 100x100 cells, n=4, 3 calls"}
                             if cpu_ms else None)}
    print(json.dumps(line))


def _prec(dg, name):
    return {"fp64": dg.DG_FP64, "mixed": dg.DG_MIXED, "mixed64": dg.DG_MIXED64, "fp64pc32": dg.DG_FP64_PC32}[name]


def run_batch(args):
    """64 uneven simulations (cells per side in {32,64,128,256}, n in {2..5}, D log-uniform in
    [1e-5, 1e-3], random phase) advanced together by the persistent batched kernel, in one
    graph-captured launch per step.  The launch configuration (block groups, per-n tiles,
    blocks per SM) is picked by the library's autotuner (dg_batch_autotune) on the first steps,
    which count as warm-up.  With --batch-compare-fp64 the same ensemble is also run in float64
    to the same step and each member's vorticity is compared."""
    import numpy as np
    import torch
    from paper_1311_7477_gb300 import build as _build
    _build.build()
    from paper_1311_7477_gb300 import dg, workloads
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    prec = _prec(dg, args.precision)
    specs = workloads.ensemble_specs()

    def ensemble(precision):
        members = []
        for sp in specs:
            g = dg.Grid(sp["N"], sp["N"], sp["n"])
            g.set_precond(args.precond)
            w0 = torch.from_numpy(workloads.initial_field(dg, g, sp)).cuda()
            dt = workloads.stable_dt(dg, sp["N"], sp["n"], sp["D"])
            members.append((g, dg.Sim(g, w0, D=sp["D"], dt=dt, precision=precision, cg_tol=1e-10,
                                      cg_maxit=100000)))
        b = dg.Batch(len(members))
        for _, s in members:
            b.admit(s)
        return members, b

    members, b = ensemble(prec)
    dof = sum(g.dof for g, _ in members)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    tuned = b.autotune(trial_steps=2)
    tune_s = time.perf_counter() - t0
    b.step(max(args.warmup, 1))
    torch.cuda.synchronize()
    before = sum(s.status().cg_iters_total for _, s in members)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        b.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = b.status()
    after = sum(s.status().cg_iters_total for _, s in members)
    steps_done = members[0][1].status().step
    line = {"metric": "Mdof·steps/s", "value": dof * args.steps / (ms / 1e3) / 1e6, "unit": "Mdof·steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "f32+f64", "mixed64": "f32+f64", "fp64": "f64", "fp64pc32": "f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": "batch64", "members": len(members), "dof_total": dof,
                       "cells": "32..256 per side", "n": "2..5", "D": "log-uniform [1e-5, 1e-3]",
                       "precision": args.precision, "cg_preconditioner": args.precond, "cg_tol": 1e-10,
                       "autotuned": tuned, "autotune_s": tune_s, "graph": st["graph"],
                       "steps_per_member": steps_done},
            "inner_cg_iters_per_member_step": (after - before) / (args.steps * len(members)),
            "gpu_launches": args.steps}
    if args.batch_compare_fp64 and prec != dg.DG_FP64:
        ref, rb = ensemble(dg.DG_FP64)
        rb.step(steps_done - 2)
        errs = []
        for (g, s), (_, r) in zip(members, ref):
            wa = torch.empty(g.shape, dtype=torch.float64, device="cuda")
            wb = torch.empty_like(wa)
            s.get(wa, None)
            r.get(wb, None)
            errs.append(float(torch.linalg.norm(wa - wb) / torch.linalg.norm(wb)))
        line["error_vs_fp64_per_member"] = {
            "steps": steps_done, "max": max(errs), "median": float(np.median(errs)),
            "what": "relative L2 of omega after the same number of steps, this precision against the same "
                    "ensemble run in float64 (the float64 path matches the FP64 oracle to 1e-12 per step)"}
        rb.close()
        for _, r in ref:
            r.close()
    print(json.dumps(line))


def run_serve(args):
    """The served workload: Poisson arrivals at 20 requests/s (seed 7), cells per side in
    {64,...,--serve-max-cells} (powers of two; 1024 by default), n in {3,4,5}, D log-uniform,
    random-phase or shear-layer fields; step counts U{100..2000} scaled by --serve-steps-scale
    (the unscaled trace is about an hour of GPU work)."""
    import torch
    from paper_1311_7477_gb300 import build as _build
    _build.build()
    from paper_1311_7477_gb300 import dg, serve, workloads
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    Ns = tuple(N for N in (64, 128, 256, 512, 1024) if N <= args.serve_max_cells)
    trace = workloads.request_trace(count=args.serve_requests, Ns=Ns)
    for r in trace:
        r["steps"] = max(3, int(round(r["steps"] * args.serve_steps_scale)))
    prec = _prec(dg, args.precision)
    # the requests carry their initial fields (generated before the clock starts, as a
    # client would send them); the server uploads them at admission
    from concurrent.futures import ThreadPoolExecutor
    nodes = {}
    for r in trace:
        key = (r["N"], r["n"])
        if key not in nodes:
            g = dg.Grid(r["N"], r["N"], r["n"])
            xn, yn, _ = g.nodes()
            nodes[key] = (xn, yn)
            g.close()
    t_gen = time.perf_counter()
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        fields_ = list(ex.map(lambda r: workloads.initial_field_from_nodes(*nodes[(r["N"], r["n"])], r), trace))
    for r, f in zip(trace, fields_):
        r["omega0"] = f
    t_gen = time.perf_counter() - t_gen
    srv = serve.Server(max_active=64, hbm_budget=200e9, precision=prec, precond=args.precond,
                       groups=args.serve_groups)
    rep = srv.run(trace)
    line = {"metric": "Mdof·steps/s", "value": rep["mdof_steps_per_s"], "unit": "Mdof·steps/s", "n_gpus": 1,
            "steps": None, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "serve", "requests": len(trace), "rate_per_s": 20, "cells": list(Ns),
                       "n": [3, 4, 5], "steps_scale": args.serve_steps_scale, "groups": args.serve_groups,
                       "precision": {0: "fp64", 1: "mixed", 2: "mixed64", 3: "fp64pc32"}[prec], "cg_preconditioner": args.precond},
            "latency_p50_s": rep["latency_p50_s"], "latency_p99_s": rep["latency_p99_s"],
            "failed_requests": rep["failed"], "fallbacks_fp64": rep["fallbacks_fp64"],
            "served": rep, "field_generation_s_before_clock": t_gen}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
