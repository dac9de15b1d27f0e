"""Benchmark: Mpoint*RHS/s of the wavelength-adaptive 27-point Helmholtz solve.

One step = one hx_solve (complex64 Krylov + CSL multigrid, FP64 iterative
refinement to a relative FP64 residual of --tol) of the linear-gradient
workload (101^3 grid incl. a 10-node PML, h = 20 m, f = 5 Hz, one source near
the surface), sources on the device to the wavefield on the device.  L2 is
flushed (512 MB write) between timed steps, outside the timed intervals.

Also reported on the same JSON line:
  e2e          same solve through the C ABI from pinned HOST buffers (velocity
               up, wavefield down) with the copies inside the timed interval;
  roofline     dominant fine-level kernel class: algorithmic bytes / CUDA-event
               time of its launches, against the measured HBM copy bandwidth in
               MEASURED_PEAKS.json; timed in a second pass over the same steps in
               which the library brackets each launch with events (it replays
               CUDA graphs in the first, value pass);
  accuracy     relative L2 error of the mixed solution against the plain FP64
               GPU solve, that FP64 form's own throughput and its dominant
               kernel class's flops against the FP64 FMA peak measured in the
               same run (FP64-ALU-bound);
  gpu_launches this library's kernel launches inside the timed steps (graph
               replays counted per kernel);
  clocks       nvidia-smi SM clocks and throttle reasons sampled during the
               timed steps;
  large        the large batched workloads (sharp contrast 64 RHS, tectonic
               16 RHS): one mixed solve each (setup time apart, iterations,
               FP64 residual, clocks) and the stencil's roofline at that size;
  serving      the serving leg: seeded requests with Poisson arrivals on the
               serving engine (smallest request first, a bound on the wait),
               p50 / p99 latency (p99 from 100 completed requests on),
               point*RHS/s, the failed requests with status and times;
  cpu_baseline the CPU oracle (banded LU, all host cores) on a bounded sample
               of the same workload: the 24^3 corner-free sub-grid around the
               source with the same model, PML and frequency; with its CSR
               matvec on the full grid and the band storage a full-size banded
               LU would need (extras).

--impl reference runs the oracle alone (rank 0), on the same metric.
Multi-GPU: one process per GPU (torchrun); every rank solves its own copy of
the workload (independent problems, no collective on the data path); the value
is all ranks' point*RHS over the slowest rank's time ("scaling": "weak").
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

METRIC = "Mpoint*RHS/s to 1e-6 rel err (mixed vs FP64 GPU)"
UNIT = "Mpoint*RHS/s"
# Algorithmic FP64 flops of the complex128 stencil: per point*RHS the class-sum
# row (26 neighbours into 4 class sums: 23 complex additions = 46 flops; 4
# real-by-complex products = 8; 3 complex additions = 6) and the sweep's update
# (b - A x and the scaled correction, about 8); per point the row formation
# (1/v, the lerp of 11 table entries, the class coefficients: about 40).
FP64_FLOPS_PER_POINT_RHS = 68
FP64_FLOPS_PER_POINT = 40
# Serving leg: the admission's bound on how long a large request is passed
# over, the omega safeguard of the served solves, and the longest span of the
# Poisson arrivals.
SERVE_MAX_WAIT_S = 240.0
SERVE_KAPPA = 0.7
SERVE_MAX_SPAN_S = 600.0


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="hx", choices=["hx", "reference"])
    p.add_argument("--tol", type=float, default=1e-10)
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison solve")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--kernel", action="store_true", help="time the operator apply alone")
    p.add_argument("--kernel-workload", default="tectonic")
    p.add_argument("--kernel-nrhs", type=int, default=4)
    p.add_argument("--kernel-prec", type=int, default=32, choices=[32, 64])
    p.add_argument("--serve-requests", type=int, default=105,
                   help="Poisson-arriving requests of the serving workload (0: skip)")
    p.add_argument("--serve-slots", type=int, default=4)
    p.add_argument("--serve-deadline", type=float, default=300.0,
                   help="runaway guard: base of the per-request solve time limit in s "
                        "(hx_solve_opts.time_limit_s); each request gets this plus its own time "
                        "at 1/slots of the measured solo capacity")
    p.add_argument("--serve-only", action="store_true", help="run the serving workload alone")
    p.add_argument("--solve-config", default=None, choices=["homogeneous", "linear_gradient",
                                                             "sharp_contrast", "tectonic"],
                   help="one mixed solve (and its autotune) of that workload with all its sources")
    p.add_argument("--solve-time-limit", type=float, default=300.0)
    p.add_argument("--kernel-mode", default="apply", choices=["apply", "jacobi", "residual"],
                   help="apply: y = A x;  jacobi / residual: the preconditioner's sweeps of the "
                        "shifted operator (beta = 1, omega = 0.6), as inside the solve")
    p.add_argument("--kernel-cfg", default="auto",
                   help="complex64 kernel configuration: auto, tune, all, or an id")
    p.add_argument("--kernel-layout", default="plain", choices=["plain", "padded"],
                   help="plain: (nrhs, nz, ny, nx) fields through hx_apply_operator / "
                        "hx_stencil_sweep;  padded: complex64 rows padded to a multiple of 4 "
                        "(the solver's layout) through hx_stencil_pitched")
    p.add_argument("--large", default="tectonic,sharp_contrast",
                   help="comma-separated large batched workloads solved once each with all their "
                        "sources (RHS split over the ranks) plus the stencil roofline at that size; "
                        "'' skips the leg")
    p.add_argument("--large-time-limit", type=float, default=300.0)
    return p.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max_ms(ms, world, device="cpu"):
    """Slowest rank's time: all-reduce MAX over the process group (identity at N = 1)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, world, steps, max_total_ms):
    """Whole-job Mpoint*RHS/s: every rank's units over the slowest rank's time
    (replicas: each rank solves its own copy of the workload)."""
    return units_per_rank * world * steps / (max_total_ms / 1e3) / 1e6


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# --------------------------------------------------------------------- oracle

def _oracle_sample(n=24):
    """Bounded CPU sample of the linear-gradient workload: an n^3 sub-grid of
    the same model (same h, f, velocity law, PML thickness and source depth)."""
    from paper_2108_08730_gb300 import synth
    wl = synth.linear_gradient(n=n, npml=10 if n >= 30 else 6)
    return wl


def oracle_rate(budget_s=12.0, n=24):
    """Time the oracle (assemble + banded LU) on the bounded sample; returns
    (Mpoint*RHS/s, seconds, repeats, sample description, threads)."""
    from oracle import operator as O
    from oracle import solve as S
    from oracle import weights as W
    nodes, T = W.fit_table()
    wl = _oracle_sample(n)
    prof = O.profiles_for(wl.shape, wl.h, wl.npml, wl.v_ref, wl.r_coef)
    t0 = time.perf_counter()
    reps = 0
    while True:
        A = O.assemble_csr(wl.v, wl.h, wl.f, prof, T, nodes)
        s = S.point_sources(wl.shape, wl.h, wl.sources)
        S.solve_banded(A, s.reshape(-1))
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 50:
            break
    rate = wl.n_points * wl.nrhs * reps / el / 1e6
    desc = (f"banded LU (scipy solve_banded, LAPACK gbsv) + CSR assembly of a {n}^3 sub-grid of the "
            f"linear-gradient model (same h, f, v law, {wl.npml[0]}-node PML), {reps} solves")
    return rate, el, reps, desc, os.cpu_count()


def banded_lu_bytes(nx, ny, nz):
    """Band storage of LAPACK's banded LU (gbsv) for the 27-point operator in
    x-fastest order: half-bandwidth nx*ny + nx + 1, (2 kl + ku + 1) rows of N
    complex128 values."""
    kl = nx * ny + nx + 1
    return (3 * kl + 1) * nx * ny * nz * 16


def oracle_extras():
    """The oracle's CSR matvec on the full linear-gradient grid (scipy, one
    thread) and the band storage that rules out the oracle's banded LU on the
    full-size workloads."""
    from oracle import operator as O
    from oracle import weights as W
    from paper_2108_08730_gb300 import synth
    import numpy as np
    nodes, T = W.fit_table()
    wl = synth.linear_gradient()
    prof = O.profiles_for(wl.shape, wl.h, wl.npml, wl.v_ref, wl.r_coef)
    t0 = time.perf_counter()
    A = O.assemble_csr(wl.v, wl.h, wl.f, prof, T, nodes)
    t_asm = time.perf_counter() - t0
    x = np.random.default_rng(0).standard_normal(A.shape[0]) + 0j
    t0 = time.perf_counter()
    n = 0
    while n < 3 or time.perf_counter() - t0 < 2.0:
        A @ x
        n += 1
    t_mv = (time.perf_counter() - t0) / n
    sizes = {"linear_gradient 101^3": (101, 101, 101), "sharp_contrast 201x201x101": (201, 201, 101),
             "tectonic 401x401x187": (401, 401, 187)}
    return {"csr_matvec": {"workload": "linear_gradient 101^3 (oracle CSR, scipy, 1 thread)",
                           "mpoint_per_s": round(wl.n_points / t_mv / 1e6, 3), "ms": round(1e3 * t_mv, 1),
                           "assembly_s": round(t_asm, 2)},
            "banded_lu_band_storage_gb": {k: round(banded_lu_bytes(*v) / 1e9, 1) for k, v in sizes.items()}}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    steps = []
    for k in range(args.warmup + args.steps):
        r, el, reps, desc, cores = oracle_rate(budget_s=4.0)
        if k >= args.warmup:
            steps.append((r, el / reps))
    value = statistics.mean(s[0] for s in steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * statistics.mean(s[1] for s in steps), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": {"workload": "linear_gradient (bounded CPU sample)", "sample": desc},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- GPU arm

class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _traffic_per_launch(kind):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
        for src, sha in rec.get("sources", {}).items():
            h = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()[:16]
            if h != sha:
                return None
        return rec.get(kind, {}).get("bytes_per_launch_full_size")
    except Exception:
        return None


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2108_08730_gb300 import binding as B
    from paper_2108_08730_gb300 import synth

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    nodes, T = B.build_weight_table()
    ctx = B.Context(local, table=T)
    wl = synth.linear_gradient()
    g = B.grid_of(wl)
    src = B.sources_of(wl)
    R = wl.nrhs
    N = wl.n_points
    units = N * R
    v_host = torch.from_numpy(wl.v).pin_memory()
    vd = v_host.to(dev)
    out = torch.zeros((R,) + wl.shape, dtype=torch.complex128, device=dev)
    out_host = torch.empty((R,) + wl.shape, dtype=torch.complex128).pin_memory()
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    opts = dict(tol=args.tol)

    def solve():
        return ctx.solve(g, vd, src, R, out, **opts)

    for _ in range(max(args.warmup, 0)):
        solve()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps():
        step_ms, reports = [], []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rep = solve()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            reports.append(rep)
        return step_ms, reports

    # ---- device-resident timed steps, run as a user runs them (graph replay on)
    clocks = Clocks(local)
    ctx.profile(False)                       # resets the launch counter
    barrier()
    clocks.start()
    step_ms, reports = timed_steps()
    barrier()
    clk = clocks.stop()
    launches = ctx.profile_read()["all"][0]
    # ---- the same steps again with every fine-level operator launch timed by
    # CUDA events on its stream (the library launches directly in this pass)
    ctx.profile(True)
    prof_step_ms, _ = timed_steps()
    prof = ctx.profile_read()
    ctx.profile(False)
    total_ms = reduce_max_ms(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = aggregate_rate(units, world, args.steps, total_ms)

    # ---- end to end through the C ABI from pinned host buffers
    e2e_ms = []
    for _ in range(max(1, args.steps)):
        flush.fill_(1.0)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vd.copy_(v_host, non_blocking=True)
        solve()
        out_host.copy_(out, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_total = reduce_max_ms(sum(e2e_ms), world, dev)
    e2e_value = aggregate_rate(units, world, len(e2e_ms), e2e_total)

    # ---- large batched workloads (all ranks: each solves its slice of the RHS)
    large = run_large(args, T, rank, world, local) if args.large else None

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- accuracy against the plain FP64 GPU form (and its throughput)
    acc = {}
    if not args.no_fp64:
        mixed = out.clone()
        ref = torch.zeros_like(out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep64 = ctx.solve(g, vd, src, R, ref, mode=B.SOLVE_FP64, tol=1e-12, max_iter=20000, check=False)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        err = float(torch.linalg.vector_norm(mixed - ref) / torch.linalg.vector_norm(ref))
        # the FP64 form's own dominant kernel class, timed per launch in a second solve
        ctx.profile(True)
        ctx.solve(g, vd, src, R, torch.zeros_like(ref), mode=B.SOLVE_FP64, tol=1e-12, max_iter=20000,
                  check=False)
        p64 = {k: v for k, v in ctx.profile_read().items() if k in ("apply64", "smooth64") and v[0] > 0}
        ctx.profile(False)
        roof64 = None
        if p64:
            k64 = max(p64, key=lambda k: p64[k][1])
            n64, ms64, by64 = p64[k64]
            peak = (_peaks() or {}).get("hbm_gbs", 6800.0)
            fp64_peak = ctx.fp64_peak()
            flops = n64 * (FP64_FLOPS_PER_POINT_RHS * N * R + FP64_FLOPS_PER_POINT * N)
            gflops = flops / (ms64 / 1e3) / 1e9
            roof64 = {"kernel": {"apply64": "stencil_kernel<double, kApply>",
                                 "smooth64": "stencil_kernel<double, kJacobi|kResidual>"}[k64],
                      "bound": "alu",
                      "flops_per_point_rhs": FP64_FLOPS_PER_POINT_RHS, "flops_per_point": FP64_FLOPS_PER_POINT,
                      "achieved_gflops": round(gflops, 1), "fp64_peak_gflops": round(fp64_peak, 1),
                      "frac_of_fp64_peak": round(gflops / fp64_peak, 4),
                      "fp64_peak_source": "hx_measure_fp64_peak (independent FMA chains, CUDA events, this run)",
                      "achieved_gbs": round(by64 / (ms64 / 1e3) / 1e9, 1),
                      "frac_of_hbm": round(by64 / (ms64 / 1e3) / 1e9 / peak, 4)}
        acc = {"rel_l2_mixed_vs_fp64": err, "fp64_status": rep64["status"],
               "fp64_rel_residual": rep64["rel_residual"], "fp64_iters": rep64["inner_iters"],
               "fp64_value": round(units / t64 / 1e6, 4), "fp64_unit": UNIT,
               "speedup_mixed_vs_fp64": round(value / world / (units / t64 / 1e6), 2),
               "fp64_dominant_kernel": roof64}

    # ---- roofline of the dominant kernel class
    peaks = _peaks()
    kinds = {k: v for k, v in prof.items() if k != "all" and v[0] > 0}
    dom = max(kinds, key=lambda k: kinds[k][1]) if kinds else None
    roof = None
    if dom:
        n, ms, by = kinds[dom]
        achieved = by / (ms / 1e3) / 1e9
        peak = peaks["hbm_gbs"] if peaks else 6800.0
        tr = _traffic_per_launch(dom)
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": tr,
                "kernel": {"apply32": "complex64 z-marching stencil, y = A x (fine level)",
                           "smooth32": "complex64 z-marching stencil, damped-Jacobi / residual sweeps of "
                                       "the shifted operator (fine level)",
                           "apply64": "stencil_kernel<double, ...>",
                           "smooth64": "stencil_kernel<double, kJacobi|kResidual>"}[dom],
                "kernel_choice": "the solver's autotuner picks the z-marching kernel and its launch "
                                 "configuration per grid size and RHS count",
                "launches": n, "algo_bytes_per_launch": by / n,
                "share_of_step": round(ms / sum(prof_step_ms), 4),
                "timed_in": "a second pass over the same steps with per-launch CUDA events",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback"}

    cpu = None
    if world == 1 and not args.no_cpu:
        r, el, reps, desc, cores = oracle_rate()
        cpu = {"value": round(r, 6), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "extras": oracle_extras()}

    serving = None
    if world == 1 and args.serve_requests > 0:
        serving = run_serving(args, T)

    rep = reports[-1]
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 (Krylov+multigrid) + f64 (residual/refinement)", "data": "synthetic",
        "config": {"workload": "linear_gradient: v=1500+0.7z, 101^3 incl. 10-node PML, h=20 m, f=5 Hz, "
                               "1 source at (50,50,13)", "nrhs": R, "points": N, "tol": args.tol,
                   "l2": "flushed between steps (512 MB write, outside the timed intervals)",
                   "parallelism": f"replicas x{world}"},
        "solve": {"outer_iters": rep["outer_iters"], "inner_iters": rep["inner_iters"],
                  "mg_levels": rep["mg_levels"], "rel_residual": rep["rel_residual"]},
        "accuracy": acc,
        "e2e": {"value": round(e2e_value, 4), "unit": UNIT,
                "h2d_bytes_per_step": int(v_host.numel() * 4),
                "d2h_bytes_per_step": int(out_host.numel() * 16)},
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": clk,
        "cpu_baseline": cpu,
        "large": large,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def run_large(args, T, rank, world, local):
    """The large batched workloads (tectonic 401x401x187 with 16 sources,
    sharp contrast 201x201x101 with 64), each solved once in mixed precision
    with all its sources as RHS (split over the ranks when world > 1): wall
    time from the call to the wavefields on the device, the library's setup
    (hierarchy, coarse inverse, autotune, first-call workspace) and solve
    times apart, iterations, the FP64 relative residual the refinement
    reached, and the clocks during the solve.  Then, at the same size, the
    complex64 stencil's CUDA-event roofline: y = A x at 1, 4 and 16 RHS and
    the damped-Jacobi sweep at 16 RHS, each autotuned, L2 flushed before every
    timed launch, median of 5."""
    import torch

    from paper_2108_08730_gb300 import binding as B
    from paper_2108_08730_gb300 import replicas as RP
    from paper_2108_08730_gb300 import synth

    dev = torch.device("cuda", local)
    peaks = _peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    res = {}
    for name in [w for w in args.large.split(",") if w]:
        wl = synth.CONFIGS[name]()
        ctx = B.Context(local, table=T)
        g = B.grid_of(wl)
        vd = torch.from_numpy(wl.v).to(dev)
        N = wl.n_points
        src, (lo, hi) = RP.local_sources(B.sources_of(wl), wl.nrhs, world, rank)
        R = hi - lo
        out = torch.zeros((R,) + wl.shape, dtype=torch.complex128, device=dev)
        clocks = Clocks(local)
        torch.cuda.synchronize(dev)
        clocks.start()
        t0 = time.perf_counter()
        rep = ctx.solve(g, vd, src, R, out, check=False, time_limit_s=args.large_time_limit)
        torch.cuda.synchronize(dev)
        wall_ms = reduce_max_ms((time.perf_counter() - t0) * 1e3, world, dev)
        clk = clocks.stop()
        solve_ms = reduce_max_ms(rep["solve_ms"], world, dev)
        del out
        entry = {
            "workload": f"{name} {wl.shape[2]}x{wl.shape[1]}x{wl.shape[0]}, h={wl.h:g} m, f={wl.f:g} Hz, "
                        f"{wl.nrhs} sources",
            "nrhs": wl.nrhs, "rhs_per_rank": R, "points": N, "status": rep["status"],
            "value": round(N * wl.nrhs / (solve_ms / 1e3) / 1e6, 4), "unit": UNIT,
            "value_incl_setup": round(N * wl.nrhs / (wall_ms / 1e3) / 1e6, 4),
            "ms": round(wall_ms, 1), "setup_ms": round(rep["setup_ms"], 1), "solve_ms": round(solve_ms, 1),
            "inner_iters": rep["inner_iters"], "outer_iters": rep["outer_iters"],
            "mg_levels": rep["mg_levels"], "rel_residual": rep["rel_residual"], "clocks": clk,
        }
        # stencil roofline at this size (rank 0 only: one GPU's kernel)
        if rank == 0:
            roof = []
            nz, ny, nx = wl.shape
            pitch = (nx + 3) // 4 * 4              # the solver's complex64 layout (padded rows)
            for mode, nr in (("apply", 1), ("apply", 4), ("apply", 16), ("jacobi", 16)):
                x = torch.randn((nr, nz, ny, pitch), dtype=torch.complex64, device=dev)
                y = torch.empty_like(x)
                b = torch.randn_like(x) if mode == "jacobi" else None

                def launch():
                    if mode == "apply":
                        ctx.stencil_pitched(g, vd, "apply", x, None, y, pitch)
                    else:
                        ctx.stencil_pitched(g, vd, "jacobi", x, b, y, pitch, shift_beta=1.0, omega=0.6)

                # the fastest configuration of the layout's kernel (ids 3.. for even pitch),
                # two timed launches each after a warm-up, then the measurement with it
                best, best_ms = -1, 1e30
                for cfg in range(3, B.lib().hx_kernel_config_info(-1, None, None)):
                    rb = B.kernel_configs()[cfg][1]
                    if rb > 1 and rb >= 2 * nr:
                        continue
                    ctx.set_kernel_config(cfg)
                    launch()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    launch()
                    launch()
                    e1.record()
                    e1.synchronize()
                    if e0.elapsed_time(e1) < best_ms:
                        best, best_ms = cfg, e0.elapsed_time(e1)
                ctx.set_kernel_config(best)
                for _ in range(2):
                    launch()
                ts = []
                for _ in range(5):
                    flush.fill_(1.0)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    launch()
                    e1.record()
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ctx.set_kernel_config(-1)
                ms = statistics.median(ts)
                algo = (16 if mode == "apply" else 24) * N * nr + 4 * N
                roof.append({"mode": mode, "nrhs": nr, "kernel_config": best, "pitch": pitch,
                             "ms": round(ms, 4), "algo_bytes": algo,
                             "achieved": round(algo / ms / 1e6, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(algo / ms / 1e6 / hbm, 4)})
                del x, y, b
            entry["stencil_roofline"] = roof
            entry["stencil_peak_source"] = "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback"
        ctx.close()
        torch.cuda.empty_cache()
        res[name] = entry
    return res


def run_serving(args, T, nreq=None, seed0=5000, log=None):
    """Serving workload (hx_server): seeded requests from synth.serving_request
    (model family uniform over the four synthetic families, sides
    log-uniform in 64..256, f ~ U(2, 10) Hz, 1..32 sources, h = 25 m, 8-node
    PML), Poisson arrivals at a rate giving an offered load of 0.8 x the solo
    capacity measured on the first requests solved one at a time (faster when
    that would spread the arrivals over more than SERVE_MAX_SPAN_S), admitted
    smallest first.  Returns the
    serving summary (latency percentiles from submission to wavefield on the
    host, point*RHS/s over the busy interval)."""
    import numpy as np

    from paper_2108_08730_gb300 import binding as B
    from paper_2108_08730_gb300 import synth

    nreq = args.serve_requests if nreq is None else nreq
    reqs = [synth.serving_request(seed0 + k) for k in range(nreq)]
    work = np.array([r.n_points * r.nrhs for r in reqs], dtype=np.float64)
    # smallest request first (a request that has waited SERVE_MAX_WAIT_S goes
    # first), and the BiCGStab omega safeguard, which removes the stalls of the
    # strongly heterogeneous requests
    srv = B.Server(T, slots=args.serve_slots, order="smallest", max_wait_s=SERVE_MAX_WAIT_S)

    def submit(k, wl, limit):
        out = np.zeros((wl.nrhs,) + wl.shape, dtype=np.complex128)
        t = srv.submit(B.grid_of(wl), wl.v, B.sources_of(wl), wl.nrhs, out, model_id=seed0 + k,
                       time_limit_s=limit, bicg_kappa=SERVE_KAPPA)
        return t, out

    # solo capacity: the first requests one at a time (also warms the engine);
    # a calibration request that stops at its limit still counts its time, so
    # the estimate can only err low
    ncal = min(6, nreq)
    t0 = time.perf_counter()
    cal_failed = []
    for k in range(ncal):
        t, _ = submit(k, reqs[k], args.serve_deadline)
        r = srv.wait(t)
        if r["status"] != 0:
            cal_failed.append({"seed": seed0 + k, "status": r["status"]})
    solo = work[:ncal].sum() / (time.perf_counter() - t0)          # point*RHS/s
    # offered load 0.8 of the calibrated capacity, the arrivals spread over at
    # most SERVE_MAX_SPAN_S (bounds the leg's length when the calibration
    # requests happen to be slow)
    rate = max(0.8 * solo / work.mean(), nreq / SERVE_MAX_SPAN_S)    # requests/s
    srv.stats(reset=True)
    rng = np.random.default_rng(seed0)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
    tickets = []
    start = time.perf_counter()
    # a runaway guard scaled to the request (not a latency target): the base
    # plus the time the request takes with the GPU shared among the slots
    limits = [args.serve_deadline + args.serve_slots * w / solo for w in work]
    for k, wl in enumerate(reqs):
        dt = arrivals[k] - (time.perf_counter() - start)
        if dt > 0:
            time.sleep(dt)
        tickets.append(submit(k, wl, limits[k]))
    res = [srv.wait(t) for t, _ in tickets]
    st = srv.stats()
    srv.close()
    bad = [seed0 + k for k, r in enumerate(res) if r["status"] != 0]
    failures = [{"seed": seed0 + k, "status": r["status"], "inner_iters": r["report"]["inner_iters"],
                 "outer_iters": r["report"]["outer_iters"], "rel_residual": r["report"]["rel_residual"],
                 "queue_ms": round(r["queue_ms"], 1), "run_ms": round(r["run_ms"], 1),
                 "limit_s": round(limits[k], 1)}
                for k, r in enumerate(res) if r["status"] != 0]
    iters = [r["report"]["inner_iters"] for r in res]
    return {"requests": nreq, "slots": args.serve_slots, "completed": st["completed"],
            "failed": len(bad), "failed_seeds": bad, "failures": failures,
            "deadline_s": f"{args.serve_deadline:g} + {args.serve_slots} x point*RHS / solo capacity "
                          f"({min(limits):.1f} .. {max(limits):.1f} s)",
            "inner_iters_median": float(np.median(iters)), "inner_iters_max": int(max(iters)),
            "arrival_rate_per_s": round(rate, 4),
            "offered_load": round(rate * work.mean() / solo, 3),
            "admission": f"smallest point*RHS first; a request waiting {SERVE_MAX_WAIT_S:g} s or "
                         "longer goes first",
            "solve_options": f"library defaults with bicg_kappa = {SERVE_KAPPA:g}",
            "solo_capacity_mpoint_rhs_s": round(solo / 1e6, 3), "calibration_failures": cal_failed,
            "p50_ms": round(st["p50_ms"], 2),
            # a 99th percentile needs at least 100 completed requests
            "p99_ms": round(st["p99_ms"], 2) if st["completed"] >= 100 else None,
            "latency": "submission to wavefield on the host, completed requests",
            "max_ms": round(st["max_ms"], 2),
            "value": round(st["point_rhs"] / st["busy_s"] / 1e6, 4) if st["busy_s"] > 0 else None,
            "unit": "Mpoint*RHS/s", "max_concurrent": st["max_concurrent"],
            "peak_committed_gb": round(st["peak_committed"] / 1e9, 2),
            "mean_point_rhs": float(work.mean()),
            "recipe": "synth.serving_request seeds 5000.., families uniform over homogeneous / linear "
                      "gradient / sharp contrast / tectonic, sides log-uniform 64..256, f U(2,10) Hz, "
                      "1..32 sources, Poisson arrivals"}


def run_solve_config(args):
    """One mixed-precision solve of a full workload (all its sources as RHS):
    throughput from sources on the device to wavefields on the device, the
    FP64 relative residual the refinement reached, iteration counts, and the
    autotuned kernel configuration (tuning done before the timed solve)."""
    import torch

    from paper_2108_08730_gb300 import binding as B
    from paper_2108_08730_gb300 import synth

    nodes, T = B.build_weight_table()
    ctx = B.Context(0, table=T)
    wl = synth.CONFIGS[args.solve_config]()
    g = B.grid_of(wl)
    vd = torch.from_numpy(wl.v).cuda()
    R = wl.nrhs
    best, tms = ctx.autotune(g, vd, R)
    out = torch.zeros((R,) + wl.shape, dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rep = ctx.solve(g, vd, B.sources_of(wl), R, out, check=False, time_limit_s=args.solve_time_limit)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"solve_config": wl.name, "shape": list(wl.shape), "nrhs": R, "points": wl.n_points,
                      "status": rep["status"], "rel_residual": rep["rel_residual"],
                      "outer_iters": rep["outer_iters"], "inner_iters": rep["inner_iters"],
                      "mg_levels": rep["mg_levels"], "ms": round(ms, 1),
                      "value": round(wl.n_points * R / ms / 1e3, 3), "unit": UNIT,
                      "kernel_config": best, "config_ms": [round(t, 3) for t in tms],
                      "G_range": [round(float(wl.v.min()) / (wl.f * wl.h), 2),
                                  round(float(wl.v.max()) / (wl.f * wl.h), 2)]}), flush=True)


def run_kernel(args):
    """Time one operator kernel alone (complex64 or complex128) on a full-size
    model: --kernel-workload (tectonic 401x401x187 by default) with
    --kernel-nrhs right-hand sides, --kernel-mode apply or a sweep, plain
    fields or the solver's padded rows (--kernel-layout); L2 flushed before
    every timed launch."""
    import torch

    from paper_2108_08730_gb300 import binding as B
    from paper_2108_08730_gb300 import synth

    nodes, T = B.build_weight_table()
    ctx = B.Context(0, table=T)
    wl = synth.CONFIGS[args.kernel_workload]()
    g = B.grid_of(wl)
    vd = torch.from_numpy(wl.v).cuda()
    R = args.kernel_nrhs
    dt = torch.complex64 if args.kernel_prec == 32 else torch.complex128
    padded = args.kernel_layout == "padded"
    if padded and args.kernel_prec != 32:
        raise SystemExit("--kernel-layout padded is complex64 only")
    nz, ny, nx = wl.shape
    pitch = (nx + 3) // 4 * 4
    fshape = (R, nz, ny, pitch) if padded else (R,) + wl.shape
    x = torch.randn(fshape, dtype=dt, device="cuda")
    y = torch.empty_like(x)
    bb = torch.randn(fshape, dtype=dt, device="cuda") if args.kernel_mode != "apply" else None
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")

    def launch():
        if padded:
            ctx.stencil_pitched(g, vd, args.kernel_mode, x, bb, y, pitch,
                                shift_beta=0.0 if args.kernel_mode == "apply" else 1.0, omega=0.6)
        elif args.kernel_mode == "apply":
            ctx.apply(g, vd, x, y)
        else:
            ctx.sweep(g, vd, args.kernel_mode, x, bb, y, shift_beta=1.0, omega=0.6)

    if args.kernel_cfg == "tune":
        best, tms = ctx.autotune(g, vd, R)
        cfgs = [-1]
    elif args.kernel_cfg == "all":
        cfgs = list(range(len(B.kernel_configs())))
    else:
        cfgs = [-1 if args.kernel_cfg == "auto" else int(args.kernel_cfg)]
    for cfg in cfgs:
        ctx.set_kernel_config(cfg)
        for _ in range(args.warmup):
            launch()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            launch()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        cb = 8 if args.kernel_prec == 32 else 16
        streams = 2 if args.kernel_mode == "apply" else 3      # x (+ b) read, y written
        algo = streams * cb * wl.n_points * R + 4 * wl.n_points
        peaks = _peaks()
        peak = peaks["hbm_gbs"] if peaks else 6800.0
        print(json.dumps({"kernel": f"{args.kernel_mode} fp{args.kernel_prec}", "workload": wl.name,
                          "layout": args.kernel_layout + (f" (pitch {pitch})" if padded else ""),
                          "nrhs": R, "cfg": cfg if cfg >= 0 else args.kernel_cfg,
                          "points": wl.n_points, "ms": round(ms, 4),
                          "Gpoint_rhs_per_s": round(wl.n_points * R / ms / 1e6, 3),
                          "algo_bytes": algo, "achieved_gbs": round(algo / ms / 1e6, 1),
                          "peak_gbs": peak, "frac": round(algo / ms / 1e6 / peak, 4)}), flush=True)


def _relaunch_distributed(n):
    """`python bench.py --gpus N` with N > 1 and no launcher: run this script
    again under torch.distributed.run, one process per GPU (127.0.0.1
    rendezvous), and return its exit code."""
    import socket
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    args = _args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ and args.impl == "hx":
        sys.exit(_relaunch_distributed(args.gpus))
    if args.kernel:
        run_kernel(args)
    elif args.solve_config:
        run_solve_config(args)
    elif args.serve_only:
        from paper_2108_08730_gb300 import binding as B
        nodes, T = B.build_weight_table()
        print(json.dumps({"serving": run_serving(args, T)}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
