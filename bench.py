"""Benchmark of the potential-field PCG solve on GB300.

One step = one full solve of the 151 x 301 x 601 problem (geometric r mesh,
ratio 1.02; flux-balanced dipole + 200-bipole synthetic Br, seed 1709;
Jacobi PCG to relative residual 1e-10) plus the field B = grad Phi, with
inputs and outputs resident in HBM.  value = PCG iterations per second over
the timed steps (all ranks).  Each rank of a multi-GPU launch solves its own
replica (weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|df|mixed]
    python bench.py --impl reference ...   # the CPU oracle as the reference arm
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("PCG iters/s + HBM GB/s (151×301×601 FP64); solves/s & p99, "
          "mixed+batched vs FP64")
SHAPE = (151, 301, 601)
RATIO = 1.02
TOL = 1e-10
SEED = 1709
DTYPES = {"fp64": "f64", "df": "f32x2", "mixed": "f32+f64"}


# ----------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend):
    ws, rank, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group(backend)
        return dist
    return None


def reduce_max(x: float, dist, device=None) -> float:
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, dist, device=None) -> float:
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(dist, device=None):
    if dist is not None:
        import torch

        t = torch.zeros(1, device=device)
        dist.all_reduce(t)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# DRAM bytes (read + write) per launch of the dominant kernel, from the ncu
# captures summarised in profiles/k_matvec_151x301x601.md (same
# kernels and tuned configuration as timed here)
TRAFFIC = {"fp64": 1.2927e9, "df": 1.2851e9, "mixed": 0.6223e9}

# FP64 FMA units: 152 SMs x 2 per clock at the 2070 MHz maximum SM clock
# (nominal; the roofline uses the rate measured by pot3d_probe_fp64_fma)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
HBM_NOMINAL_GBS = 7900.0

_fp64_peak = None


def fp64_peak(pot3d):
    """Measured FP64 peak (TFLOP/s) from the library's DFMA throughput probe,
    with the SM clock sampled while it ran; measured once per process."""
    global _fp64_peak
    if _fp64_peak is None:
        pot3d.probe_fp64_fma(0.1)  # warm-up
        clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
        clk.start()
        rate, el = pot3d.probe_fp64_fma(1.0)
        c = clk.stop()
        _fp64_peak = {"tflops": 2.0 * rate / 1e12, "seconds": el, "clocks": c,
                      "how": "pot3d_probe_fp64_fma: 8 independent DFMA chains per thread, "
                             "2048 threads per SM, CUDA events"}
    return _fp64_peak


# FP64 FMAs per point of the matvec kernel (p~ and x~ updates, 6-term
# scaled stencil, sigma term): the algorithmic count, halo work excluded
FP64_FMA_PER_POINT_MATVEC = 9.0


# ------------------------------------------------------------- workloads
def make_br():
    import pot3d_synth as syn

    return syn.bipole_br(SHAPE[1], SHAPE[2], seed=SEED)


def cpu_baseline(br, iters=60):
    """The oracle as it stands, on the host cores, for a bounded sample:
    the first `iters` PCG iterations of the same 151x301x601 solve."""
    import oracle

    oracle.build()
    n = os.cpu_count() or 1
    oracle.set_threads(n)
    g = oracle.Grid(*SHAPE, ratio=RATIO)
    b = g.rhs(br)
    g.pcg(b, 1e-300, maxit=2)  # warm the pages
    t = time.perf_counter()
    x, it, st = g.pcg(b, 1e-300, maxit=iters)
    dt = time.perf_counter() - t
    cores = oracle.get_threads()
    # the same oracle on one thread, over a shorter sample
    oracle.set_threads(1)
    t1 = time.perf_counter()
    x1, it1, st1 = g.pcg(b, 1e-300, maxit=max(2, iters // 10))
    dt1 = time.perf_counter() - t1
    oracle.set_threads(n)
    return {"value": it / dt, "unit": "iters/s", "cores": cores, "kind": "oracle",
            "sample": "first %d PCG iterations of the 151x301x601 solve (of ~6000 to 1e-10), "
                      "FP64, OpenMP" % it, "seconds": dt,
            "single_thread": {"value": it1 / dt1, "unit": "iters/s", "cores": 1,
                              "sample": "first %d PCG iterations" % it1, "seconds": dt1}}


GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_151x301x601.json")


def sampled_error_vs_oracle(phi):
    """Relative L2 error of Phi on the stratified sample of cells stored with
    the oracle's own solve of this workload to 1e-10 (None if the file is
    absent)."""
    try:
        with open(GOLDEN) as f:
            gold = json.load(f)
        idx = np.asarray(gold["sample_index"], dtype=np.int64)
        ref = np.asarray(gold["tol_1e-10"]["sample_phi"])
    except (OSError, ValueError, KeyError):
        return None
    x = phi.reshape(-1)[idx.tolist()].cpu().numpy()
    return {"value": float(np.linalg.norm(x - ref) / np.linalg.norm(ref)), "samples": int(idx.size),
            "source": "tests/golden/oracle_151x301x601.json (oracle PCG to 1e-10, stratified "
                      "sample incl. boundary layers, pole rings, phi-wrap columns)"}


def workload_config(prec, ws):
    """The benchmark workload, identical on the GPU arm and the reference arm."""
    return {"workload": "potential-field PCG 151x301x601, r geometric 1.02, "
                        "dipole + 200 bipoles (seed 1709), tol 1e-10, + field",
            "grid": list(SHAPE), "tol": TOL, "precision": prec,
            "l2": "inputs larger than L2 (each vector %.0f MB)"
                  % ((4 if prec == "mixed" else 8) * SHAPE[0] * SHAPE[1] * SHAPE[2] / 1e6),
            "parallelism": "replicas x%d" % ws}


def run_reference(args):
    ws, rank, _ = dist_env()
    dist = dist_init("gloo")
    if rank != 0:
        barrier(dist)
        return 0
    br = make_br()
    import oracle

    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    g = oracle.Grid(*SHAPE, ratio=RATIO)
    b = g.rhs(br)
    per_step = 20
    for _ in range(args.warmup):
        g.pcg(b, 1e-300, maxit=per_step)
    t = time.perf_counter()
    total = 0
    for _ in range(args.steps):
        x, it, st = g.pcg(b, 1e-300, maxit=per_step)
        total += it
    dt = time.perf_counter() - t
    v = total / dt
    line = {"metric": METRIC, "value": v, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": workload_config(args.prec, 1),
            "cpu_baseline": {"value": v, "unit": "iters/s", "kind": "oracle",
                             "cores": oracle.get_threads(),
                             "sample": "each step: the first %d PCG iterations of this solve "
                                       "(FP64 oracle, OpenMP)" % per_step},
            "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    barrier(dist)
    return 0


KT_ITERS = 300


def kernel_times(plan, prec, br_d, phi, torch, dev):
    """Average duration of the matvec and update kernels, from CUDA events
    around every launch (time_kernels) over the first KT_ITERS iterations of
    the same solve, on the plan's tuned configuration."""
    if prec == "mixed":
        plan.set_opts(time_kernels=1, max_iters=KT_ITERS, max_outer=1)
        plan.solve_mixed(br_d, TOL, phi, check=False)
    else:
        plan.set_opts(time_kernels=1, max_iters=KT_ITERS)
        plan.solve(br_d, TOL, phi, check=False)
    torch.cuda.synchronize(dev)
    km = plan.stats()["kernel_ms"]
    plan.set_opts()
    return km[0] / max(km[2], 1), km[1] / max(km[3], 1)


def field_time(plan, br_d, phi, B, torch, dev, reps=5):
    """Device time of pot3d_field (pole averages + staggered B = grad Phi)
    between CUDA events on the plan's stream, averaged over `reps` calls,
    against its algorithmic bytes: Phi and Br read once, the three face
    components written once (about 32 B per unknown)."""
    nr, nt, np_ = SHAPE
    n = nr * nt * np_
    nbytes = 8.0 * (n + nt * np_) + 8.0 * sum(plan.field_sizes())
    stream = torch.cuda.current_stream(dev)
    plan.field(phi, br_d, B)  # warm
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        plan.field(phi, br_d, B)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    peaks, _ = measured_peaks()
    return {"avg_call_ms": ms, "algorithmic_bytes": nbytes, "GB_s": nbytes / (ms * 1e-3) / 1e9,
            "frac_of_measured_hbm": nbytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "launches_per_call": 2}


def measure(pot3d, torch, dev, dist, br, br_d, prec, steps, warmup, with_e2e=True):
    """Times `steps` solves (+ field) of one precision after `warmup` solves."""
    ws, rank, local = dist_env()
    # the library's default path: chunks of iterations as CUDA graphs
    plan = pot3d.Plan(*SHAPE, ratio=RATIO, precision=prec)
    # kernel variant and r-chunking chosen by the autotuner (before timing)
    tuned = plan.autotune(4 if prec == "mixed" else 0)
    info = plan.info()
    phi = torch.zeros(SHAPE, dtype=torch.float64, device=dev)
    B = torch.empty(sum(plan.field_sizes()), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        if prec == "mixed":
            rc, o, it = plan.solve_mixed(br_d, TOL, phi)
        else:
            rc, it = plan.solve(br_d, TOL, phi)
        st = plan.stats()
        plan.field(phi, br_d, B)
        return it, st

    last = {}

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(dist, dev)
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    iters, launches = 0, 0
    for _ in range(steps):
        it, st = step()
        last = st
        iters += it
        launches += st["launches"] + 2  # + the field's two kernels
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(dist, dev)
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    ms_max = reduce_max(ms, dist, dev)
    iters_all = reduce_sum(iters, dist, dev)
    value = iters_all / (ms_max * 1e-3)
    es = 4 if prec == "mixed" else 8
    n = SHAPE[0] * SHAPE[1] * SHAPE[2]
    bytes_per_iter = 9.0 * es * n  # 6 vectors touched by the matvec + 3 by the update
    peaks, src = measured_peaks()
    # Phi of the last timed solve, before the kernel-time pass reuses phi
    err = sampled_error_vs_oracle(phi)
    mv_ms, up_ms = kernel_times(plan, prec, br_d, phi, torch, dev)
    hbm_mv = info["bytes_matvec"] / (mv_ms * 1e-3) / 1e9
    if prec == "fp64":
        achieved = 2 * FP64_FMA_PER_POINT_MATVEC * n / (mv_ms * 1e-3) / 1e12
        pk = fp64_peak(pot3d)
        roof = {"bound": "alu", "kernel": "k_matvec<PF64>", "achieved": achieved,
                "peak": pk["tflops"], "unit": "TFLOP/s", "frac": achieved / pk["tflops"],
                "traffic": TRAFFIC.get(prec), "peak_source": "measured",
                "peak_measurement": pk,
                "nominal_peak": FP64_PEAK_TFLOPS,
                "frac_of_nominal": achieved / FP64_PEAK_TFLOPS,
                "nominal_source": "FP64 FMA units x max SM clock: 152 x 2/clk x 2 flop x 2.07 GHz",
                "hbm_GB_s": hbm_mv,
                "hbm_frac_of_measured": hbm_mv / peaks["hbm_gbs"],
                "hbm_frac_of_nominal": hbm_mv / HBM_NOMINAL_GBS}
    else:
        achieved = hbm_mv
        roof = {"bound": "hbm", "kernel": "k_matvec<%s>" % ("PDF" if prec == "df" else "PF32"),
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": TRAFFIC.get(prec),
                "peak_source": "%s: MEASURED_PEAKS.json hbm_gbs" % src,
                "frac_of_nominal": achieved / HBM_NOMINAL_GBS,
                "nominal_peak": HBM_NOMINAL_GBS}
    roof["avg_launch_ms"] = mv_ms
    roof["algorithmic_bytes_per_launch"] = info["bytes_matvec"]
    up_gbs = info["bytes_update"] / (up_ms * 1e-3) / 1e9 if up_ms else None
    roof["update_kernel"] = {"avg_launch_ms": up_ms, "GB_s": up_gbs,
                             "frac_of_measured_hbm": up_gbs / peaks["hbm_gbs"] if up_gbs else None,
                             "frac_of_nominal_hbm": up_gbs / HBM_NOMINAL_GBS if up_gbs else None}
    roof["field_kernels"] = field_time(plan, br_d, phi, B, torch, dev)
    out = {"value": value, "unit": "iters/s", "ms_per_step": ms_max / steps, "dtype": DTYPES[prec],
           "autotune": {"matvec_variant": tuned[0], "r_chunks": tuned[1], "matvec_ms": tuned[2]},
           "iters_per_solve": iters / steps, "hbm_gbs": value / ws * bytes_per_iter / 1e9,
           "bytes_per_iter": bytes_per_iter, "roofline": roof, "gpu_launches": launches,
           "clocks": clk, "steps": steps, "warmup": warmup,
           "final_relres": last.get("relres"),
           "final_relres_kind": ("FP64 residual recomputed" if prec == "mixed"
                                 else "PCG recurrence residual")}
    if prec == "mixed":
        out["outer_per_solve"] = last.get("outer_iters")
    if err is not None:
        out["sampled_rel_error_vs_oracle"] = err
    if with_e2e:
        # end to end through the same C ABI with pinned host buffers
        br_h = torch.from_numpy(br).pin_memory().numpy()
        phi_h = torch.zeros(SHAPE, dtype=torch.float64).pin_memory().numpy()
        B_h = torch.zeros(B.numel(), dtype=torch.float64).pin_memory().numpy()
        e2e_steps = max(1, min(steps, 2))
        barrier(dist, dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e_iters = 0
        for _ in range(e2e_steps):
            if prec == "mixed":
                rc, o, it = plan.solve_mixed(br_h, TOL, phi_h)
            else:
                rc, it = plan.solve(br_h, TOL, phi_h)
            plan.field(phi_h, br_h, B_h)
            e_iters += it
        torch.cuda.synchronize(dev)
        e_dt = reduce_max(time.perf_counter() - t0, dist, dev)
        e_iters = reduce_sum(e_iters, dist, dev)
        out["e2e"] = {"value": e_iters / e_dt, "unit": "iters/s",
                      "h2d_bytes_per_step": br_h.nbytes * 2 + phi_h.nbytes,  # solve Br; field Br, Phi
                      "d2h_bytes_per_step": phi_h.nbytes + B_h.nbytes}
    plan.close()
    return out


def run_gpu(args):
    import torch

    from paper_1709_01126_gb300 import pot3d

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init("nccl")
    pot3d.load()
    br = make_br()
    br_d = torch.from_numpy(br).to(dev)
    head = measure(pot3d, torch, dev, dist, br, br_d, args.prec, args.steps, args.warmup)
    result = {
        "metric": METRIC, "value": head["value"], "unit": "iters/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": head["dtype"],
        "data": "synthetic",
        "config": dict(workload_config(args.prec, ws), iters_per_solve=head["iters_per_solve"]),
        "hbm_gbs": head["hbm_gbs"], "bytes_per_iter": head["bytes_per_iter"],
        "roofline": head["roofline"], "e2e": head["e2e"], "gpu_launches": head["gpu_launches"],
        "autotune": head["autotune"],
        "clocks": head["clocks"],
        "final_relres": head.get("final_relres"), "final_relres_kind": head.get("final_relres_kind"),
        "sampled_rel_error_vs_oracle": head.get("sampled_rel_error_vs_oracle"),
    }
    variants = {}
    for pv in args.variants:
        if pv == args.prec:
            continue
        v = measure(pot3d, torch, dev, dist, br, br_d, pv, steps=4, warmup=2, with_e2e=False)
        variants[pv] = v
    if variants:
        result["variants"] = variants
    if ws == 1 and args.precond_compare:
        result["precond_comparison"] = precond_record(pot3d, torch, dev, br_d)
    if ws == 1 and args.serve_requests > 0:
        # the second half of the metric: mixed + batched serving vs FP64
        # one-at-a-time on one seeded stream (not part of the timed PCG steps)
        result["serve"] = serve_record(args.serve_requests, args.batch_k, args.inner_tol)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(br)
    if rank == 0:
        print(json.dumps(result), flush=True)
    barrier(dist, dev)
    return 0


def precond_record(pot3d, torch, dev, br_d, steps=1):
    """Time to solution of the same 151x301x601 solve to 1e-10 with diagonal
    scaling (PC1, the paper's), with the line preconditioners (phi lines,
    radial lines, both directions) and with PC2 (the paper's subdomain
    ILU(0)), in FP64 and in the mixed path: PCG
    iterations, seconds per solve (CUDA events on torch's stream, after one
    warm-up solve) and the FP64 residual of the result."""
    out = {}
    stream = torch.cuda.current_stream(dev)
    phi = torch.zeros(SHAPE, dtype=torch.float64, device=dev)
    for prec in ("fp64", "mixed"):
        out[prec] = {}
        for pc in ("jacobi", "philine", "rline", "lines", "ilu"):
            plan = pot3d.Plan(*SHAPE, ratio=RATIO, precision=prec, precond=pc)
            plan.autotune(4 if prec == "mixed" else 0)
            plan.set_opts(precond=pc)

            def solve():
                if prec == "mixed":
                    rc, o, it = plan.solve_mixed(br_d, TOL, phi)
                else:
                    rc, it = plan.solve(br_d, TOL, phi)
                return it

            solve()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            its = [solve() for _ in range(steps)]
            e1.record(stream)
            torch.cuda.synchronize(dev)
            sec = e0.elapsed_time(e1) / 1e3 / steps
            st = plan.stats()
            out[prec][pc] = {"iters": its[-1], "outer": st["outer_iters"], "s_per_solve": sec,
                             "relres_fp64": st["relres_fp64"],
                             "iters_per_s": its[-1] / sec}
            plan.close()
        j = out[prec]["jacobi"]
        for pc in ("philine", "rline", "lines", "ilu"):
            l = out[prec][pc]
            l["speedup_time_to_solution"] = j["s_per_solve"] / l["s_per_solve"]
            l["iteration_ratio"] = j["iters"] / l["iters"]
    return out


def serve_record(requests, batch_k=16, inner_tol=0.0):
    """Serving stream: seeded Poisson arrivals of solves on grids drawn from
    41x61x121, 81x121x241, 101x181x361 and 151x301x601 (bipole Br with seed
    1709 + request id, tol 1e-10), served by the continuous-batching mixed
    path and by FP64 one-at-a-time solves (opts.verify: they stop on the FP64
    residual, as the refinement path does) on the same trace.  The arrival
    rate is 1.5x the calibrated FP64 one-at-a-time solve rate over the grid
    mix.  Every served Phi's FP64 residual is recomputed after the stream
    (pot3d_residual) and the largest is reported per server.  Capacity: the
    same requests all present at t = 0, batched, against the calibrated FP64
    one-at-a-time rate."""
    import torch

    from paper_1709_01126_gb300 import pot3d, serve

    pot3d.load()
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    rate64, times = serve.calibrate_fp64_rate()
    rate = 1.5 * rate64
    reqs = serve.make_requests(requests, rate)
    inputs = serve.prepare_inputs(reqs)
    free, total = torch.cuda.mem_get_info()
    budget = int(min(0.5 * free, 96e9))
    batched = serve.run_batched(reqs, inputs, batch_bytes=budget, k=batch_k,
                                inner_tol=inner_tol)
    batched_l = serve.run_batched(reqs, inputs, batch_bytes=budget, k=batch_k,
                                  inner_tol=inner_tol, precond="philine")
    base = serve.run_fp64_serial(reqs, inputs)
    # capacity: the same requests all present at t = 0
    sat_reqs = [serve.Request(r.rid, r.grid, 0.0, r.seed) for r in reqs]
    sat = serve.run_batched(sat_reqs, inputs, batch_bytes=budget, k=batch_k,
                            inner_tol=inner_tol).summary()
    sat_l = serve.run_batched(sat_reqs, inputs, batch_bytes=budget, k=batch_k,
                              inner_tol=inner_tol, precond="philine").summary()
    clocks = clk.stop()
    b, bl, f = batched.summary(), batched_l.summary(), base.summary()
    return {"requests": requests, "arrival_rate_per_s": rate,
            "workload": "serving stream of %d solves, Poisson arrivals at %.3f/s (1.5x FP64 "
                        "rate), grids %s, tol 1e-10" % (requests, rate, serve.GRIDS),
            "batch_arena_bytes": budget, "step_iters": batch_k,
            "batched": b, "batched_phi_line": bl, "fp64_one_at_a_time": f,
            "speedup_solves_per_s": b["solves_per_s"] / f["solves_per_s"],
            "p99_ratio_fp64_over_batched": f["p99_latency_s"] / b["p99_latency_s"],
            "p99_ratio_fp64_over_batched_phi_line": f["p99_latency_s"] / bl["p99_latency_s"],
            "capacity_solves_per_s": {"batched_all_at_t0": sat["solves_per_s"],
                                      "batched_all_at_t0_max_relres_fp64": sat["max_relres_fp64"],
                                      "batched_phi_line_all_at_t0": sat_l["solves_per_s"],
                                      "batched_phi_line_all_at_t0_max_relres_fp64":
                                          sat_l["max_relres_fp64"],
                                      "fp64_one_at_a_time": rate64,
                                      "ratio": sat["solves_per_s"] / rate64,
                                      "ratio_phi_line": sat_l["solves_per_s"] / rate64},
            "fp64_calibration_s": dict(zip(["x".join(map(str, g)) for g in serve.GRIDS], times)),
            "clocks": clocks}


def run_serve(args):
    rec = serve_record(args.requests, args.batch_k, args.inner_tol)
    b = rec["batched"]
    line = {"metric": METRIC, "value": b["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": args.requests, "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "workload_kind": "serve",
            "config": {"workload": rec["workload"], "batch_arena_bytes": rec["batch_arena_bytes"],
                       "step_iters": rec["step_iters"]},
            "clocks": rec["clocks"], "serve": rec}
    print(json.dumps(line), flush=True)
    return 0


def run_large(args):
    """The largest single-GPU case, 401 x 801 x 1601 (514 M unknowns, same
    stretching and Br generator): PCG iterations/s over a fixed number of
    iterations per step (the full solve needs far more iterations than a
    benchmark run can afford), FP64 and double-float."""
    import torch

    from paper_1709_01126_gb300 import pot3d
    import pot3d_synth as syn

    pot3d.load()
    shape = (401, 801, 1601)
    br_d = torch.from_numpy(syn.bipole_br(shape[1], shape[2], seed=SEED)).cuda()
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    n = shape[0] * shape[1] * shape[2]
    out = {}
    peaks, src = measured_peaks()
    for prec in ("fp64", "df"):
        plan = pot3d.Plan(*shape, ratio=RATIO, precision=prec, max_iters=args.large_iters)
        tuned = plan.autotune(0)
        plan.solve(br_d, 1e-300, phi, check=False)  # warm-up
        torch.cuda.synchronize()
        t = time.perf_counter()
        iters = 0
        for _ in range(args.steps):
            rc, it = plan.solve(br_d, 1e-300, phi, check=False)
            iters += it
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        # per-kernel durations: event-timed launches of the same iterations
        plan.set_opts(max_iters=min(args.large_iters, 50), time_kernels=1)
        plan.solve(br_d, 1e-300, phi, check=False)
        torch.cuda.synchronize()
        st = plan.stats()
        info = plan.info()
        mv = st["kernel_ms"][0] / max(st["kernel_ms"][2], 1)
        up = st["kernel_ms"][1] / max(st["kernel_ms"][3], 1)
        out[prec] = {"iters_per_s": iters / dt, "matvec_ms": mv, "update_ms": up,
                     "matvec_GB_s": info["bytes_matvec"] / (mv * 1e-3) / 1e9,
                     "update_GB_s": info["bytes_update"] / (up * 1e-3) / 1e9,
                     "hbm_GB_s_per_iter_model": 72.0 * n * iters / dt / 1e9,
                     "workspace_GB": info["workspace_bytes"] / 1e9,
                     "autotune": {"matvec_variant": tuned[0], "r_chunks": tuned[1]}}
        plan.close()
    line = {"metric": METRIC, "value": out["fp64"]["iters_per_s"], "unit": "iters/s",
            "n_gpus": 1, "steps": args.steps, "warmup": 1, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "workload_kind": "large",
            "config": {"workload": "401x801x1601 (514M unknowns), r geometric 1.02, 200 bipoles, "
                                   "%d PCG iterations per step" % args.large_iters,
                       "hbm_peak_GB_s": peaks["hbm_gbs"]},
            "fp64": out["fp64"], "df": out["df"]}
    print(json.dumps(line), flush=True)
    return 0


def run_profile_case(args):
    """Short solve for ncu: the same 151x301x601 problem, capped at a few
    PCG iterations so a capture ends quickly."""
    import torch

    from paper_1709_01126_gb300 import pot3d

    pot3d.load()
    br_d = torch.from_numpy(make_br()).cuda()
    plan = pot3d.Plan(*SHAPE, ratio=RATIO, precision=args.profile_case,
                      max_iters=args.profile_iters, use_graphs=-1, precond=args.precond)
    plan.autotune(4 if args.profile_case == "mixed" else 0)  # the bench's kernel configuration
    phi = torch.zeros(SHAPE, dtype=torch.float64, device="cuda")
    if args.profile_case == "mixed":
        plan.set_opts(max_iters=args.profile_iters, use_graphs=-1, max_outer=1,
                      precond=args.precond)
        plan.solve_mixed(br_d, TOL, phi, check=False)
    else:
        plan.solve(br_d, TOL, phi, check=False)
    torch.cuda.synchronize()
    if args.profile_field:
        B = torch.empty(sum(plan.field_sizes()), dtype=torch.float64, device="cuda")
        for _ in range(3):
            plan.field(phi, br_d, B)
        torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "iters": plan.stats()["iters"]}))
    plan.close()
    return 0


def run_large_solve(args):
    """Full solves of the 401 x 801 x 1601 case to the benchmark tolerance:
    time to solution, iterations and the FP64 relative residual of the
    result, per precision (the r stretching ratio is a flag: the literal
    1.02 over 401 cells makes a first-to-last cell ratio of 2755)."""
    import torch

    from paper_1709_01126_gb300 import pot3d
    import pot3d_synth as syn

    pot3d.load()
    shape = (401, 801, 1601)
    br_d = torch.from_numpy(syn.bipole_br(shape[1], shape[2], seed=SEED)).cuda()
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    out = {}
    for prec in [p for p in args.large_precs.split(",") if p]:
        plan = pot3d.Plan(*shape, ratio=args.large_ratio, precision=prec,
                          max_iters=args.large_maxit, verify=1 if args.large_verify else 0,
                          precond=args.precond)
        tuned = plan.autotune(4 if prec == "mixed" else 0)
        phi.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        if prec == "mixed":
            rc, outer, it = plan.solve_mixed(br_d, TOL, phi, check=False)
        else:
            rc, it = plan.solve(br_d, TOL, phi, check=False)
            outer = 0
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        if prec != "mixed":
            outer = plan.stats()["outer_iters"]  # residual replacements (verify)
        out[prec] = {"status": rc, "seconds": dt, "iters": it, "outer": outer,
                     "precond": args.precond,
                     "verify": bool(args.large_verify) and prec != "mixed",
                     "iters_per_s": it / dt, "relres_fp64": plan.residual(br_d, phi),
                     "autotune": {"matvec_variant": tuned[0], "r_chunks": tuned[1]}}
        plan.close()
        print(json.dumps({"large_solve": prec, **out[prec]}), file=sys.stderr, flush=True)
    first = next(iter(out.values()))
    line = {"metric": "time to solution (401x801x1601 to %g)" % TOL, "value": first["seconds"],
            "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES.get(next(iter(out)), "f64"),
            "data": "synthetic", "workload_kind": "large-solve",
            "config": {"workload": "401x801x1601 (514M unknowns), r geometric %g, 200 bipoles "
                                   "(seed 1709), tol %g" % (args.large_ratio, TOL)},
            "solves": out}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "df", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", default="df,mixed",
                    help="other precisions measured briefly on the same line ('' for none)")
    ap.add_argument("--profile-case", choices=["fp64", "df", "mixed"], default=None,
                    help="run a short capped solve for ncu and exit")
    ap.add_argument("--profile-iters", type=int, default=6)
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "philine", "rline", "lines", "ilu"],
                    help="the preconditioner of --profile-case and --workload large-solve")
    ap.add_argument("--profile-field", action="store_true",
                    help="with --profile-case: also three field evaluations")
    ap.add_argument("--workload", default="pcg", choices=["pcg", "serve", "large", "large-solve"])
    ap.add_argument("--large-precs", default="df,mixed",
                    help="precisions of --workload large-solve, comma-separated")
    ap.add_argument("--large-ratio", type=float, default=RATIO)
    ap.add_argument("--large-maxit", type=int, default=60000)
    ap.add_argument("--large-verify", action="store_true",
                    help="large-solve: FP64/double-float restart on the FP64 residual (opts.verify)")
    ap.add_argument("--large-iters", type=int, default=200)
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--no-precond-compare", dest="precond_compare", action="store_false",
                    help="skip the diagonal vs phi-line preconditioner comparison")
    ap.add_argument("--serve-requests", type=int, default=64,
                    help="requests of the serving record in the default run (0: none)")
    ap.add_argument("--batch-k", type=int, default=16)
    ap.add_argument("--inner-tol", type=float, default=0.0)
    args = ap.parse_args()
    args.variants = [v for v in args.variants.split(",") if v]
    if args.profile_case:
        return run_profile_case(args)
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "large":
        return run_large(args)
    if args.workload == "large-solve":
        return run_large_solve(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
