"""Serving loop: a stream of potential-field solves of mixed grid sizes.

Requests arrive at seeded Poisson times.  The continuous-batching server
admits each request into a pot3d batch as soon as a slot and device memory are
free, advances every admitted solve together (persistent graph-captured
kernels, FP32 PCG inside FP64 refinement) and retires solves as they finish,
which frees memory for the next admissions.  The baseline solves the same
requests one at a time in arrival order with native FP64 PCG.  Both record,
per request, completion time minus arrival time.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import pot3d

GRIDS = [(41, 61, 121), (81, 121, 241), (101, 181, 361), (151, 301, 601)]
RATIO = 1.02
TOL = 1e-10
SEED = 1709


@dataclass
class Request:
    rid: int
    grid: tuple
    arrival: float  # seconds after the start of the stream
    seed: int


@dataclass
class Outcome:
    rid: int
    grid: tuple
    arrival: float
    done: float
    status: int
    relres: float
    iters: int
    outer: int = 0
    relres_fp64: float = float("nan")  # ||b - L Phi|| / ||b|| of the served Phi

    @property
    def latency(self):
        return self.done - self.arrival


@dataclass
class ServeStats:
    kind: str
    outcomes: list = field(default_factory=list)
    wall: float = 0.0
    results: dict = field(default_factory=dict)  # rid -> (br, phi) device tensors, if kept

    def summary(self):
        lat = np.array([o.latency for o in self.outcomes])
        span = max(o.done for o in self.outcomes) - min(o.arrival for o in self.outcomes)
        true = [o.relres_fp64 for o in self.outcomes]
        return {"kind": self.kind, "solves": len(self.outcomes),
                "solves_per_s": len(self.outcomes) / span if span > 0 else None,
                "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)),
                "mean_latency_s": float(lat.mean()),
                "max_relres": float(max(o.relres for o in self.outcomes)),
                "max_relres_fp64": (None if any(np.isnan(t) for t in true)
                                    else float(max(true))),
                "all_ok": all(o.status == 0 for o in self.outcomes),
                "span_s": span}


def check_residuals(stats: ServeStats, plans):
    """After the stream: the FP64 residual ||b - L Phi|| / ||b|| of every
    served Phi, recomputed by the library's FP64 operator (outside the timed
    stream)."""
    for o in stats.outcomes:
        br, phi = stats.results[o.rid]
        o.relres_fp64 = plans[o.grid].residual(br, phi)


def make_requests(n: int, rate: float, grids=GRIDS, seed: int = SEED):
    """n requests, grids drawn uniformly from `grids`, exponential gaps of
    mean 1/rate; request i uses bipole seed `seed + i`."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n)
    gaps[0] = 0.0
    t = np.cumsum(gaps)
    gi = rng.integers(0, len(grids), n)
    return [Request(i, tuple(grids[gi[i]]), float(t[i]), seed + i) for i in range(n)]


def _br(req: Request):
    import pot3d_synth as syn

    return syn.bipole_br(req.grid[1], req.grid[2], seed=req.seed)


def prepare_inputs(requests):
    """Br maps of every request, made before the stream starts (input
    generation is not part of the served work)."""
    return {r.rid: _br(r) for r in requests}


def run_batched(requests, inputs, batch_bytes: int, k: int = 16, max_slots: int = 256,
                inner_tol: float = 0.0, verify: bool = True, keep: bool = False,
                precond: str = "jacobi"):
    """Serves `requests` with the continuous-batching mixed-precision path.
    verify: recompute every served Phi's FP64 residual after the stream;
    keep: keep the (Br, Phi) device tensors in the returned stats;
    precond: the inner solves' preconditioner ("jacobi" or "philine")."""
    import torch

    plans = {g: pot3d.Plan(*g, ratio=RATIO, precision="mixed") for g in {r.grid for r in requests}}
    for p in plans.values():
        p.autotune(4)  # FP32 kernels: tile variant, r-chunks, update rows
    batch = pot3d.Batch(batch_bytes, max_slots=max_slots, inner_tol=inner_tol, precond=precond)
    stats = ServeStats("mixed+batched" + ("" if precond == "jacobi" else " (%s)" % precond))
    pending = sorted(requests, key=lambda r: r.arrival)
    waiting, live = [], {}
    t0 = time.perf_counter()
    now = 0.0
    while pending or waiting or live:
        now = time.perf_counter() - t0
        while pending and pending[0].arrival <= now:
            waiting.append(pending.pop(0))
        while waiting:
            r = waiting[0]
            br = torch.from_numpy(inputs[r.rid]).cuda()
            phi = torch.empty(r.grid, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            if not batch.submit(plans[r.grid], br, TOL, phi, r.rid):
                break
            live[r.rid] = (r, br, phi)
            waiting.pop(0)
        if live:
            batch.step(k)
            for tag, st, outer, inner, relres in batch.poll():
                r, br, phi = live.pop(tag)
                stats.outcomes.append(Outcome(r.rid, r.grid, r.arrival, time.perf_counter() - t0,
                                              st, relres, inner, outer))
                if verify or keep:
                    stats.results[r.rid] = (br, phi)
        elif pending:
            time.sleep(max(0.0, min(0.002, pending[0].arrival - now)))
    stats.wall = time.perf_counter() - t0
    batch.close()
    torch.cuda.synchronize()
    if verify:
        check_residuals(stats, plans)
    if not keep:
        stats.results = {}
    for p in plans.values():
        p.close()
    return stats


def run_fp64_serial(requests, inputs, verify: bool = True, keep: bool = False):
    """Serves `requests` one at a time in arrival order with native FP64 PCG.
    Each solve runs with opts.verify, so it stops on the recomputed FP64
    residual, the same criterion as the refinement path (equal final
    accuracy by construction)."""
    import torch

    plans = {g: pot3d.Plan(*g, ratio=RATIO, precision="fp64", verify=1)
             for g in {r.grid for r in requests}}
    for p in plans.values():
        p.autotune(1)
    stats = ServeStats("fp64 one-at-a-time")
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda q: q.arrival):
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        br = torch.from_numpy(inputs[r.rid]).cuda()
        phi = torch.empty(r.grid, dtype=torch.float64, device="cuda")
        rc, it = plans[r.grid].solve(br, TOL, phi, check=False)
        torch.cuda.synchronize()
        st = plans[r.grid].stats()
        stats.outcomes.append(Outcome(r.rid, r.grid, r.arrival, time.perf_counter() - t0, rc,
                                      st["relres"], it, st["outer_iters"]))
        if verify or keep:
            stats.results[r.rid] = (br, phi)
    stats.wall = time.perf_counter() - t0
    if verify:
        check_residuals(stats, plans)
    if not keep:
        stats.results = {}
    for p in plans.values():
        p.close()
    return stats


def calibrate_fp64_rate(grids=GRIDS):
    """FP64 one-at-a-time solve rate over the grid mix (solves per second),
    from one solve of each grid."""
    import torch

    import pot3d_synth as syn

    times = []
    for g in grids:
        plan = pot3d.Plan(*g, ratio=RATIO, precision="fp64")
        plan.autotune(1)
        br = torch.from_numpy(syn.bipole_br(g[1], g[2], seed=SEED)).cuda()
        phi = torch.empty(g, dtype=torch.float64, device="cuda")
        plan.solve(br, TOL, phi)  # warm
        torch.cuda.synchronize()
        t = time.perf_counter()
        plan.solve(br, TOL, phi)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
        plan.close()
    return 1.0 / float(np.mean(times)), times
