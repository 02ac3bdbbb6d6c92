"""Writes tests/golden/oracle_151x301x601.json from the CPU oracle only.

The 151 x 301 x 601 problem (geometric r, ratio 1.02; dipole + 200 bipoles,
seed 1709; the benchmark's workload) takes the oracle minutes per solve, so
its results are stored for the GPU tests:

- for tol 1e-10 and 1e-12: the stopping iteration and Phi at a stratified
  sample of cells (every boundary-folded layer is represented: the inner
  layer i = 0, the source-surface layer i = nr-1, both pole rings j = 0 and
  j = nt-1, the phi-wrap columns k = 0 and k = np-1, the eight corners, and
  interior cells);
- the oracle's own residual history ||r_k|| / ||b|| from k = 0 to 30
  iterations past the 1e-12 stop (PCG continued with tol = 0), so that a
  test can read the oracle's residual on both sides of any stop;
- the same history under other OpenMP thread counts, whose reductions add in
  other orders (equally valid roundings of the same method): the iteration
  at which each crosses 1e-10 and 1e-12, and the largest relative difference
  between its history and the main one.

Run from the repo root:  python tests/golden/make_golden_large.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import pot3d_synth as syn  # noqa: E402

SHAPE, RATIO, SEED = (151, 301, 601), 1.02, 1709
TOLS = (1e-10, 1e-12)
MAIN_THREADS = 8
OTHER_THREADS = (4, 6)
EXTRA = 30


def stratified_index(shape, seed=1, per_face=16, interior=64):
    """Flat indices of a stratified sample of cells (C order, phi fastest)."""
    nr, nt, np_ = shape
    rng = np.random.default_rng(seed)
    cells = []

    def some(n, fix):
        for _ in range(n):
            c = [int(rng.integers(0, nr)), int(rng.integers(0, nt)), int(rng.integers(0, np_))]
            for ax, v in fix.items():
                c[ax] = v
            cells.append(tuple(c))

    some(per_face, {0: 0})            # inner layer (Br folded into b, Eq. 2)
    some(per_face, {0: nr - 1})       # source-surface layer (mirror ghost)
    some(per_face, {1: 0})            # north pole ring (zero-area pole face)
    some(per_face, {1: nt - 1})       # south pole ring
    some(per_face, {2: 0})            # phi wrap, k = 0
    some(per_face, {2: np_ - 1})      # phi wrap, k = np-1
    for i in (0, nr - 1):
        for j in (0, nt - 1):
            for k in (0, np_ - 1):
                cells.append((i, j, k))
    some(interior, {})
    seen, out = set(), []
    for c in cells:
        f = (c[0] * nt + c[1]) * np_ + c[2]
        if f not in seen:
            seen.add(f)
            out.append(f)
    return out


def first_crossing(hist, tol):
    for k, v in enumerate(hist):
        if v <= tol:
            return k
    return None


def make():
    br = syn.bipole_br(SHAPE[1], SHAPE[2], seed=SEED)
    g = oracle.Grid(*SHAPE, ratio=RATIO)
    b = g.rhs(br)
    idx = stratified_index(SHAPE)
    out = {"shape": list(SHAPE), "ratio": RATIO, "br": "bipole_br(seed=1709, 200 bipoles)",
           "sample": "stratified: i=0, i=nr-1, j=0, j=nt-1, k=0, k=np-1 (16 each), "
                     "8 corners, 64 interior; seed 1",
           "sample_index": idx}
    oracle.set_threads(MAIN_THREADS)
    for tol in TOLS:
        t = time.time()
        x, it, st = g.pcg(b, tol)
        out["tol_%g" % tol] = {"iters": it, "status": st, "seconds": time.time() - t,
                               "sample_phi": [float(v) for v in x.ravel()[idx]],
                               "phi_norm2": float(np.linalg.norm(x)),
                               "threads": oracle.get_threads()}
        print("tol %g: %d iterations, %.0f s" % (tol, it, time.time() - t), flush=True)
    it12 = out["tol_1e-12"]["iters"]
    _, _, _, hist = g.pcg(b, 0.0, maxit=it12 + EXTRA, history=True)
    out["relres_history"] = {"threads": MAIN_THREADS, "values": [float(v) for v in hist]}
    for tol in TOLS:
        assert first_crossing(hist, tol) == out["tol_%g" % tol]["iters"]
    spread = {}
    for nth in OTHER_THREADS:
        oracle.set_threads(nth)
        _, _, _, h = g.pcg(b, 0.0, maxit=it12 + EXTRA, history=True)
        n = min(len(h), len(hist))
        dev = np.abs(h[:n] - hist[:n]) / hist[:n]
        spread[str(oracle.get_threads())] = {
            "stop_1e-10": first_crossing(h, 1e-10), "stop_1e-12": first_crossing(h, 1e-12),
            "max_rel_history_diff": float(dev.max())}
        print("threads %d:" % nth, spread[str(oracle.get_threads())], flush=True)
    out["other_thread_counts"] = spread
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_151x301x601.json")
    res = make()
    with open(path, "w") as f:
        json.dump(res, f, indent=0)
    print("wrote", path)
