"""Writes tests/golden/oracle_151x301x601.json from the CPU oracle only.

The full 151 x 301 x 601 oracle solve (geometric r, ratio 1.02; dipole + 200
bipoles, seed 1709; the benchmark's workload) takes minutes on a CPU, so its
iteration counts and a sample of its solution are stored for the GPU tests.
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


def make():
    oracle.set_threads(os.cpu_count() or 1)
    shape, ratio = (151, 301, 601), 1.02
    br = syn.bipole_br(shape[1], shape[2], seed=1709)
    g = oracle.Grid(*shape, ratio=ratio)
    b = g.rhs(br)
    out = {"shape": list(shape), "ratio": ratio, "br": "bipole_br(seed=1709, 200 bipoles)"}
    for tol in (1e-10,):
        t = time.time()
        x, it, st, hist = g.pcg(b, tol, history=True)
        idx = np.random.default_rng(1).integers(0, g.n, 64)
        tail0 = max(0, it - 40)
        out["tol_%g" % tol] = {"iters": it, "status": st, "seconds": time.time() - t,
                               "sample_index": idx.tolist(),
                               "sample_phi": [float(v) for v in x.ravel()[idx]],
                               "phi_norm2": float(np.linalg.norm(x)),
                               "relres_tail_start": tail0,
                               "relres_tail": [float(v) for v in hist[tail0:]],
                               "threads": oracle.get_threads()}
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_151x301x601.json")
    res = make()
    with open(path, "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", path, {k: v["iters"] for k, v in res.items() if isinstance(v, dict)})
