"""Writes tests/golden/oracle_small.json from the CPU oracle only.

Fixtures: iteration counts and solution samples of small seeded solves, used
by the tests as stored expected values (regression of the oracle itself and
iteration-count targets for the GPU parity tests).  Run from the repo root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import pot3d_synth as syn  # noqa: E402

CASES = [
    # name, (nr, nt, np), ratio, Br kind, tol
    ("ylm32_40x40x80", (40, 40, 80), 1.0, "ylm", 1e-12),
    ("bip_13x21x37_g1.05", (13, 21, 37), 1.05, "bip", 1e-12),
    ("bip_24x33x65_g1.02", (24, 33, 65), 1.02, "bip", 1e-10),
]


def make():
    oracle.set_threads(1)
    out = {}
    for name, shape, ratio, kind, tol in CASES:
        g = oracle.Grid(*shape, ratio=ratio)
        if kind == "ylm":
            br = syn.ylm_br(shape[1], shape[2], 3, 2)[0]
        else:
            br = syn.bipole_br(shape[1], shape[2], seed=1709, n_bipoles=40)
        x, it, st = g.solve(br, tol)
        idx = np.random.default_rng(0).integers(0, g.n, 16)
        out[name] = {"shape": list(shape), "ratio": ratio, "br": kind, "tol": tol, "iters": it,
                     "status": st, "sample_index": idx.tolist(),
                     "sample_phi": [float(v) for v in x.ravel()[idx]],
                     "phi_norm2": float(np.linalg.norm(x))}
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json")
    with open(path, "w") as f:
        json.dump(make(), f, indent=1)
    print("wrote", path)
