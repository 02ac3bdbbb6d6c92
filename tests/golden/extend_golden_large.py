"""Adds oracle data to tests/golden/oracle_151x301x601.json (oracle only):

  --threads T ...   the residual history of the same PCG run under T OpenMP
                    threads (its reductions add in another order): where it
                    crosses 1e-10 and 1e-12, and its largest relative
                    difference from the stored main history
  --true-residual   for tol 1e-10 and 1e-12: the oracle's own solve (under
                    the stored main thread count, so the same iterates as the
                    stored sample, which is checked) and the true residual
                    ||b - L Phi|| / ||b|| of its result
  --precond PC ...  the solve to 1e-10 with the oracle's preconditioner PC
                    ("philine", "rline", "lines", "ilu"; PC2 with its default
                    boxes): stopping iteration, Phi on the stored sample and
                    the true residual under the main thread count, and the
                    stopping iteration under each --stop-threads count

Several processes may run at once (different thread counts); each updates
the file under a lock.  Run from the repo root, e.g.
    python tests/golden/extend_golden_large.py --threads 2 5
    python tests/golden/extend_golden_large.py --threads 3 7 --true-residual
"""
import argparse
import fcntl
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import oracle  # noqa: E402
import pot3d_synth as syn  # noqa: E402
from make_golden_large import EXTRA, RATIO, SEED, SHAPE, first_crossing  # noqa: E402

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_151x301x601.json")


def update(fn):
    with open(PATH + ".lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        with open(PATH) as f:
            gold = json.load(f)
        fn(gold)
        with open(PATH + ".tmp", "w") as f:
            json.dump(gold, f, indent=0)
        os.replace(PATH + ".tmp", PATH)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, nargs="*", default=[])
    ap.add_argument("--true-residual", action="store_true")
    ap.add_argument("--precond", nargs="*", default=[])
    ap.add_argument("--stop-threads", type=int, nargs="*", default=[])
    args = ap.parse_args()
    with open(PATH) as f:
        gold = json.load(f)
    br = syn.bipole_br(SHAPE[1], SHAPE[2], seed=SEED)
    g = oracle.Grid(*SHAPE, ratio=RATIO)
    b = g.rhs(br)
    main_h = np.array(gold["relres_history"]["values"])
    it12 = gold["tol_1e-12"]["iters"]
    for nth in args.threads:
        oracle.set_threads(nth)
        _, _, _, h = g.pcg(b, 0.0, maxit=it12 + EXTRA, history=True)
        n = min(len(h), len(main_h))
        rec = {"stop_1e-10": first_crossing(h, 1e-10), "stop_1e-12": first_crossing(h, 1e-12),
               "max_rel_history_diff": float(np.max(np.abs(h[:n] - main_h[:n]) / main_h[:n]))}
        key = str(oracle.get_threads())
        update(lambda gd: gd["other_thread_counts"].__setitem__(key, rec))
        print("threads %s:" % key, rec, flush=True)
    if args.true_residual:
        oracle.set_threads(gold["relres_history"]["threads"])
        idx = gold["sample_index"]
        for tol in (1e-10, 1e-12):
            x, it, st = g.pcg(b, tol)
            ref = gold["tol_%g" % tol]
            assert it == ref["iters"] and np.array_equal(x.ravel()[idx], np.array(ref["sample_phi"]))
            tr = float(np.linalg.norm(b - g.apply(x)) / np.linalg.norm(b))
            update(lambda gd: gd["tol_%g" % tol].__setitem__("true_relres", tr))
            print("tol %g: true residual %.3e" % (tol, tr), flush=True)
    for pc in args.precond:
        gp = oracle.Grid(*SHAPE, ratio=RATIO, precond=pc)
        main_t = gold["relres_history"]["threads"]
        oracle.set_threads(main_t)
        x, it, st = gp.pcg(b, 1e-10)
        assert st == oracle.OK
        tr = float(np.linalg.norm(b - g.apply(x)) / np.linalg.norm(b))
        rec = {"tol": 1e-10, "iters": it, "threads": main_t, "true_relres": tr,
               "sample_phi": x.ravel()[gold["sample_index"]].tolist(), "other_stops": {}}
        if pc == "ilu":
            rec["blocks"] = list(gp.blocks)
        for nth in args.stop_threads:
            oracle.set_threads(nth)
            _, it_t, _ = gp.pcg(b, 1e-10)
            rec["other_stops"][str(oracle.get_threads())] = it_t
        update(lambda gd: gd.setdefault("precond", {}).__setitem__(pc, rec))
        print("precond %s: %d iterations, true residual %.3e, other stops %s"
              % (pc, it, tr, rec["other_stops"]), flush=True)


if __name__ == "__main__":
    main()
