"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times.

- 151 x 301 x 601 (the benchmark workload):
  * the first 200 PCG iterates against the oracle's;
  * full solves to 1e-10 and to 1e-12 against the stored oracle solves
    (tests/golden/oracle_151x301x601.json, written by make_golden_large.py
    from the oracle alone): Phi on a stratified sample of cells (every
    boundary-folded layer: inner and source-surface layers, both pole rings,
    the phi-wrap columns), the stopping iteration, the whole residual
    history, and the true residual recomputed by the oracle's operator;
  * full FP64 solves to 1e-10 with phi lines, both line directions, PC2 and
    radial lines against the stored oracle solves with the same
    preconditioner;
- 401 x 801 x 1601 (514 M unknowns, the largest single-GPU case): the first
  200 iterates against the oracle's.

Rounding-order bars.  Two correct FP64 PCG runs that add their dot products
in different orders drift apart: the oracle itself, run with other OpenMP
thread counts (its reductions then add in other orders), gives iterates 200
that differ by up to about 3e-11 (relative L2) here, residual histories that
differ by up to the stored max_rel_history_diff, and stopping iterations that
differ by the stored spread.  Each bar below is a small multiple of the
oracle's own spread, measured (live, or stored with the golden solve), never
a fixed allowance.  Iterates after 200 steps are still in the regime where
the deviation scales with the unit roundoff, so double-float (2^-48) gets 32
times FP64's bar there; the deviation of whole histories saturates at a level
set by the problem's sensitivity, not by the unit roundoff (measured: FP64
11%, double-float 9% at 1e-12; 0.9% both at 1e-10), so both get the same
history bar.
"""
import json
import os

import numpy as np
import pytest

import pot3d_synth as syn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                    "oracle_151x301x601.json")
C2 = (151, 301, 601)
# double-float's unit roundoff (2^-48) is 32 times FP64's
ARITH_FACTOR = {"fp64": 1.0, "df": 32.0}


@pytest.fixture(scope="module")
def p3():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_01126_gb300 import pot3d

    pot3d.load(build_if_missing=True)
    return pot3d


@pytest.fixture(scope="module")
def c2(oracle_mod):
    oracle_mod.set_threads(os.cpu_count() or 1)
    br = syn.bipole_br(C2[1], C2[2], seed=1709)
    g = oracle_mod.Grid(*C2, ratio=1.02)
    return g, br, g.rhs(br)


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as f:
        return json.load(f)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def oracle_iterates(oracle_mod, g, b, k, others):
    """The oracle's k-th iterate with all host threads, and the largest
    relative distance to the same iterate under the thread counts `others`
    (reductions in other orders): the oracle's own rounding spread.  Thread
    counts whose chunkings differ strongly from n's give the spread (at
    151 x 301 x 601 on 8 threads: 8 vs 7 gives 3.3e-12, vs 5, 4, 3 give
    1.3e-11, 2.0e-11, 2.6e-11)."""
    n = os.cpu_count() or 1
    oracle_mod.set_threads(n)
    x, _, _ = g.pcg(b, 1e-300, maxit=k)
    spread = 0.0
    for t in sorted({t for t in others if 1 <= t < n}):
        oracle_mod.set_threads(t)
        y, _, _ = g.pcg(b, 1e-300, maxit=k)
        spread = max(spread, rel(y, x))
    oracle_mod.set_threads(n)
    return x, spread


@pytest.fixture(scope="module")
def c2_iterates(oracle_mod, c2):
    g, br, b = c2
    n = os.cpu_count() or 1
    return oracle_iterates(oracle_mod, g, b, 200, (n // 2 + 1, 5, 3))


@pytest.mark.parametrize("prec", ["fp64", "df"])
def test_c2_first_200_iterates(p3, oracle_mod, c2, c2_iterates, prec):
    g, br, b = c2
    x, spread = c2_iterates
    plan = p3.Plan(*C2, ratio=1.02, precision=prec, max_iters=200)
    plan.autotune(0)  # the benchmark's kernel configuration
    phi = torch.zeros(C2, dtype=torch.float64, device="cuda")
    rc, it_gpu = plan.solve(torch.from_numpy(br).cuda(), 1e-300, phi, check=False)
    assert rc == p3.POT3D_ERR_NOT_CONVERGED and it_gpu == 200
    d = rel(phi.cpu().numpy(), x)
    assert d <= 4.0 * ARITH_FACTOR[prec] * max(spread, 1e-14), (d, spread)
    plan.close()


def stop_band(gold, tol):
    """Stopping iterations of the oracle under its stored reduction orders."""
    key = "%g" % tol
    stops = [gold["tol_" + key]["iters"]]
    stops += [v["stop_" + key] for v in gold["other_thread_counts"].values()]
    return min(stops), max(stops)


@pytest.mark.parametrize("tol", [1e-10, 1e-12])
@pytest.mark.parametrize("prec", ["fp64", "df", "mixed"])
def test_c2_full_solve(p3, oracle_mod, c2, gold, prec, tol):
    g, br, b = c2
    ref = gold["tol_%g" % tol]
    idx = gold["sample_index"]
    plan = p3.Plan(*C2, ratio=1.02, precision=prec, history=1)
    plan.autotune(4 if prec == "mixed" else 0)
    phi = torch.zeros(C2, dtype=torch.float64, device="cuda")
    rc, it = plan.solve(torch.from_numpy(br).cuda(), tol, phi)
    st = plan.stats()
    x = phi.cpu().numpy()
    true_rel = np.linalg.norm(b - g.apply(x)) / np.linalg.norm(b)
    xs = x.ravel()[idx]
    rs = np.array(ref["sample_phi"])
    err = np.linalg.norm(xs - rs) / np.linalg.norm(rs)
    # the library's own FP64 residual agrees with the oracle's recomputation
    # within their rounding: each side evaluates b - A x with per-element
    # error at most gamma_16 (|b| + |A||x|) (8 terms, coefficients formed in
    # up to 8 operations).  b is nonzero on the inner layer only, so the
    # interior rows are pure cancellation and the bound is about 1e-13 here
    u = 2.0 ** -53
    ax = np.abs(x)
    abs_a_x = 2.0 * g.diag()[:, :, None] * ax - g.apply(ax)  # |A| |x|: A = D - C, C >= 0
    noise = 2.0 * 16 * u / (1 - 16 * u) * np.linalg.norm(np.abs(b) + abs_a_x) / np.linalg.norm(b)
    assert abs(st["relres_fp64"] - true_rel) <= noise, (st["relres_fp64"], true_rel, noise)
    if prec == "mixed":
        # refinement stops on the FP64 residual itself
        assert true_rel <= tol * 1.0001, true_rel
        assert err <= (1e-6 if tol >= 1e-10 else 1e-8), err
        plan.close()
        return
    # Phi on the stratified sample: within 1e-9 of the oracle's
    assert err <= 1e-9, err
    # the residual history follows the oracle's, within a small multiple of
    # the oracle's own history spread between reduction orders
    ho = np.array(gold["relres_history"]["values"])
    spread = max(v["max_rel_history_diff"] for v in gold["other_thread_counts"].values())
    band = 4.0 * spread
    h = plan.history()
    m = min(len(h), len(ho))
    dev = np.max(np.abs(h[:m] - ho[:m]) / ho[:m])
    assert dev <= band, (dev, spread)
    # the stopping iteration: +-1 of the oracle's; or inside the oracle's
    # own stops under other reduction orders, +-1; or, what the history bar
    # implies, a crossing of tol by the oracle's stored history within that
    # band (the oracle at it-1 not below tol / (1 + band), at it not above
    # tol (1 + band))
    lo, hi = stop_band(gold, tol)
    crossing = (it < len(ho) and ho[it - 1] >= tol / (1 + band) and ho[it] <= tol * (1 + band))
    assert abs(it - ref["iters"]) <= 1 or lo - 1 <= it <= hi + 1 or crossing, (
        it, ref["iters"], lo, hi, ho[it - 1:it + 1])
    # the true residual.  Near 1e-12 the recurrence residual of FP64 PCG
    # (the oracle's too) runs below the true one, which stalls at the
    # attainable accuracy; the bar is 4 x the larger of tol and the oracle's
    # own true residual at its stop (stored), 32 x more for double-float,
    # whose attainable accuracy is set by a 32 x larger unit roundoff
    floor = max(tol, ref["true_relres"])
    assert true_rel <= 4.0 * ARITH_FACTOR[prec] * floor, (true_rel, ref["true_relres"])
    plan.close()


def test_c2_df_verify_restarts_to_true_residual(p3, oracle_mod, c2, gold):
    """Double-float PCG stopped by its recurrence residual at 1e-10 leaves a
    true residual slightly above 1e-10 here; with opts.verify it restarts
    from Phi with the FP64 residual and returns a true residual within tol
    (recomputed by the oracle)."""
    g, br, b = c2
    ref = gold["tol_1e-10"]
    plan = p3.Plan(*C2, ratio=1.02, precision="df", verify=1)
    phi = torch.zeros(C2, dtype=torch.float64, device="cuda")
    rc, it = plan.solve(torch.from_numpy(br).cuda(), 1e-10, phi)
    st = plan.stats()
    x = phi.cpu().numpy()
    true_rel = np.linalg.norm(b - g.apply(x)) / np.linalg.norm(b)
    assert rc == 0 and true_rel <= 1.001e-10, (true_rel, st)
    assert abs(st["relres"] - true_rel) <= 1e-13
    assert st["outer_iters"] >= 1 and it > ref["iters"]
    xs = x.ravel()[gold["sample_index"]]
    rs = np.array(ref["sample_phi"])
    assert np.linalg.norm(xs - rs) / np.linalg.norm(rs) <= 1e-9
    plan.close()


def test_c2_mixed_inner_dots_match_fp64_accumulation(p3, oracle_mod):
    """The FP32 inner PCG forms its dot products from exact float products
    summed in compensated float pairs per thread and row, then in FP64
    across rows and blocks.  At 151 x 301 x 601, after 50 inner iterations,
    sigma = sum D^-1 p~ q and ||r||^2 as the kernels summed them agree with
    the same sums accumulated in FP64 from the FP32 vectors left in the
    workspace, to 1e-12 relative."""
    nr, nt, np_ = C2
    br = syn.bipole_br(nt, np_, seed=1709)
    # the inner solve runs 50 iterations (no refinement hand-over before)
    plan = p3.Plan(*C2, ratio=1.02, precision="mixed", torch_workspace=True, max_iters=50,
                   max_outer=1, use_graphs=-1, inner_tol=1e-20)
    phi = torch.zeros(C2, dtype=torch.float64, device="cuda")
    rc, outer, inner = plan.solve_mixed(torch.from_numpy(br).cuda(), 1e-10, phi, check=False)
    assert inner == 50
    st = plan.stats()
    pitch = plan.info()["pitch"]
    v4 = (nr * nt * pitch * 4 + 255) // 256 * 256
    ws = plan._ws[plan._ws_offset:]

    def vec(i):
        return ws[i * v4: i * v4 + nr * nt * pitch * 4].view(torch.float32).reshape(
            nr, nt, pitch)[:, :, :np_].cpu().numpy().astype(np.float64)

    r, p_k, q = vec(1), vec(2 + (50 & 1)), vec(4)
    g = oracle_mod.Grid(*C2, ratio=1.02)
    dinv = (1.0 / g.diag()).astype(np.float32).astype(np.float64)
    sigma_ref = np.sum(dinv * np.sum(p_k * q, axis=2))
    rr_ref = np.sum(r * r)
    assert abs(st["sigma"] - sigma_ref) <= 1e-12 * abs(sigma_ref), (st["sigma"], sigma_ref)
    assert abs(st["rr"] - rr_ref) <= 1e-12 * rr_ref, (st["rr"], rr_ref)
    plan.close()


def test_c3_first_200_iterates(p3, oracle_mod):
    shape = (401, 801, 1601)
    free, total = torch.cuda.mem_get_info()
    if free < 30e9:
        pytest.skip("needs about 25 GB of free device memory")
    br = syn.bipole_br(shape[1], shape[2], seed=1709)
    g = oracle_mod.Grid(*shape, ratio=1.02)
    n = os.cpu_count() or 1
    x, spread = oracle_iterates(oracle_mod, g, g.rhs(br), 200, (n // 2 + 1,))
    brd = torch.from_numpy(br).cuda()
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    for prec in ("fp64", "df"):
        plan = p3.Plan(*shape, ratio=1.02, precision=prec, max_iters=200)
        rc, it = plan.solve(brd, 1e-300, phi, check=False)
        assert rc == p3.POT3D_ERR_NOT_CONVERGED and it == 200
        d = rel(phi.cpu().numpy(), x)
        assert d <= 4.0 * ARITH_FACTOR[prec] * max(spread, 1e-14), (prec, d, spread)
        plan.close()


@pytest.mark.parametrize("pc", ["philine", "lines", "ilu", "rline"])
def test_c2_preconditioned_full_solve(p3, oracle_mod, c2, gold, pc):
    """151 x 301 x 601 to 1e-10 in FP64 with each stronger preconditioner
    (phi lines, both line directions, PC2, radial lines), in the benchmark's
    kernel configuration, against the oracle's solve with the same
    preconditioner (stored by extend_golden_large.py --precond): the stopping
    iteration within +-1 of the oracle's stops under its stored reduction
    orders, Phi on the stratified sample within 1e-9, and the true residual
    (recomputed by the oracle) within 4 x the larger of tol and the oracle's
    own true residual at its stop."""
    rec = gold.get("precond", {}).get(pc)
    if rec is None:
        pytest.skip("no stored oracle solve with %s" % pc)
    g, br, b = c2
    plan = p3.Plan(*C2, ratio=1.02, precision="fp64", precond=pc)
    plan.autotune(0)
    plan.set_opts(precond=pc)
    phi = torch.zeros(C2, dtype=torch.float64, device="cuda")
    rc, it = plan.solve(torch.from_numpy(br).cuda(), rec["tol"], phi)
    stops = [rec["iters"]] + list(rec["other_stops"].values())
    assert min(stops) - 1 <= it <= max(stops) + 1, (it, stops)
    x = phi.cpu().numpy()
    xs = x.ravel()[gold["sample_index"]]
    rs = np.array(rec["sample_phi"])
    assert np.linalg.norm(xs - rs) / np.linalg.norm(rs) <= 1e-9
    true_rel = np.linalg.norm(b - g.apply(x)) / np.linalg.norm(b)
    assert true_rel <= 4.0 * max(rec["tol"], rec["true_relres"]), (true_rel, rec["true_relres"])
    plan.close()
