"""Batched solves (continuous batching): a solve gives the same bits alone,
in a mix, and through pot3d_solve_mixed; admission is bounded by the
arena's memory; the serving loop completes a small stream."""
import numpy as np
import pytest

import pot3d_synth as syn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GRIDS = [(12, 16, 40), (9, 21, 37), (14, 11, 70), (7, 9, 130)]


@pytest.fixture(scope="module")
def p3():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_01126_gb300 import pot3d

    pot3d.load(build_if_missing=True)
    return pot3d


def run_batch(p3, plans, brs, tol=1e-10, k=8, nbytes=1 << 30, precond="jacobi"):
    b = p3.Batch(nbytes, max_slots=16, precond=precond)
    phis = []
    for t, (pl, br) in enumerate(zip(plans, brs)):
        phi = torch.full(pl.shape, np.nan, dtype=torch.float64, device="cuda")
        assert b.submit(pl, br, tol, phi, t)
        phis.append(phi)
    done = {}
    for _ in range(10000):
        b.step(k)
        for tag, st, outer, inner, rr in b.poll():
            done[tag] = (st, outer, inner, rr)
        if len(done) == len(plans):
            break
    b.close()
    torch.cuda.synchronize()
    return [p.cpu().numpy() for p in phis], done


def test_batch_matches_solve_mixed_and_is_mix_independent(p3, oracle_mod):
    plans = [p3.Plan(*g, ratio=1.03, precision="mixed") for g in GRIDS]
    brs = [torch.from_numpy(syn.bipole_br(g[1], g[2], seed=50 + u, n_bipoles=15)).cuda()
           for u, g in enumerate(GRIDS)]
    mixed, info = run_batch(p3, plans, brs)
    for u, (pl, br) in enumerate(zip(plans, brs)):
        st, outer, inner, rr = info[u]
        assert st == 0 and rr <= 1e-10
        # alone in its own batch: the same bits
        alone, _ = run_batch(p3, [pl], [br])
        assert np.array_equal(alone[0], mixed[u])
        # the single-solve entry point: the same bits
        phi = torch.zeros(pl.shape, dtype=torch.float64, device="cuda")
        rc, o2, i2 = pl.solve_mixed(br, 1e-10, phi)
        assert (o2, i2) == (outer, inner)
        assert np.array_equal(phi.cpu().numpy(), mixed[u])
        # and the FP64 residual, recomputed by the oracle, meets the tolerance
        g = oracle_mod.Grid(*pl.shape, ratio=1.03)
        b = g.rhs(br.cpu().numpy())
        assert np.linalg.norm(b - g.apply(mixed[u])) / np.linalg.norm(b) <= 1.01e-10


def test_admission_is_bounded_by_memory(p3):
    pl = p3.Plan(10, 12, 33, ratio=1.02, precision="mixed")
    probe = p3.Batch(1 << 20, max_slots=4)
    need = probe.bytes_needed(pl)
    probe.close()
    b = p3.Batch(need + need // 2, max_slots=4)  # room for one solve only
    br = torch.from_numpy(syn.bipole_br(12, 33, seed=3, n_bipoles=5)).cuda()
    phis = [torch.zeros(pl.shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    assert b.submit(pl, br, 1e-10, phis[0], 0)
    assert not b.submit(pl, br, 1e-10, phis[1], 1)  # busy: no memory
    done = []
    while not done:
        b.step(16)
        done += b.poll()
    assert b.info()["bytes_used"] == 0
    assert b.submit(pl, br, 1e-10, phis[1], 1)  # memory came back
    while len(done) < 2:
        b.step(16)
        done += b.poll()
    torch.cuda.synchronize()
    assert torch.equal(phis[0], phis[1])
    b.close()


def test_serving_loop_small_stream(p3, oracle_mod):
    """Both servers complete a small stream; every served Phi's FP64
    residual, recomputed by the library, meets the tolerance; and one served
    Phi of each server is checked with the oracle's own operator."""
    from paper_1709_01126_gb300 import serve

    grids = [(9, 13, 27), (12, 17, 35)]
    reqs = serve.make_requests(8, rate=200.0, grids=grids)
    inputs = serve.prepare_inputs(reqs)
    for run in (serve.run_batched, serve.run_fp64_serial):
        if run is serve.run_batched:
            st = run(reqs, inputs, batch_bytes=1 << 28, k=8, keep=True)
        else:
            st = run(reqs, inputs, keep=True)
        s = st.summary()
        assert s["solves"] == 8 and s["all_ok"], s
        assert s["max_relres_fp64"] <= 1e-10, s
        assert s["p99_latency_s"] >= s["p50_latency_s"] > 0
        o = max(st.outcomes, key=lambda q: q.grid)
        br, phi = st.results[o.rid]
        g = oracle_mod.Grid(*o.grid, ratio=serve.RATIO)
        b = g.rhs(br.cpu().numpy())
        true_rel = np.linalg.norm(b - g.apply(phi.cpu().numpy())) / np.linalg.norm(b)
        assert true_rel <= 1.001e-10, (run.__name__, true_rel)
        assert abs(true_rel - o.relres_fp64) <= 1e-3 * true_rel + 1e-15


def test_batch_phi_line_matches_solve_mixed(p3, oracle_mod):
    """With the phi-line preconditioner a batched solve gives the same bits
    alone, in a mix and through pot3d_solve_mixed, meets the tolerance in
    the oracle's FP64 residual, and needs fewer inner iterations than with
    diagonal scaling."""
    plans = [p3.Plan(*g, ratio=1.03, precision="mixed", precond="philine") for g in GRIDS]
    brs = [torch.from_numpy(syn.bipole_br(g[1], g[2], seed=50 + u, n_bipoles=15)).cuda()
           for u, g in enumerate(GRIDS)]
    mixed, info = run_batch(p3, plans, brs, precond="philine")
    _, info_j = run_batch(p3, plans, brs)
    for u, (pl, br) in enumerate(zip(plans, brs)):
        st, outer, inner, rr = info[u]
        assert st == 0 and rr <= 1e-10
        assert inner < info_j[u][2], (inner, info_j[u][2])
        alone, _ = run_batch(p3, [pl], [br], precond="philine")
        assert np.array_equal(alone[0], mixed[u])
        phi = torch.zeros(pl.shape, dtype=torch.float64, device="cuda")
        rc, o2, i2 = pl.solve_mixed(br, 1e-10, phi)
        assert (o2, i2) == (outer, inner)
        assert np.array_equal(phi.cpu().numpy(), mixed[u])
        g = oracle_mod.Grid(*pl.shape, ratio=1.03)
        b = g.rhs(br.cpu().numpy())
        assert np.linalg.norm(b - g.apply(mixed[u])) / np.linalg.norm(b) <= 1.01e-10


@pytest.mark.parametrize("precond", ["jacobi", "philine"])
def test_batch_closed_wall_in_a_mix(p3, oracle_mod, precond):
    """Closed-wall plans (Br = 0 at r1: balanced Br, zero-mean gauge) batched
    together with source-surface plans: each gives the bits of
    pot3d_solve_mixed, its mean is zero, and the oracle's FP64 residual of
    the balanced system meets the tolerance."""
    outers = ["closed", "source", "closed", "source"]
    plans = [p3.Plan(*g, ratio=1.03, precision="mixed", outer=o, precond=precond)
             for g, o in zip(GRIDS, outers)]
    brs = [torch.from_numpy(syn.bipole_br(g[1], g[2], seed=70 + u, n_bipoles=15) + 0.3).cuda()
           for u, g in enumerate(GRIDS)]
    mixed, info = run_batch(p3, plans, brs, precond=precond)
    for u, (pl, br, o) in enumerate(zip(plans, brs, outers)):
        st, outer, inner, rr = info[u]
        assert st == 0 and rr <= 1e-10
        phi = torch.zeros(pl.shape, dtype=torch.float64, device="cuda")
        rc, o2, i2 = pl.solve_mixed(br, 1e-10, phi)
        assert (o2, i2) == (outer, inner)
        assert np.array_equal(phi.cpu().numpy(), mixed[u])
        g = oracle_mod.Grid(*pl.shape, ratio=1.03, outer=o)
        b = g.rhs(br.cpu().numpy())
        assert np.linalg.norm(b - g.apply(mixed[u])) / np.linalg.norm(b) <= 1.01e-10
        if o == "closed":
            assert abs(mixed[u].mean()) <= 1e-12 * np.abs(mixed[u]).max()
