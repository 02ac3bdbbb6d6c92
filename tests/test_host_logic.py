"""Host-side logic that needs no GPU: the serving trace generator and its
statistics, and bench.py's workload description and oracle-error check."""
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_requests_are_seeded_poisson_over_the_grid_mix():
    from paper_1709_01126_gb300 import serve

    a = serve.make_requests(4000, rate=2.0)
    b = serve.make_requests(4000, rate=2.0)
    assert [(r.grid, r.arrival, r.seed) for r in a] == [(r.grid, r.arrival, r.seed) for r in b]
    t = np.array([r.arrival for r in a])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    # exponential gaps of mean 1/rate: mean and coefficient of variation near 1/2 and 1
    assert abs(gaps.mean() - 0.5) < 0.05 and abs(gaps.std() / gaps.mean() - 1.0) < 0.08
    assert {r.grid for r in a} == set(serve.GRIDS)
    counts = np.array([sum(r.grid == g for r in a) for g in serve.GRIDS])
    assert counts.min() > 0.8 * len(a) / len(serve.GRIDS)
    assert [r.seed for r in a[:3]] == [serve.SEED, serve.SEED + 1, serve.SEED + 2]
    assert serve.make_requests(10, rate=2.0, seed=7)[0].seed == 7


def test_serve_summary_percentiles_and_rate():
    from paper_1709_01126_gb300 import serve

    st = serve.ServeStats("x")
    for i in range(101):
        # arrival i, latency i / 100 s
        st.outcomes.append(serve.Outcome(i, (1, 1, 1), float(i), float(i) + i / 100.0, 0,
                                         1e-11 * i, 10))
    s = st.summary()
    assert s["solves"] == 101 and s["all_ok"]
    assert s["p50_latency_s"] == pytest.approx(0.5) and s["p99_latency_s"] == pytest.approx(0.99)
    # span: first arrival (0 s) to last completion (100 + 1.00 s)
    assert s["span_s"] == pytest.approx(101.0) and s["solves_per_s"] == pytest.approx(1.0)
    assert s["max_relres"] == pytest.approx(1e-9)
    st.outcomes[3].status = -4
    assert not st.summary()["all_ok"]


def test_bench_arms_share_the_workload_config():
    import bench

    c = bench.workload_config("fp64", 1)
    assert c["grid"] == [151, 301, 601] and c["tol"] == 1e-10 and c["precision"] == "fp64"
    assert "inputs larger than L2" in c["l2"]
    assert bench.workload_config("mixed", 2)["parallelism"] == "replicas x2"


def test_bench_error_vs_oracle_samples():
    torch = pytest.importorskip("torch")
    import bench

    with open(bench.GOLDEN) as f:
        gold = json.load(f)
    idx = torch.tensor(gold["sample_index"])
    phi = torch.zeros(bench.SHAPE, dtype=torch.float64)
    flat = phi.view(-1)
    flat[idx] = torch.tensor(gold["tol_1e-10"]["sample_phi"], dtype=torch.float64)
    e = bench.sampled_error_vs_oracle(phi)
    assert e["value"] == 0.0 and e["samples"] == len(gold["sample_index"])
    flat[idx] *= 1.0 + 1e-6
    assert bench.sampled_error_vs_oracle(phi)["value"] == pytest.approx(1e-6, rel=1e-6)
