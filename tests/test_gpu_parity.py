"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs.  Bar: Phi relative L2 <= 1e-9
at relative residual 1e-12, iteration counts within +-1; the operator and
the field elementwise to FP64 rounding."""
import numpy as np
import pytest

import pot3d_synth as syn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def p3():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_01126_gb300 import pot3d

    pot3d.load(build_if_missing=True)
    return pot3d


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


GRIDS = [
    # (nr, nt, np), ratio, Br kind -- tiles: 8 theta rows x 64 phi columns, ragged tails
    ((40, 40, 80), 1.0, "ylm"),
    ((13, 21, 37), 1.05, "bip"),
    ((9, 8, 64), 1.1, "bip"),
    ((17, 35, 129), 1.02, "bip"),
    ((2, 2, 3), 1.0, "bip"),
]


def make_br(kind, nt, np_, seed=1709):
    if kind == "ylm":
        return syn.ylm_br(nt, np_, 3, 2)[0]
    return syn.bipole_br(nt, np_, seed=seed, n_bipoles=30)


@pytest.mark.parametrize("shape,ratio,kind", GRIDS)
def test_operator_matches_oracle(p3, oracle_mod, shape, ratio, kind):
    g = oracle_mod.Grid(*shape, ratio=ratio)
    plan = p3.Plan(*shape, ratio=ratio)
    x = syn.random_field(shape, seed=5)
    y = torch.empty(shape, dtype=torch.float64, device="cuda")
    plan.apply(dev(x), y)
    yo = g.apply(x)
    np.testing.assert_allclose(host(y), yo, rtol=0, atol=1e-13 * np.abs(yo).max())


def test_gpu_operator_symmetric_spd(p3):
    shape = (11, 19, 45)
    plan = p3.Plan(*shape, ratio=1.03)
    x, y = syn.random_field(shape, 1), syn.random_field(shape, 2)
    Lx = torch.empty(shape, dtype=torch.float64, device="cuda")
    Ly = torch.empty_like(Lx)
    plan.apply(dev(x), Lx)
    plan.apply(dev(y), Ly)
    Lx, Ly = host(Lx), host(Ly)
    assert abs(np.vdot(x, Ly) - np.vdot(y, Lx)) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(Ly)
    assert np.vdot(x, Lx) > 0 and np.vdot(y, Ly) > 0


@pytest.mark.parametrize("prec", ["fp64", "df"])
@pytest.mark.parametrize("shape,ratio,kind", GRIDS)
def test_solve_parity(p3, oracle_mod, prec, shape, ratio, kind):
    nr, nt, np_ = shape
    br = make_br(kind, nt, np_)
    g = oracle_mod.Grid(*shape, ratio=ratio)
    ref, it_ref, st = g.solve(br, 1e-12)
    assert st == oracle_mod.OK
    plan = p3.Plan(*shape, ratio=ratio, precision=prec)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    rc, it = plan.solve(dev(br), 1e-12, phi)
    x = host(phi)
    assert abs(it - it_ref) <= 1, (it, it_ref)
    assert rel(x, ref) <= 1e-9, rel(x, ref)
    # the GPU's convergence claim holds for the true residual, recomputed by
    # the oracle, up to the residual gap of the arithmetic (about 2^-48 per
    # operation for double-float, 2^-53 for FP64)
    r = g.rhs(br) - g.apply(x)
    gap = 2e-12 if prec == "fp64" else 2e-11
    true_rel = np.linalg.norm(r) / np.linalg.norm(g.rhs(br))
    assert true_rel <= 1e-12 + gap
    # the library's own FP64 residual of the returned Phi, and its flag
    st = plan.stats()
    assert abs(st["relres_fp64"] - true_rel) <= 0.02 * max(true_rel, 1e-13), (st, true_rel)
    assert (st["flags"] & p3.POT3D_FLAG_ABOVE_TOL) == (st["relres_fp64"] > 1e-12)


@pytest.mark.parametrize("prec", ["fp64", "df"])
def test_field_parity(p3, oracle_mod, prec):
    shape, ratio = (14, 23, 70), 1.04
    br = make_br("bip", shape[1], shape[2], seed=3)
    g = oracle_mod.Grid(*shape, ratio=ratio)
    plan = p3.Plan(*shape, ratio=ratio, precision=prec)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    plan.solve(dev(br), 1e-12, phi)
    x = host(phi)
    B = torch.empty(sum(plan.field_sizes()), dtype=torch.float64, device="cuda")
    plan.field(phi, None, B)  # Br of the last solve
    Bo = np.concatenate([a.ravel() for a in g.field(x, br)])
    Bg = host(B)
    np.testing.assert_allclose(Bg, Bo, rtol=0, atol=1e-12 * np.abs(Bo).max())
    assert np.array_equal(Bg[: shape[1] * shape[2]], br.ravel())


def test_host_pointer_path_matches_device_path(p3):
    shape = (10, 12, 33)
    br = make_br("bip", 12, 33)
    plan = p3.Plan(*shape, ratio=1.05, precision="df")
    phi_d = torch.zeros(shape, dtype=torch.float64, device="cuda")
    rc, it_d = plan.solve(dev(br), 1e-11, phi_d)
    phi_h = np.zeros(shape)
    rc, it_h = plan.solve(br, 1e-11, phi_h)
    assert it_d == it_h
    assert np.array_equal(host(phi_d), phi_h)


@pytest.mark.parametrize("prec", ["fp64", "df"])
def test_deterministic(p3, prec):
    shape = (16, 30, 100)
    br = dev(make_br("bip", 30, 100))
    plan = p3.Plan(*shape, ratio=1.02, precision=prec)
    a = torch.zeros(shape, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    plan.solve(br, 1e-10, a)
    plan.solve(br, 1e-10, b)
    assert torch.equal(a, b)


def test_graphs_timing_and_plain_launches_agree(p3):
    shape = (12, 20, 50)
    br = dev(make_br("bip", 20, 50))
    outs = []
    for opts in ({}, {"use_graphs": -1}, {"time_kernels": 1}, {"chunk": 3}):
        plan = p3.Plan(*shape, ratio=1.02, precision="fp64", **opts)
        phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
        rc, it = plan.solve(br, 1e-10, phi)
        outs.append((it, host(phi)))
        if opts.get("time_kernels"):
            st = plan.stats()
            assert st["kernel_ms"][2] == it and st["kernel_ms"][0] > 0
    for it, x in outs[1:]:
        assert it == outs[0][0] and np.array_equal(x, outs[0][1])


@pytest.mark.parametrize("prec", ["fp64", "df"])
def test_initial_guess_restart(p3, oracle_mod, prec):
    shape, ratio = (12, 16, 40), 1.05
    br = make_br("bip", 16, 40)
    g = oracle_mod.Grid(*shape, ratio=ratio)
    ref, it_ref, _ = g.solve(br, 1e-12)
    plan = p3.Plan(*shape, ratio=ratio, precision=prec, use_x0=1)
    phi = dev(ref)
    rc, it = plan.solve(dev(br), 1e-12, phi)
    assert it <= 2
    assert rel(host(phi), ref) <= 1e-10
    # restart from a partial solve gives the same answer as a cold solve
    x5, _, _ = g.pcg(g.rhs(br), 1e-300, maxit=5)
    phi = dev(x5)
    plan.solve(dev(br), 1e-12, phi)
    assert rel(host(phi), ref) <= 1e-9


def test_iteration_cap_returns_last_iterate(p3, oracle_mod):
    shape, ratio = (10, 14, 30), 1.05
    br = make_br("bip", 14, 30)
    g = oracle_mod.Grid(*shape, ratio=ratio)
    x7, _, st = g.pcg(g.rhs(br), 1e-300, maxit=7)
    for prec in ("fp64", "df"):
        plan = p3.Plan(*shape, ratio=ratio, precision=prec, max_iters=7)
        phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
        rc, it = plan.solve(dev(br), 1e-14, phi, check=False)
        assert rc == p3.POT3D_ERR_NOT_CONVERGED and it == 7
        assert rel(host(phi), x7) <= 1e-12


def test_zero_and_nan_inputs(p3):
    shape = (5, 6, 9)
    plan = p3.Plan(*shape, ratio=1.0)
    phi = torch.full(shape, 3.0, dtype=torch.float64, device="cuda")
    rc, it = plan.solve(torch.zeros((6, 9), dtype=torch.float64, device="cuda"), 1e-10, phi)
    assert rc == 0 and it == 0 and torch.count_nonzero(phi) == 0
    br = np.ones((6, 9))
    br[2, 3] = np.nan
    rc, it = plan.solve(dev(br), 1e-10, phi, check=False)
    assert rc == p3.POT3D_ERR_BREAKDOWN


def test_invalid_arguments(p3):
    with pytest.raises(p3.Pot3dError):
        p3.Plan(4, 4, 2)
    with pytest.raises(p3.Pot3dError):
        p3.Plan(4, 1, 8)
    plan = p3.Plan(4, 4, 8)
    phi = torch.zeros((4, 4, 8), dtype=torch.float64, device="cuda")
    br = torch.zeros((4, 8), dtype=torch.float64, device="cuda")
    rc, _ = plan.solve(br, -1.0, phi, check=False)
    assert rc == p3.POT3D_ERR_INVALID_ARG
    rc, _ = plan.solve(br, float("nan"), phi, check=False)
    assert rc == p3.POT3D_ERR_INVALID_ARG


def test_torch_workspace(p3, oracle_mod):
    shape = (9, 11, 31)
    br = make_br("bip", 11, 31)
    g = oracle_mod.Grid(*shape, ratio=1.05)
    ref, it_ref, _ = g.solve(br, 1e-12)
    plan = p3.Plan(*shape, ratio=1.05, precision="df", torch_workspace=True)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    rc, it = plan.solve(dev(br), 1e-12, phi)
    assert abs(it - it_ref) <= 1 and rel(host(phi), ref) <= 1e-9


@pytest.mark.parametrize("prec,flags", [("fp64", 1), ("df", 2), ("mixed", 4)])
def test_autotune_keeps_parity(p3, oracle_mod, prec, flags):
    shape, ratio = (14, 37, 150), 1.03
    br = make_br("bip", 37, 150)
    g = oracle_mod.Grid(*shape, ratio=ratio)
    ref, it_ref, _ = g.solve(br, 1e-12)
    plan = p3.Plan(*shape, ratio=ratio, precision=prec)
    var, chunks, ms = plan.autotune(flags)
    assert var >= 0 and chunks >= 1 and ms > 0
    # a second plan of the same dimensions takes the cached choice
    plan2 = p3.Plan(*shape, ratio=ratio, precision=prec)
    assert plan2.autotune(flags)[:2] == (var, chunks)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    if prec == "mixed":
        plan.solve_mixed(dev(br), 1e-11, phi)
        b = g.rhs(br)
        assert np.linalg.norm(b - g.apply(host(phi))) / np.linalg.norm(b) <= 1e-11
    else:
        rc, it = plan.solve(dev(br), 1e-12, phi)
        assert abs(it - it_ref) <= 1 and rel(host(phi), ref) <= 1e-9


@pytest.mark.parametrize("prec", ["fp64", "df", "mixed"])
def test_gpu_closed_form_second_order(p3, prec):
    """The GPU solution itself converges to the analytic shell potential of
    Br = Y_3^2 at second order (Sec. 2.2), independently of the oracle."""
    l, m, R1 = 3, 2, 2.5
    M = np.array([[l, -(l + 1.0)], [R1 ** l, R1 ** (-(l + 1.0))]])
    a, b = np.linalg.solve(M, np.array([1.0, 0.0]))
    errs = []
    for n in (10, 20, 40):
        shape = (n, n, 2 * n)
        br, scale = syn.ylm_br(n, 2 * n, l, m)
        plan = p3.Plan(*shape, ratio=1.0, precision=prec)
        phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
        plan.solve(dev(br), 1e-12, phi)
        rc = (np.arange(n) + 0.5) * (1.5 / n) + 1.0
        tc = (np.arange(n) + 0.5) * (np.pi / n)
        pc = (np.arange(2 * n) + 0.5) * (2 * np.pi / (2 * n))
        R, T, P = np.meshgrid(rc, tc, pc, indexing="ij")
        ex = (a * R ** l + b * R ** (-(l + 1.0))) * syn.ylm_shape(l, m, T, P, scale)
        errs.append(rel(host(phi), ex))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.9), (errs, orders)


def test_explicit_faces_match_oracle(p3, oracle_mod):
    """Explicit nonuniform r and theta faces (Sec. 2.2: nonuniform in r and
    theta) give the oracle's solution."""
    nr, nt, np_ = 11, 17, 40
    rf = 1.0 + 1.5 * (np.linspace(0, 1, nr + 1) ** 1.3)
    u = np.linspace(0, 1, nt + 1)
    tf = np.pi * (u + 0.12 * np.sin(2 * np.pi * u) / (2 * np.pi))
    tf[0], tf[-1] = 0.0, np.pi
    br = make_br("bip", nt, np_)
    g = oracle_mod.Grid(nr, nt, np_, r_faces=rf, t_faces=tf)
    ref, it_ref, _ = g.solve(br, 1e-12)
    for prec in ("fp64", "df"):
        plan = p3.Plan(nr, nt, np_, r_faces=rf, t_faces=tf, precision=prec)
        phi = torch.zeros((nr, nt, np_), dtype=torch.float64, device="cuda")
        rc, it = plan.solve(dev(br), 1e-12, phi)
        assert abs(it - it_ref) <= 1 and rel(host(phi), ref) <= 1e-9


@pytest.mark.parametrize("arith", ["fp64", "df", "f32"])
def test_every_variant_keeps_parity(p3, oracle_mod, arith):
    """Every matvec variant, with one and three r-chunks and with 16 and 150
    update rows per item, on a grid with ragged tails in every dimension
    for every tile shape (37 theta rows, 150 phi columns), against the
    oracle's solve."""
    shape, ratio = (14, 37, 150), 1.03
    br = make_br("bip", 37, 150)
    g = oracle_mod.Grid(*shape, ratio=ratio)
    ref, it_ref, _ = g.solve(br, 1e-12)
    b = g.rhs(br)
    prec = {"fp64": "fp64", "df": "df", "f32": "mixed"}[arith]
    vs = p3.variants(arith)
    assert len(vs) >= 2
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    for v in range(len(vs)):
        for chunks, rows in ((1, 16), (3, 150)):
            plan = p3.Plan(*shape, ratio=ratio, precision=prec)
            plan.set_decomposition(arith, v, chunks, rows)
            info = plan.info()
            if arith != "f32":
                assert info["tiles_update"] == -(-14 * 37 // rows)
            if prec == "mixed":
                plan.solve_mixed(dev(br), 1e-11, phi)
                x = host(phi)
                assert np.linalg.norm(b - g.apply(x)) / np.linalg.norm(b) <= 1e-11, (v, chunks)
                assert rel(x, ref) <= 1e-8, (v, chunks)
            else:
                rc, it = plan.solve(dev(br), 1e-12, phi)
                assert abs(it - it_ref) <= 1 and rel(host(phi), ref) <= 1e-9, (v, chunks, it)
            plan.close()


def test_set_decomposition_rejects_bad_arguments(p3):
    plan = p3.Plan(9, 8, 64)
    n = len(p3.variants("fp64"))
    for args in (("fp64", n, 0, 0), ("fp64", -1, 0, 0), (3, 0, 0, 0), ("df", 0, -1, 0),
                 ("df", 0, 0, -1)):
        with pytest.raises(p3.Pot3dError):
            plan.set_decomposition(*args)
    plan.set_decomposition("df", 0, 100, 1000)  # counts are clamped, not rejected
    plan.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("df", 1e-13)])
def test_verify_stops_on_true_residual(p3, oracle_mod, prec, tol):
    """opts.verify: the returned Phi's FP64 residual, recomputed by the
    oracle's own operator, is within tol.  Without verify the solve stops on
    the recurrence residual; with it the solve restarts from Phi exactly
    when that left the true residual above tol."""
    shape, ratio = (17, 35, 129), 1.05
    br = make_br("bip", 35, 129)
    g = oracle_mod.Grid(*shape, ratio=ratio)
    b = g.rhs(br)
    true_rel = lambda x: np.linalg.norm(b - g.apply(x)) / np.linalg.norm(b)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    plain = p3.Plan(*shape, ratio=ratio, precision=prec)
    rc0, it0 = plain.solve(dev(br), tol, phi)
    t0 = true_rel(host(phi))
    plan = p3.Plan(*shape, ratio=ratio, precision=prec, verify=1)
    rc, it = plan.solve(dev(br), tol, phi)
    st = plan.stats()
    t1 = true_rel(host(phi))
    assert rc == 0 and t1 <= tol * 1.001, (t0, t1)
    # both residuals carry FP64 rounding of b - L Phi, about 1e-16 here
    assert abs(st["relres"] - t1) <= 0.02 * tol
    if t0 <= tol * 0.999:
        assert st["outer_iters"] == 0 and it == it0
    elif t0 > tol * 1.001:
        assert st["outer_iters"] >= 1 and it > it0


@pytest.mark.parametrize("prec,factor", [("fp64", 4.0), ("df", 4.0 * 32)])
def test_residual_history_matches_oracle(p3, oracle_mod, prec, factor):
    """opts.history: the recurrence residual ||r_k|| / ||b|| of every
    iteration, against the oracle's own history of the same solve.  The bar
    is the oracle's own spread: the largest relative difference between its
    histories under other thread counts (reductions added in other orders,
    all valid roundings of the same method), times 4 for FP64 and times a
    further 32 for double-float, whose unit roundoff (2^-48) is 32 times
    FP64's."""
    import os

    shape, ratio = (17, 35, 129), 1.02
    br = make_br("bip", 35, 129)
    g = oracle_mod.Grid(*shape, ratio=ratio)
    hs = []
    for t in (1, 2, 3, 5):
        oracle_mod.set_threads(t)
        hs.append(g.pcg(g.rhs(br), 1e-12, history=True)[3])
    oracle_mod.set_threads(os.cpu_count() or 1)
    h_ref = hs[0]
    it_ref = len(h_ref) - 1
    spread = max(np.max(np.abs(h[:min(len(h), len(h_ref))] - h_ref[:min(len(h), len(h_ref))])
                        / h_ref[:min(len(h), len(h_ref))]) for h in hs[1:])
    bound = factor * max(spread, 1e-14)
    plan = p3.Plan(*shape, ratio=ratio, precision=prec, history=1)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    rc, it = plan.solve(dev(br), 1e-12, phi)
    h = plan.history()
    assert len(h) == it + 1 and h[0] == 1.0 and h[-1] <= 1e-12 < h[-2]
    m = min(len(h), len(h_ref))
    dev_rel = np.abs(h[:m] - h_ref[:m]) / h_ref[:m]
    assert dev_rel.max() <= bound, (dev_rel.max(), spread)
    assert abs(it - it_ref) <= 1
    plan.set_opts()  # history off: nothing recorded
    plan.solve(dev(br), 1e-12, phi)
    with pytest.raises(p3.Pot3dError):
        plan.history()
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "df", "mixed"])
@pytest.mark.parametrize("shape", [(5, 7, 700), (4, 5, 1601), (6, 9, 321)])
def test_long_rows_keep_parity(p3, oracle_mod, prec, shape):
    """Rows longer than one update unit (the register-staged update takes
    640 FP32 or 320 double-float elements per unit, the bulk-copy update
    2560 bytes per segment): several units per row, a ragged last one."""
    nr, nt, np_ = shape
    br = make_br("bip", nt, np_)
    g = oracle_mod.Grid(*shape, ratio=1.04)
    ref, it_ref, st = g.solve(br, 1e-12)
    assert st == oracle_mod.OK
    plan = p3.Plan(*shape, ratio=1.04, precision=prec)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    rc, it = plan.solve(dev(br), 1e-12, phi)
    x = host(phi)
    b = g.rhs(br)
    true_rel = np.linalg.norm(b - g.apply(x)) / np.linalg.norm(b)
    if prec == "mixed":
        assert true_rel <= 1.001e-12 and rel(x, ref) <= 1e-8, (true_rel, rel(x, ref))
    else:
        assert abs(it - it_ref) <= 1, (it, it_ref)
        assert rel(x, ref) <= 1e-9, rel(x, ref)
    plan.close()


@pytest.mark.parametrize("pc", ["philine", "rline", "lines", "ilu"])
@pytest.mark.parametrize("outer", ["source", "closed"])
def test_explicit_faces_every_preconditioner(p3, oracle_mod, pc, outer):
    """Explicit nonuniform r and theta faces with each stronger
    preconditioner and both outer boundaries: every preconditioner builds
    its tables (ring factors, column factors, PC2 pivots) from the plan's
    own coefficients, which here come from the given faces."""
    nr, nt, np_ = 11, 17, 40
    rf = 1.0 + 1.5 * (np.linspace(0, 1, nr + 1) ** 1.3)
    u = np.linspace(0, 1, nt + 1)
    tf = np.pi * (u + 0.12 * np.sin(2 * np.pi * u) / (2 * np.pi))
    tf[0], tf[-1] = 0.0, np.pi
    br = make_br("bip", nt, np_)
    g = oracle_mod.Grid(nr, nt, np_, r_faces=rf, t_faces=tf, outer=outer, precond=pc)
    ref, it_ref, st = g.solve(br, 1e-12)
    assert st == oracle_mod.OK
    for prec in ("fp64", "mixed"):
        plan = p3.Plan(nr, nt, np_, r_faces=rf, t_faces=tf, precision=prec, outer=outer,
                       precond=pc)
        phi = torch.zeros((nr, nt, np_), dtype=torch.float64, device="cuda")
        rc, it = plan.solve(dev(br), 1e-12, phi)
        x = host(phi)
        if prec == "fp64":
            assert abs(it - it_ref) <= 1 and rel(x, ref) <= 1e-9, (prec, it, it_ref, rel(x, ref))
        else:
            b = g.rhs(br)
            true_rel = np.linalg.norm(b - g.apply(x)) / np.linalg.norm(b)
            assert true_rel <= 1.001e-12 and rel(x, ref) <= 1e-8, (true_rel, rel(x, ref))
        plan.close()


@pytest.mark.parametrize("pc", ["philine", "rline", "lines", "ilu"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_initial_guess_every_preconditioner(p3, oracle_mod, pc, prec):
    """A solve started from a given Phi (opts.use_x0, also what verify's
    restarts use) with each stronger preconditioner: from the oracle's
    solution it stops at once (FP64) or keeps it (mixed), from the oracle's
    5th PCG iterate (with the same preconditioner) it reaches the oracle's
    solution (the preconditioners' setup launches run on the residual of the
    given Phi)."""
    shape, ratio = (12, 16, 40), 1.05
    br = make_br("bip", 16, 40)
    g = oracle_mod.Grid(*shape, ratio=ratio, precond=pc)
    ref, it_ref, _ = g.solve(br, 1e-12)
    plan = p3.Plan(*shape, ratio=ratio, precision=prec, use_x0=1, precond=pc)
    phi = dev(ref)
    if prec == "mixed":
        rc, outer, it = plan.solve_mixed(dev(br), 1e-12, phi)
    else:
        rc, it = plan.solve(dev(br), 1e-12, phi)
    if prec == "fp64":
        assert it <= 2, it
        assert rel(host(phi), ref) <= 1e-10
    else:
        # refinement stops on the FP64 residual of the given Phi, which may
        # sit just above tol: at most one short refinement step
        assert rel(host(phi), ref) <= 1e-8
    x5, _, _ = g.pcg(g.rhs(br), 1e-300, maxit=5)
    phi = dev(x5)
    if prec == "mixed":
        plan.solve_mixed(dev(br), 1e-12, phi)
    else:
        plan.solve(dev(br), 1e-12, phi)
    assert rel(host(phi), ref) <= (1e-9 if prec == "fp64" else 1e-8)
    plan.close()
