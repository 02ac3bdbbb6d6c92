"""GPU parity of the phi-line preconditioner (opts.precond =
POT3D_PC_PHI_LINE: one cyclic tridiagonal solve per (r, theta) ring, the
stronger line preconditioner of the kind Sec. 6 calls for) through the C ABI
against the oracle's phi-line PCG, which solves its rings by a different
algorithm (Sherman-Morrison around a Thomas solve; the GPU factors the ring
into two first-order recurrences)."""
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
    ((40, 40, 80), 1.0, "ylm", "source"),
    ((13, 21, 37), 1.05, "bip", "source"),
    ((9, 8, 64), 1.1, "bip", "source"),
    ((17, 35, 129), 1.02, "bip", "source"),
    ((5, 6, 3), 1.0, "bip", "source"),
    ((12, 17, 40), 1.03, "bip", "closed"),
]


def make_br(kind, nt, np_):
    if kind == "ylm":
        return syn.ylm_br(nt, np_, 3, 2)[0]
    return syn.bipole_br(nt, np_, seed=1709, n_bipoles=30)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape,ratio,kind,outer", GRIDS)
def test_phi_line_solve_parity(p3, oracle_mod, prec, shape, ratio, kind, outer):
    nr, nt, np_ = shape
    br = make_br(kind, nt, np_)
    g = oracle_mod.Grid(*shape, ratio=ratio, outer=outer, precond="philine")
    ref, it_ref, st = g.solve(br, 1e-12)
    assert st == oracle_mod.OK
    plan = p3.Plan(*shape, ratio=ratio, precision=prec, outer=outer, precond="philine")
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
        assert true_rel <= 1e-12 + 2e-12
    plan.close()


def test_phi_line_history_and_fewer_iterations(p3, oracle_mod):
    """The residual history follows the oracle's phi-line history; the
    same solution is reached in fewer iterations than with diagonal
    scaling."""
    shape, ratio = (17, 35, 129), 1.02
    br = make_br("bip", 35, 129)
    g = oracle_mod.Grid(*shape, ratio=ratio, precond="philine")
    _, it_ref, _, h_ref = g.pcg(g.rhs(br), 1e-12, history=True)
    plan = p3.Plan(*shape, ratio=ratio, precision="fp64", precond="philine", history=1)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    rc, it = plan.solve(dev(br), 1e-12, phi)
    h = plan.history()
    m = min(len(h), len(h_ref))
    assert np.max(np.abs(h[:m] - h_ref[:m]) / h_ref[:m]) <= 1e-6
    pj = p3.Plan(*shape, ratio=ratio, precision="fp64")
    phj = torch.zeros(shape, dtype=torch.float64, device="cuda")
    rc, itj = pj.solve(dev(br), 1e-12, phj)
    assert it < 0.8 * itj, (it, itj)
    assert rel(host(phi), host(phj)) <= 1e-9
    plan.close()
    pj.close()


@pytest.mark.parametrize("arith", ["fp64", "f32"])
def test_phi_line_every_decomposition(p3, oracle_mod, arith):
    """Every matvec variant and update work-item size keeps parity with the
    phi-line preconditioner (the ring solve runs inside the update kernel,
    so its work items must hold whole rings)."""
    shape, ratio = (14, 37, 150), 1.03
    br = make_br("bip", 37, 150)
    g = oracle_mod.Grid(*shape, ratio=ratio, precond="philine")
    ref, it_ref, _ = g.solve(br, 1e-12)
    b = g.rhs(br)
    prec = {"fp64": "fp64", "f32": "mixed"}[arith]
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    for v in range(len(p3.variants(arith))):
        for chunks, rows in ((1, 16), (3, 150)):
            plan = p3.Plan(*shape, ratio=ratio, precision=prec, precond="philine")
            plan.set_decomposition(arith, v, chunks, rows)
            rc, it = plan.solve(dev(br), 1e-12 if prec == "fp64" else 1e-11, phi)
            x = host(phi)
            if prec == "fp64":
                assert abs(it - it_ref) <= 1 and rel(x, ref) <= 1e-9, (v, chunks, it)
            else:
                assert np.linalg.norm(b - g.apply(x)) / np.linalg.norm(b) <= 1e-11, (v, chunks)
            plan.close()


def test_phi_line_unsupported_paths(p3):
    plan = p3.Plan(6, 7, 9, precision="df", precond="philine")
    phi = torch.zeros((6, 7, 9), dtype=torch.float64, device="cuda")
    br = torch.ones((7, 9), dtype=torch.float64, device="cuda")
    rc, _ = plan.solve(br, 1e-10, phi, check=False)
    assert rc == p3.POT3D_ERR_UNSUPPORTED
    plan.close()
