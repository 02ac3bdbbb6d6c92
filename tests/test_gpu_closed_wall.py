"""GPU parity of the closed-wall outer boundary (Sec. 2.1: Br = 0 at R_1)
through the C ABI against the oracle: the singular system with zero-net-flux
Br and the zero-mean gauge, in every arithmetic, the field, the residual
entry points and the batched path."""
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


GRIDS = [((40, 40, 80), 1.0, "ylm"), ((13, 21, 37), 1.05, "bip"), ((17, 35, 129), 1.02, "bip")]


def make_br(kind, nt, np_):
    if kind == "ylm":
        return syn.ylm_br(nt, np_, 3, 2)[0]
    # bipoles plus a monopole, which the closed wall must remove
    return syn.bipole_br(nt, np_, seed=1709, n_bipoles=30) + 0.3


@pytest.mark.parametrize("prec", ["fp64", "df", "mixed"])
@pytest.mark.parametrize("shape,ratio,kind", GRIDS)
def test_closed_wall_solve_parity(p3, oracle_mod, prec, shape, ratio, kind):
    nr, nt, np_ = shape
    br = make_br(kind, nt, np_)
    g = oracle_mod.Grid(*shape, ratio=ratio, outer="closed")
    ref, it_ref, st = g.solve(br, 1e-12)
    assert st == oracle_mod.OK
    plan = p3.Plan(*shape, ratio=ratio, precision=prec, outer="closed")
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    rc, it = plan.solve(dev(br), 1e-12, phi)
    x = host(phi)
    assert abs(x.sum()) <= 1e-12 * np.abs(x).sum()  # the zero-mean gauge
    b = g.rhs(br)
    true_rel = np.linalg.norm(b - g.apply(x)) / np.linalg.norm(b)
    if prec == "mixed":
        assert true_rel <= 1.001e-12 and rel(x, ref) <= 1e-8, (true_rel, rel(x, ref))
    else:
        assert abs(it - it_ref) <= 1, (it, it_ref)
        assert rel(x, ref) <= 1e-9, rel(x, ref)
        assert true_rel <= 1e-12 + (2e-12 if prec == "fp64" else 2e-11)
    assert abs(plan.stats()["relres_fp64"] - true_rel) <= 0.02 * max(true_rel, 1e-13)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_closed_wall_gpu_closed_form_second_order(p3, prec):
    """The GPU solution itself converges to the analytic closed-wall shell
    potential of Br = Y_3^2 (dPhi/dr = 0 at 2.5) at second order."""
    l, m, R1 = 3, 2, 2.5
    M = np.array([[l, -(l + 1.0)], [l * R1 ** (l - 1.0), -(l + 1.0) * R1 ** (-(l + 2.0))]])
    a, b = np.linalg.solve(M, np.array([1.0, 0.0]))
    errs = []
    for n in (10, 20, 40):
        shape = (n, n, 2 * n)
        br, scale = syn.ylm_br(n, 2 * n, l, m)
        plan = p3.Plan(*shape, ratio=1.0, precision=prec, outer="closed")
        phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
        plan.solve(dev(br), 1e-12, phi)
        rc = (np.arange(n) + 0.5) * (1.5 / n) + 1.0
        tc = (np.arange(n) + 0.5) * (np.pi / n)
        pc = (np.arange(2 * n) + 0.5) * (2 * np.pi / (2 * n))
        R, T, P = np.meshgrid(rc, tc, pc, indexing="ij")
        ex = (a * R ** l + b * R ** (-(l + 1.0))) * syn.ylm_shape(l, m, T, P, scale)
        errs.append(rel(host(phi), ex - ex.mean()))
        plan.close()
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.85), (errs, orders)


def test_closed_wall_field_and_residuals(p3, oracle_mod):
    shape, ratio = (14, 23, 70), 1.04
    br = make_br("bip", shape[1], shape[2])
    g = oracle_mod.Grid(*shape, ratio=ratio, outer="closed")
    plan = p3.Plan(*shape, ratio=ratio, precision="fp64", outer="closed")
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    plan.solve(dev(br), 1e-12, phi)
    x = host(phi)
    bb = g.balanced_br(br)
    Bo = np.concatenate([a.ravel() for a in g.field(x, bb)])
    tol = 1e-12 * np.abs(Bo).max()
    for given in (None, dev(br)):  # the last solve's Br, or Br given again
        B = torch.empty(sum(plan.field_sizes()), dtype=torch.float64, device="cuda")
        plan.field(phi, given, B)
        Bg = host(B)
        np.testing.assert_allclose(Bg, Bo, rtol=0, atol=tol)
        nf = shape[1] * shape[2]
        assert np.all(Bg[shape[0] * nf: (shape[0] + 1) * nf] == 0.0)  # outer face
        np.testing.assert_allclose(Bg[:nf], bb.ravel(), rtol=0, atol=1e-14 * np.abs(bb).max())
    # both residual entry points balance Br as the solve did
    b = g.rhs(br)
    true_rel = np.linalg.norm(b - g.apply(x)) / np.linalg.norm(b)
    r1 = plan.residual(dev(br), phi)
    r2 = plan.residual_noalloc(dev(br), phi)
    for r in (r1, r2):
        assert abs(r - true_rel) <= 0.02 * max(true_rel, 1e-13), (r, true_rel)
    plan.close()


def test_closed_wall_batch_matches_solve_mixed(p3, oracle_mod):
    shape, ratio = (12, 16, 40), 1.03
    br = dev(make_br("bip", 16, 40))
    pl = p3.Plan(*shape, ratio=ratio, precision="mixed", outer="closed")
    b = p3.Batch(1 << 28, max_slots=4)
    phi_b = torch.full(shape, np.nan, dtype=torch.float64, device="cuda")
    assert b.submit(pl, br, 1e-10, phi_b, 3)
    done = []
    for _ in range(2000):
        b.step(16)
        done += b.poll()
        if done:
            break
    b.close()
    assert done and done[0][1] == 0 and done[0][4] <= 1e-10
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    rc, o, i = pl.solve_mixed(br, 1e-10, phi)
    assert (o, i) == (done[0][2], done[0][3])
    assert torch.equal(phi, phi_b)
    g = oracle_mod.Grid(*shape, ratio=ratio, outer="closed")
    rhs = g.rhs(br.cpu().numpy())
    x = host(phi)
    assert abs(x.sum()) <= 1e-12 * np.abs(x).sum()
    assert np.linalg.norm(rhs - g.apply(x)) / np.linalg.norm(rhs) <= 1.01e-10
    pl.close()
