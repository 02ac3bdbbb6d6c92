"""Pins of the oracle's line preconditioners (stronger than diagonal
scaling yet line-parallel, of the kind Sec. 6 asks for), on the CPU.

Radial lines: M is the part of L that couples cells of one (theta, phi)
column (the full diagonal and the two radial neighbours).  Phi lines: M is
the part of L that couples cells of one (r, theta) ring (the full diagonal
and the two periodic phi neighbours).  z = M^-1 r is checked against a dense
solve with M cut out of the assembled L, and PCG with it against the dense
direct solve of L Phi = b.
"""
import numpy as np
import pytest

import pot3d_synth as syn


def line_part(A, shape, kind="rline"):
    """The entries of A that couple cells of the same (theta, phi) column
    (rline) or of the same (r, theta) ring (philine)."""
    nr, nt, np_ = shape
    idx = np.arange(A.shape[0])
    key = idx % (nt * np_) if kind == "rline" else idx // np_
    return np.where(key[:, None] == key[None, :], A, 0.0)


@pytest.mark.parametrize("outer", ["source", "closed"])
@pytest.mark.parametrize("shape,ratio", [((4, 5, 7), 1.1), ((6, 4, 8), 1.0), ((2, 3, 4), 1.3)])
def test_precond_is_the_radial_line_solve(oracle_mod, shape, ratio, outer):
    g = oracle_mod.Grid(*shape, ratio=ratio, outer=outer, precond="rline")
    A = g.dense()
    M = line_part(A, shape)
    # tridiagonal in i within a column, the diagonal of L on its diagonal
    assert np.array_equal(np.diag(M), np.diag(A))
    assert np.count_nonzero(M) == g.n + 2 * (shape[0] - 1) * shape[1] * shape[2]
    r = syn.random_field(shape, seed=4)
    z = g.apply_precond(r)
    zd = np.linalg.solve(M, r.ravel())
    np.testing.assert_allclose(z.ravel(), zd, rtol=1e-13, atol=1e-13 * np.abs(zd).max())
    # the default preconditioner is the diagonal
    gj = oracle_mod.Grid(*shape, ratio=ratio, outer=outer)
    np.testing.assert_allclose(gj.apply_precond(r).ravel(), r.ravel() / np.diag(A), rtol=1e-15)


@pytest.mark.parametrize("outer", ["source", "closed"])
@pytest.mark.parametrize("shape,ratio", [((4, 5, 7), 1.1), ((3, 6, 3), 1.0), ((2, 3, 2), 1.3),
                                         ((3, 4, 16), 1.05)])
def test_precond_is_the_phi_line_solve(oracle_mod, shape, ratio, outer):
    g = oracle_mod.Grid(*shape, ratio=ratio, outer=outer, precond="philine")
    A = g.dense()
    M = line_part(A, shape, "philine")
    assert np.array_equal(np.diag(M), np.diag(A))
    # cyclic tridiagonal in k within a ring (np = 2: one merged neighbour)
    nnz_ring = 3 * shape[2] if shape[2] > 2 else 4
    assert np.count_nonzero(M) == shape[0] * shape[1] * nnz_ring
    r = syn.random_field(shape, seed=6)
    z = g.apply_precond(r)
    zd = np.linalg.solve(M, r.ravel())
    np.testing.assert_allclose(z.ravel(), zd, rtol=1e-12, atol=1e-13 * np.abs(zd).max())


@pytest.mark.parametrize("kind", ["rline", "philine"])
@pytest.mark.parametrize("shape,ratio", [((4, 4, 8), 1.0), ((3, 5, 6), 1.2), ((6, 6, 12), 1.05)])
def test_pcg_line_matches_dense_direct_solve(oracle_mod, shape, ratio, kind):
    g = oracle_mod.Grid(*shape, ratio=ratio, precond=kind)
    br = syn.random_field(shape[1:], seed=11)
    b = g.rhs(br)
    x, it, st = g.pcg(b, 1e-13)
    assert st == oracle_mod.OK
    xd = np.linalg.solve(g.dense(), b.ravel())
    assert np.linalg.norm(x.ravel() - xd) / np.linalg.norm(xd) < 1e-11


@pytest.mark.parametrize("kind", ["rline", "philine"])
def test_pcg_line_first_step_closed_form(oracle_mod, kind):
    """One step from x0 = 0 is alpha_1 M^-1 b with alpha_1 = (b.z)/(z.Lz),
    z = M^-1 b (M cut out of the dense L)."""
    shape = (4, 5, 6)
    g = oracle_mod.Grid(*shape, ratio=1.1, precond=kind)
    A = g.dense()
    b = g.rhs(syn.random_field((5, 6), seed=8)).ravel()
    z = np.linalg.solve(line_part(A, shape, kind), b)
    alpha = (b @ z) / (z @ A @ z)
    x1, it, st = g.pcg(b, 1e-300, maxit=1)
    assert it == 1 and st == oracle_mod.NOT_CONVERGED
    np.testing.assert_allclose(x1.ravel(), alpha * z, rtol=1e-12, atol=1e-14 * np.abs(z).max())


def test_line_preconditioners_same_solution_fewer_iterations(oracle_mod):
    """Both line preconditioners reach the same discrete solution as
    diagonal scaling.  Phi lines cut the iteration count by far the most:
    near the poles the phi couplings dr dth / (sin th dphi) dwarf the others
    (by about 860 times at r = 1 on the 151 x 301 x 601 mesh), and a
    phi-line solve removes exactly that anisotropy; radial lines help little
    (measured with this oracle at 24 x 33 x 65, ratio 1.05: 383, 323 and 197
    iterations to 1e-10 for diagonal, radial-line and phi-line)."""
    shape, ratio = (24, 33, 65), 1.05
    br = syn.bipole_br(33, 65, seed=1709, n_bipoles=40)
    xj, itj, _ = oracle_mod.Grid(*shape, ratio=ratio).solve(br, 1e-12)
    xr, itr, _ = oracle_mod.Grid(*shape, ratio=ratio, precond="rline").solve(br, 1e-12)
    xp, itp, _ = oracle_mod.Grid(*shape, ratio=ratio, precond="philine").solve(br, 1e-12)
    for x in (xr, xp):
        assert np.linalg.norm(x - xj) / np.linalg.norm(xj) <= 1e-10
    assert itp < 0.6 * itj and itp < itr < itj, (itj, itr, itp)


@pytest.mark.parametrize("outer", ["source", "closed"])
@pytest.mark.parametrize("shape,ratio", [((4, 5, 7), 1.1), ((3, 6, 3), 1.0), ((5, 4, 8), 1.3)])
def test_precond_both_lines_is_the_additive_combination(oracle_mod, shape, ratio, outer):
    """Both line directions: M^-1 = T_r^-1 + T_phi^-1 - D^-1 with T_r, T_phi
    cut out of the dense L; M^-1 is symmetric positive definite."""
    g = oracle_mod.Grid(*shape, ratio=ratio, outer=outer, precond="lines")
    A = g.dense()
    Minv = (np.linalg.inv(line_part(A, shape, "rline")) + np.linalg.inv(line_part(A, shape, "philine"))
            - np.diag(1.0 / np.diag(A)))
    np.testing.assert_allclose(Minv, Minv.T, rtol=0, atol=1e-13 * np.abs(Minv).max())
    assert np.linalg.eigvalsh(0.5 * (Minv + Minv.T)).min() > 0
    r = syn.random_field(shape, seed=7)
    z = g.apply_precond(r)
    zd = Minv @ r.ravel()
    np.testing.assert_allclose(z.ravel(), zd, rtol=1e-12, atol=1e-13 * np.abs(zd).max())


def test_pcg_both_lines_matches_dense_and_first_step(oracle_mod):
    shape = (4, 5, 6)
    g = oracle_mod.Grid(*shape, ratio=1.1, precond="lines")
    A = g.dense()
    br = syn.random_field((5, 6), seed=11)
    b = g.rhs(br)
    x, it, st = g.pcg(b, 1e-13)
    assert st == oracle_mod.OK
    xd = np.linalg.solve(A, b.ravel())
    assert np.linalg.norm(x.ravel() - xd) / np.linalg.norm(xd) < 1e-11
    Minv = (np.linalg.inv(line_part(A, shape, "rline")) + np.linalg.inv(line_part(A, shape, "philine"))
            - np.diag(1.0 / np.diag(A)))
    z = Minv @ b.ravel()
    alpha = (b.ravel() @ z) / (z @ A @ z)
    x1, it1, st1 = g.pcg(b, 1e-300, maxit=1)
    np.testing.assert_allclose(x1.ravel(), alpha * z, rtol=1e-12, atol=1e-14 * np.abs(z).max())


def test_both_lines_beat_either_under_strong_radial_stretching(oracle_mod):
    """With a first radial cell 1000 times thinner than the angular cells
    the radial couplings dominate almost everywhere and phi lines alone help
    little; adding radial lines removes that anisotropy as well."""
    shape, ratio = (41, 31, 61), 1.15
    br = syn.bipole_br(31, 61, seed=1709, n_bipoles=30)
    its = {}
    xs = {}
    for pc in ("jacobi", "rline", "philine", "lines"):
        xs[pc], its[pc], st = oracle_mod.Grid(*shape, ratio=ratio, precond=pc).solve(br, 1e-10)
        assert st == oracle_mod.OK
    for pc in ("rline", "philine", "lines"):
        assert np.linalg.norm(xs[pc] - xs["jacobi"]) / np.linalg.norm(xs["jacobi"]) <= 1e-8
    assert its["lines"] < its["rline"] < its["philine"] < its["jacobi"], its
