"""Pins of the oracle's closed-wall outer boundary (Sec. 2.1: the alternative
to the source surface, Br = dPhi/dr = 0 at r = R_1), on the CPU.

With no flux through either radial boundary the operator is singular: its
null space is the constants.  The right-hand side then needs zero net flux
(the inner Br loses its area-weighted mean), and the solution is defined up
to a constant (the oracle returns the representative with zero cell mean).
Each test would fail for a plausible slip: a leftover source-surface term on
the outer diagonal, a wrong balancing weight, a wrong ghost in the field.
"""
import numpy as np
import pytest

import pot3d_synth as syn


def closed_shell_coeffs(l, R1):
    """a, b of Phi = (a r^l + b r^-(l+1)) Y with dPhi/dr = Y at r = 1 (Eq. 2)
    and dPhi/dr = 0 at r = R1 (closed wall)."""
    M = np.array([[l, -(l + 1.0)], [l * R1 ** (l - 1.0), -(l + 1.0) * R1 ** (-(l + 2.0))]])
    return np.linalg.solve(M, np.array([1.0, 0.0]))


@pytest.mark.parametrize("shape,ratio,tstretch", [((3, 4, 6), 1.1, False), ((4, 5, 7), 1.0, True)])
def test_operator_symmetric_semidefinite_with_constant_null_space(oracle_mod, shape, ratio,
                                                                  tstretch):
    nr, nt, np_ = shape
    tf = None
    if tstretch:
        u = np.linspace(0, 1, nt + 1)
        tf = np.pi * (u + 0.15 * np.sin(2 * np.pi * u) / (2 * np.pi))
    g = oracle_mod.Grid(nr, nt, np_, ratio=ratio, t_faces=tf, outer="closed")
    A = g.dense()
    assert np.array_equal(A, A.T)
    scale = np.abs(A).max()
    assert np.abs(A @ np.ones(g.n)).max() <= 1e-14 * scale
    w = np.linalg.eigvalsh(A)
    assert abs(w[0]) <= 1e-12 * w[-1]          # one zero eigenvalue ...
    assert w[1] > 1e-6 * w[-1]                 # ... and only one
    # every row is a pure difference now: diagonal = sum of |off-diagonal|
    off = np.abs(A - np.diag(np.diag(A))).sum(axis=1)
    np.testing.assert_allclose(np.diag(A), off, rtol=1e-13)
    # the source-surface operator differs exactly on the outer layer's diagonal
    S = oracle_mod.Grid(nr, nt, np_, ratio=ratio, t_faces=tf, outer="source").dense()
    assert np.all(np.diagonal(S - A).reshape(shape)[:-1] == 0)
    assert np.all(np.diagonal(S - A).reshape(shape)[-1] > 0)
    assert np.count_nonzero(S - A - np.diag(np.diag(S - A))) == 0


def test_rhs_has_zero_net_flux(oracle_mod):
    g = oracle_mod.Grid(5, 6, 8, ratio=1.05, outer="closed")
    br = syn.random_field((6, 8), seed=5)
    b = g.rhs(br)
    assert abs(b.sum()) <= 1e-14 * np.abs(b).sum()
    # a uniform Br (pure monopole) is removed entirely
    np.testing.assert_allclose(g.rhs(br + 3.0), b, rtol=0, atol=1e-14 * np.abs(b).max())
    # the balanced Br has zero area-weighted mean
    bb = g.balanced_br(br)
    area = (np.sin(g.tc) * np.diff(g.tf))[:, None] * np.ones((1, 8))
    assert abs((area * bb).sum()) <= 1e-14 * (area * np.abs(bb)).sum()
    # source surface: Br untouched
    s = oracle_mod.Grid(5, 6, 8, ratio=1.05, outer="source")
    assert np.array_equal(s.balanced_br(br), br)


@pytest.mark.parametrize("shape,ratio", [((4, 4, 8), 1.0), ((3, 5, 6), 1.2), ((6, 6, 12), 1.05)])
def test_pcg_matches_minimum_norm_direct_solve(oracle_mod, shape, ratio):
    """The singular system's solution with zero mean (its null space is the
    constants), from a dense solve of the bordered system
    [[A, 1], [1^T, 0]] [x, lam] = [b, 0]: PCG plus the gauge must reproduce
    it."""
    g = oracle_mod.Grid(*shape, ratio=ratio, outer="closed")
    br = syn.random_field(shape[1:], seed=11)
    x, it, st = g.solve(br, 1e-13)
    assert st == oracle_mod.OK
    b = g.rhs(br).ravel()
    n = g.n
    K = np.zeros((n + 1, n + 1))
    K[:n, :n] = g.dense()
    K[:n, n] = K[n, :n] = 1.0
    sol = np.linalg.solve(K, np.concatenate([b, [0.0]]))
    xd = sol[:n]
    assert abs(sol[n]) <= 1e-12 * np.abs(b).max()  # b is compatible: no multiplier
    assert abs(xd.sum()) <= 1e-12 * np.abs(xd).sum()
    assert abs(x.sum()) <= 1e-12 * np.abs(x).sum()
    assert np.linalg.norm(x.ravel() - xd) / np.linalg.norm(xd) < 1e-10


def _closed_shell_error(oracle_mod, n, l, m, ratio=1.0):
    g = oracle_mod.Grid(n, n, 2 * n, ratio=ratio, outer="closed")
    br, scale = syn.ylm_br(g.nt, g.np, l, m)
    x, it, st = g.solve(br, 1e-12)
    assert st == oracle_mod.OK
    a, b = closed_shell_coeffs(l, 2.5)
    R, T, P = np.meshgrid(g.rc, g.tc, g.pc, indexing="ij")
    ex = (a * R ** l + b * R ** (-(l + 1.0))) * syn.ylm_shape(l, m, T, P, scale)
    ex = ex - ex.mean()
    return np.linalg.norm(x - ex) / np.linalg.norm(ex), g, x, br


@pytest.mark.parametrize("l,m", [(3, 2), (1, 1)])
def test_closed_form_shell_second_order(oracle_mod, l, m):
    """Phi = (a r^l + b r^-(l+1)) Y_l^m with dPhi/dr = Y at r = 1 and 0 at
    r = 2.5: the discrete solution converges at second order."""
    errs = [_closed_shell_error(oracle_mod, n, l, m)[0] for n in (10, 20, 40)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 5e-3, errs
    assert np.all(orders > 1.85), (errs, orders)


def test_closed_wall_field(oracle_mod):
    """Outer face Br = 0 exactly; inner face = the balanced Br; the
    volume-weighted divergence of B equals the residual b - L Phi."""
    nr, nt, np_ = 9, 12, 20
    g = oracle_mod.Grid(nr, nt, np_, ratio=1.05, outer="closed")
    br = syn.bipole_br(nt, np_, seed=21, n_bipoles=6) + 0.7  # add a monopole
    phi, it, st = g.solve(br, 1e-11)
    bb = g.balanced_br(br)
    Br, Bt, Bp = g.field(phi, bb)
    assert np.all(Br[-1] == 0.0)
    assert np.array_equal(Br[0], bb)
    dphi = 2 * np.pi / np_
    dr, dt = np.diff(g.rf), np.diff(g.tf)
    st_f = np.sin(g.tf)
    st_f[0] = st_f[-1] = 0.0
    Ar = (g.rf ** 2)[:, None, None] * (np.sin(g.tc) * dt)[None, :, None] * dphi
    At = (g.rc * dr)[:, None, None] * st_f[None, :, None] * dphi
    Ap = (g.rc * dr)[:, None, None] * dt[None, :, None]
    Fr, Ft, Fp = Br * Ar, Bt * At, Bp * Ap
    div = (Fr[1:] - Fr[:-1]) + (Ft[:, 1:] - Ft[:, :-1]) + (Fp - np.roll(Fp, 1, axis=2))
    resid = g.rhs(br) - g.apply(phi)
    np.testing.assert_allclose(div, resid, rtol=0, atol=1e-11 * np.abs(g.rhs(br)).max())
