"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(no GPU).  Each test would fail for a plausible slip in the oracle: a
dropped metric factor, a wrong sign or index, a transposed coefficient, a
wrong pole or ghost treatment, or a wrong PCG step.

Paper references: Sec. 2.1 (Eqs. 1-3), Sec. 2.2 (stencil, Eq. 4), Sec. 2.3 (PCG, PC1).
"""
import numpy as np
import pytest

import pot3d_synth as syn


def shell_coeffs(l, R1):
    """a, b of Phi = (a r^l + b r^-(l+1)) Y with dPhi/dr(1) = Y (Eq. 2) and
    Phi(R1) = 0 (source surface): a 2x2 linear solve."""
    M = np.array([[l, -(l + 1.0)], [R1 ** l, R1 ** (-(l + 1.0))]])
    return np.linalg.solve(M, np.array([1.0, 0.0]))


def ylm_grad(l, m, scale, r, th, ph, a, b):
    """Analytic grad of (a r^l + b r^-(l+1)) * scale P_l^m(cos th) cos(m ph)."""
    from scipy.special import lpmv

    f = a * r ** l + b * r ** (-(l + 1.0))
    fp = a * l * r ** (l - 1.0) - b * (l + 1.0) * r ** (-(l + 2.0))
    x = np.cos(th)
    P = lpmv(m, l, x)
    # dP/dth = -sin th dP/dx; (1-x^2) dP/dx = (l+1) x P_l^m - (l-m+1) P_{l+1}^m
    dPdx_times = (l + 1.0) * x * P - (l - m + 1.0) * lpmv(m, l + 1, x)
    dPdth = -dPdx_times / np.sin(th)
    Y = scale * P * np.cos(m * ph)
    Br = fp * Y
    Bt = f / r * scale * dPdth * np.cos(m * ph)
    Bp = f / (r * np.sin(th)) * scale * P * (-m * np.sin(m * ph))
    return Br, Bt, Bp


def test_radial_mesh_geometric(oracle_mod):
    g = oracle_mod.Grid(151, 8, 8, ratio=1.02)
    dr = np.diff(g.rf)
    assert g.rf[0] == 1.0 and g.rf[-1] == 2.5
    np.testing.assert_allclose(dr[1:] / dr[:-1], 1.02, rtol=1e-9)
    assert abs(dr.sum() - 1.5) < 1e-13
    # finest cell at the photosphere
    assert dr.argmin() == 0
    u = oracle_mod.Grid(10, 8, 8, ratio=1.0)
    np.testing.assert_allclose(np.diff(u.rf), 0.15, rtol=1e-12)


def test_theta_mesh_and_centres(oracle_mod):
    g = oracle_mod.Grid(4, 6, 8)
    np.testing.assert_allclose(g.tf, np.pi * np.arange(7) / 6, rtol=0, atol=1e-15)
    # epsilon of Eq. 3: the first centre sits half a cell from the pole
    assert abs(g.tc[0] - 0.5 * (g.tf[1] - g.tf[0])) < 1e-15


@pytest.mark.parametrize("shape,ratio,tstretch", [((3, 4, 6), 1.1, False), ((4, 5, 7), 1.0, True),
                                                   ((2, 3, 4), 1.3, True)])
def test_operator_symmetric_positive_definite(oracle_mod, shape, ratio, tstretch):
    nr, nt, np_ = shape
    tf = None
    if tstretch:
        # nonuniform theta faces, symmetric about the equator
        u = np.linspace(0, 1, nt + 1)
        tf = np.pi * (u + 0.15 * np.sin(2 * np.pi * u) / (2 * np.pi))
    g = oracle_mod.Grid(nr, nt, np_, ratio=ratio, t_faces=tf)
    A = g.dense()
    assert np.array_equal(A, A.T), "L must be exactly symmetric (Sec. 2.3)"
    w = np.linalg.eigvalsh(A)
    assert w.min() > 0, "L must be positive definite"
    np.linalg.cholesky(A)
    # matrix-free apply agrees with the assembled matrix
    x = syn.random_field(shape, seed=3)
    np.testing.assert_allclose(g.apply(x).ravel(), A @ x.ravel(), rtol=1e-13, atol=1e-15)
    # diagonal: sum of the row's couplings; strictly dominant on the outer layer only
    off = np.abs(A - np.diag(np.diag(A))).sum(axis=1).reshape(shape)
    d = np.diag(A).reshape(shape)
    np.testing.assert_allclose(d[:-1], off[:-1], rtol=1e-13)
    assert np.all(d[-1] > off[-1] * (1 + 1e-12))
    np.testing.assert_allclose(g.diag(), d[:, :, 0], rtol=0, atol=0)


def test_constant_is_harmonic_except_source_surface(oracle_mod):
    """L 1 = 0 wherever the stencil is a pure difference (interior, inner
    flux face, poles, phi wrap); only the Phi = 0 ghost of the source surface
    leaves a residual, and it is positive there."""
    g = oracle_mod.Grid(6, 7, 9, ratio=1.07)
    y = g.apply(np.ones(g.shape))
    assert np.max(np.abs(y[:-1])) < 1e-14 * np.max(np.abs(y[-1]))
    assert np.all(y[-1] > 0)


def test_rhs_is_inner_flux(oracle_mod):
    """b = -r0^2 sin(th) dth dphi Br on the first layer only (Eq. 2)."""
    g = oracle_mod.Grid(5, 6, 8)
    br = syn.random_field((6, 8), seed=5)
    b = g.rhs(br)
    assert np.all(b[1:] == 0)
    area = (np.sin(g.tc) * np.diff(g.tf))[:, None] * (2 * np.pi / 8)
    np.testing.assert_allclose(b[0], -area * br, rtol=1e-14)
    # total inner flux = sum of b: the discrete Gauss law of the solution
    np.testing.assert_allclose(b.sum(), -(area * br).sum(), rtol=1e-12)


def _shell_error(oracle_mod, n, l, m, ratio=1.0, tf=None, tol=1e-12):
    g = oracle_mod.Grid(n, n, 2 * n, ratio=ratio, t_faces=tf)
    br, scale = syn.ylm_br(g.nt, g.np, l, m, t_faces=tf)
    x, it, st = g.solve(br, tol)
    assert st == oracle_mod.OK
    a, b = shell_coeffs(l, 2.5)
    R, T, P = np.meshgrid(g.rc, g.tc, g.pc, indexing="ij")
    ex = (a * R ** l + b * R ** (-(l + 1.0))) * syn.ylm_shape(l, m, T, P, scale)
    return np.linalg.norm(x - ex) / np.linalg.norm(ex), g, x, br, scale


def test_closed_form_shell_second_order(oracle_mod):
    """Y_3^2 on the shell: discrete Phi converges to the exact potential at
    second order (Sec. 2.2: globally second-order)."""
    errs = [_shell_error(oracle_mod, n, 3, 2)[0] for n in (10, 20, 40)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 3e-3
    assert np.all(orders > 1.9), (errs, orders)


def test_closed_form_stretched_meshes(oracle_mod):
    """Same, on a geometric r mesh and a nonuniform theta mesh."""
    def tfaces(nt):
        u = np.linspace(0, 1, nt + 1)
        return np.pi * (u + 0.1 * np.sin(2 * np.pi * u) / (2 * np.pi))

    errs = []
    for n, g in ((10, 1.08), (20, 1.08 ** 0.5), (40, 1.08 ** 0.25)):
        errs.append(_shell_error(oracle_mod, n, 3, 2, ratio=g, tf=tfaces(n))[0])
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), (errs, orders)


@pytest.mark.parametrize("l,m", [(1, 0), (1, 1), (2, 1), (4, 3)])
def test_closed_form_other_harmonics(oracle_mod, l, m):
    e1 = _shell_error(oracle_mod, 12, l, m)[0]
    e2 = _shell_error(oracle_mod, 24, l, m)[0]
    assert np.log2(e1 / e2) > 1.8, (l, m, e1, e2)


@pytest.mark.parametrize("shape,ratio", [((4, 4, 8), 1.0), ((3, 5, 6), 1.2), ((6, 6, 12), 1.05)])
def test_pcg_matches_dense_direct_solve(oracle_mod, shape, ratio):
    g = oracle_mod.Grid(*shape, ratio=ratio)
    br = syn.random_field(shape[1:], seed=11)
    b = g.rhs(br)
    x, it, st = g.pcg(b, 1e-13)
    assert st == oracle_mod.OK
    xd = np.linalg.solve(g.dense(), b.ravel())
    assert np.linalg.norm(x.ravel() - xd) / np.linalg.norm(xd) < 1e-11


def test_pcg_finite_termination(oracle_mod):
    """In exact arithmetic CG ends in at most n steps (n = unknowns)."""
    g = oracle_mod.Grid(2, 3, 4, ratio=1.1)
    b = g.rhs(syn.random_field((3, 4), seed=2))
    x, it, st, hist = g.pcg(b, 1e-12, history=True)
    assert st == oracle_mod.OK and it <= g.n + 2
    assert hist[0] == 1.0 and hist[-1] <= 1e-12


def test_pcg_is_jacobi_preconditioned(oracle_mod):
    """One PCG step from x0 = 0 equals the closed form alpha_1 D^-1 b with
    alpha_1 = (b.D^-1 b) / (z.Lz), z = D^-1 b (Sec. 2.3, PC1)."""
    g = oracle_mod.Grid(4, 5, 6, ratio=1.1)
    A = g.dense()
    b = g.rhs(syn.random_field((5, 6), seed=8)).ravel()
    z = b / np.diag(A)
    alpha = (b @ z) / (z @ A @ z)
    x1, it, st = g.pcg(b, 1e-300, maxit=1)
    assert it == 1 and st == oracle_mod.NOT_CONVERGED
    np.testing.assert_allclose(x1.ravel(), alpha * z, rtol=1e-13)


def test_pcg_initial_guess_restart(oracle_mod):
    g = oracle_mod.Grid(6, 8, 12, ratio=1.05)
    b = g.rhs(syn.bipole_br(8, 12, seed=4, n_bipoles=5))
    x, it, st = g.pcg(b, 1e-12)
    x2, it2, st2 = g.pcg(b, 1e-12, x0=x)
    assert st2 == oracle_mod.OK and it2 <= 2
    np.testing.assert_allclose(x2, x, rtol=1e-10, atol=1e-14 * np.abs(x).max())


def test_field_invariants(oracle_mod):
    """B = grad Phi on faces: (i) the inner face carries the input Br
    (Eq. 2); (ii) the volume-weighted discrete divergence of B equals the
    residual b - L Phi; (iii) Btheta on each pole face has zero phi-mean
    (Eq. 3: the pole value is the ring average)."""
    nr, nt, np_ = 10, 12, 20
    g = oracle_mod.Grid(nr, nt, np_, ratio=1.05)
    br = syn.bipole_br(nt, np_, seed=21, n_bipoles=6)
    phi, it, st = g.solve(br, 1e-10)
    Br, Bt, Bp = g.field(phi, br)
    assert np.array_equal(Br[0], br)
    # fluxes through faces
    dphi = 2 * np.pi / np_
    dr, dt = np.diff(g.rf), np.diff(g.tf)
    st_c = np.sin(g.tc)
    st_f = np.sin(g.tf)
    st_f[0] = st_f[-1] = 0.0
    Ar = (g.rf ** 2)[:, None, None] * (st_c * dt)[None, :, None] * dphi
    At = (g.rc * dr)[:, None, None] * st_f[None, :, None] * dphi
    Ap = (g.rc * dr)[:, None, None] * dt[None, :, None]
    Fr = Br * Ar
    Ft = Bt * At
    Fp = Bp * Ap
    div = (Fr[1:] - Fr[:-1]) + (Ft[:, 1:] - Ft[:, :-1]) + (Fp - np.roll(Fp, 1, axis=2))
    resid = g.rhs(br) - g.apply(phi)
    scale = np.abs(g.rhs(br)).max()
    np.testing.assert_allclose(div, resid, rtol=0, atol=1e-11 * scale)
    assert np.linalg.norm(div) <= 2e-10 * np.linalg.norm(g.rhs(br))
    for f in (0, nt):
        m = Bt[:, f, :].mean(axis=1)
        assert np.all(np.abs(m) <= 1e-13 * np.abs(Bt).max())


def test_field_matches_analytic_gradient(oracle_mod):
    """Face fields of the Y_3^2 solution converge to grad Phi at second order."""
    l, m = 3, 2
    a, b = shell_coeffs(l, 2.5)
    errs = []
    for n in (10, 20, 40):
        e, g, phi, br, scale = _shell_error(oracle_mod, n, l, m)
        Br, Bt, Bp = g.field(phi, br)
        # radial faces between centres (skip the two boundary faces)
        R, T, P = np.meshgrid(g.rf[1:-1], g.tc, g.pc, indexing="ij")
        ex_r = ylm_grad(l, m, scale, R, T, P, a, b)[0]
        # theta faces away from the poles
        R2, T2, P2 = np.meshgrid(g.rc, g.tf[1:-1], g.pc, indexing="ij")
        ex_t = ylm_grad(l, m, scale, R2, T2, P2, a, b)[1]
        # phi faces between k and k+1
        R3, T3, P3 = np.meshgrid(g.rc, g.tc, g.pc + np.pi / g.np, indexing="ij")
        ex_p = ylm_grad(l, m, scale, R3, T3, P3, a, b)[2]
        num = np.concatenate([(Br[1:-1] - ex_r).ravel(), (Bt[:, 1:-1] - ex_t).ravel(),
                              (Bp - ex_p).ravel()])
        den = np.concatenate([ex_r.ravel(), ex_t.ravel(), ex_p.ravel()])
        errs.append(np.linalg.norm(num) / np.linalg.norm(den))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), (errs, orders)


@pytest.mark.parametrize("l", [1, 2])
def test_pole_face_btheta_matches_analytic(oracle_mod, l):
    """Btheta on the two pole faces (Eq. 3: the ghost across the pole makes
    the face value the ring's phi-average) converges to the analytic
    dPhi/(r dtheta) at theta = 0 and pi for the m = 1 harmonics, whose
    pole-face Btheta is non-zero and varies with phi.  The face value divides
    the first ring's error by the half-cell distance to the pole, so it
    converges at about order 1.6 (measured for l = 1 from 10 to 80 cells:
    1.57, 1.64, 1.63), not 2.  A dropped factor 2 in the mirror spacing, or a
    flipped sign, makes the error O(1)."""
    from scipy.special import lpmv

    m = 1
    a, b = shell_coeffs(l, 2.5)
    h = 1e-6
    # d/dtheta of P_l^1(cos theta) just inside each pole (P_l^1 vanishes there)
    dn = lpmv(m, l, np.cos(h)) / h
    ds = -lpmv(m, l, np.cos(np.pi - h)) / h
    errs = []
    for n in (10, 20, 40):
        e, g, phi, br, scale = _shell_error(oracle_mod, n, l, m)
        Br, Bt, Bp = g.field(phi, br)
        f = a * g.rc ** l + b * g.rc ** (-(l + 1.0))
        ang = np.cos(m * g.pc)
        ex_n = (f / g.rc)[:, None] * scale * dn * ang[None, :]
        ex_s = (f / g.rc)[:, None] * scale * ds * ang[None, :]
        num = np.concatenate([(Bt[:, 0, :] - ex_n).ravel(), (Bt[:, -1, :] - ex_s).ravel()])
        den = np.concatenate([ex_n.ravel(), ex_s.ravel()])
        errs.append(np.linalg.norm(num) / np.linalg.norm(den))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-2, errs
    assert np.all(orders > 1.35), (errs, orders)


def test_pole_average(oracle_mod):
    g = oracle_mod.Grid(3, 4, 5)
    phi = syn.random_field(g.shape, seed=9)
    north, south = g.pole_avg(phi)
    np.testing.assert_allclose(north, phi[:, 0, :].mean(axis=1), rtol=1e-15)
    np.testing.assert_allclose(south, phi[:, -1, :].mean(axis=1), rtol=1e-15)


def test_bipole_generator_deterministic_and_balanced():
    a = syn.bipole_br(61, 121, seed=1709)
    b = syn.bipole_br(61, 121, seed=1709)
    c = syn.bipole_br(61, 121, seed=1710)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    tf = syn.theta_faces(61)
    area = (np.sin(0.5 * (tf[1:] + tf[:-1])) * np.diff(tf))[:, None] * (2 * np.pi / 121)
    assert abs(np.sum(a * area)) <= 1e-12 * np.sum(np.abs(a) * area)
    assert 1.0 < np.abs(a).max() < 2000.0


def test_ylm_unit_amplitude():
    br, scale = syn.ylm_br(400, 400, 3, 2)
    assert 0.99 < np.abs(br).max() <= 1.0 + 1e-12
