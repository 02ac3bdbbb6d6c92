"""Pins of the oracle's PC2 (Sec. 2.3: non-overlapping domain decomposition
with a zero-fill incomplete LU factorisation of every subdomain block), on
the CPU, against what ILU(0) is by definition rather than against the
oracle's own loops:

- M = L U is block diagonal over the subdomain boxes, L is unit lower and U
  upper triangular with the sparsity pattern of the box's block of A, and
  (L U)_ij = a_ij wherever a_ij != 0 (the defining property of ILU(0),
  Saad, Iterative Methods for Sparse Linear Systems, Sec. 10.3.2);
- a box of one radial column is a tridiagonal block, whose ILU(0) is its
  exact LU: M^-1 is then the radial-line solve;
- for the 7-point pattern only the diagonal changes: the pivots follow
  d_c = a_cc - sum over lower neighbours m in the box of a_cm a_mc / d_m;
- the paper's r-fastest numbering gives the same M (a plain dense ILU(0)
  written here, run in that numbering);
- PCG with PC2 reaches the dense direct solution in fewer iterations.
"""
import numpy as np
import pytest

import pot3d_synth as syn


def dense_inverse_of_precond(g):
    """M^-1 column by column from the oracle's z = M^-1 r."""
    n = g.n
    Mi = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        Mi[:, c] = g.apply_precond(e.reshape(g.shape)).ravel()
    return Mi


def box_ids(shape, blocks):
    """Subdomain box of every cell (C order), boxes of `blocks` cells (0 =
    the whole extent; the last box of an axis takes the remainder)."""
    idx = np.indices(shape).reshape(3, -1)
    key = np.zeros(idx.shape[1], dtype=np.int64)
    for ax in range(3):
        b = blocks[ax] if 0 < blocks[ax] < shape[ax] else shape[ax]
        key = key * (shape[ax] + 1) + idx[ax] // b
    return key


def lu_nopivot(M):
    """Doolittle LU without pivoting: M = L U, L unit lower."""
    n = M.shape[0]
    U = M.astype(np.float64).copy()
    L = np.eye(n)
    for k in range(n - 1):
        f = U[k + 1:, k] / U[k, k]
        L[k + 1:, k] = f
        U[k + 1:, k:] -= np.outer(f, U[k, k:])
        U[k + 1:, k] = 0.0
    return L, U


def ilu0_dense(A):
    """Plain ILU(0) of a dense matrix, pattern = nonzeros of A (the IKJ
    form: a_ik /= a_kk, then a_ij -= a_ik a_kj for j > k inside the
    pattern).  Returns M = L U."""
    n = A.shape[0]
    nz = A != 0
    a = A.astype(np.float64).copy()
    for i in range(1, n):
        for k in range(i):
            if not nz[i, k]:
                continue
            a[i, k] /= a[k, k]
            for j in range(k + 1, n):
                if nz[i, j]:
                    a[i, j] -= a[i, k] * a[k, j]
    L = np.tril(a, -1) + np.eye(n)
    U = np.triu(a)
    return L @ U


CASES = [((5, 6, 7), 1.05, (0, 2, 3)), ((4, 5, 9), 1.1, (2, 3, 4)), ((4, 3, 8), 1.0, (0, 1, 3)),
         ((3, 4, 5), 1.2, (0, 0, 0)), ((4, 4, 6), 1.02, (0, 1, 0))]


@pytest.mark.parametrize("outer", ["source", "closed"])
@pytest.mark.parametrize("shape,ratio,blocks", CASES)
def test_ilu0_defining_property(oracle_mod, shape, ratio, blocks, outer):
    if outer == "closed" and blocks == (0, 0, 0):
        pytest.skip("one box holding the whole singular closed-wall operator")
    g = oracle_mod.Grid(*shape, ratio=ratio, outer=outer, precond="ilu", blocks=blocks)
    A = g.dense()
    M = np.linalg.inv(dense_inverse_of_precond(g))
    scale = np.abs(A).max()
    box = box_ids(shape, blocks)
    same = box[:, None] == box[None, :]
    nz = A != 0
    # block diagonal over the boxes; equal to A on A's pattern inside a box
    if (~same).any():
        assert np.abs(M[~same]).max() <= 1e-13 * scale
    assert np.abs((M - A)[nz & same]).max() <= 1e-13 * scale
    # M = L U with L and U inside the pattern of the box blocks of A
    L, U = lu_nopivot(M)
    pat = nz & same
    off = 1e-11 * scale
    assert np.abs(np.tril(L, -1)[~pat]).max(initial=0.0) <= off / scale
    assert np.abs(np.triu(U, 1)[~pat]).max(initial=0.0) <= off
    # symmetric positive definite (A symmetric M-matrix: positive pivots)
    assert np.abs(M - M.T).max() <= 1e-13 * scale
    assert np.diag(U).min() > 0.0


@pytest.mark.parametrize("outer", ["source", "closed"])
@pytest.mark.parametrize("shape,ratio", [((6, 4, 5), 1.1), ((9, 3, 4), 1.0)])
def test_radial_column_box_is_the_radial_line_solve(oracle_mod, shape, ratio, outer):
    """One radial column per box: the block is tridiagonal, ILU(0) drops
    nothing, M^-1 r is the radial-line (Thomas) solve."""
    r = syn.random_field(shape, seed=11)
    gi = oracle_mod.Grid(*shape, ratio=ratio, outer=outer, precond="ilu", blocks=(0, 1, 1))
    gl = oracle_mod.Grid(*shape, ratio=ratio, outer=outer, precond="rline")
    zi, zl = gi.apply_precond(r), gl.apply_precond(r)
    np.testing.assert_allclose(zi, zl, rtol=1e-13, atol=1e-14 * np.abs(zl).max())


@pytest.mark.parametrize("shape,ratio,blocks", [((5, 6, 7), 1.05, (0, 2, 3)),
                                                ((4, 5, 9), 1.1, (0, 1, 4)),
                                                ((4, 5, 9), 1.1, (2, 3, 4))])
def test_pivots_follow_the_seven_point_recurrence(oracle_mod, shape, ratio, blocks):
    """For the 7-point pattern ILU(0) changes only the diagonal: the pivot
    of cell c is a_cc minus a_cm a_mc / d_m over its lower neighbours m
    (r-1, theta-1, phi-1) that lie in its box."""
    g = oracle_mod.Grid(*shape, ratio=ratio, precond="ilu", blocks=blocks)
    A = g.dense()
    M = np.linalg.inv(dense_inverse_of_precond(g))
    _, U = lu_nopivot(M)
    nr, nt, np_ = shape
    box = box_ids(shape, blocks).reshape(shape)
    d = np.zeros(shape)
    for i in range(nr):
        for j in range(nt):
            for k in range(np_):
                c = (i * nt + j) * np_ + k
                v = A[c, c]
                for (ii, jj, kk) in ((i - 1, j, k), (i, j - 1, k), (i, j, k - 1)):
                    if min(ii, jj, kk) < 0 or box[ii, jj, kk] != box[i, j, k]:
                        continue
                    m = (ii * nt + jj) * np_ + kk
                    v -= A[c, m] * A[m, c] / d[ii, jj, kk]
                d[i, j, k] = v
    np.testing.assert_allclose(np.diag(U), d.ravel(), rtol=1e-12)
    # and the off-diagonal factors are A's own couplings: U = D~ + strict upper of A
    off = np.triu(A, 1) * (box.ravel()[:, None] == box.ravel()[None, :])
    np.testing.assert_allclose(np.triu(U, 1), off, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("shape,blocks", [((3, 4, 5), (0, 2, 3)), ((4, 3, 4), (0, 0, 0))])
def test_r_fastest_numbering_gives_the_same_preconditioner(oracle_mod, shape, blocks):
    """The paper's FORTRAN arrays put r fastest.  ILU(0) of each box block
    in that numbering (a plain dense ILU(0), run here) gives the M of the
    oracle's C-order numbering."""
    g = oracle_mod.Grid(*shape, ratio=1.07, precond="ilu", blocks=blocks)
    A = g.dense()
    box = box_ids(shape, blocks)
    Ab = np.where(box[:, None] == box[None, :], A, 0.0)
    nr, nt, np_ = shape
    # position in the r-fastest numbering of each C-order cell
    i, j, k = np.indices(shape).reshape(3, -1)
    order = np.argsort(i + nr * (j + nt * k), kind="stable")
    Mf = ilu0_dense(Ab[np.ix_(order, order)])
    M = np.empty_like(Mf)
    M[np.ix_(order, order)] = Mf
    Mo = np.linalg.inv(dense_inverse_of_precond(g))
    np.testing.assert_allclose(Mo, M, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("outer", ["source", "closed"])
def test_pcg_with_pc2_matches_direct_solve_in_fewer_iterations(oracle_mod, outer):
    shape = (8, 12, 40)
    br = syn.bipole_br(shape[1], shape[2], seed=5, n_bipoles=8)
    g1 = oracle_mod.Grid(*shape, ratio=1.05, outer=outer)
    g2 = oracle_mod.Grid(*shape, ratio=1.05, outer=outer, precond="ilu", blocks=(0, 1, 32))
    b = g1.rhs(br)
    A = g1.dense()
    if outer == "closed":
        # bordered system [[L, 1], [1^T, 0]]: the zero-mean solution
        n = g1.n
        K = np.zeros((n + 1, n + 1))
        K[:n, :n] = A
        K[:n, n] = K[n, :n] = 1.0
        xd = np.linalg.solve(K, np.append(b.ravel(), 0.0))[:n]
    else:
        xd = np.linalg.solve(A, b.ravel())
    x1, it1, st1 = g1.solve(br, 1e-12)
    x2, it2, st2 = g2.solve(br, 1e-12)
    assert st1 == st2 == 0
    assert np.linalg.norm(x2.ravel() - xd) <= 1e-10 * np.linalg.norm(xd)
    assert it2 < it1, (it2, it1)
