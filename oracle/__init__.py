"""Plain FP64 CPU oracle for the POT3D potential-field solve (arXiv:1709.01126).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the GPU library: the C source next to this
file (``pot3d_oracle.c``) has its own mesh, coefficient, operator, PCG and
field code, written step by step from the paper:

- Sec. 2.1, Eqs. 1-3: Laplace equation, inner Br condition, source surface
  (or its alternative, the closed wall Br = 0), periodic phi and the polar
  average.
- Sec. 2.2 (finite-difference stencil) and Eq. 4: the 7-point operator, in
  its symmetric volume-weighted form with the r^2 metric factors restored.
- Sec. 2.3: PCG with point-Jacobi / diagonal scaling (PC1) and with PC2,
  the non-overlapping domain decomposition with a zero-fill incomplete LU
  factorisation (ILU(0), Saad Algorithm 10.4) of each subdomain's block;
  as the stronger preconditioners Sec. 6 asks for, radial-line Jacobi (one
  tridiagonal solve per (theta, phi) column) and phi-line Jacobi (one cyclic
  tridiagonal solve per (r, theta) ring).

The wrapper below only marshals numpy arrays into the C routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pot3d_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, NOT_CONVERGED, BREAKDOWN, BAD_ARG = 0, 1, 2, 3

_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C, OpenMP) into oracle/_build."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i, d = ctypes.c_int, ctypes.c_double
            lib.orc_r_faces.argtypes = [i, d, d, d, _dp]
            lib.orc_t_faces.argtypes = [i, _dp]
            lib.orc_apply.argtypes = [i, i, i, _dp, _dp, _dp, _dp]
            lib.orc_diag.argtypes = [i, i, i, _dp, _dp, _dp]
            lib.orc_coeffs.argtypes = [i, i, i, _dp, _dp, _dp, _dp, _dp]
            lib.orc_rhs.argtypes = [i, i, i, _dp, _dp, _dp, _dp]
            lib.orc_pcg.argtypes = [i, i, i, _dp, _dp, _dp, d, i, i, _dp,
                                    ctypes.POINTER(ctypes.c_int), _dp]
            lib.orc_pole_avg.argtypes = [i, i, i, _dp, _dp, _dp]
            lib.orc_field.argtypes = [i, i, i, _dp, _dp, _dp, _dp, _dp]
            lib.orc_csr.argtypes = [i, i, i, _dp, _dp, _lp, _lp, _dp]
            lib.orc_csr.restype = ctypes.c_long
            lib.orc_set_outer.argtypes = [i]
            lib.orc_set_precond.argtypes = [i]
            lib.orc_set_blocks.argtypes = [i, i, i]
            lib.orc_precond.argtypes = [i, i, i, _dp, _dp, _dp, _dp]
            lib.orc_balance_br.argtypes = [i, i, i, _dp, _dp, _dp, _dp]
            lib.orc_remove_mean.argtypes = [ctypes.c_long, _dp]
            lib.orc_remove_mean.restype = None
            lib.orc_set_threads.argtypes = [i]
            lib.orc_get_threads.restype = i
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


OUTER = {"source": 0, "closed": 1}
PRECOND = {"jacobi": 0, "rline": 1, "philine": 2, "lines": 3, "ilu": 4}


class Grid:
    """Mesh of nr x nt x np cell-centred unknowns (Sec. 2.2: nonuniform in r
    and theta, periodic in phi).  r faces run from r0 (the photosphere) to r1
    (the outer boundary), geometric with cell-width ratio ``ratio`` (1 =
    uniform) unless ``r_faces`` is given; theta faces are uniform unless
    ``t_faces`` is given.  ``outer``: "source" (source surface, Phi = 0 at r1)
    or "closed" (closed wall, Br = 0 at r1), Sec. 2.1.  ``precond``: "jacobi"
    (diagonal scaling, PC1 of Sec. 2.3), "rline" (radial-line Jacobi) or
    "philine" (phi-line Jacobi: one cyclic tridiagonal solve per ring),
    "lines" (both: M^-1 = T_r^-1 + T_phi^-1 - D^-1) or "ilu" (PC2: ILU(0)
    of every subdomain box of ``blocks`` = (cells in r, theta, phi; 0 = the
    whole extent), couplings between boxes dropped)."""

    def __init__(self, nr, nt, np_, r0=1.0, r1=2.5, ratio=1.0, r_faces=None, t_faces=None,
                 outer="source", precond="jacobi", blocks=(0, 1, 32)):
        self.nr, self.nt, self.np = int(nr), int(nt), int(np_)
        self.outer = outer
        self.precond = precond
        self.blocks = tuple(int(b) for b in blocks)
        lib = _load()
        if r_faces is None:
            rf = np.empty(self.nr + 1)
            if lib.orc_r_faces(self.nr, float(r0), float(r1), float(ratio), _p(rf)) != OK:
                raise ValueError("bad radial mesh")
        else:
            rf = np.ascontiguousarray(r_faces, dtype=np.float64)
            assert rf.shape == (self.nr + 1,)
        if t_faces is None:
            tf = np.empty(self.nt + 1)
            lib.orc_t_faces(self.nt, _p(tf))
        else:
            tf = np.ascontiguousarray(t_faces, dtype=np.float64)
            assert tf.shape == (self.nt + 1,)
        self.rf, self.tf = rf, tf

    @property
    def shape(self):
        return (self.nr, self.nt, self.np)

    @property
    def n(self):
        return self.nr * self.nt * self.np

    @property
    def rc(self):
        return 0.5 * (self.rf[1:] + self.rf[:-1])

    @property
    def tc(self):
        return 0.5 * (self.tf[1:] + self.tf[:-1])

    @property
    def pc(self):
        return (np.arange(self.np) + 0.5) * (2 * np.pi / self.np)

    def _dims(self):
        _load().orc_set_outer(OUTER[self.outer])
        _load().orc_set_precond(PRECOND[self.precond])
        _load().orc_set_blocks(*self.blocks)
        return self.nr, self.nt, self.np, _p(self.rf), _p(self.tf)

    # -- operator (Sec. 2.2, Eq. 4) --------------------------------------
    def apply(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.shape)
        y = np.empty_like(x)
        _load().orc_apply(*self._dims(), _p(x), _p(y))
        return y

    def diag(self) -> np.ndarray:
        d = np.empty((self.nr, self.nt))
        _load().orc_diag(*self._dims(), _p(d))
        return d

    def coeffs(self):
        cr = np.empty((self.nr, self.nt))
        ct = np.empty((self.nr, self.nt - 1))
        cp = np.empty((self.nr, self.nt))
        _load().orc_coeffs(*self._dims(), _p(cr), _p(ct), _p(cp))
        return cr, ct, cp

    def apply_precond(self, r: np.ndarray) -> np.ndarray:
        """z = M^-1 r with this grid's preconditioner."""
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(self.shape)
        z = np.empty_like(r)
        _load().orc_precond(*self._dims(), _p(r), _p(z))
        return z

    def rhs(self, br: np.ndarray) -> np.ndarray:
        br = np.ascontiguousarray(br, dtype=np.float64).reshape(self.nt, self.np)
        b = np.empty(self.shape)
        _load().orc_rhs(*self._dims(), _p(br), _p(b))
        return b

    def csr(self):
        """Assembled (rowptr, col, val) of L (small grids only)."""
        n = self.n
        rowptr = np.empty(n + 1, dtype=np.int64)
        col = np.empty(7 * n, dtype=np.int64)
        val = np.empty(7 * n)
        nnz = _load().orc_csr(*self._dims(), rowptr.ctypes.data_as(_lp), col.ctypes.data_as(_lp),
                              _p(val))
        if nnz < 0:
            raise ValueError("bad grid")
        return rowptr, col[:nnz].copy(), val[:nnz].copy()

    def dense(self) -> np.ndarray:
        rowptr, col, val = self.csr()
        A = np.zeros((self.n, self.n))
        for r in range(self.n):
            A[r, col[rowptr[r]:rowptr[r + 1]]] = val[rowptr[r]:rowptr[r + 1]]
        return A

    # -- solve (Sec. 2.3, PC1) -------------------------------------------
    def pcg(self, b: np.ndarray, tol: float, maxit: int = 1_000_000, x0: np.ndarray | None = None,
            history: bool = False):
        """Returns (x, iters, status[, relres history])."""
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(self.shape)
        if x0 is None:
            x = np.zeros(self.shape)
            given = 0
        else:
            x = np.array(x0, dtype=np.float64).reshape(self.shape).copy()
            given = 1
        it = ctypes.c_int(0)
        hist = np.zeros(maxit + 1) if history else None
        st = _load().orc_pcg(*self._dims(), _p(b), float(tol), int(maxit), given, _p(x),
                             ctypes.byref(it), _p(hist) if history else None)
        if history:
            return x, it.value, st, hist[: it.value + 1].copy()
        return x, it.value, st

    def balanced_br(self, br: np.ndarray) -> np.ndarray:
        """The Br the right-hand side uses: for the closed wall, without its
        area-weighted mean (zero net flux); else unchanged."""
        br = np.ascontiguousarray(br, dtype=np.float64).reshape(self.nt, self.np)
        out = np.empty_like(br)
        _load().orc_balance_br(*self._dims(), _p(br), _p(out))
        return out

    def remove_mean(self, x: np.ndarray) -> np.ndarray:
        """x minus its mean over the cells (the closed-wall gauge)."""
        y = np.array(x, dtype=np.float64, order="C", copy=True)
        _load().orc_remove_mean(y.size, _p(y))
        return y

    def solve(self, br: np.ndarray, tol: float, maxit: int = 1_000_000):
        """PCG on b(Br); for the closed wall the result is gauged to zero
        mean over the cells."""
        x, it, st = self.pcg(self.rhs(br), tol, maxit)
        if self.outer == "closed":
            x = self.remove_mean(x)
        return x, it, st

    # -- field (Sec. 2.1: B = grad Phi; Eq. 3 at the poles) ----------------
    def pole_avg(self, phi: np.ndarray):
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(self.shape)
        north = np.empty(self.nr)
        south = np.empty(self.nr)
        _load().orc_pole_avg(self.nr, self.nt, self.np, _p(phi), _p(north), _p(south))
        return north, south

    def field_sizes(self):
        nr, nt, np_ = self.shape
        return ((nr + 1) * nt * np_, nr * (nt + 1) * np_, nr * nt * np_)

    def field(self, phi: np.ndarray, br: np.ndarray):
        """Returns (Br, Bth, Bph) on the staggered faces."""
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(self.shape)
        br = np.ascontiguousarray(br, dtype=np.float64).reshape(self.nt, self.np)
        sizes = self.field_sizes()
        B = np.empty(sum(sizes))
        _load().orc_field(*self._dims(), _p(phi), _p(br), _p(B))
        nr, nt, np_ = self.shape
        Br = B[: sizes[0]].reshape(nr + 1, nt, np_)
        Bt = B[sizes[0]: sizes[0] + sizes[1]].reshape(nr, nt + 1, np_)
        Bp = B[sizes[0] + sizes[1]:].reshape(nr, nt, np_)
        return Br, Bt, Bp
