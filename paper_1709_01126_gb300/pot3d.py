"""Thin ctypes binding of libpot3d (include/pot3d.h).

The functions keep the C names and only marshal arguments: torch CUDA
tensors pass their device pointers (and torch's current stream), numpy
arrays pass host pointers, which the library stages through device memory.
Every step of the solve runs in the library's CUDA kernels; there is no
Python or CPU fallback: if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

POT3D_OK = 0
POT3D_ERR_INVALID_ARG = -1
POT3D_ERR_OOM = -2
POT3D_ERR_CUDA = -3
POT3D_ERR_NOT_CONVERGED = -4
POT3D_ERR_BREAKDOWN = -5
POT3D_ERR_TIMEOUT = -6
POT3D_ERR_UNSUPPORTED = -7
POT3D_ERR_BUSY = -8
POT3D_ERR_TOO_LARGE = -9

POT3D_PREC_FP64 = 0
POT3D_PREC_FP64_DF = 1
POT3D_PREC_MIXED = 2
POT3D_OUTER_SOURCE_SURFACE = 0
POT3D_OUTER_CLOSED_WALL = 1
POT3D_POLE_AVERAGE = 0

PRECISIONS = {"fp64": POT3D_PREC_FP64, "df": POT3D_PREC_FP64_DF, "mixed": POT3D_PREC_MIXED}
OUTER = {"source": POT3D_OUTER_SOURCE_SURFACE, "closed": POT3D_OUTER_CLOSED_WALL}
POT3D_PC_JACOBI = 0
POT3D_PC_PHI_LINE = 1
POT3D_PC_R_LINE = 2
POT3D_PC_LINES = 3
POT3D_PC_ILU = 4
PRECONDS = {"jacobi": POT3D_PC_JACOBI, "philine": POT3D_PC_PHI_LINE, "rline": POT3D_PC_R_LINE,
            "lines": POT3D_PC_LINES, "ilu": POT3D_PC_ILU}


class pot3d_grid_t(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("nt", ctypes.c_int), ("np", ctypes.c_int),
                ("r0", ctypes.c_double), ("r1", ctypes.c_double), ("r_ratio", ctypes.c_double),
                ("r_faces", ctypes.POINTER(ctypes.c_double)),
                ("t_faces", ctypes.POINTER(ctypes.c_double)), ("precision", ctypes.c_int)]


class pot3d_bc_t(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int), ("pole", ctypes.c_int)]


class pot3d_opts_t(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("use_x0", ctypes.c_int), ("chunk", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("time_kernels", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("mixed_restart", ctypes.c_int), ("verify", ctypes.c_int),
                ("precond", ctypes.c_int), ("history", ctypes.c_int)]


POT3D_FLAG_ABOVE_TOL = 1


class pot3d_stats_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("relres", ctypes.c_double), ("kernel_ms", ctypes.c_double * 4),
                ("launches", ctypes.c_longlong), ("relres_fp64", ctypes.c_double),
                ("flags", ctypes.c_int), ("sigma", ctypes.c_double), ("rr", ctypes.c_double)]


class pot3d_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_longlong), ("pitch", ctypes.c_int), ("tiles_matvec", ctypes.c_int),
                ("tiles_update", ctypes.c_int), ("workspace_bytes", ctypes.c_size_t),
                ("bytes_matvec", ctypes.c_double), ("bytes_update", ctypes.c_double)]


EXPORTS = ["pot3d_plan", "pot3d_autotune", "pot3d_variant_info", "pot3d_set_decomposition", "pot3d_destroy", "pot3d_set_stream", "pot3d_set_opts", "pot3d_get_info",
           "pot3d_last_stats", "pot3d_workspace_bytes", "pot3d_set_workspace", "pot3d_solve",
           "pot3d_solve_mixed", "pot3d_field", "pot3d_apply", "pot3d_residual",
           "pot3d_residual_noalloc", "pot3d_batch_create", "pot3d_batch_destroy",
           "pot3d_batch_set_stream", "pot3d_batch_set_opts", "pot3d_batch_bytes_needed",
           "pot3d_batch_submit", "pot3d_batch_step", "pot3d_batch_poll", "pot3d_batch_info",
           "pot3d_last_error", "pot3d_strerror", "pot3d_selftest_wait", "pot3d_probe_fp64_fma",
           "pot3d_test_freeze_poll", "pot3d_get_history"]

_lib = None


def lib_path() -> str:
    return _build.LIB


def selftest_wait(limit_s: float):
    """pot3d_selftest_wait: (device status code, elapsed seconds) of a bounded
    device wait on a barrier that nothing completes."""
    st, el = ctypes.c_int(0), ctypes.c_double(0.0)
    _check(load().pot3d_selftest_wait(float(limit_s), ctypes.byref(st), ctypes.byref(el)),
           "pot3d_selftest_wait")
    return st.value, el.value


def probe_fp64_fma(min_seconds: float = 0.5):
    """pot3d_probe_fp64_fma: (DFMA per second, timed device seconds)."""
    r, el = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().pot3d_probe_fp64_fma(float(min_seconds), ctypes.byref(r), ctypes.byref(el)),
           "pot3d_probe_fp64_fma")
    return r.value, el.value


ARITHS = {"fp64": 0, "df": 1, "f32": 2}


def _arith(a):
    return ARITHS[a] if isinstance(a, str) else int(a)


def variants(arith):
    """pot3d_variant_info for every matvec variant of an arithmetic:
    [{'tile_rows', 'tile_cols', 'stages', 'blocks_per_sm'}, ...]."""
    out = []
    L = load()
    while True:
        v = [ctypes.c_int(0) for _ in range(4)]
        if L.pot3d_variant_info(_arith(arith), len(out), *[ctypes.byref(x) for x in v]) != 0:
            return out
        out.append(dict(zip(("tile_rows", "tile_cols", "stages", "blocks_per_sm"),
                            (x.value for x in v))))


def load(build_if_missing: bool = False):
    """Loads libpot3d.so; raises if it is absent (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError("libpot3d.so is not built (%s); run __graft_entry__.build()"
                               % _build.LIB)
    L = ctypes.CDLL(_build.LIB)
    P, D, I, V = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p
    L.pot3d_plan.argtypes = [ctypes.POINTER(pot3d_grid_t), ctypes.POINTER(pot3d_bc_t)]
    L.pot3d_plan.restype = P
    L.pot3d_destroy.argtypes = [P]
    L.pot3d_destroy.restype = None
    L.pot3d_set_stream.argtypes = [P, V]
    L.pot3d_set_opts.argtypes = [P, ctypes.POINTER(pot3d_opts_t)]
    L.pot3d_get_info.argtypes = [P, ctypes.POINTER(pot3d_info_t)]
    L.pot3d_last_stats.argtypes = [P, ctypes.POINTER(pot3d_stats_t)]
    L.pot3d_autotune.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(I), D]
    L.pot3d_variant_info.argtypes = [I, I] + [ctypes.POINTER(I)] * 4
    L.pot3d_set_decomposition.argtypes = [P, I, I, I, I]
    L.pot3d_workspace_bytes.argtypes = [P]
    L.pot3d_workspace_bytes.restype = ctypes.c_size_t
    L.pot3d_set_workspace.argtypes = [P, V, ctypes.c_size_t]
    L.pot3d_solve.argtypes = [P, V, ctypes.c_double, V, ctypes.POINTER(I)]
    L.pot3d_solve_mixed.argtypes = [P, V, ctypes.c_double, V, ctypes.POINTER(I), ctypes.POINTER(I)]
    L.pot3d_field.argtypes = [P, V, V, V]
    L.pot3d_apply.argtypes = [P, V, V]
    L.pot3d_residual.argtypes = [P, V, V, D]
    L.pot3d_residual_noalloc.argtypes = [P, V, V, D]
    L.pot3d_batch_create.argtypes = [ctypes.c_size_t, I]
    L.pot3d_batch_create.restype = P
    L.pot3d_batch_destroy.argtypes = [P]
    L.pot3d_batch_destroy.restype = None
    L.pot3d_batch_set_stream.argtypes = [P, V]
    L.pot3d_batch_set_opts.argtypes = [P, ctypes.POINTER(pot3d_opts_t)]
    L.pot3d_batch_bytes_needed.argtypes = [P, P]
    L.pot3d_batch_bytes_needed.restype = ctypes.c_size_t
    L.pot3d_batch_submit.argtypes = [P, P, V, ctypes.c_double, V, ctypes.c_longlong]
    L.pot3d_batch_step.argtypes = [P, I]
    L.pot3d_batch_poll.argtypes = [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(I),
                                   ctypes.POINTER(I), ctypes.POINTER(I), D, I, ctypes.POINTER(I)]
    L.pot3d_batch_info.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_size_t),
                                   ctypes.POINTER(ctypes.c_size_t)]
    L.pot3d_selftest_wait.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_double)]
    L.pot3d_probe_fp64_fma.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
    L.pot3d_test_freeze_poll.argtypes = [P, I]
    L.pot3d_get_history.argtypes = [P, D, I, ctypes.POINTER(I)]
    L.pot3d_last_error.argtypes = []
    L.pot3d_strerror.argtypes = [I]
    L.pot3d_strerror.restype = ctypes.c_char_p
    _lib = L
    return L


class Pot3dError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = load().pot3d_strerror(code).decode()
        super().__init__("%s: %s (%d)" % (what, msg, code) if what else "%s (%d)" % (msg, code))


def _check(code: int, what: str):
    if code != POT3D_OK:
        raise Pot3dError(code, what)
    return code


def _ptr(a):
    """Device pointer of a torch tensor, host pointer of a numpy array."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "float64 C-contiguous required"
        return a.ctypes.data
    # torch tensor
    assert a.is_contiguous() and str(a.dtype) == "torch.float64", "float64 contiguous required"
    return a.data_ptr()


def _stream_of(*arrays):
    for a in arrays:
        if a is not None and not isinstance(a, np.ndarray) and a.is_cuda:
            import torch

            return torch.cuda.current_stream(a.device).cuda_stream
    return None


class Plan:
    """Owns a pot3d_plan_t.  Optional torch-allocated workspace: with
    ``torch_workspace=True`` the device workspace is a torch uint8 tensor
    (PyTorch's allocator) handed to pot3d_set_workspace."""

    def __init__(self, nr, nt, np_, r0=1.0, r1=2.5, ratio=1.0, precision="fp64", r_faces=None,
                 t_faces=None, torch_workspace=False, outer="source", **opts):
        L = load()
        self._rf = None if r_faces is None else np.ascontiguousarray(r_faces, dtype=np.float64)
        self._tf = None if t_faces is None else np.ascontiguousarray(t_faces, dtype=np.float64)
        g = pot3d_grid_t(int(nr), int(nt), int(np_), float(r0), float(r1), float(ratio),
                         None if self._rf is None else self._rf.ctypes.data_as(
                             ctypes.POINTER(ctypes.c_double)),
                         None if self._tf is None else self._tf.ctypes.data_as(
                             ctypes.POINTER(ctypes.c_double)),
                         PRECISIONS.get(precision, precision))
        bc = pot3d_bc_t(OUTER.get(outer, outer), POT3D_POLE_AVERAGE)
        h = L.pot3d_plan(ctypes.byref(g), ctypes.byref(bc))
        if not h:
            raise Pot3dError(L.pot3d_last_error(), "pot3d_plan")
        self.h = h
        self.nr, self.nt, self.np = int(nr), int(nt), int(np_)
        self.precision = precision
        self.outer = outer
        self._ws = None
        if opts:
            self.set_opts(**opts)
        if torch_workspace:
            import torch

            nbytes = L.pot3d_workspace_bytes(h)
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            aligned = (base + 255) // 256 * 256
            self._ws_offset = aligned - base  # workspace starts here in self._ws
            _check(L.pot3d_set_workspace(h, aligned, nbytes), "pot3d_set_workspace")

    @property
    def shape(self):
        return (self.nr, self.nt, self.np)

    def close(self):
        if getattr(self, "h", None):
            load().pot3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_opts(self, max_iters=0, use_x0=0, chunk=0, use_graphs=0, time_kernels=0,
                 inner_tol=0.0, max_outer=0, mixed_restart=0, verify=0, precond=0, history=0):
        """pot3d_set_opts; precond: a POT3D_PC_* value or its name ("jacobi",
        "philine", "rline", "lines")."""
        pc = PRECONDS.get(precond, precond)
        o = pot3d_opts_t(int(max_iters), int(use_x0), int(chunk), int(use_graphs), int(time_kernels),
                         float(inner_tol), int(max_outer), int(mixed_restart), int(verify),
                         int(pc), int(history))
        _check(load().pot3d_set_opts(self.h, ctypes.byref(o)), "pot3d_set_opts")

    def set_stream(self, stream_handle):
        _check(load().pot3d_set_stream(self.h, stream_handle), "pot3d_set_stream")

    def autotune(self, flags: int = 0):
        """pot3d_autotune: returns (variant, r-chunks, matvec ms) of the last
        arithmetic tuned."""
        v, c, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
        _check(load().pot3d_autotune(self.h, int(flags), ctypes.byref(v), ctypes.byref(c),
                                     ctypes.byref(ms)), "pot3d_autotune")
        return v.value, c.value, ms.value

    def set_decomposition(self, arith, variant, chunks=0, update_rows=0):
        """pot3d_set_decomposition: arith 'fp64' / 'df' / 'f32' (or 0 / 1 / 2)."""
        _check(load().pot3d_set_decomposition(self.h, _arith(arith), int(variant), int(chunks),
                                              int(update_rows)), "pot3d_set_decomposition")

    def info(self):
        i = pot3d_info_t()
        _check(load().pot3d_get_info(self.h, ctypes.byref(i)), "pot3d_get_info")
        return {f: getattr(i, f) for f, _ in pot3d_info_t._fields_}

    def stats(self):
        s = pot3d_stats_t()
        _check(load().pot3d_last_stats(self.h, ctypes.byref(s)), "pot3d_last_stats")
        return {"status": s.status, "iters": s.iters, "outer_iters": s.outer_iters,
                "relres": s.relres, "kernel_ms": list(s.kernel_ms), "launches": s.launches,
                "relres_fp64": s.relres_fp64, "flags": s.flags, "sigma": s.sigma, "rr": s.rr}

    def test_freeze_poll(self, on: bool):
        """pot3d_test_freeze_poll (testing hook of the host progress guard)."""
        _check(load().pot3d_test_freeze_poll(self.h, 1 if on else 0), "pot3d_test_freeze_poll")

    def _bind_stream(self, *arrays):
        st = _stream_of(*arrays)
        if st is not None:
            self.set_stream(st)

    def solve(self, br, tol, phi, check=True):
        """pot3d_solve: returns (status, iters)."""
        self._bind_stream(br, phi)
        it = ctypes.c_int(0)
        rc = load().pot3d_solve(self.h, _ptr(br), float(tol), _ptr(phi), ctypes.byref(it))
        if check and rc not in (POT3D_OK,):
            raise Pot3dError(rc, "pot3d_solve")
        return rc, it.value

    def solve_mixed(self, br, tol, phi, check=True):
        """pot3d_solve_mixed: returns (status, outer, inner)."""
        self._bind_stream(br, phi)
        o, i = ctypes.c_int(0), ctypes.c_int(0)
        rc = load().pot3d_solve_mixed(self.h, _ptr(br), float(tol), _ptr(phi), ctypes.byref(o),
                                      ctypes.byref(i))
        if check and rc != POT3D_OK:
            raise Pot3dError(rc, "pot3d_solve_mixed")
        return rc, o.value, i.value

    def field(self, phi, br, B):
        self._bind_stream(phi, br, B)
        _check(load().pot3d_field(self.h, _ptr(phi), _ptr(br), _ptr(B)), "pot3d_field")

    def apply(self, x, y):
        self._bind_stream(x, y)
        _check(load().pot3d_apply(self.h, _ptr(x), _ptr(y)), "pot3d_apply")

    def residual(self, br, phi):
        self._bind_stream(br, phi)
        r = ctypes.c_double(0.0)
        _check(load().pot3d_residual(self.h, _ptr(br), _ptr(phi), ctypes.byref(r)),
               "pot3d_residual")
        return r.value

    def residual_noalloc(self, br, phi, check=True):
        """pot3d_residual_noalloc: device arrays only; allocates nothing."""
        self._bind_stream(br, phi)
        r = ctypes.c_double(0.0)
        rc = load().pot3d_residual_noalloc(self.h, _ptr(br), _ptr(phi), ctypes.byref(r))
        if check:
            _check(rc, "pot3d_residual_noalloc")
            return r.value
        return rc, r.value

    def history(self):
        """pot3d_get_history: the residual history of the last solve run with
        history=1, as a numpy array (k = 0 .. iters)."""
        cap = 1 << 22
        buf = np.zeros(cap)
        n = ctypes.c_int(0)
        _check(load().pot3d_get_history(self.h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        cap, ctypes.byref(n)), "pot3d_get_history")
        return buf[: n.value].copy()

    def field_sizes(self):
        nr, nt, np_ = self.shape
        return ((nr + 1) * nt * np_, nr * (nt + 1) * np_, nr * nt * np_)


class Batch:
    """Owns a pot3d_batch_t (continuous batching of mixed-precision solves)."""

    def __init__(self, max_bytes: int, max_slots: int = 256, inner_tol=0.0, max_outer=0,
                 max_iters=0, mixed_restart=0, precond=0):
        L = load()
        h = L.pot3d_batch_create(int(max_bytes), int(max_slots))
        if not h:
            raise Pot3dError(L.pot3d_last_error(), "pot3d_batch_create")
        self.h = h
        self.max_slots = int(max_slots)
        o = pot3d_opts_t(int(max_iters), 0, 0, 0, 0, float(inner_tol), int(max_outer),
                         int(mixed_restart), 0, int(PRECONDS.get(precond, precond)), 0)
        rc = L.pot3d_batch_set_opts(h, ctypes.byref(o))
        if rc != POT3D_OK:
            L.pot3d_batch_destroy(h)
            self.h = None
            raise Pot3dError(rc, "pot3d_batch_set_opts")

    def close(self):
        if getattr(self, "h", None):
            load().pot3d_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle):
        _check(load().pot3d_batch_set_stream(self.h, stream_handle), "pot3d_batch_set_stream")

    def bytes_needed(self, plan: "Plan") -> int:
        return int(load().pot3d_batch_bytes_needed(self.h, plan.h))

    def submit(self, plan: "Plan", br, tol, phi, tag: int) -> bool:
        """True if admitted, False if busy (no slot or memory)."""
        rc = load().pot3d_batch_submit(self.h, plan.h, _ptr(br), float(tol), _ptr(phi), int(tag))
        if rc == POT3D_ERR_BUSY:
            return False
        _check(rc, "pot3d_batch_submit")
        return True

    def step(self, k: int) -> int:
        rc = load().pot3d_batch_step(self.h, int(k))
        if rc < 0:
            raise Pot3dError(rc, "pot3d_batch_step")
        return rc

    def poll(self, max_n: int = 1024):
        """List of (tag, status, outer, inner, relres) of retired solves."""
        n = max(1, min(max_n, self.max_slots))
        tags = (ctypes.c_longlong * n)()
        st, o, i = (ctypes.c_int * n)(), (ctypes.c_int * n)(), (ctypes.c_int * n)()
        rr = (ctypes.c_double * n)()
        nd = ctypes.c_int(0)
        _check(load().pot3d_batch_poll(self.h, tags, st, o, i, rr, n, ctypes.byref(nd)),
               "pot3d_batch_poll")
        return [(tags[u], st[u], o[u], i[u], rr[u]) for u in range(nd.value)]

    def info(self):
        a, u, c = ctypes.c_int(0), ctypes.c_size_t(0), ctypes.c_size_t(0)
        _check(load().pot3d_batch_info(self.h, ctypes.byref(a), ctypes.byref(u), ctypes.byref(c)),
               "pot3d_batch_info")
        return {"active": a.value, "bytes_used": u.value, "bytes_cap": c.value}


# C-named entry points (argument marshalling only)
def pot3d_plan(nr, nt, np_, **kw) -> Plan:
    return Plan(nr, nt, np_, **kw)


def pot3d_solve(plan: Plan, br, tol, phi):
    return plan.solve(br, tol, phi)


def pot3d_solve_mixed(plan: Plan, br, tol, phi):
    return plan.solve_mixed(br, tol, phi)


def pot3d_field(plan: Plan, phi, br, B):
    return plan.field(phi, br, B)


def pot3d_apply(plan: Plan, x, y):
    return plan.apply(x, y)


def pot3d_residual(plan: Plan, br, phi):
    return plan.residual(br, phi)


def pot3d_destroy(plan: Plan):
    plan.close()
