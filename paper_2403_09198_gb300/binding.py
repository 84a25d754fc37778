"""ctypes binding of ``libsts.so`` (C ABI in ``include/sts.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch supplies device memory and the current stream.  There is no
CPU fallback: if the library is not built, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsts.so")

STS_OK = 0
STATUS_NAMES = {0: "STS_OK", 1: "STS_ERR_INVALID_ARG", 2: "STS_ERR_ALLOC", 3: "STS_ERR_CUDA",
                4: "STS_ERR_SINGULAR", 5: "STS_ERR_NOT_CONVERGED", 6: "STS_ERR_NUMERIC",
                7: "STS_ERR_TIMEOUT", 8: "STS_ERR_NOT_SETUP", 9: "STS_ERR_COMM"}
STS_F64, STS_MIXED = 0, 2
STS_LAYOUT_CELL_MAJOR, STS_LAYOUT_COMPONENT_MAJOR = 0, 1
STS_REP_FACTORED, STS_REP_DENSE_BSR = 0, 1
STS_PRECOND_BJ, STS_PRECOND_NONE = 0, 1

# Every entry point declared in include/sts.h.
ABI_FUNCTIONS = ["sts_last_error", "sts_version", "sts_jac_create", "sts_jac_update_values",
                 "sts_jac_matvec", "sts_jac_matvec_noalloc", "sts_jac_matvec_f32", "sts_jac_bjacobi_setup",
                 "sts_jac_bjacobi_apply", "sts_jac_bjacobi_apply_f32", "sts_gmres_solve",
                 "sts_jac_grad", "sts_jac_memory", "sts_launch_count", "sts_selftest_bounded_wait",
                 "sts_jac_destroy", "sts_flow_create", "sts_flow_get_sizes", "sts_flow_get_layout",
                 "sts_flow_residual", "sts_flow_jacobian", "sts_flow_newton", "sts_flow_destroy",
                 "sts_dd_plan_create", "sts_dd_plan_sizes", "sts_dd_plan_get", "sts_dd_plan_value_sizes",
                 "sts_dd_plan_gather", "sts_dd_plan_destroy", "sts_dd_create", "sts_dd_matvec",
                 "sts_dd_bjacobi_apply", "sts_dd_gmres_solve", "sts_dd_destroy", "sts_dd_gmres_ops"]


class sts_jac_desc(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int), ("block_size", ctypes.c_int),
                ("n_levels", ctypes.c_int), ("dtype", ctypes.c_int), ("vec_layout", ctypes.c_int),
                ("representation", ctypes.c_int),
                ("block_indptr", ctypes.c_void_p), ("block_indices", ctypes.c_void_p),
                ("d_indptr", ctypes.c_void_p), ("d_indices", ctypes.c_void_p),
                ("o_indptr", ctypes.c_void_p), ("o_indices", ctypes.c_void_p),
                ("r_diag", ctypes.c_int), ("r_off", ctypes.c_int), ("pair_indptr", ctypes.c_void_p),
                ("S", ctypes.c_void_p), ("U", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("values_on_host", ctypes.c_int), ("enable_transpose", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class sts_flow_desc(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("n_species", ctypes.c_int), ("band", ctypes.c_int),
                ("r", ctypes.c_void_p), ("cv", ctypes.c_void_p), ("e0", ctypes.c_void_p),
                ("beta", ctypes.c_void_p), ("ws", ctypes.c_void_p), ("K", ctypes.c_void_p),
                ("A", ctypes.c_double), ("theta", ctypes.c_double), ("dt", ctypes.c_double),
                ("stream", ctypes.c_void_p)]


class sts_flow_sizes(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int), ("block_size", ctypes.c_int), ("nnzb", ctypes.c_int),
                ("nnz_d", ctypes.c_int), ("nnz_o", ctypes.c_int), ("n_pairs", ctypes.c_int),
                ("nnz_S", ctypes.c_longlong)]


class sts_gmres_opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_iters", ctypes.c_int), ("rtol", ctypes.c_double),
                ("precond", ctypes.c_int), ("flexible", ctypes.c_int), ("trans", ctypes.c_int),
                ("mixed", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("vectors_on_host", ctypes.c_int), ("history", ctypes.c_void_p), ("left", ctypes.c_int),
                ("arnoldi", ctypes.c_int)]


class sts_newton_opts(ctypes.Structure):
    _fields_ = [("max_newton", ctypes.c_int), ("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("max_halvings", ctypes.c_int), ("gmres", sts_gmres_opts), ("history", ctypes.c_void_p),
                ("forcing", ctypes.c_int)]


class sts_newton_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("linear_iterations", ctypes.c_int), ("halvings", ctypes.c_int),
                ("converged", ctypes.c_int), ("res0", ctypes.c_double), ("res", ctypes.c_double)]


class sts_gmres_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("converged", ctypes.c_int), ("true_rel_residual", ctypes.c_double),
                ("matvecs", ctypes.c_int), ("applies", ctypes.c_int)]


class sts_dd_sizes(ctypes.Structure):
    _fields_ = [("n_owned", ctypes.c_int), ("n_ghost", ctypes.c_int), ("n_local", ctypes.c_int),
                ("nnzb", ctypes.c_int), ("n_neighbors", ctypes.c_int), ("n_send", ctypes.c_int),
                ("n_recv", ctypes.c_int)]


_IP = ctypes.POINTER(ctypes.c_int)
_DPP = ctypes.POINTER(ctypes.c_void_p)
DD_EXCHANGE = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, _IP, _IP, _DPP, _IP, ctypes.c_int,
                               _IP, _IP, _DPP, _IP, ctypes.c_void_p)
DD_ALLREDUCE = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int)


class sts_dd_comm(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("exchange", DD_EXCHANGE), ("allreduce", DD_ALLREDUCE)]


class sts_dd_desc(ctypes.Structure):
    _fields_ = [("n_parts", ctypes.c_int), ("part_ids", ctypes.c_void_p), ("jac", ctypes.c_void_p),
                ("plans", ctypes.c_void_p), ("comm", ctypes.POINTER(sts_dd_comm))]


_I, _V, _D = ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
DD_OPS_FIELDS = [("matvec", ctypes.CFUNCTYPE(_I, _V, _I, _I)), ("apply", ctypes.CFUNCTYPE(_I, _V, _I, _I)),
                 ("copy", ctypes.CFUNCTYPE(_I, _V, _I, _I)), ("sub", ctypes.CFUNCTYPE(_I, _V, _I, _I, _I)),
                 ("scale", ctypes.CFUNCTYPE(_I, _V, _I, _I, ctypes.c_double)),
                 ("dots", ctypes.CFUNCTYPE(_I, _V, _I, _I, _I, _I, _D)),
                 ("update", ctypes.CFUNCTYPE(_I, _V, _I, _I, _I, _D, _I, _D)),
                 ("norm2", ctypes.CFUNCTYPE(_I, _V, _I, _D)),
                 ("axpy", ctypes.CFUNCTYPE(_I, _V, _I, _I, _I, _D)),
                 ("allreduce", ctypes.CFUNCTYPE(_I, _V, _D, _I))]


class sts_dd_ops(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p)] + DD_OPS_FIELDS


class StsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"{path} is missing: build it with paper_2403_09198_gb300.build.build()")
            lib = ctypes.CDLL(path)
            P, I = ctypes.c_void_p, ctypes.c_int
            lib.sts_last_error.restype = ctypes.c_char_p
            lib.sts_last_error.argtypes = []
            lib.sts_version.restype = ctypes.c_char_p
            lib.sts_version.argtypes = []
            sig = {
                "sts_jac_create": [ctypes.POINTER(sts_jac_desc), ctypes.POINTER(P)],
                "sts_jac_update_values": [P, P, P, P, I],
                "sts_jac_matvec": [P, P, P, I],
                "sts_jac_matvec_noalloc": [P, P, P, I],
                "sts_jac_matvec_f32": [P, P, P, I],
                "sts_jac_bjacobi_setup": [P],
                "sts_jac_bjacobi_apply": [P, P, P, I],
                "sts_jac_bjacobi_apply_f32": [P, P, P, I],
                "sts_gmres_solve": [P, P, P, ctypes.POINTER(sts_gmres_opts),
                                    ctypes.POINTER(sts_gmres_info)],
                "sts_jac_grad": [P, P, P, P, P, P],
                "sts_jac_memory": [P, ctypes.POINTER(ctypes.c_size_t)],
                "sts_launch_count": [ctypes.POINTER(ctypes.c_ulonglong)],
                "sts_selftest_bounded_wait": [P],
                "sts_jac_destroy": [P],
                "sts_flow_create": [ctypes.POINTER(sts_flow_desc), ctypes.POINTER(P)],
                "sts_flow_get_sizes": [P, ctypes.POINTER(sts_flow_sizes)],
                "sts_flow_get_layout": [P, P, P, P, P, P, P, P],
                "sts_flow_residual": [P, P, P, P],
                "sts_flow_jacobian": [P, P, P, P, P],
                "sts_flow_newton": [P, P, P, P, ctypes.POINTER(sts_newton_opts), ctypes.POINTER(sts_newton_info)],
                "sts_flow_destroy": [P],
                "sts_dd_plan_create": [I, P, P, I, P, I, ctypes.POINTER(P)],
                "sts_dd_plan_sizes": [P, ctypes.POINTER(sts_dd_sizes)],
                "sts_dd_plan_get": [P, P, P, P, P, P, P, P, P, P],
                "sts_dd_plan_value_sizes": [P, I, I, P, I, I, ctypes.POINTER(ctypes.c_longlong),
                                            ctypes.POINTER(ctypes.c_int), P],
                "sts_dd_plan_gather": [P, I, I, I, P, I, I, P, P, P, P, P, P, I, P],
                "sts_dd_plan_destroy": [P],
                "sts_dd_create": [ctypes.POINTER(sts_dd_desc), ctypes.POINTER(P)],
                "sts_dd_matvec": [P, P, P, I],
                "sts_dd_bjacobi_apply": [P, P, P, I],
                "sts_dd_gmres_solve": [P, P, P, ctypes.POINTER(sts_gmres_opts), ctypes.POINTER(sts_gmres_info)],
                "sts_dd_destroy": [P],
                "sts_dd_gmres_ops": [ctypes.POINTER(sts_dd_ops), ctypes.POINTER(sts_gmres_opts),
                                     ctypes.POINTER(sts_gmres_info)],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = I
            _lib = lib
    return _lib


def check(status: int, allow=()) -> int:
    if status != STS_OK and status not in allow:
        raise StsError(status, load().sts_last_error().decode(errors="replace"))
    return status


def launch_count() -> int:
    """Kernels launched by the CUDA library since it was loaded."""
    n = ctypes.c_ulonglong()
    check(load().sts_launch_count(ctypes.byref(n)))
    return int(n.value)


def _ptr(t) -> int:
    """Device pointer of a torch tensor or host pointer of a numpy array."""
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_ptr(stream) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


@dataclass
class GmresInfo:
    iterations: int
    restarts: int
    converged: bool
    true_rel_residual: float
    history: np.ndarray | None = None
    matvecs: int = 0          # FP64 J x products the solve made
    applies: int = 0          # FP64 block-Jacobi applies the solve made


def gmres_info(info, hist=None) -> GmresInfo:
    """GmresInfo from an sts_gmres_info (history cut to the iterations taken)."""
    return GmresInfo(info.iterations, info.restarts, bool(info.converged), info.true_rel_residual,
                     hist[:info.iterations].copy() if hist is not None else None, info.matvecs, info.applies)


class StsJacobian:
    """Owner of one ``sts_jac_t`` handle.

    ``w`` is any object exposing the public layout arrays (``block_indptr``,
    ``block_indices``, ``d_indptr``, ``d_indices``, ``o_indptr``, ``o_indices``,
    ``r_diag``, ``r_off``, ``b``, and optionally ``pair_indptr`` for per-block pair
    counts); ``S``, ``U``, ``V`` are FP64 torch CUDA tensors or numpy arrays
    (host), in the public layout.
    """

    def __init__(self, w, S, U, V, *, mixed: bool = False, layout: str = "cell",
                 dense: bool = False, transpose: bool = False, stream=None, n_levels: int = 0):
        import torch
        self.lib = load()
        self.b = int(w.b)
        self.n_cells = int(np.asarray(w.block_indptr).shape[0] - 1)
        self.layout = layout
        self._idx = [np.ascontiguousarray(a, dtype=np.int32) for a in
                     (w.block_indptr, w.block_indices, w.d_indptr, w.d_indices, w.o_indptr,
                      w.o_indices)]
        pip = getattr(w, "pair_indptr", None)
        self._pip = None if pip is None else np.ascontiguousarray(pip, dtype=np.int32)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        on_host = isinstance(S, np.ndarray)
        if on_host:
            S, U, V = (np.ascontiguousarray(a, dtype=np.float64) for a in (S, U, V))
        else:
            for a in (S, U, V):
                if a.dtype != torch.float64 or not a.is_cuda or not a.is_contiguous():
                    raise ValueError("S, U, V must be contiguous float64 CUDA tensors or numpy arrays")
        d = sts_jac_desc()
        d.n_cells = self.n_cells
        d.block_size = self.b
        d.n_levels = int(n_levels or getattr(w, "N", 0))
        d.dtype = STS_MIXED if mixed else STS_F64
        d.vec_layout = STS_LAYOUT_CELL_MAJOR if layout == "cell" else STS_LAYOUT_COMPONENT_MAJOR
        d.representation = STS_REP_DENSE_BSR if dense else STS_REP_FACTORED
        (d.block_indptr, d.block_indices, d.d_indptr, d.d_indices, d.o_indptr,
         d.o_indices) = [a.ctypes.data for a in self._idx]
        d.r_diag = int(w.r_diag)
        d.r_off = int(w.r_off)
        d.pair_indptr = None if self._pip is None else self._pip.ctypes.data
        d.S, d.U, d.V = _ptr(S), _ptr(U), _ptr(V)
        d.values_on_host = 1 if on_host else 0
        d.enable_transpose = 1 if transpose else 0
        d.stream = self.stream.cuda_stream
        h = ctypes.c_void_p()
        check(self.lib.sts_jac_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        # bumped whenever the handle's values change (update_values, a Newton step)
        self.values_version = 0
        self.mixed = mixed
        self.n = self.n_cells * self.b
        # sizes of the public value arrays (index bookkeeping only)
        bptr, bidx = self._idx[0], self._idx[1]
        rows = np.repeat(np.arange(self.n_cells), np.diff(bptr))
        n_diag = int(np.sum(rows == bidx))
        n_off = int(bidx.shape[0]) - n_diag
        self.nnz_S = n_diag * int(self._idx[2][-1]) + n_off * int(self._idx[4][-1])
        self.n_pairs = (int(self._pip[-1]) if self._pip is not None
                        else n_diag * int(w.r_diag) + n_off * int(w.r_off))

    # -- lifetime
    def close(self):
        if getattr(self, "h", None):
            self.lib.sts_jac_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls
    def update_values(self, S, U, V):
        on_host = isinstance(S, np.ndarray)
        if on_host:
            S, U, V = (np.ascontiguousarray(a, dtype=np.float64) for a in (S, U, V))
        self.values_version += 1
        check(self.lib.sts_jac_update_values(self.h, _ptr(S), _ptr(U), _ptr(V), int(on_host)))
        if on_host:
            self.stream.synchronize()   # host arrays must outlive the copies

    def matvec(self, x, out=None, trans: bool = False):
        import torch
        y = torch.empty_like(x) if out is None else out
        if x.dtype == torch.float32:
            check(self.lib.sts_jac_matvec_f32(self.h, _ptr(x), _ptr(y), int(trans)))
        else:
            check(self.lib.sts_jac_matvec(self.h, _ptr(x), _ptr(y), int(trans)))
        return y

    def bjacobi_setup(self):
        check(self.lib.sts_jac_bjacobi_setup(self.h))

    def bjacobi_apply(self, x, out=None, trans: bool = False):
        import torch
        z = torch.empty_like(x) if out is None else out
        if x.dtype == torch.float32:
            check(self.lib.sts_jac_bjacobi_apply_f32(self.h, _ptr(x), _ptr(z), int(trans)))
        else:
            check(self.lib.sts_jac_bjacobi_apply(self.h, _ptr(x), _ptr(z), int(trans)))
        return z

    def gmres(self, b, x0=None, *, restart: int = 30, rtol: float = 1e-10, max_iters: int = 1000,
              precond: str = "bj", trans: bool = False, mixed: bool = False,
              inner_rtol: float = 0.0, history: bool = False, raise_on_fail: bool = True,
              left: bool = False, graph: bool = True):
        """Solve J x = b (J^T x = b).  ``b``: CUDA tensor or numpy array (host).
        ``graph=False`` rotates on the host after every Arnoldi step instead of
        running each cycle as one CUDA graph."""
        import torch
        on_host = isinstance(b, np.ndarray)
        if on_host:
            b = np.ascontiguousarray(b, dtype=np.float64)
            x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        else:
            x = torch.zeros_like(b) if x0 is None else x0.clone()
        o = sts_gmres_opts()
        o.restart, o.max_iters, o.rtol = restart, max_iters, rtol
        o.precond = STS_PRECOND_BJ if precond == "bj" else STS_PRECOND_NONE
        o.trans, o.mixed, o.inner_rtol, o.left = int(trans), int(mixed), inner_rtol, int(left)
        o.arnoldi = 0 if graph else 1       # STS_ARNOLDI_GRAPH / STS_ARNOLDI_HOST
        o.vectors_on_host = int(on_host)
        hist = np.zeros(max_iters) if history else None
        o.history = hist.ctypes.data if history else None
        info = sts_gmres_info()
        st = self.lib.sts_gmres_solve(self.h, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(info))
        if raise_on_fail:
            check(st)
        return x, gmres_info(info, hist if history else None)

    def grad(self, lam, x):
        """Adjoint outer products (gS, gU, gV) in the public S / U / V layouts."""
        import torch
        gS = torch.empty(self.nnz_S, dtype=torch.float64, device=lam.device)
        gU = torch.empty((self.n_pairs, self.b), dtype=torch.float64, device=lam.device)
        gV = torch.empty_like(gU)
        check(self.lib.sts_jac_grad(self.h, _ptr(lam), _ptr(x), _ptr(gS), _ptr(gU), _ptr(gV)))
        return gS, gU, gV

    def memory_bytes(self) -> int:
        n = ctypes.c_size_t()
        check(self.lib.sts_jac_memory(self.h, ctypes.byref(n)))
        return int(n.value)


@dataclass
class FlowLayout:
    """BR1-BSR layout of the flow Jacobian, accepted by ``StsJacobian`` as it is."""
    N: int
    b: int
    r_diag: int
    r_off: int
    block_indptr: np.ndarray
    block_indices: np.ndarray
    d_indptr: np.ndarray
    d_indices: np.ndarray
    o_indptr: np.ndarray
    o_indices: np.ndarray
    pair_indptr: np.ndarray
    nnz_S: int

    @property
    def n_pairs(self) -> int:
        return int(self.pair_indptr[-1])


class StsFlow:
    """Owner of one ``sts_flow_t``: residual and r1-sparse Jacobian of the toy
    HLL-flux model for the constants and grid of ``case`` (an
    ``inputs.FlowCase``, or any object with the same fields)."""

    def __init__(self, case, stream=None):
        import torch
        self.lib = load()
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self._c = [np.ascontiguousarray(a, dtype=np.float64) for a in
                   (case.r, case.cv, case.e0, case.beta, case.ws, case.K)]
        d = sts_flow_desc()
        d.Lx, d.Ly, d.n_species, d.band = int(case.Lx), int(case.Ly), int(case.N), int(case.w)
        d.r, d.cv, d.e0, d.beta, d.ws, d.K = [a.ctypes.data for a in self._c]
        d.A, d.theta, d.dt = float(case.A), float(case.theta), float(case.dt)
        d.stream = self.stream.cuda_stream
        h = ctypes.c_void_p()
        check(self.lib.sts_flow_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        z = sts_flow_sizes()
        check(self.lib.sts_flow_get_sizes(self.h, ctypes.byref(z)))
        self.sizes = z
        nc, b = z.n_cells, z.block_size
        arrs = [np.zeros(n, dtype=np.int32) for n in (nc + 1, z.nnzb, b + 1, z.nnz_d, b + 1, z.nnz_o, z.nnzb + 1)]
        check(self.lib.sts_flow_get_layout(self.h, *[a.ctypes.data for a in arrs]))
        counts = np.diff(arrs[6])
        rows = np.repeat(np.arange(nc), np.diff(arrs[0]))
        diag = rows == arrs[1]
        self.layout = FlowLayout(N=int(case.N), b=b, r_diag=int(counts[diag].max(initial=0)),
                                 r_off=int(counts[~diag].max(initial=0)), block_indptr=arrs[0],
                                 block_indices=arrs[1], d_indptr=arrs[2], d_indices=arrs[3],
                                 o_indptr=arrs[4], o_indices=arrs[5], pair_indptr=arrs[6],
                                 nnz_S=int(z.nnz_S))

    def close(self):
        if getattr(self, "h", None):
            self.lib.sts_flow_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _states(self, *ts):
        import torch
        n = self.sizes.n_cells * self.sizes.block_size
        for t in ts:
            if (not torch.is_tensor(t) or t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous()
                    or t.numel() != n):
                raise ValueError(f"states must be contiguous float64 CUDA tensors of {n} values")

    def residual(self, Q, Qn, out=None):
        """R(Q) given the previous level Qn; CUDA float64 tensors [n_cells, b]."""
        import torch
        self._states(Q, Qn)
        R = torch.empty_like(Q) if out is None else out
        self._states(R)
        check(self.lib.sts_flow_residual(self.h, _ptr(Q), _ptr(Qn), _ptr(R)))
        return R

    def jacobian(self, Q, S=None, U=None, V=None):
        """(S, U, V) of dR/dQ at Q in ``self.layout``; CUDA float64 tensors."""
        import torch
        self._states(Q)
        z, dev = self.sizes, Q.device
        S = torch.empty(z.nnz_S, dtype=torch.float64, device=dev) if S is None else S
        U = torch.empty((z.n_pairs, z.block_size), dtype=torch.float64, device=dev) if U is None else U
        V = torch.empty_like(U) if V is None else V
        check(self.lib.sts_flow_jacobian(self.h, _ptr(Q), _ptr(S), _ptr(U), _ptr(V)))
        return S, U, V

    def jacobian_handle(self, **kw):
        """A cell-major ``StsJacobian`` of this layout for ``newton`` (``dense=True``
        for the dense-BSR storage), holding the flow Jacobian at the states
        ``Q=...`` if given, else zeros (``newton`` writes its own values)."""
        import torch
        Q = kw.pop("Q", None)
        if Q is None:
            z = self.sizes
            S = torch.zeros(z.nnz_S, dtype=torch.float64, device="cuda")
            U = torch.zeros((z.n_pairs, z.block_size), dtype=torch.float64, device="cuda")
            V = torch.zeros_like(U)
        else:
            S, U, V = self.jacobian(Q)
        return StsJacobian(self.layout, S, U, V, layout="cell", n_levels=self.layout.N, **kw)

    def newton(self, jac, Q, Qn, *, max_newton: int = 20, rtol: float = 1e-10, atol: float = 0.0,
               max_halvings: int = 8, gmres_rtol: float = 1e-10, restart: int = 30, gmres_max_iters: int = 1000,
               precond: str = "bj", left: bool = False, forcing: bool = False, raise_on_fail: bool = True,
               graph: bool = True):
        """One pseudo-time step by Newton's method; Q (CUDA [n_cells, b]) is updated
        in place.  Returns (info dict, history of ||R||)."""
        self._states(Q, Qn)
        o = sts_newton_opts()
        o.max_newton, o.rtol, o.atol, o.max_halvings = max_newton, rtol, atol, max_halvings
        o.gmres.restart, o.gmres.max_iters, o.gmres.rtol = restart, gmres_max_iters, gmres_rtol
        o.gmres.precond = STS_PRECOND_BJ if precond == "bj" else STS_PRECOND_NONE
        o.gmres.left = int(left)
        o.gmres.arnoldi = 0 if graph else 1
        o.forcing = int(forcing)
        hist = np.zeros(max_newton + 1)
        o.history = hist.ctypes.data
        info = sts_newton_info()
        jac.values_version += 1          # the step writes its own Jacobians into jac
        st = self.lib.sts_flow_newton(self.h, jac.h, _ptr(Q), _ptr(Qn), ctypes.byref(o), ctypes.byref(info))
        if raise_on_fail:
            check(st)
        d = dict(iterations=info.iterations, linear_iterations=info.linear_iterations, halvings=info.halvings,
                 converged=bool(info.converged), res0=info.res0, res=info.res, status=st)
        return d, hist[:info.iterations + 1].copy()
