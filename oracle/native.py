"""ctypes front end of ``oracle.c`` (test infrastructure only).

``build()`` compiles ``oracle.c`` with gcc into ``liboracle.so`` next to it; the
library is loaded on first use.  All arrays are checked for dtype and
contiguity before their pointers are passed.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP, no FP contraction) and return its path."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            common = [I, I, P, P, P, P, P, P, P]
            lib.orc_matvec.argtypes = common + [P, P, P, P, P, I]
            lib.orc_matvec.restype = None
            lib.orc_matvec_rows.argtypes = common + [P, P, P, P, I, I, P, P]
            lib.orc_matvec_rows.restype = None
            lib.orc_bj_setup.argtypes = common + [P, P, P, P, P]
            lib.orc_bj_setup.restype = I
            lib.orc_bj_apply.argtypes = [I, I, P, P, P, P, I]
            lib.orc_bj_apply.restype = None
            lib.orc_bj_cells.argtypes = common + [P, P, P, P, I, I, P, P]
            lib.orc_bj_cells.restype = I
            lib.orc_grad.argtypes = common + [P, P, P, P, P, P, P]
            lib.orc_grad.restype = None
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = I
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().orc_max_threads())


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleSingular(RuntimeError):
    """A diagonal block has a zero pivot under partial pivoting."""

    def __init__(self, cell: int):
        super().__init__(f"diagonal block of cell {cell} is singular")
        self.cell = cell


@dataclasses.dataclass
class Jacobian:
    """Block r1-sparse Jacobian in the public BR1-BSR layout (Section 5.1)."""

    n_cells: int
    b: int
    block_indptr: np.ndarray
    block_indices: np.ndarray
    d_indptr: np.ndarray
    d_indices: np.ndarray
    o_indptr: np.ndarray
    o_indices: np.ndarray
    pair_indptr: np.ndarray
    S: np.ndarray
    U: np.ndarray
    V: np.ndarray

    def __post_init__(self):
        self.block_indptr = _i32(self.block_indptr)
        self.block_indices = _i32(self.block_indices)
        self.d_indptr = _i32(self.d_indptr)
        self.d_indices = _i32(self.d_indices)
        self.o_indptr = _i32(self.o_indptr)
        self.o_indices = _i32(self.o_indices)
        self.pair_indptr = _i32(self.pair_indptr)
        self.S = _f64(self.S).ravel()
        self.U = _f64(self.U).reshape(-1)
        self.V = _f64(self.V).reshape(-1)
        if self.block_indptr.shape[0] != self.n_cells + 1:
            raise ValueError("block_indptr must have n_cells + 1 entries")
        if self.d_indptr.shape[0] != self.b + 1 or self.o_indptr.shape[0] != self.b + 1:
            raise ValueError("pattern indptr arrays must have b + 1 entries")

    @classmethod
    def from_workload(cls, w, S=None, U=None, V=None) -> "Jacobian":
        """Read the arrays of any object exposing the public layout attributes."""
        return cls(n_cells=int(w.block_indptr.shape[0] - 1), b=int(w.b),
                   block_indptr=w.block_indptr, block_indices=w.block_indices,
                   d_indptr=w.d_indptr, d_indices=w.d_indices,
                   o_indptr=w.o_indptr, o_indices=w.o_indices,
                   pair_indptr=w.pair_indptr,
                   S=w.S if S is None else S, U=w.U if U is None else U,
                   V=w.V if V is None else V)

    @property
    def n(self) -> int:
        return self.n_cells * self.b

    def _common(self):
        return (self.n_cells, self.b, _p(self.block_indptr), _p(self.block_indices),
                _p(self.d_indptr), _p(self.d_indices), _p(self.o_indptr), _p(self.o_indices),
                _p(self.pair_indptr))


def matvec(J: Jacobian, x, trans: bool = False) -> np.ndarray:
    """y = D x (or D^T x) with every block assembled densely."""
    x = _f64(x).ravel()
    if x.shape[0] != J.n:
        raise ValueError("x has the wrong length")
    y = np.empty(J.n, dtype=np.float64)
    _load().orc_matvec(*J._common(), _p(J.S), _p(J.U), _p(J.V), _p(x), _p(y), int(bool(trans)))
    return y


def matvec_rows(J: Jacobian, x, rows, trans: bool = False) -> np.ndarray:
    """Selected entries y[rows] of D x (or D^T x); rows are global indices cell*b + p."""
    x = _f64(x).ravel()
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(rows.shape[0], dtype=np.float64)
    _load().orc_matvec_rows(*J._common(), _p(J.S), _p(J.U), _p(J.V), _p(x), int(bool(trans)),
                            int(rows.shape[0]), _p(rows), _p(out))
    return out


@dataclasses.dataclass
class BJFactors:
    """Per-cell LU factors of the diagonal blocks (partial pivoting)."""

    n_cells: int
    b: int
    LU: np.ndarray
    piv: np.ndarray


def bj_setup(J: Jacobian) -> BJFactors:
    LU = np.empty(J.n_cells * J.b * J.b, dtype=np.float64)
    piv = np.empty(J.n_cells * J.b, dtype=np.int32)
    rc = _load().orc_bj_setup(*J._common(), _p(J.S), _p(J.U), _p(J.V), _p(LU), _p(piv))
    if rc < 0:
        raise OracleSingular(-rc - 1)
    return BJFactors(J.n_cells, J.b, LU, piv)


def bj_apply(F: BJFactors, x, trans: bool = False) -> np.ndarray:
    """z_i = D_ii^-1 x_i (or D_ii^-T x_i) for every cell."""
    x = _f64(x).ravel()
    z = np.empty_like(x)
    _load().orc_bj_apply(F.n_cells, F.b, _p(F.LU), _p(F.piv), _p(x), _p(z), int(bool(trans)))
    return z


def bj_cells(J: Jacobian, x, cells, trans: bool = False) -> np.ndarray:
    """Block-Jacobi output of the listed cells only: array [len(cells), b]."""
    x = _f64(x).ravel()
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    out = np.empty((cells.shape[0], J.b), dtype=np.float64)
    rc = _load().orc_bj_cells(*J._common(), _p(J.S), _p(J.U), _p(J.V), _p(x), int(bool(trans)),
                              int(cells.shape[0]), _p(cells), _p(out))
    if rc < 0:
        raise OracleSingular(int(cells[-rc - 1]))
    return out


def grad(J: Jacobian, lam, x):
    """Adjoint outer products (gS, gU, gV) in the public layout for cotangent lambda."""
    lam = _f64(lam).ravel()
    x = _f64(x).ravel()
    gS = np.empty_like(J.S)
    gU = np.empty_like(J.U)
    gV = np.empty_like(J.V)
    _load().orc_grad(*J._common(), _p(J.U), _p(J.V), _p(lam), _p(x), _p(gS), _p(gU), _p(gV))
    return gS, gU.reshape(-1, J.b), gV.reshape(-1, J.b)
