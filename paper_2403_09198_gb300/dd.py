"""Domain decomposition through the C ABI (``sts_dd_*`` in ``include/sts.h``).

Argument marshalling only: the partition plan, the halo exchange kernels and
the GMRES driver are in the CUDA library.  This module wraps them, builds the
local layout a sub-domain handle is created from, and offers a communicator
over ``torch.distributed`` for parts held by other processes (NCCL for device
buffers, gloo for host buffers).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from .binding import (DD_ALLREDUCE, DD_EXCHANGE, DD_OPS_FIELDS, STS_PRECOND_BJ, STS_PRECOND_NONE,
                      StsJacobian, _ptr, check, gmres_info, load, sts_dd_comm, sts_dd_desc, sts_dd_ops,
                      sts_dd_sizes, sts_gmres_info, sts_gmres_opts)


def grid_partition(Lx: int, Ly: int, px: int, py: int) -> np.ndarray:
    """Part of every cell (id iy*Lx + ix) of an Lx x Ly grid cut into px x py
    rectangular tiles of near-equal size, numbered row by row."""
    ix = np.arange(Lx) * px // Lx
    iy = np.arange(Ly) * py // Ly
    return (iy[:, None] * px + ix[None, :]).ravel().astype(np.int32)


@dataclass
class LocalLayout:
    """BR1-BSR layout of one sub-domain, accepted by ``StsJacobian`` as it is."""
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
    def n_cells(self) -> int:
        return int(self.block_indptr.shape[0] - 1)

    @property
    def n(self) -> int:
        return self.n_cells * self.b

    @property
    def n_pairs(self) -> int:
        return int(self.pair_indptr[-1])


class DdPlan:
    """Owner of one ``sts_dd_plan_t``: part ``part`` of the partition
    ``part_of_cell`` of the block CSR (``block_indptr``, ``block_indices``)."""

    def __init__(self, block_indptr, block_indices, part_of_cell, n_parts: int, part: int):
        self.lib = load()
        bp = np.ascontiguousarray(block_indptr, dtype=np.int32)
        bi = np.ascontiguousarray(block_indices, dtype=np.int32)
        pc = np.ascontiguousarray(part_of_cell, dtype=np.int32)
        h = ctypes.c_void_p()
        check(self.lib.sts_dd_plan_create(int(bp.shape[0] - 1), bp.ctypes.data, bi.ctypes.data, int(n_parts),
                                          pc.ctypes.data, int(part), ctypes.byref(h)))
        self.h = h
        self.part = int(part)
        z = sts_dd_sizes()
        check(self.lib.sts_dd_plan_sizes(self.h, ctypes.byref(z)))
        self.sizes = z
        self.n_owned, self.n_ghost, self.n_local = z.n_owned, z.n_ghost, z.n_local
        nn = z.n_neighbors
        a = [np.zeros(n, dtype=np.int32) for n in (z.n_local, z.n_local + 1, z.nnzb, z.nnzb, nn, nn + 1, z.n_send,
                                                    nn + 1, z.n_recv)]
        check(self.lib.sts_dd_plan_get(self.h, *[x.ctypes.data for x in a]))
        (self.local_to_global, self.block_indptr, self.block_indices, self.block_map, self.neighbors,
         self.send_ptr, self.send_cells, self.recv_ptr, self.recv_cells) = a

    def close(self):
        if getattr(self, "h", None):
            self.lib.sts_dd_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _pairs(self, w):
        pip = getattr(w, "pair_indptr", None)
        return None if pip is None else np.ascontiguousarray(pip, dtype=np.int32)

    def local_layout(self, w) -> LocalLayout:
        """The sub-domain's layout for the global layout ``w`` (patterns, pair counts)."""
        pip = self._pairs(w)
        nnz_d, nnz_o = int(w.d_indptr[-1]), int(w.o_indptr[-1])
        lp = np.zeros(self.block_map.shape[0] + 1, dtype=np.int32)
        nS, npairs = ctypes.c_longlong(), ctypes.c_int()
        check(self.lib.sts_dd_plan_value_sizes(self.h, nnz_d, nnz_o, None if pip is None else pip.ctypes.data,
                                               int(w.r_diag), int(w.r_off), ctypes.byref(nS), ctypes.byref(npairs),
                                               lp.ctypes.data))
        rows = np.repeat(np.arange(self.n_local), np.diff(self.block_indptr))
        diag = rows == self.block_indices
        cnt = np.diff(lp)
        return LocalLayout(N=int(getattr(w, "N", 0)), b=int(w.b), r_diag=int(cnt[diag].max(initial=0)),
                           r_off=int(cnt[~diag].max(initial=0)), block_indptr=self.block_indptr,
                           block_indices=self.block_indices, d_indptr=np.asarray(w.d_indptr, dtype=np.int32),
                           d_indices=np.asarray(w.d_indices, dtype=np.int32),
                           o_indptr=np.asarray(w.o_indptr, dtype=np.int32),
                           o_indices=np.asarray(w.o_indices, dtype=np.int32), pair_indptr=lp, nnz_S=int(nS.value))

    def gather(self, w, S, U, V, stream=None):
        """The sub-domain's values from the global (S, U, V): CUDA float64 tensors
        (gathered by a kernel) or numpy arrays (gathered on the host)."""
        L = self.local_layout(w)
        pip = self._pairs(w)
        nnz_d, nnz_o = int(w.d_indptr[-1]), int(w.o_indptr[-1])
        if isinstance(S, np.ndarray):
            S, U, V = (np.ascontiguousarray(a, dtype=np.float64) for a in (S, U, V))
            out = [np.zeros(L.nnz_S), np.zeros((L.n_pairs, L.b)), np.zeros((L.n_pairs, L.b))]
            on_host, st = 1, None
        else:
            import torch
            out = [torch.empty(L.nnz_S, dtype=torch.float64, device=S.device),
                   torch.empty((L.n_pairs, L.b), dtype=torch.float64, device=S.device),
                   torch.empty((L.n_pairs, L.b), dtype=torch.float64, device=S.device)]
            on_host = 0
            st = (torch.cuda.current_stream() if stream is None else stream).cuda_stream
        check(self.lib.sts_dd_plan_gather(self.h, L.b, nnz_d, nnz_o, None if pip is None else pip.ctypes.data,
                                          int(w.r_diag), int(w.r_off), _ptr(S), _ptr(U), _ptr(V),
                                          _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), on_host, st))
        return L, out


def _tensor_at(ptr: int, n: int, device):
    """A float64 tensor viewing n values at address ptr (device memory when
    ``device`` is CUDA, host memory otherwise); no copy."""
    import torch
    if device.type == "cuda":
        class _View:
            pass
        v = _View()
        v.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False), "version": 3}
        return torch.as_tensor(v, device=device)
    return torch.from_numpy(np.ctypeslib.as_array((ctypes.c_double * max(n, 1)).from_address(ptr))[:n])


class TorchComm:
    """Exchange and allreduce callbacks over ``torch.distributed``.

    ``part_rank[p]`` is the process rank holding part p.  Messages between two
    processes are posted in (from part, to part) order on both sides, so the
    point-to-point operations pair up.  Buffers live on ``device`` (CUDA for
    the library's GPU path, with a NCCL group; CPU with a gloo group).  A
    failure (for instance a peer that left) makes the callback return 1, which
    the library reports as STS_ERR_COMM; the exception is kept in ``error``.
    """

    def __init__(self, part_rank, device="cuda", group=None):
        import torch
        self.part_rank = {int(p): int(r) for p, r in dict(part_rank).items()}
        self.device = torch.device(device)
        self.group = group
        self.error = None
        self._ex = DD_EXCHANGE(self._exchange)
        self._ar = DD_ALLREDUCE(self._allreduce)
        self.c = sts_dd_comm(None, self._ex, self._ar)

    def exchange_tensors(self, sends, recvs):
        """sends / recvs: lists of (from_part, to_part, tensor); every receive
        tensor is filled in place."""
        import torch.distributed as dist
        ops = []
        for f, t, x in sorted(sends, key=lambda e: (e[0], e[1])):
            ops.append(dist.P2POp(dist.isend, x, self.part_rank[t], group=self.group))
        for f, t, x in sorted(recvs, key=lambda e: (e[0], e[1])):
            ops.append(dist.P2POp(dist.irecv, x, self.part_rank[f], group=self.group))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()

    def _exchange(self, ctx, n_send, s_from, s_to, s_buf, s_len, n_recv, r_from, r_to, r_buf, r_len, stream):
        try:
            import torch
            sends = [(s_from[k], s_to[k], _tensor_at(s_buf[k], s_len[k], self.device)) for k in range(n_send)]
            recvs = [(r_from[k], r_to[k], _tensor_at(r_buf[k], r_len[k], self.device)) for k in range(n_recv)]
            if self.device.type == "cuda":
                with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
                    self.exchange_tensors(sends, recvs)
            else:
                self.exchange_tensors(sends, recvs)
            return 0
        except Exception as e:        # reported to the library as a failed callback
            self.error = e
            return 1

    def allreduce_array(self, vals: np.ndarray):
        import torch
        import torch.distributed as dist
        t = torch.from_numpy(vals)
        if dist.get_backend(self.group) == "nccl":
            td = t.to(self.device)
            dist.all_reduce(td, group=self.group)
            t.copy_(td.cpu())
        else:
            dist.all_reduce(t, group=self.group)

    def _allreduce(self, ctx, vals, count):
        try:
            self.allreduce_array(np.ctypeslib.as_array(vals, shape=(count,)))
            return 0
        except Exception as e:
            self.error = e
            return 1


def _opts(restart, max_iters, rtol, precond, trans, history):
    o = sts_gmres_opts()
    o.restart, o.max_iters, o.rtol = restart, max_iters, rtol
    o.precond = STS_PRECOND_BJ if precond == "bj" else STS_PRECOND_NONE
    o.trans = int(trans)
    hist = np.zeros(max_iters) if history else None
    o.history = hist.ctypes.data if history else None
    return o, hist


class DdSolver:
    """Owner of one ``sts_dd_t`` over the parts of this process.

    ``jacs``: the parts' ``StsJacobian`` handles (created from
    ``DdPlan.local_layout`` and ``DdPlan.gather``, one stream), ``plans``: their
    ``DdPlan``s, ``comm``: a ``TorchComm`` when other processes hold parts.
    Vectors are lists with one CUDA tensor per part (n_local * b values)."""

    def __init__(self, jacs, plans, comm: TorchComm | None = None):
        self.lib = load()
        self.jacs, self.plans, self.comm = list(jacs), list(plans), comm
        n = len(self.jacs)
        self._ids = np.array([p.part for p in self.plans], dtype=np.int32)
        self._jh = (ctypes.c_void_p * n)(*[j.h.value for j in self.jacs])
        self._ph = (ctypes.c_void_p * n)(*[p.h.value for p in self.plans])
        d = sts_dd_desc()
        d.n_parts = n
        d.part_ids = self._ids.ctypes.data
        d.jac = ctypes.cast(self._jh, ctypes.c_void_p)
        d.plans = ctypes.cast(self._ph, ctypes.c_void_p)
        d.comm = ctypes.pointer(comm.c) if comm is not None else None
        h = ctypes.c_void_p()
        check(self.lib.sts_dd_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.sts_dd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _arr(ts):
        return (ctypes.c_void_p * len(ts))(*[_ptr(t) for t in ts])

    def matvec(self, xs, trans: bool = False):
        import torch
        ys = [torch.empty_like(x) for x in xs]
        check(self.lib.sts_dd_matvec(self.h, self._arr(xs), self._arr(ys), int(trans)))
        return ys

    def bjacobi_apply(self, xs, trans: bool = False):
        import torch
        zs = [torch.empty_like(x) for x in xs]
        check(self.lib.sts_dd_bjacobi_apply(self.h, self._arr(xs), self._arr(zs), int(trans)))
        return zs

    def gmres(self, bs, x0s=None, *, restart: int = 30, rtol: float = 1e-10, max_iters: int = 1000,
              precond: str = "bj", trans: bool = False, history: bool = False, raise_on_fail: bool = True):
        import torch
        xs = [torch.zeros_like(b) for b in bs] if x0s is None else [x.clone() for x in x0s]
        o, hist = _opts(restart, max_iters, rtol, precond, trans, history)
        info = sts_gmres_info()
        st = self.lib.sts_dd_gmres_solve(self.h, self._arr(bs), self._arr(xs), ctypes.byref(o), ctypes.byref(info))
        if raise_on_fail:
            check(st)
        return xs, gmres_info(info, hist if history else None)


def gmres_ops(ops, *, restart: int = 30, rtol: float = 1e-10, max_iters: int = 1000, precond: str = "bj",
              history: bool = False, raise_on_fail: bool = True):
    """Run the library's distributed GMRES driver over the operations of the
    Python object ``ops`` (methods named as the ``sts_dd_ops`` callbacks; vector
    indices as documented there; ``dots`` returns a sequence, ``update`` returns
    the local squared norm when asked, ``norm2`` a float, ``allreduce`` sums a
    float64 numpy array in place).  An exception in a method is reported as
    STS_ERR_COMM and kept in the returned info's ``error``."""
    err = []

    def guard(fn):
        def call(*a):
            try:
                fn(*a)
                return 0
            except Exception as e:        # reported to the driver as a failed callback
                err.append(e)
                return 1
        return call

    def dots(ctx, v0, k, w, self_, out):
        r = np.asarray(ops.dots(v0, k, w, bool(self_)), dtype=np.float64)
        out_a = np.ctypeslib.as_array(out, shape=(k + (1 if self_ else 0),))
        out_a[:] = r

    def update(ctx, w, v0, k, h, norm, out):
        r = ops.update(w, v0, k, np.ctypeslib.as_array(h, shape=(k,)).copy(), bool(norm))
        if norm:
            out[0] = float(r)

    def norm2(ctx, v, out):
        out[0] = float(ops.norm2(v))

    def axpy(ctx, x, v0, k, y):
        ops.axpy(x, v0, k, np.ctypeslib.as_array(y, shape=(k,)).copy())

    def allreduce(ctx, vals, n):
        ops.allreduce(np.ctypeslib.as_array(vals, shape=(n,)))

    impl = {"matvec": lambda c, i, o: ops.matvec(i, o), "apply": lambda c, i, o: ops.apply(i, o),
            "copy": lambda c, o, i: ops.copy(o, i), "sub": lambda c, o, a, b: ops.sub(o, a, b),
            "scale": lambda c, o, i, s: ops.scale(o, i, s), "dots": dots, "update": update, "norm2": norm2,
            "axpy": axpy, "allreduce": allreduce}
    cbs = [t(guard(impl[name])) for name, t in DD_OPS_FIELDS]
    st_ops = sts_dd_ops(None, *cbs)
    o, hist = _opts(restart, max_iters, rtol, precond, False, history)
    info = sts_gmres_info()
    st = load().sts_dd_gmres_ops(ctypes.byref(st_ops), ctypes.byref(o), ctypes.byref(info))
    gi = gmres_info(info, hist if history else None)
    gi.error = err[0] if err else None
    gi.status = st
    if raise_on_fail and st != 0:
        check(st)
    return gi


__all__ = ["DdPlan", "DdSolver", "LocalLayout", "TorchComm", "gmres_ops", "grid_partition", "StsJacobian"]
