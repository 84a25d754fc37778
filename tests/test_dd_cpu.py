"""Domain decomposition on the CPU: the sub-domain plans (host code of the C
library) against the global problem, and the library's distributed GMRES
driver (sts_dd_gmres_ops) run on world_size-2 gloo ranks, each rank's local
operator being the FP64 oracle applied to its sub-domain (test harness only).

The plans are pinned by the oracle: the owned rows of every sub-domain product
(J x and J^T x, after the ghost entries are filled from the global vector)
equal the rows of the global product, and the distributed solve equals the
oracle's serial GMRES solution.
"""
import datetime
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_2403_09198_gb300 import dd, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    "strips": dict(Lx=7, Ly=6, N=4, w=1, r_diag=2, r_off=1, seed=3, px=1, py=2),
    "tiles2x2": dict(Lx=9, Ly=7, N=5, w=2, r_diag=2, r_off=1, seed=4, px=2, py=2),
    "faces_3x1": dict(Lx=8, Ly=5, N=4, w=1, r_diag=1, r_off=2, pairs_per_face=2, seed=5, px=3, py=1),
    "random_parts": dict(Lx=6, Ly=6, N=3, w=1, r_diag=2, r_off=1, seed=6, px=0, py=0),
}


def _case(name):
    kw = dict(CASES[name])
    px, py = kw.pop("px"), kw.pop("py")
    w = inputs.make_workload(**kw)
    if px == 0:                       # an irregular partition into 3 parts, every part non-empty
        part = np.random.default_rng(kw["seed"]).integers(0, 3, w.n_cells).astype(np.int32)
        part[:3] = [0, 1, 2]
        n_parts = 3
    else:
        part = dd.grid_partition(kw["Lx"], kw["Ly"], px, py)
        n_parts = px * py
    return w, part, n_parts


def _local(w, P):
    L, (S, U, V) = P.gather(w, w.S, w.U, w.V)
    return L, oracle.Jacobian.from_workload(L, S=S, U=U, V=V)


@pytest.mark.parametrize("name", sorted(CASES))
def test_plans_cover_the_mesh_and_agree_on_the_halo(name):
    w, part, n_parts = _case(name)
    plans = [dd.DdPlan(w.block_indptr, w.block_indices, part, n_parts, p) for p in range(n_parts)]
    owned = np.concatenate([P.local_to_global[:P.n_owned] for P in plans])
    assert np.array_equal(np.sort(owned), np.arange(w.n_cells))
    for P in plans:
        assert np.all(part[P.local_to_global[:P.n_owned]] == P.part)
        assert np.all(part[P.local_to_global[P.n_owned:]] != P.part)
        for k, q in enumerate(P.neighbors):
            Q = plans[q]
            kq = int(np.where(Q.neighbors == P.part)[0][0])
            recv = P.local_to_global[P.recv_cells[P.recv_ptr[k]:P.recv_ptr[k + 1]]]
            sent = Q.local_to_global[Q.send_cells[Q.send_ptr[kq]:Q.send_ptr[kq + 1]]]
            assert np.array_equal(recv, sent)           # same cells, same order
            assert np.all(np.diff(recv) > 0)
        # every ghost arrives from exactly one neighbour
        assert np.array_equal(np.sort(P.recv_cells), np.arange(P.n_owned, P.n_local))


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("trans", [False, True])
def test_subdomain_products_equal_the_global_rows(name, trans):
    w, part, n_parts = _case(name)
    J = oracle.Jacobian.from_workload(w)
    x = np.random.default_rng(1).standard_normal(w.n)
    y = oracle.matvec(J, x, trans=trans)
    F = oracle.bj_setup(J)
    z = oracle.bj_apply(F, x, trans=trans)
    for p in range(n_parts):
        P = dd.DdPlan(w.block_indptr, w.block_indices, part, n_parts, p)
        L, Jl = _local(w, P)
        xl = x.reshape(w.n_cells, w.b)[P.local_to_global].ravel()      # ghosts filled from the global x
        yl = oracle.matvec(Jl, xl, trans=trans).reshape(P.n_local, w.b)
        own = P.local_to_global[:P.n_owned]
        ref = y.reshape(w.n_cells, w.b)[own]
        assert np.abs(yl[:P.n_owned] - ref).max() <= 1e-13 * np.abs(ref).max()
        zl = oracle.bj_apply(oracle.bj_setup(Jl), xl, trans=trans).reshape(P.n_local, w.b)
        assert np.array_equal(zl[:P.n_owned], z.reshape(w.n_cells, w.b)[own])   # per-cell, same arithmetic


@pytest.mark.parametrize("px,py", [(2, 2), (3, 1)])
def test_plans_on_a_non_symmetric_block_pattern(px, py):
    """A block pattern that is not symmetric (lower neighbours only, plus one
    full row): a cell is a ghost of a part when it shares a block with an owned
    cell in either direction, so the owned rows of J x and J^T x still equal the
    global rows, and the halos agree."""
    from tests._workloads import nonsymmetric
    w = nonsymmetric()
    part = dd.grid_partition(7, 6, px, py)
    n_parts = px * py
    J = oracle.Jacobian.from_workload(w)
    x = np.random.default_rng(4).standard_normal(w.n)
    plans = [dd.DdPlan(w.block_indptr, w.block_indices, part, n_parts, p) for p in range(n_parts)]
    owned = np.concatenate([P.local_to_global[:P.n_owned] for P in plans])
    assert np.array_equal(np.sort(owned), np.arange(w.n_cells))
    for P in plans:
        for k, q in enumerate(P.neighbors):
            Q = plans[q]
            kq = int(np.where(Q.neighbors == P.part)[0][0])
            recv = P.local_to_global[P.recv_cells[P.recv_ptr[k]:P.recv_ptr[k + 1]]]
            sent = Q.local_to_global[Q.send_cells[Q.send_ptr[kq]:Q.send_ptr[kq + 1]]]
            assert np.array_equal(recv, sent)
        assert np.array_equal(np.sort(P.recv_cells), np.arange(P.n_owned, P.n_local))
    for trans in (False, True):
        y = oracle.matvec(J, x, trans=trans).reshape(w.n_cells, w.b)
        for P in plans:
            _, Jl = _local(w, P)
            xl = x.reshape(w.n_cells, w.b)[P.local_to_global].ravel()
            yl = oracle.matvec(Jl, xl, trans=trans).reshape(P.n_local, w.b)
            ref = y[P.local_to_global[:P.n_owned]]
            assert np.abs(yl[:P.n_owned] - ref).max() <= 1e-13 * np.abs(ref).max(), (P.part, trans)


def test_plan_rejects_bad_partitions():
    from paper_2403_09198_gb300.binding import StsError
    w = inputs.make_workload(4, 3, N=2, w=1, seed=0)
    part = np.zeros(w.n_cells, dtype=np.int32)
    with pytest.raises(StsError, match="owns no cell"):
        dd.DdPlan(w.block_indptr, w.block_indices, part, 2, 1)
    part[0] = 5
    with pytest.raises(StsError, match="out of range"):
        dd.DdPlan(w.block_indptr, w.block_indices, part, 2, 0)


# ---------------------------------------------------------------- gloo ranks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleOps:
    """The sts_dd_ops of one rank: its sub-domain's vectors as numpy arrays
    (cell-major, owned cells first), the oracle as local operator, gloo for the
    halo exchange and the sums."""

    def __init__(self, w, P, comm, m, trans, rhs):
        self.P, self.comm, self.trans, self.b = P, comm, trans, w.b
        L, self.J = _local(w, P)
        self.F = oracle.bj_setup(self.J)
        self.no = P.n_owned * w.b
        self.v = np.zeros((2 * m + 5, P.n_local * w.b))
        bl = rhs.reshape(w.n_cells, w.b)[P.local_to_global].ravel()
        bl[self.no:] = 0.0
        self.v[2 * m + 4] = bl
        self.n_mv = self.n_ap = 0

    def halo(self, x):
        import torch
        P, b = self.P, self.b
        X = x.reshape(P.n_local, b)
        sends, recvs = [], []
        for k, q in enumerate(P.neighbors):
            cells = P.send_cells[P.send_ptr[k]:P.send_ptr[k + 1]]
            sends.append((P.part, int(q), torch.from_numpy(X[cells].ravel().copy())))
            n = P.recv_ptr[k + 1] - P.recv_ptr[k]
            recvs.append((int(q), P.part, torch.empty(n * b, dtype=torch.float64)))
        self.comm.exchange_tensors(sends, recvs)
        for k, (_, _, t) in enumerate(recvs):
            X[P.recv_cells[P.recv_ptr[k]:P.recv_ptr[k + 1]]] = t.numpy().reshape(-1, b)

    def matvec(self, i, o):
        self.n_mv += 1
        x = self.v[i].copy()
        self.halo(x)
        y = oracle.matvec(self.J, x, trans=self.trans)
        y[self.no:] = 0.0
        self.v[o] = y

    def apply(self, i, o):
        self.n_ap += 1
        z = oracle.bj_apply(self.F, self.v[i], trans=self.trans)
        z[self.no:] = 0.0
        self.v[o] = z

    def copy(self, o, i):
        self.v[o] = self.v[i]

    def sub(self, o, a, b):
        self.v[o] = self.v[a] - self.v[b]

    def scale(self, o, i, s):
        self.v[o] = 0.0 if s == 0.0 else s * self.v[i]

    def dots(self, v0, k, w, self_):
        ww = self.v[w][:self.no]
        r = [float(self.v[v0 + i][:self.no] @ ww) for i in range(k)]
        return r + ([float(ww @ ww)] if self_ else [])

    def update(self, w, v0, k, h, norm):
        for i in range(k):
            self.v[w] -= h[i] * self.v[v0 + i]
        if norm:
            ww = self.v[w][:self.no]
            return float(ww @ ww)

    def norm2(self, v):
        x = self.v[v][:self.no]
        return float(x @ x)

    def axpy(self, x, v0, k, y):
        for i in range(k):
            self.v[x] += y[i] * self.v[v0 + i]

    def allreduce(self, vals):
        self.comm.allreduce_array(vals)


def _worker(rank, world, port, q, name, trans, die_rank, guess_rank=-1):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    try:
        from paper_2403_09198_gb300 import dd as ddm
        w, part, n_parts = _case(name)
        part = (part % world).astype(np.int32)
        P = ddm.DdPlan(w.block_indptr, w.block_indices, part, world, rank)
        comm = ddm.TorchComm({p: p for p in range(world)}, device="cpu")
        m = 30
        ops = OracleOps(w, P, comm, m, trans, w.rhs)
        if rank == guess_rank:             # a nonzero initial guess on this rank's owned rows only
            ops.v[2 * m + 3][:ops.no] = 1e-3 * np.random.default_rng(rank).standard_normal(ops.no)
        if rank == die_rank:
            os._exit(0)                       # leaves before the solve, nothing in flight
        info = ddm.gmres_ops(ops, restart=m, rtol=1e-14, raise_on_fail=False)
        x = ops.v[2 * m + 3][:ops.no].reshape(P.n_owned, w.b)
        q.put((rank, "ok", info.status, info.iterations, info.true_rel_residual,
               P.local_to_global[:P.n_owned].tolist(), x.tolist(),
               (info.matvecs, info.applies, ops.n_mv, ops.n_ap, info.restarts)))
    except Exception as e:                    # pragma: no cover - reported to the test
        q.put((rank, "error", repr(e)))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, name, trans=False, die_rank=-1, guess_rank=-1):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, name, trans, die_rank, guess_rank))
             for r in range(world)]
    for p in procs:
        p.start()
    out = []
    for p in procs:
        p.join(timeout=180)
        if p.is_alive():
            p.kill()
            pytest.fail("a rank hung")
    while not q.empty():
        out.append(q.get())
    return sorted(out, key=lambda r: r[0])


@pytest.mark.parametrize("name,trans", [("tiles2x2", False), ("faces_3x1", True)])
def test_distributed_gmres_on_two_gloo_ranks_equals_the_oracle(name, trans):
    out = _run(2, name, trans)
    assert [r[0] for r in out] == [0, 1] and all(r[1] == "ok" for r in out), out
    w, _, _ = _case(name)
    J = oracle.Jacobian.from_workload(w)
    xo, io = oracle.gmres(J, w.rhs, rtol=1e-14, trans=trans)
    x = np.zeros((w.n_cells, w.b))
    for r in out:
        assert r[2] == 0 and r[4] <= 1e-14
        x[np.array(r[5])] = np.array(r[6])
        assert abs(r[3] - io["iterations"]) <= 1
        # reported operator calls equal the callbacks made; the zero guess
        # starts from r = b, so each cycle's residual check but the first costs
        # a product, and every Arnoldi step one product and one apply
        mv, ap, n_mv, n_ap, restarts = r[7]
        assert (mv, ap) == (n_mv, n_ap)
        assert mv == r[3] + restarts and ap == r[3]
    assert np.linalg.norm(x.ravel() - xo) <= 1e-12 * np.linalg.norm(xo)


def test_killed_rank_makes_the_driver_return_an_error():
    out = _run(2, "tiles2x2", die_rank=1)
    assert len(out) == 1 and out[0][1] == "ok", out
    assert out[0][2] == 9                  # STS_ERR_COMM: the allreduce callback failed, no hang


def test_initial_guess_on_one_rank_is_seen_by_all():
    """A nonzero initial guess on rank 0 only: the zero-guess test sums
    ||x0||^2 over the ranks, so both ranks compute the initial product (one
    more than the iterations and restarts) and reach the oracle's solution."""
    out = _run(2, "tiles2x2", guess_rank=0)
    assert [r[0] for r in out] == [0, 1] and all(r[1] == "ok" for r in out), out
    w, _, _ = _case("tiles2x2")
    J = oracle.Jacobian.from_workload(w)
    xo, _ = oracle.gmres(J, w.rhs, rtol=1e-14)
    x = np.zeros((w.n_cells, w.b))
    for r in out:
        assert r[2] == 0 and r[4] <= 1e-14
        x[np.array(r[5])] = np.array(r[6])
        mv, ap, n_mv, n_ap, restarts = r[7]
        assert (mv, ap) == (n_mv, n_ap) and mv == r[3] + restarts + 1
    assert out[0][3] == out[1][3]
    assert np.linalg.norm(x.ravel() - xo) <= 1e-12 * np.linalg.norm(xo)
