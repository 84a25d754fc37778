"""Domain decomposition on the GPU, several parts in one process (their halos
copied on the device): matvec, transposed matvec, block-Jacobi and GMRES over
the partition against the FP64 oracle of the whole problem, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2403_09198_gb300 import inputs
from paper_2403_09198_gb300.binding import StsJacobian
from paper_2403_09198_gb300.dd import DdPlan, DdSolver, grid_partition
from tests._gpu import TOL64, dev, host, rel_err, sol_err
from tests.test_dd_cpu import CASES, _case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _parts(w, part, n_parts, layout="cell"):
    plans, jacs = [], []
    for p in range(n_parts):
        P = DdPlan(w.block_indptr, w.block_indices, part, n_parts, p)
        L, (S, U, V) = P.gather(w, dev(w.S), dev(w.U), dev(w.V))
        j = StsJacobian(L, S, U, V, transpose=True, layout=layout)
        j.bjacobi_setup()
        plans.append(P)
        jacs.append(j)
    return plans, jacs, DdSolver(jacs, plans)


def _scatter(w, plans, v, layout="cell"):
    out = []
    for P in plans:
        loc = v.reshape(w.n_cells, w.b)[P.local_to_global]
        out.append(dev(np.ascontiguousarray(loc if layout == "cell" else loc.T).ravel()))
    return out


def _gather(w, plans, vs, layout="cell"):
    """The owned rows of every part, assembled into a global vector; also
    checks that the ghost rows are zero."""
    x = np.full((w.n_cells, w.b), np.nan)
    for P, v in zip(plans, vs):
        a = host(v).reshape(P.n_local, w.b) if layout == "cell" else host(v).reshape(w.b, P.n_local).T
        assert not a[P.n_owned:].any()
        x[P.local_to_global[:P.n_owned]] = a[:P.n_owned]
    return x.ravel()


@pytest.mark.parametrize("name", sorted(CASES))
def test_dd_operators_equal_the_oracle(name):
    w, part, n_parts = _case(name)
    J = oracle.Jacobian.from_workload(w)
    F = oracle.bj_setup(J)
    plans, jacs, S = _parts(w, part, n_parts)
    x = np.random.default_rng(2).standard_normal(w.n)
    xs = _scatter(w, plans, x)
    for trans in (False, True):
        assert rel_err(_gather(w, plans, S.matvec(xs, trans=trans)), oracle.matvec(J, x, trans=trans)) <= TOL64
        assert rel_err(_gather(w, plans, S.bjacobi_apply(xs, trans=trans)), oracle.bj_apply(F, x, trans=trans)) <= TOL64
    S.close()
    for j in jacs:
        j.close()


@pytest.mark.parametrize("name,layout", [("strips", "cell"), ("tiles2x2", "component"), ("faces_3x1", "cell"),
                                         ("random_parts", "component")])
def test_dd_gmres_equals_the_oracle(name, layout):
    """Right-preconditioned GMRES over the parts (one halo exchange per matvec,
    sums over the parts per Arnoldi step): to rtol 1e-14 the solution equals the
    oracle's serial GMRES solution to 1e-12 in both directions."""
    w, part, n_parts = _case(name)
    J = oracle.Jacobian.from_workload(w)
    plans, jacs, S = _parts(w, part, n_parts, layout)
    for trans in (False, True):
        xs, info = S.gmres(_scatter(w, plans, w.rhs, layout), rtol=1e-14, trans=trans)
        assert info.converged and info.true_rel_residual <= 1e-14
        xo, io = oracle.gmres(J, w.rhs, rtol=1e-14, trans=trans)
        assert sol_err(_gather(w, plans, xs, layout), xo) <= TOL64
        assert abs(info.iterations - io["iterations"]) <= 1
    S.close()
    for j in jacs:
        j.close()


def test_dd_single_part_is_bit_identical_to_the_handle_solver():
    """With the whole mesh as one part the driver runs the single-handle
    solver's arithmetic (host-driven steps): same iterations, same history,
    same bits."""
    w = inputs.make_workload(9, 7, N=5, w=2, r_diag=2, r_off=1, seed=7, dt=0.2)
    part = np.zeros(w.n_cells, dtype=np.int32)
    plans, jacs, S = _parts(w, part, 1)
    ref = StsJacobian(w, dev(w.S), dev(w.U), dev(w.V))
    ref.bjacobi_setup()
    xr, ir = ref.gmres(dev(w.rhs), rtol=1e-12, restart=10, history=True, graph=False)
    xs, info = S.gmres(_scatter(w, plans, w.rhs), rtol=1e-12, restart=10, history=True)
    assert info.iterations == ir.iterations and info.restarts == ir.restarts
    assert np.array_equal(info.history, ir.history)
    assert np.array_equal(_gather(w, plans, xs), host(xr))
    S.close()
    ref.close()
    for j in jacs:
        j.close()


def test_dd_full_size_four_parts():
    """128 x 128 cells, N = 60 (the benchmark workload) in 2 x 2 parts: sampled
    rows of J x against the oracle, and GMRES to rtol 1e-14 against the oracle's
    solution."""
    w = inputs.named_workload("grid128_N60")
    part = grid_partition(128, 128, 2, 2)
    J = oracle.Jacobian.from_workload(w)
    plans, jacs, S = _parts(w, part, 4, "component")
    x = np.random.default_rng(3).standard_normal(w.n)
    y = _gather(w, plans, S.matvec(_scatter(w, plans, x, "component")), "component")
    rows = np.random.default_rng(4).choice(w.n, 3000, replace=False)
    assert rel_err(y[rows], oracle.matvec_rows(J, x, rows)) <= TOL64
    xs, info = S.gmres(_scatter(w, plans, w.rhs, "component"), rtol=1e-14)
    xo, io = oracle.gmres(J, w.rhs, rtol=1e-14)
    assert info.converged and sol_err(_gather(w, plans, xs, "component"), xo) <= TOL64
    S.close()
    for j in jacs:
        j.close()


@pytest.mark.parametrize("layout", ["cell", "component"])
def test_dd_non_symmetric_block_pattern(layout):
    """A block pattern that is not symmetric, in 2 x 2 parts: J x, J^T x, the
    block-Jacobi applies and GMRES in both directions against the oracle."""
    from tests._workloads import nonsymmetric
    w = nonsymmetric()
    part = grid_partition(7, 6, 2, 2)
    J = oracle.Jacobian.from_workload(w)
    F = oracle.bj_setup(J)
    plans, jacs, S = _parts(w, part, 4, layout)
    x = np.random.default_rng(5).standard_normal(w.n)
    xs = _scatter(w, plans, x, layout)
    for trans in (False, True):
        assert rel_err(_gather(w, plans, S.matvec(xs, trans=trans), layout), oracle.matvec(J, x, trans=trans)) <= TOL64
        assert rel_err(_gather(w, plans, S.bjacobi_apply(xs, trans=trans), layout),
                       oracle.bj_apply(F, x, trans=trans)) <= TOL64
        xg, info = S.gmres(_scatter(w, plans, w.rhs, layout), rtol=1e-14, trans=trans)
        xo, _ = oracle.gmres(J, w.rhs, rtol=1e-14, trans=trans)
        assert info.converged and sol_err(_gather(w, plans, xg, layout), xo) <= TOL64
        assert info.matvecs == info.iterations + info.restarts and info.applies == info.iterations
    S.close()
    for j in jacs:
        j.close()
