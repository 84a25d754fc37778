"""Parity of the CUDA path against the FP64 oracle, through the C ABI.

Small workloads are compared element by element on whole outputs; the
128 x 128, N = 60 and 256 x 256, N = 200 workloads are compared on sampled
outputs the oracle computes one by one, in the launch configuration the
benchmark times.
"""
import numpy as np
import pytest

import oracle
from paper_2403_09198_gb300 import inputs
from paper_2403_09198_gb300.binding import StsError, StsJacobian
from tests._gpu import (SMALL, TOL64, dev, from_component_major, full, host, oracle_jac, rel_err,
                        sol_err, to_component_major, workload)
from tests._workloads import nonsymmetric

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _jac(w, **kw):
    return StsJacobian(w, dev(w.S), dev(w.U), dev(w.V), **kw)


# ---------------------------------------------------------------- matvec


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("layout", ["cell", "component"])
def test_matvec_small(name, layout):
    w = workload(name)
    J = oracle_jac(w)
    jac = _jac(w, transpose=True, layout=layout)
    x = np.random.default_rng(1).standard_normal(w.n)
    for trans in (False, True):
        ref = oracle.matvec(J, x, trans=trans)
        if layout == "cell":
            got = host(jac.matvec(dev(x), trans=trans))
        else:
            got = from_component_major(
                host(jac.matvec(dev(to_component_major(x, w.n_cells, w.b)), trans=trans)),
                w.n_cells, w.b)
        assert rel_err(got, ref) <= TOL64, (name, trans)
    jac.close()


def test_matvec_worked_example_bit_exact():
    """Section 5.1 r1-sparse example on one cell: integer x keeps every product
    exact, so the GPU result equals the oracle bit for bit."""
    from tests._golden import load
    g, r1 = load("csr_example"), load("r1_sparse_example")

    class W:
        b = 4
        block_indptr = np.array([0, 1])
        block_indices = np.array([0])
        d_indptr = np.array(g["indptr"])
        d_indices = np.array(g["indices"])
        o_indptr = np.zeros(5, dtype=np.int32)
        o_indices = np.zeros(0, dtype=np.int32)
        r_diag, r_off = 2, 0
        pair_indptr = np.array([0, 2])
        S = np.array(g["data"], dtype=float)
        U = np.array(r1["r1_columns"], dtype=float)
        V = np.array(r1["r1_rows"], dtype=float)

    jac = StsJacobian(W, dev(W.S), dev(W.U), dev(W.V), transpose=True)
    J = oracle.Jacobian.from_workload(W)
    for x in ([1.0, -2.0, 3.0, 5.0], [0.0, 0.0, 0.0, 1.0]):
        x = np.array(x)
        for trans in (False, True):
            assert np.array_equal(host(jac.matvec(dev(x), trans=trans)), oracle.matvec(J, x, trans=trans))


def _sample_rows(w, rng, n_rand=3000):
    nc, b = w.n_cells, w.b
    special = [0, w.Lx - 1, nc - w.Lx, nc - 1, nc // 2]
    rows = [c * b + p for c in special for p in range(b)]
    rows += list(rng.choice(nc * b, n_rand, replace=False))
    return np.unique(np.array(rows, dtype=np.int64))


@pytest.mark.parametrize("name", ["grid128_N60", "grid256_N200", "grid512_N60", "grid128_N60_pairs9"])
def test_matvec_full_size_sampled(name):
    w = full(name)
    J = oracle_jac(w)
    both = name.startswith("grid128")
    jac = _jac(w, transpose=both, layout="component")
    rng = np.random.default_rng(11)
    x = rng.standard_normal(w.n)
    rows = _sample_rows(w, rng)
    xi = to_component_major(x, w.n_cells, w.b)
    for trans in ((False, True) if both else (False,)):
        y = from_component_major(host(jac.matvec(dev(xi), trans=trans)), w.n_cells, w.b)
        ref = oracle.matvec_rows(J, x, rows, trans=trans)
        assert rel_err(y[rows], ref) <= TOL64, trans
    jac.close()


# ---------------------------------------------------------------- block-Jacobi


@pytest.mark.parametrize("name", sorted(SMALL))
def test_bjacobi_small(name):
    w = workload(name)
    J = oracle_jac(w)
    F = oracle.bj_setup(J)
    jac = _jac(w, transpose=True)
    jac.bjacobi_setup()
    x = np.random.default_rng(2).standard_normal(w.n)
    for trans in (False, True):
        got = host(jac.bjacobi_apply(dev(x), trans=trans))
        assert rel_err(got, oracle.bj_apply(F, x, trans=trans)) <= TOL64, (name, trans)
    jac.close()


def _sample_cells(w, rng):
    """First and last cells of the first tiles, of every 97th tile and of the
    last tile, plus 300 random cells."""
    nc = w.n_cells
    ends = [c for t in list(range(0, (nc + 31) // 32, 97)) + [0, 1, 2, (nc - 1) // 32]
            for c in (32 * t, min(32 * t + 31, nc - 1))]
    return np.unique(np.concatenate([ends, rng.choice(nc, 300, replace=False)]))


@pytest.mark.parametrize("name", ["grid128_N60", "grid256_N200", "grid512_N60", "grid128_N60_pairs9"])
def test_bjacobi_full_size_sampled(name):
    """Full-size workloads on sampled cells.  On 256 x 256 and 512 x 512 cells
    each apply warp streams several tiles in a row (its ring runs on across
    tiles and it copies the next tile's x during the tail), which no small
    workload does; 512 x 512 also checks the FP32 apply at full size."""
    w = full(name)
    J = oracle_jac(w)
    big = name == "grid512_N60"
    jac = _jac(w, transpose=not big, mixed=big, layout="component")
    jac.bjacobi_setup()
    rng = np.random.default_rng(12)
    x = rng.standard_normal(w.n)
    cells = _sample_cells(w, rng)
    xi = dev(to_component_major(x, w.n_cells, w.b))
    for trans in ((False,) if big else (False, True)):
        z = from_component_major(host(jac.bjacobi_apply(xi, trans=trans)), w.n_cells, w.b)
        ref = oracle.bj_cells(J, x, cells, trans=trans)
        got = z.reshape(w.n_cells, w.b)[cells]
        assert rel_err(got, ref) <= TOL64, trans
    if big:
        z32 = host(jac.bjacobi_apply(xi.float())).astype(np.float64)
        got = from_component_major(z32, w.n_cells, w.b).reshape(w.n_cells, w.b)[cells]
        ref = oracle.bj_cells(J, x, cells)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-6
    jac.close()


def test_bjacobi_working_vector_in_y():
    """b = 143 (N = 140, band +-4, 3 pairs): b rows per warp would leave fewer
    than four consumers per SM in FP64 and in FP32, so both applies keep their
    working vector in y.  Every cell against the oracle, both directions in
    FP64, and the FP32 apply."""
    w = inputs.make_workload(12, 11, N=140, w=4, r_diag=3, r_off=1, seed=41)
    J = oracle_jac(w)
    F = oracle.bj_setup(J)
    jac = _jac(w, transpose=True, mixed=True, layout="component")
    jac.bjacobi_setup()
    x = np.random.default_rng(14).standard_normal(w.n)
    xi = dev(to_component_major(x, w.n_cells, w.b))
    for trans in (False, True):
        z = from_component_major(host(jac.bjacobi_apply(xi, trans=trans)), w.n_cells, w.b)
        assert rel_err(z, oracle.bj_apply(F, x, trans=trans)) <= TOL64, trans
    z32 = from_component_major(host(jac.bjacobi_apply(xi.float())).astype(np.float64), w.n_cells, w.b)
    ref = oracle.bj_apply(F, x)
    assert np.linalg.norm(z32 - ref) / np.linalg.norm(ref) <= 1e-6
    jac.close()


@pytest.mark.parametrize("N", [61, 60])
def test_bjacobi_two_tiles_per_warp(N):
    """160 x 160 cells: 800 tiles on 608 apply warps, so 192 warps apply two
    tiles and copy the second tile's x during the first tile's tail, one row
    group at a time.  b = 64 fills every tail group (no ragged rows); b = 63
    leaves a ragged last group, copied after the section.  FP64 in both
    directions and FP32, on sampled cells against the oracle."""
    w = inputs.make_workload(160, 160, N=N, w=2, r_diag=2, r_off=1, seed=31)
    J = oracle_jac(w)
    jac = _jac(w, transpose=True, mixed=True, layout="component")
    jac.bjacobi_setup()
    rng = np.random.default_rng(13)
    x = rng.standard_normal(w.n)
    # the cells of the tiles that a warp takes second, and of the first tiles
    cells = np.unique(np.concatenate([np.arange(608 * 32, 609 * 32), np.arange(w.n_cells - 64, w.n_cells),
                                      np.arange(0, 32), _sample_cells(w, rng)]))
    xi = dev(to_component_major(x, w.n_cells, w.b))
    for trans in (False, True):
        z = from_component_major(host(jac.bjacobi_apply(xi, trans=trans)), w.n_cells, w.b)
        ref = oracle.bj_cells(J, x, cells, trans=trans)
        assert rel_err(z.reshape(w.n_cells, w.b)[cells], ref) <= TOL64, trans
    z32 = host(jac.bjacobi_apply(xi.float())).astype(np.float64)
    got = from_component_major(z32, w.n_cells, w.b).reshape(w.n_cells, w.b)[cells]
    ref = oracle.bj_cells(J, x, cells)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-6
    jac.close()


def test_bjacobi_errors():
    w = workload("ragged5x3")
    jac = _jac(w)
    with pytest.raises(StsError) as e:
        jac.bjacobi_apply(dev(np.zeros(w.n)))
    assert e.value.status == 8                     # STS_ERR_NOT_SETUP
    S = w.S.copy()
    offs = w.s_offsets()
    k = np.flatnonzero(w.is_diag_block())[7]       # cell 7
    S[offs[k]:offs[k + 1]] = 0.0
    jac.update_values(dev(S), dev(w.U), dev(w.V))
    with pytest.raises(StsError) as e:
        jac.bjacobi_setup()
    assert e.value.status == 4 and "cell 7" in e.value.message
    jac.close()


# ---------------------------------------------------------------- GMRES


@pytest.mark.parametrize("case", ["grid16_N10", "weak_diag_restart", "long_cycle", "pairs_random", "left_restart"])
def test_gmres_parity(case):
    """GMRES against the oracle's textbook GMRES.  long_cycle runs 25 Arnoldi
    steps in one cycle (no preconditioner, restart 40), so the multi-dot
    sweeps over more than one chunk of 16 basis vectors."""
    pc, left = "bj", case.startswith("left")
    if case == "grid16_N10":
        w, m = workload("grid16_N10"), 20
    elif case == "weak_diag_restart":
        w, m = inputs.make_workload(6, 5, N=4, w=2, r_diag=2, r_off=1, seed=9, dt=0.5), 4
    elif case == "pairs_random":
        w, m = inputs.make_workload(6, 5, N=4, w=2, random_pair_max=4, seed=9, dt=0.5), 4
    elif case == "left_restart":
        w, m = inputs.make_workload(6, 5, N=4, w=2, r_diag=2, r_off=1, seed=9, dt=0.5), 4
    else:
        w, m, pc = inputs.make_workload(6, 5, N=4, w=2, r_diag=2, r_off=1, seed=9, dt=0.5), 40, "none"
    J = oracle_jac(w)
    jac = _jac(w)
    jac.bjacobi_setup()
    xg, ig = jac.gmres(dev(w.rhs), restart=m, rtol=1e-10, history=True, precond=pc, left=left)
    xo, io = oracle.gmres(J, w.rhs, restart=m, rtol=1e-10, precond=pc, left=left)
    if case == "long_cycle":
        assert ig.restarts == 1 and ig.iterations > 17
    if left:
        assert ig.restarts > 1
    assert ig.converged and io["converged"]
    assert ig.true_rel_residual <= 1e-10 and io["true_rel"] <= 1e-10
    r = w.rhs - oracle.matvec(J, host(xg))
    assert np.linalg.norm(r) / np.linalg.norm(w.rhs) <= 1e-10
    assert abs(ig.iterations - io["iterations"]) <= 1
    ho = np.array(io["history"])
    n = min(len(ho), len(ig.history))
    keep = ho[:n] > 1e-13
    # 1e-8 relative while the residual is above 1e-13, plus an absolute floor of
    # 1e-15 (about 5 eps in units of ||b||): two backward-stable solvers that
    # orthogonalise differently (CGS2 here, MGS in the oracle) may differ by
    # O(eps ||b||) in the rotated residual, and that difference survives restarts
    np.testing.assert_allclose(ig.history[:n][keep], ho[:n][keep], rtol=1e-8, atol=1e-15)
    xg2, _ = jac.gmres(dev(w.rhs), restart=m, rtol=1e-14, max_iters=400, precond=pc, left=left)
    xo2, _ = oracle.gmres(J, w.rhs, restart=m, rtol=1e-14, max_iters=400, precond=pc, left=left)
    assert sol_err(host(xg2), xo2) <= TOL64
    # the reductions are deterministic: a second solve is bit-identical
    xg3, ig3 = jac.gmres(dev(w.rhs), restart=m, rtol=1e-10, history=True, precond=pc, left=left)
    assert np.array_equal(host(xg3), host(xg)) and np.array_equal(ig3.history, ig.history)
    jac.close()


@pytest.mark.parametrize("case", ["bj_restart4", "none_long", "trans", "dense", "max_iters"])
def test_gmres_cycle_graph(case):
    """Each cycle as one CUDA graph (device-side Givens rotations, conditional
    steps; the default): the same iterations and rotated residuals as the
    host-driven solver, the oracle's solution at rtol 1e-14, and across cycles, the
    transposed and unpreconditioned solves, dense storage and a step budget
    that ends inside a cycle."""
    w = inputs.make_workload(6, 5, N=4, w=2, r_diag=2, r_off=1, seed=9, dt=0.5)
    J = oracle_jac(w)
    kw, jkw = dict(restart=4), dict(transpose=True)
    if case == "none_long":
        kw = dict(restart=40, precond="none")
    elif case == "trans":
        kw = dict(restart=6, trans=True)
    elif case == "dense":
        jkw = dict(dense=True)
    jac = _jac(w, **jkw)
    jac.bjacobi_setup()
    if case == "max_iters":
        xg, ig = jac.gmres(dev(w.rhs), rtol=1e-14, max_iters=6, restart=4, graph=True, history=True,
                           raise_on_fail=False)
        xh, ih = jac.gmres(dev(w.rhs), rtol=1e-14, max_iters=6, restart=4, history=True, raise_on_fail=False,
                           graph=False)
        assert not ig.converged and ig.iterations == ih.iterations == 6 and ig.restarts == ih.restarts == 2
        np.testing.assert_allclose(ig.history, ih.history, rtol=1e-12, atol=0)
        assert sol_err(host(xg), host(xh)) <= 1e-13
        jac.close()
        return
    trans = kw.get("trans", False)
    xg, ig = jac.gmres(dev(w.rhs), rtol=1e-10, graph=True, history=True, **kw)
    xh, ih = jac.gmres(dev(w.rhs), rtol=1e-10, history=True, graph=False, **kw)
    assert ig.converged and ig.iterations == ih.iterations and ig.restarts == ih.restarts
    np.testing.assert_allclose(ig.history, ih.history, rtol=1e-12, atol=1e-16)
    r = w.rhs - oracle.matvec(J, host(xg), trans=trans)
    assert np.linalg.norm(r) / np.linalg.norm(w.rhs) <= 1e-10
    xg2, i2 = jac.gmres(dev(w.rhs), rtol=1e-14, max_iters=400, graph=True, **kw)
    xo2, _ = oracle.gmres(J, w.rhs, rtol=1e-14, max_iters=400, precond=kw.get("precond", "bj"), trans=trans,
                          restart=kw["restart"])
    assert i2.converged and sol_err(host(xg2), xo2) <= TOL64
    jac.close()


def test_gmres_host_vectors_transposed_and_unpreconditioned():
    w = workload("ragged5x3")
    J = oracle_jac(w)
    jac = _jac(w, transpose=True)
    jac.bjacobi_setup()
    # solutions: both solvers to rtol 1e-14, norm-wise agreement 1e-12
    x, info = jac.gmres(w.rhs.copy(), rtol=1e-14)                 # host vectors
    assert isinstance(x, np.ndarray) and info.converged
    assert sol_err(x, oracle.gmres(J, w.rhs, rtol=1e-14)[0]) <= TOL64
    xt, it = jac.gmres(dev(w.rhs), rtol=1e-14, trans=True)
    assert it.converged
    assert sol_err(host(xt), oracle.gmres(J, w.rhs, rtol=1e-14, trans=True)[0]) <= TOL64
    xn, inn = jac.gmres(dev(w.rhs), rtol=1e-14, precond="none", restart=60)
    assert inn.converged
    assert sol_err(host(xn), oracle.gmres(J, w.rhs, rtol=1e-14)[0]) <= TOL64
    jac.close()


def test_gmres_not_converged_keeps_x():
    w = inputs.make_workload(6, 5, N=4, w=2, seed=9, dt=0.5)
    jac = _jac(w)
    jac.bjacobi_setup()
    x, info = jac.gmres(dev(w.rhs), rtol=1e-14, max_iters=1, raise_on_fail=False)
    assert not info.converged and info.iterations == 1
    r = w.rhs - oracle.matvec(oracle_jac(w), host(x))
    assert abs(np.linalg.norm(r) / np.linalg.norm(w.rhs) - info.true_rel_residual) <= 1e-12
    with pytest.raises(StsError) as e:
        jac.gmres(dev(w.rhs), rtol=1e-14, max_iters=1)
    assert e.value.status == 5
    jac.close()


def test_gmres_nan_is_reported():
    """NaN in the right-hand side or in the Jacobian values ends the solve with
    STS_ERR_NUMERIC instead of returning garbage."""
    w = workload("ragged5x3")
    jac = _jac(w)
    jac.bjacobi_setup()
    rhs = w.rhs.copy()
    rhs[5] = np.nan
    with pytest.raises(StsError) as e:
        jac.gmres(dev(rhs))
    assert e.value.status == 6
    U = w.U.copy()
    U[3, 1] = np.nan
    jac.update_values(dev(w.S), dev(U), dev(w.V))
    with pytest.raises(StsError) as e:
        jac.bjacobi_setup()
        jac.gmres(dev(w.rhs))
    assert e.value.status in (4, 6)
    jac.close()


def test_gmres_operator_counts_and_zero_guess():
    """The solver reports the FP64 products and applies it made.  A zero guess
    starts from r = b with no product; a nonzero guess costs one more and
    reaches the oracle's solution too.  Left preconditioning adds one apply per
    cycle; the mixed solve's inner operators are FP32 and not counted."""
    w = workload("grid16_N10")
    J = oracle_jac(w)
    jac = _jac(w, transpose=True, mixed=True)
    jac.bjacobi_setup()
    xo, _ = oracle.gmres(J, w.rhs, rtol=1e-14)
    for graph in (True, False):
        x, info = jac.gmres(dev(w.rhs), rtol=1e-14, graph=graph)
        assert info.converged and sol_err(host(x), xo) <= TOL64
        assert info.matvecs == info.iterations + info.restarts and info.applies == info.iterations
    x0 = dev(1e-3 * np.random.default_rng(3).standard_normal(w.n))
    x1, i1 = jac.gmres(dev(w.rhs), x0, rtol=1e-14)
    assert i1.converged and sol_err(host(x1), xo) <= TOL64
    assert i1.matvecs == i1.iterations + i1.restarts + 1 and i1.applies == i1.iterations
    _, il = jac.gmres(dev(w.rhs), rtol=1e-12, left=True)
    assert il.matvecs == il.iterations + il.restarts and il.applies == il.iterations + il.restarts
    _, im = jac.gmres(dev(w.rhs), rtol=1e-10, mixed=True)
    assert im.converged and im.applies == 0 and im.matvecs == im.restarts
    _, inone = jac.gmres(dev(w.rhs), rtol=1e-12, precond="none")
    assert inone.applies == 0 and inone.matvecs == inone.iterations + inone.restarts
    jac.close()


@pytest.mark.parametrize("layout", ["cell", "component"])
def test_non_symmetric_block_pattern(layout):
    """A block pattern that is not symmetric: every row keeps its diagonal and
    its lower neighbours, one interior cell keeps its whole row.  The widest
    row then holds 5 blocks and the widest column 4, so the forward and the
    transposed plans get different slot counts (and kernel instances).  J x,
    J^T x, the block-Jacobi applies and GMRES in both directions against the
    oracle."""
    w = nonsymmetric()
    counts_r = np.diff(w.block_indptr)
    counts_c = np.bincount(w.block_indices, minlength=w.n_cells)
    assert counts_r.max() == 5 and counts_c.max() == 4
    J = oracle_jac(w)
    F = oracle.bj_setup(J)
    jac = _jac(w, transpose=True, layout=layout)
    jac.bjacobi_setup()
    cm = (lambda v: to_component_major(v, w.n_cells, w.b)) if layout == "component" else (lambda v: v)
    cc = (lambda v: from_component_major(v, w.n_cells, w.b)) if layout == "component" else (lambda v: v)
    x = np.random.default_rng(5).standard_normal(w.n)
    for trans in (False, True):
        assert rel_err(cc(host(jac.matvec(dev(cm(x)), trans=trans))), oracle.matvec(J, x, trans=trans)) <= TOL64
        assert rel_err(cc(host(jac.bjacobi_apply(dev(cm(x)), trans=trans))),
                       oracle.bj_apply(F, x, trans=trans)) <= TOL64
        xs, info = jac.gmres(dev(cm(w.rhs)), rtol=1e-14, trans=trans)
        xo, io = oracle.gmres(J, w.rhs, rtol=1e-14, trans=trans)
        assert info.converged and abs(info.iterations - io["iterations"]) <= 1
        assert sol_err(cc(host(xs)), xo) <= TOL64
    jac.close()


def test_values_from_host_memory():
    """Values handed over in host memory (values_on_host = 1) give the same operator."""
    w = workload("grid16_N10")
    J = oracle_jac(w)
    jac = StsJacobian(w, w.S, w.U, w.V, transpose=True)       # numpy arrays: host path
    x = np.random.default_rng(9).standard_normal(w.n)
    for trans in (False, True):
        assert rel_err(host(jac.matvec(dev(x), trans=trans)), oracle.matvec(J, x, trans=trans)) <= TOL64
    jac.update_values(w.S * 2.0, w.U, w.V)
    J2 = oracle_jac(w, S=w.S * 2.0)
    assert rel_err(host(jac.matvec(dev(x))), oracle.matvec(J2, x)) <= TOL64
    # device values in between, then host values again: the staging buffer
    # kept by the handle is reused and every update lands
    jac.update_values(dev(w.S), dev(w.U), dev(w.V))
    assert rel_err(host(jac.matvec(dev(x))), oracle.matvec(J, x)) <= TOL64
    jac.update_values(w.S * 3.0, w.U * 0.5, w.V)
    J3 = oracle_jac(w, S=w.S * 3.0, U=w.U * 0.5)
    for trans in (False, True):
        assert rel_err(host(jac.matvec(dev(x), trans=trans)), oracle.matvec(J3, x, trans=trans)) <= TOL64
    jac.close()


def test_gmres_zero_rhs():
    w = workload("ragged5x3")
    jac = _jac(w)
    jac.bjacobi_setup()
    x, info = jac.gmres(dev(np.zeros(w.n)))
    assert info.converged and info.iterations == 0 and not host(x).any()


def test_gmres_full_size_true_residual():
    """128 x 128, N = 60: GMRES(30) to 1e-10; the oracle recomputes the residual
    of the GPU solution and solves the same system for the iteration count."""
    w = inputs.named_workload("grid128_N60")
    J = oracle_jac(w)
    jac = _jac(w)
    jac.bjacobi_setup()
    x, info = jac.gmres(dev(w.rhs), restart=30, rtol=1e-10, history=True)
    r = w.rhs - oracle.matvec(J, host(x))
    assert info.converged and np.linalg.norm(r) / np.linalg.norm(w.rhs) <= 1e-10
    xo, io = oracle.gmres(J, w.rhs, restart=30, rtol=1e-10)
    assert abs(info.iterations - io["iterations"]) <= 1
    jac.close()


def test_gmres_full_size_solution_parity():
    """128 x 128, N = 60: both solvers run to rtol 1e-14, where the solution is
    determined to about kappa 1e-14; the GPU and oracle solutions then agree to
    1e-12 (reading (iv) of GMRES parity)."""
    w = full("grid128_N60")
    J = oracle_jac(w)
    jac = _jac(w)
    jac.bjacobi_setup()
    x, info = jac.gmres(dev(w.rhs), restart=30, rtol=1e-14)
    assert info.converged
    xo, io = oracle.gmres(J, w.rhs, restart=30, rtol=1e-14)
    assert io["true_rel"] <= 1e-14
    assert sol_err(host(x), xo) <= TOL64
    assert abs(info.iterations - io["iterations"]) <= 1
    jac.close()


# ---------------------------------------------------------------- mixed precision


@pytest.mark.parametrize("dt", [1e-3, 1.0])
def test_mixed_precision_fgmres(dt):
    """FP32 matvec and block-Jacobi inside FP64 flexible GMRES: the true FP64
    residual reaches 1e-10 and the error against the FP64 oracle stays within
    kappa(J) * 1e-10 (kappa from numpy on this small system).  dt = 1 weakens
    the diagonal (kappa about 12, 30 block-Jacobi GMRES steps), so several
    flexible cycles with FP32 operators are needed."""
    w = inputs.make_workload(8, 8, N=10, w=2, seed=13, dt=dt)
    J = oracle_jac(w)
    jac = _jac(w, mixed=True)
    jac.bjacobi_setup()
    x, info = jac.gmres(dev(w.rhs), rtol=1e-10, mixed=True)
    assert info.converged and info.true_rel_residual <= 1e-10
    r = w.rhs - oracle.matvec(J, host(x))
    assert np.linalg.norm(r) / np.linalg.norm(w.rhs) <= 1e-10
    D = np.stack([oracle.matvec(J, e) for e in np.eye(w.n)], axis=1)
    kappa = np.linalg.cond(D)
    x64 = np.linalg.solve(D, w.rhs)
    assert np.linalg.norm(host(x) - x64) <= 1.01 * kappa * 1e-10 * np.linalg.norm(x64)
    # FP32 operators themselves: within FP32 rounding of the FP64 oracle
    import torch
    xx = np.random.default_rng(3).standard_normal(w.n)
    y32 = host(jac.matvec(dev(xx).float())).astype(np.float64)
    yo = oracle.matvec(J, xx)
    assert np.linalg.norm(y32 - yo) / np.linalg.norm(yo) <= 1e-6
    z32 = host(jac.bjacobi_apply(dev(xx).float())).astype(np.float64)
    zo = oracle.bj_apply(oracle.bj_setup(J), xx)
    assert np.linalg.norm(z32 - zo) / np.linalg.norm(zo) <= 1e-6
    del torch
    jac.close()


def test_mixed_precision_full_size_weak_diagonal():
    """512 x 512 cells, N = 60 (the mixed-precision workload's mesh and levels,
    seed 3) with dt = 1 instead of 1e-3, so that J is far from a scaled identity:
    FP32 matvec and block-Jacobi inside FP64 flexible GMRES reach a true FP64
    residual of 1e-10 (recomputed by the oracle), and the solution differs from
    the oracle's FP64 GMRES solution (rtol 1e-12) by at most kappa * 1e-10.
    kappa is estimated from below by the oracle alone: sigma_max by power
    iterations on J^T J, 1 / sigma_min by ||x|| / ||b||; a smaller estimate only
    tightens the bound."""
    w = inputs.make_workload(512, 512, N=60, w=2, r_diag=2, r_off=1, seed=3, dt=1.0)
    J = oracle_jac(w)
    jac = _jac(w, mixed=True)
    jac.bjacobi_setup()
    x, info = jac.gmres(dev(w.rhs), rtol=1e-10, restart=30, mixed=True)
    xm = host(x)
    jac.close()
    assert info.converged
    bn = np.linalg.norm(w.rhs)
    assert np.linalg.norm(w.rhs - oracle.matvec(J, xm)) <= 1e-10 * bn * (1 + 1e-6)
    xo, io = oracle.gmres(J, w.rhs, restart=30, rtol=1e-12)
    assert io["true_rel"] <= 1e-12
    rng = np.random.default_rng(31)
    v = rng.standard_normal(w.n)
    for _ in range(6):
        v = oracle.matvec(J, oracle.matvec(J, v), trans=True)
        v /= np.linalg.norm(v)
    smax = np.sqrt(np.linalg.norm(oracle.matvec(J, oracle.matvec(J, v), trans=True)))
    kappa = smax * np.linalg.norm(xo) / bn
    assert kappa > 2.0, kappa          # the bound is not vacuous
    err = np.linalg.norm(xm - xo) / np.linalg.norm(xo)
    assert err <= kappa * (1e-10 + 1e-12), (err, kappa)


# ---------------------------------------------------------------- adjoint


def test_grad_matches_oracle_outer_products():
    for name in ("ragged5x3", "pairs9_2", "band4_r3", "pairs_faces", "pairs_random"):
        w = workload(name)
        J = oracle_jac(w)
        jac = _jac(w, transpose=True)
        rng = np.random.default_rng(4)
        lam, x = rng.standard_normal(w.n), rng.standard_normal(w.n)
        gS, gU, gV = jac.grad(dev(lam), dev(x))
        rS, rU, rV = oracle.grad(J, lam, x)
        assert rel_err(host(gS), rS) <= TOL64
        assert rel_err(host(gU), rU) <= TOL64
        assert rel_err(host(gV), rV) <= TOL64
        jac.close()


def test_implicit_solve_autograd_vs_oracle_and_fd():
    import torch
    from paper_2403_09198_gb300.autograd import ImplicitSolve
    w = inputs.make_workload(3, 2, N=3, w=1, r_diag=2, r_off=1, seed=21, dt=0.2)
    J = oracle_jac(w)
    jac = _jac(w, transpose=True)
    Wd = dev(w.W)
    params = [dev(a).requires_grad_(True) for a in (w.rhs, w.S, w.U, w.V)]

    def loss_of(b, S, U, V):
        x = ImplicitSolve.apply(b, S, U, V, jac, 1e-14, 30)
        return 0.5 * torch.sum((Wd * x) ** 2)

    L = loss_of(*params)
    L.backward()
    grads = [host(p.grad) for p in params]
    ref = oracle.adjoint(J, w.rhs, w.W)
    for g, r in zip(grads, (ref["gb"], ref["gS"], ref["gU"], ref["gV"])):
        assert rel_err(g, r) <= 1e-10
    rng = np.random.default_rng(22)
    h = 1e-6
    base = [host(p.detach()) for p in params]
    with torch.no_grad():
        for _ in range(64):
            d = [rng.standard_normal(a.shape) for a in base]
            d = [di / np.linalg.norm(di) for di in d]
            tot = np.sqrt(sum(float(np.sum(di * di)) for di in d))
            d = [di / tot for di in d]
            gd = sum(float(np.sum(g * di)) for g, di in zip(grads, d))
            Lp = float(loss_of(*[dev(a + h * di) for a, di in zip(base, d)]))
            Lm = float(loss_of(*[dev(a - h * di) for a, di in zip(base, d)]))
            fd = (Lp - Lm) / (2 * h)
            assert abs(gd - fd) <= 1e-6 * max(abs(fd), 1e-12 * np.sqrt(sum(np.sum(g * g) for g in grads)))
    jac.close()


def test_implicit_solve_two_solves_share_one_handle():
    """Two ImplicitSolve calls with different values on one handle in one graph
    (as in unrolled pseudo-time steps): each solve's gradients equal the oracle
    adjoint of its own Jacobian, although the handle holds the second solve's
    values when the first one's backward runs."""
    import torch
    from paper_2403_09198_gb300.autograd import ImplicitSolve
    w = inputs.make_workload(4, 3, N=3, w=1, r_diag=2, r_off=1, seed=23, dt=0.2)
    S2, U2, V2 = 1.1 * w.S, 0.9 * w.U, 1.2 * w.V
    J1, J2 = oracle_jac(w), oracle_jac(w, S=S2, U=U2, V=V2)
    rhs2 = np.random.default_rng(24).standard_normal(w.n)
    jac = _jac(w, transpose=True)
    Wd = dev(w.W)
    p1 = [dev(a).requires_grad_(True) for a in (w.rhs, w.S, w.U, w.V)]
    p2 = [dev(a).requires_grad_(True) for a in (rhs2, S2, U2, V2)]
    x1 = ImplicitSolve.apply(*p1, jac, 1e-14, 30)
    x2 = ImplicitSolve.apply(*p2, jac, 1e-14, 30)
    L = 0.5 * torch.sum((Wd * x1) ** 2) + 0.5 * torch.sum((Wd * x2) ** 2)
    L.backward()
    for params, J, rhs in ((p1, J1, w.rhs), (p2, J2, rhs2)):
        ref = oracle.adjoint(J, rhs, w.W)
        for p, r in zip(params, (ref["gb"], ref["gS"], ref["gU"], ref["gV"])):
            assert rel_err(host(p.grad), r) <= 1e-10
    jac.close()


def test_adjoint_full_size_sampled():
    """128 x 128, N = 60, seed 4: adjoint GMRES on the transposed operators; the
    oracle checks J^T lambda = W^2 x on sampled rows and the outer products."""
    w = inputs.named_workload("grid128_N60_adjoint")
    J = oracle_jac(w)
    jac = _jac(w, transpose=True)
    jac.bjacobi_setup()
    x, info = jac.gmres(dev(w.rhs), rtol=1e-12)
    assert info.converged
    xh = host(x)
    g = w.W * w.W * xh
    lam, it = jac.gmres(dev(g), rtol=1e-12, trans=True)
    assert it.converged
    lh = host(lam)
    rng = np.random.default_rng(5)
    rows = rng.choice(w.n, 2000, replace=False)
    res = oracle.matvec_rows(J, lh, rows, trans=True) - g[rows]
    assert np.linalg.norm(res) <= 1e-11 * np.linalg.norm(g[rows]) * 10
    gS, gU, gV = jac.grad(lam, x)
    rS, rU, rV = oracle.grad(J, lh, xh)
    for a, b in ((gS, rS), (gU, rU), (gV, rV)):
        assert rel_err(host(a), b) <= TOL64
    jac.close()


def test_adjoint_full_size_fd_and_oracle_gradient():
    """128 x 128, N = 60, seed 4 (the adjoint workload): ImplicitSolve's
    gradients with respect to b, S, U and V equal the oracle's adjoint gradient
    element by element, and 64 central finite differences (16 per parameter
    group) agree with g . d to 1e-6 relative.  Directions have N(0, 1) entries
    and the step is h = 1e-3 per entry: a solve determines L only to about
    eps L, so a central difference carries an error near eps L / h, which at
    h = 1e-6 is 1e-5 of the directional derivatives here (about 1e-5); at
    h = 1e-3 it is 1e-8 of them, while J moves by about 1e-6 of its diagonal,
    so the O(h^2) truncation stays near 1e-9 relative.  L(p + h d) - L(p - h d)
    is formed as 0.5 sum W^2 (x+ - x-)(x+ + x-).  Each solve runs a fixed
    number of Arnoldi steps (that of the base solve to rtol 1e-14, plus two),
    so the computed solution is a smooth function of the data."""
    import torch
    from paper_2403_09198_gb300.autograd import ImplicitSolve
    w = full("grid128_N60_adjoint")
    jac = _jac(w, transpose=True)
    Wd = dev(w.W)
    params = [dev(a).requires_grad_(True) for a in (w.rhs, w.S, w.U, w.V)]
    x = ImplicitSolve.apply(*params, jac, 1e-14, 30)
    L = 0.5 * torch.sum((Wd * x) ** 2)
    L.backward()
    grads = [p.grad.detach().clone() for p in params]
    J = oracle_jac(w)
    ref = oracle.adjoint(J, w.rhs, w.W)
    for g, r in zip(grads, (ref["gb"], ref["gS"], ref["gU"], ref["gV"])):
        assert rel_err(host(g), r) <= 1e-10
    base = [p.detach() for p in params]
    jac.update_values(base[1], base[2], base[3])
    jac.bjacobi_setup()
    _, info0 = jac.gmres(base[0], rtol=1e-14)
    steps = min(info0.iterations + 2, 30)

    def solve(ps):
        jac.update_values(ps[1], ps[2], ps[3])
        jac.bjacobi_setup()
        xs, _ = jac.gmres(ps[0], rtol=1e-300, restart=30, max_iters=steps, raise_on_fail=False)
        return xs

    gnorm = float(torch.sqrt(sum(torch.sum(g * g) for g in grads)))
    gen = torch.Generator(device="cuda").manual_seed(41)
    h = 1e-3
    W2 = Wd * Wd
    for k in range(64):
        grp = k % 4
        d = torch.randn(base[grp].shape, generator=gen, device="cuda", dtype=torch.float64)
        gd = float(torch.sum(grads[grp] * d))
        pp, pm = list(base), list(base)
        pp[grp] = base[grp] + h * d
        pm[grp] = base[grp] - h * d
        xp = solve(pp)
        xm = solve(pm)
        fd = float(0.5 * torch.sum(W2 * (xp - xm) * (xp + xm))) / (2 * h)
        assert abs(gd - fd) <= 1e-6 * max(abs(fd), 1e-12 * gnorm), (k, grp, gd, fd)
    jac.close()


# ---------------------------------------------------------------- dense-BSR baseline


@pytest.mark.parametrize("name", ["grid16_N10", "ragged5x3", "pairs9_2", "band4_r3", "pairs_random"])
def test_dense_bsr_baseline(name):
    w = workload(name)
    J = oracle_jac(w)
    jac = _jac(w, dense=True)
    x = np.random.default_rng(6).standard_normal(w.n)
    assert rel_err(host(jac.matvec(dev(x))), oracle.matvec(J, x)) <= TOL64
    jac.bjacobi_setup()
    assert rel_err(host(jac.bjacobi_apply(dev(x))), oracle.bj_apply(oracle.bj_setup(J), x)) <= TOL64
    xs, info = jac.gmres(dev(w.rhs), rtol=1e-14)
    assert info.converged
    assert sol_err(host(xs), oracle.gmres(J, w.rhs, rtol=1e-14)[0]) <= TOL64
    jac.close()


def test_memory_linear_in_N():
    """Bytes held by a factored handle grow linearly in N, dense ones quadratically."""
    sizes = {}
    for N in (10, 20, 40):
        w = inputs.make_workload(16, 16, N=N, w=2, seed=0)
        f = _jac(w)
        d = _jac(w, dense=True)
        sizes[N] = (f.memory_bytes(), d.memory_bytes())
        f.close()
        d.close()
    bs = np.log([13, 23, 43])                     # block size b = N + 3
    f_slope = np.polyfit(bs, np.log([sizes[n][0] for n in (10, 20, 40)]), 1)[0]
    d_slope = np.polyfit(bs, np.log([sizes[n][1] for n in (10, 20, 40)]), 1)[0]
    assert f_slope < 1.2 and d_slope > 1.7, (f_slope, d_slope)
