"""Pins of the FP64 oracle against things other than itself (no GPU needed).

Each test checks the oracle against values the paper prints for its worked
examples, exact arithmetic on a different computation route, a library routine
for a special case, an invariant, or brute force on tiny inputs.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle.gmres import gmres_operator
from paper_2403_09198_gb300 import inputs
from tests._golden import load


def _single_block_jacobian(b, indptr, indices, S, U=None, V=None):
    r = 0 if U is None else len(U)
    return oracle.Jacobian(
        n_cells=1, b=b, block_indptr=[0, 1], block_indices=[0],
        d_indptr=indptr, d_indices=indices, o_indptr=[0] * (b + 1), o_indices=[],
        pair_indptr=[0, r], S=S,
        U=np.zeros((0, b)) if U is None else U, V=np.zeros((0, b)) if V is None else V)


def _dense_of(J, trans=False):
    """Columns of the operator from the oracle's own matvec on unit vectors."""
    n = J.n
    return np.stack([oracle.matvec(J, np.eye(n)[k], trans=trans) for k in range(n)], axis=1)


def _tiny(Lx=3, Ly=2, N=3, w=1, r_diag=2, r_off=1, seed=7, **kw):
    return inputs.make_workload(Lx, Ly, N=N, w=w, r_diag=r_diag, r_off=r_off, seed=seed, **kw)


def _global_csr(wl):
    """scipy CSR of S alone, built from the public layout by index bookkeeping only."""
    rows, cols = [], []
    is_diag = wl.is_diag_block()
    k = 0
    for i in range(wl.n_cells):
        for blk in range(wl.block_indptr[i], wl.block_indptr[i + 1]):
            j = wl.block_indices[blk]
            ip, ix = (wl.d_indptr, wl.d_indices) if is_diag[blk] else (wl.o_indptr, wl.o_indices)
            for p in range(wl.b):
                for e in range(ip[p], ip[p + 1]):
                    rows.append(i * wl.b + p)
                    cols.append(j * wl.b + ix[e])
                    k += 1
    assert k == wl.S.shape[0]
    return sp.csr_array(sp.coo_array((wl.S, (rows, cols)), shape=(wl.n, wl.n)))


# ---------------------------------------------------------------- worked examples


def test_csr_example_scatter():
    """Section 5.1 CSR example: the oracle scatters data/indices/indptr to the printed matrix."""
    g = load("csr_example")
    J = _single_block_jacobian(4, g["indptr"], g["indices"], g["data"])
    np.testing.assert_array_equal(_dense_of(J), np.array(g["matrix"], dtype=float))


def test_r1_sparse_example_exact():
    """Section 5.1 r1-sparse example: (A + sum u v^T) x, computed exactly in rationals
    in the factored form A x + sum u (v . x), equals the oracle's dense product bit for bit."""
    g = load("csr_example")
    r1 = load("r1_sparse_example")
    U = np.array(r1["r1_columns"], dtype=float)
    V = np.array(r1["r1_rows"], dtype=float)
    J = _single_block_jacobian(4, g["indptr"], g["indices"], g["data"], U, V)
    A = [[Fraction(v) for v in row] for row in g["matrix"]]
    Uf = [[Fraction(v) for v in row] for row in r1["r1_columns"]]
    Vf = [[Fraction(str(v)) for v in row] for row in r1["r1_rows"]]
    rng = np.random.default_rng(0)
    for x in [np.eye(4)[k] for k in range(4)] + [rng.integers(-9, 10, 4).astype(float)]:
        xf = [Fraction(int(v)) for v in x]
        exact = []
        for p in range(4):
            acc = sum(A[p][q] * xf[q] for q in range(4))
            for k in range(2):
                acc += Uf[k][p] * sum(Vf[k][q] * xf[q] for q in range(4))
            exact.append(float(acc))
        np.testing.assert_array_equal(oracle.matvec(J, x), np.array(exact))
    # a transposed operand (v u^T instead of u v^T) would change the result
    Jt = _single_block_jacobian(4, g["indptr"], g["indices"], g["data"], V, U)
    assert not np.array_equal(_dense_of(Jt), _dense_of(J))


def test_bsr_example_blocks():
    """Section 5.1 BSR example: block placement reproduces the printed 8x8 matrix."""
    g = load("bsr_example")
    dense_pat = ([0, 2, 4], [0, 1, 0, 1])
    J = oracle.Jacobian(
        n_cells=4, b=2, block_indptr=g["block_indptr"], block_indices=g["block_indices"],
        d_indptr=dense_pat[0], d_indices=dense_pat[1], o_indptr=dense_pat[0],
        o_indices=dense_pat[1], pair_indptr=[0] * 9, S=np.array(g["data"], float).ravel(),
        U=np.zeros((0, 2)), V=np.zeros((0, 2)))
    M = np.array(g["matrix"], dtype=float)
    np.testing.assert_array_equal(_dense_of(J), M)
    np.testing.assert_array_equal(_dense_of(J, trans=True), M.T)


def test_br1_bsr_index_example():
    """Section 5.1 BR1-BSR example: pair_indptr and column_pair_indptr for 3 / 1 pairs."""
    g = load("br1_bsr_example")
    pip = inputs.pair_indptr_for(g["block_indptr"], g["block_indices"],
                                 g["pairs_per_diagonal_block"], g["pairs_per_off_diagonal_block"])
    assert pip.tolist() == g["pair_indptr"]
    assert pip[np.array(g["block_indptr"])].tolist() == g["column_pair_indptr"]


def test_br1_product_example_integer():
    """Section 5.2 example: with S = 0 the product is, per block row i,
    sum_j U_ij (V_ij^T x_j); integer data keeps every sum exact."""
    g = load("br1_bsr_example")
    bi, bp = np.array(g["block_indices"]), np.array(g["block_indptr"])
    pip = np.array(g["pair_indptr"])
    rng = np.random.default_rng(3)
    b = 2
    U = rng.integers(-5, 6, (16, b)).astype(float)
    V = rng.integers(-5, 6, (16, b)).astype(float)
    x = rng.integers(-5, 6, 4 * b).astype(float)
    dense_pat = ([0, 2, 4], [0, 1, 0, 1])
    J = oracle.Jacobian(n_cells=4, b=b, block_indptr=bp, block_indices=bi,
                        d_indptr=dense_pat[0], d_indices=dense_pat[1], o_indptr=dense_pat[0],
                        o_indices=dense_pat[1], pair_indptr=pip, S=np.zeros(8 * 4), U=U, V=V)
    expect = np.zeros(4 * b)
    for i in range(4):
        for k in range(bp[i], bp[i + 1]):
            j = bi[k]
            Uk, Vk = U[pip[k]:pip[k + 1]].T, V[pip[k]:pip[k + 1]].T   # b x r
            expect[i * b:(i + 1) * b] += Uk @ (Vk.T @ x[j * b:(j + 1) * b])
    np.testing.assert_array_equal(oracle.matvec(J, x), expect)


# ---------------------------------------------------------------- matvec


def test_matvec_r0_is_csr_spmv():
    """With no rank-one pairs the operator is the CSR matrix S (scipy as the check)."""
    wl = _tiny(r_diag=0, r_off=0)
    J = oracle.Jacobian.from_workload(wl)
    A = _global_csr(wl)
    x = np.random.default_rng(1).standard_normal(wl.n)
    np.testing.assert_allclose(oracle.matvec(J, x), A @ x, rtol=1e-14, atol=1e-12)
    np.testing.assert_allclose(oracle.matvec(J, x, trans=True), A.T @ x, rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("kw", [{}, dict(same_pattern=True),
                                dict(r_diag=1, r_off=2, pairs_per_face=2),
                                dict(random_pair_max=3)],
                         ids=["uniform", "same_pattern", "pairs_per_face", "random_counts"])
def test_matvec_factored_route(kw):
    """Dense assembly equals the factored route S x + sum_p u_p (v_p . x_j),
    also with pair counts that differ from block to block (Section 5.1)."""
    wl = _tiny(Lx=4, Ly=3, N=4, w=2, **kw)
    J = oracle.Jacobian.from_workload(wl)
    A = _global_csr(wl)
    x = np.random.default_rng(2).standard_normal(wl.n)
    y = A @ x
    yt = A.T @ x
    is_diag = wl.is_diag_block()
    b = wl.b
    for i in range(wl.n_cells):
        for k in range(wl.block_indptr[i], wl.block_indptr[i + 1]):
            j = wl.block_indices[k]
            for p in range(wl.pair_indptr[k], wl.pair_indptr[k + 1]):
                y[i * b:(i + 1) * b] += wl.U[p] * np.dot(wl.V[p], x[j * b:(j + 1) * b])
                yt[j * b:(j + 1) * b] += wl.V[p] * np.dot(wl.U[p], x[i * b:(i + 1) * b])
    assert is_diag.sum() == wl.n_cells
    np.testing.assert_allclose(oracle.matvec(J, x), y, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(oracle.matvec(J, x, trans=True), yt, rtol=1e-13, atol=1e-12)


def _pad_pairs(wl, r_diag, r_off):
    """The same Jacobian with every block padded to r_diag / r_off pairs by zero pairs."""
    counts = np.diff(wl.pair_indptr)
    target = np.where(wl.is_diag_block(), r_diag, r_off)
    assert np.all(target >= counts)
    pip = np.zeros(wl.nnzb + 1, dtype=np.int64)
    np.cumsum(target, out=pip[1:])
    U = np.zeros((pip[-1], wl.b))
    V = np.zeros((pip[-1], wl.b))
    for k in range(wl.nnzb):
        c = counts[k]
        U[pip[k]:pip[k] + c] = wl.U[wl.pair_indptr[k]:wl.pair_indptr[k + 1]]
        V[pip[k]:pip[k] + c] = wl.V[wl.pair_indptr[k]:wl.pair_indptr[k + 1]]
    return oracle.Jacobian(n_cells=wl.n_cells, b=wl.b, block_indptr=wl.block_indptr,
                           block_indices=wl.block_indices, d_indptr=wl.d_indptr,
                           d_indices=wl.d_indices, o_indptr=wl.o_indptr, o_indices=wl.o_indices,
                           pair_indptr=pip.astype(np.int32), S=wl.S, U=U, V=V)


def test_non_uniform_pairs_equal_zero_padding():
    """Per-block pair counts: padding every block with zero pairs to a uniform
    count leaves the operator and its block-Jacobi inverse unchanged (u v^T = 0)."""
    wl = _tiny(Lx=4, Ly=3, N=4, w=2, seed=13, random_pair_max=3)
    assert len(set(np.diff(wl.pair_indptr).tolist())) > 1 and np.min(np.diff(wl.pair_indptr)) == 0
    J = oracle.Jacobian.from_workload(wl)
    Jp = _pad_pairs(wl, wl.r_diag + 1, wl.r_off + 2)
    x = np.random.default_rng(3).standard_normal(wl.n)
    for trans in (False, True):
        np.testing.assert_array_equal(oracle.matvec(Jp, x, trans=trans), oracle.matvec(J, x, trans=trans))
        np.testing.assert_array_equal(oracle.bj_apply(oracle.bj_setup(Jp), x, trans=trans),
                                      oracle.bj_apply(oracle.bj_setup(J), x, trans=trans))


def test_matvec_adjoint_identity():
    wl = _tiny(Lx=5, Ly=4, N=5, w=2, seed=11)
    J = oracle.Jacobian.from_workload(wl)
    rng = np.random.default_rng(4)
    x, z = rng.standard_normal(wl.n), rng.standard_normal(wl.n)
    lhs = np.dot(z, oracle.matvec(J, x))
    rhs = np.dot(oracle.matvec(J, z, trans=True), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("trans", [False, True])
def test_matvec_rows_sample(trans):
    wl = _tiny(Lx=6, Ly=5, N=6, w=2, seed=5)
    J = oracle.Jacobian.from_workload(wl)
    x = np.random.default_rng(6).standard_normal(wl.n)
    y = oracle.matvec(J, x, trans=trans)
    rows = np.random.default_rng(7).choice(wl.n, 40, replace=False)
    np.testing.assert_allclose(oracle.matvec_rows(J, x, rows, trans=trans), y[rows],
                               rtol=1e-14, atol=1e-13)


# ---------------------------------------------------------------- block-Jacobi


def test_bj_single_cell_is_exact_inverse():
    """On a 1x1 mesh block-Jacobi is J^-1: J (M x) = x, and M x matches numpy's solve."""
    wl = _tiny(Lx=1, Ly=1, N=6, w=2)
    J = oracle.Jacobian.from_workload(wl)
    F = oracle.bj_setup(J)
    x = np.random.default_rng(8).standard_normal(wl.n)
    z = oracle.bj_apply(F, x)
    np.testing.assert_allclose(oracle.matvec(J, z), x, rtol=1e-13, atol=1e-13)
    D = _dense_of(J)
    np.testing.assert_allclose(z, np.linalg.solve(D, x), rtol=1e-13, atol=1e-16)
    zt = oracle.bj_apply(F, x, trans=True)
    np.testing.assert_allclose(zt, np.linalg.solve(D.T, x), rtol=1e-13, atol=1e-16)


def test_bj_inverse_identity_and_cells():
    """(S + U V^T)^-1 (S + U V^T) = I per cell, and the subset routine agrees."""
    wl = _tiny(Lx=3, Ly=3, N=5, w=2, seed=9)
    J = oracle.Jacobian.from_workload(wl)
    F = oracle.bj_setup(J)
    b = wl.b
    for c in range(wl.n_cells):
        LU = F.LU[c * b * b:(c + 1) * b * b]
        assert np.all(np.isfinite(LU))
    # block inverse times block = identity, through unit vectors on each cell
    D = _dense_of(J)
    for c in [0, 4, 8]:
        Dii = D[c * b:(c + 1) * b, c * b:(c + 1) * b]
        Minv = np.stack([oracle.bj_apply(F, np.concatenate(
            [np.zeros(c * b), Dii[:, q], np.zeros((wl.n_cells - c - 1) * b)]))[c * b:(c + 1) * b]
            for q in range(b)], axis=1)
        np.testing.assert_allclose(Minv, np.eye(b), atol=1e-13)
    x = np.random.default_rng(10).standard_normal(wl.n)
    z = oracle.bj_apply(F, x)
    cells = np.array([8, 0, 5])
    for trans in (False, True):
        zz = oracle.bj_apply(F, x, trans=trans)
        out = oracle.bj_cells(J, x, cells, trans=trans)
        for s, c in enumerate(cells):
            np.testing.assert_allclose(out[s], zz[c * b:(c + 1) * b], rtol=1e-15, atol=1e-18)
    assert z.shape == x.shape


def test_bj_partial_pivoting_needed():
    """A diagonal block whose leading entry is zero still solves (row exchange)."""
    b = 3
    indptr, indices = [0, 3, 6, 9], [0, 1, 2] * 3
    S = np.array([0.0, 2.0, 1.0, 3.0, 1.0, 0.5, 1.0, 1.0, 4.0])
    J = _single_block_jacobian(b, indptr, indices, S)
    F = oracle.bj_setup(J)
    x = np.array([1.0, -2.0, 0.5])
    np.testing.assert_allclose(oracle.bj_apply(F, x), np.linalg.solve(S.reshape(3, 3), x),
                               rtol=1e-14)
    np.testing.assert_allclose(oracle.bj_apply(F, x, trans=True),
                               np.linalg.solve(S.reshape(3, 3).T, x), rtol=1e-14)


def test_bj_singular_block_reported():
    wl = _tiny(Lx=2, Ly=2, N=2, w=1, r_diag=0, r_off=0)
    S = wl.S.copy()
    offs = wl.s_offsets()
    diag_blocks = np.flatnonzero(wl.is_diag_block())
    k = diag_blocks[2]                      # cell 2
    S[offs[k]:offs[k + 1]] = 0.0
    J = oracle.Jacobian.from_workload(wl, S=S)
    with pytest.raises(oracle.OracleSingular) as e:
        oracle.bj_setup(J)
    assert e.value.cell == 2


def test_smw_reading_of_section6_sign():
    """Section 6 steps SMW-1/2/3 reproduce the block inverse only with x = x0 - W z.

    The paper prints x = x0 + W z (and a '+' in the inverse formula); with
    C = I + V^T A0^-1 U the Woodbury identity needs the minus sign.  Here the steps
    run in numpy on one cell; the oracle's dense LU is the reference."""
    wl = _tiny(Lx=1, Ly=1, N=6, w=2, r_diag=3, seed=12)
    J = oracle.Jacobian.from_workload(wl)
    b = wl.b
    A0 = _dense_of(_single_block_jacobian(b, wl.d_indptr, wl.d_indices, wl.S))
    Uk, Vk = wl.U.T, wl.V.T                       # b x r
    rhs = np.random.default_rng(13).standard_normal(b)
    x0 = np.linalg.solve(A0, rhs)                 # SMW-1
    Wk = np.linalg.solve(A0, Uk)
    Ck = np.eye(Uk.shape[1]) + Vk.T @ Wk
    z = np.linalg.solve(Ck, Vk.T @ x0)            # SMW-2
    ref = oracle.bj_apply(oracle.bj_setup(J), rhs)
    np.testing.assert_allclose(x0 - Wk @ z, ref, rtol=1e-12)       # SMW-3, minus sign
    assert np.linalg.norm((x0 + Wk @ z) - ref) > 1e-6 * np.linalg.norm(ref)


def test_sherman_morrison_r1():
    """r = 1: x = x0 - S^-1 u (v . x0) / (1 + v . S^-1 u)."""
    wl = _tiny(Lx=1, Ly=1, N=5, w=2, r_diag=1, seed=14)
    J = oracle.Jacobian.from_workload(wl)
    b = wl.b
    A0 = _dense_of(_single_block_jacobian(b, wl.d_indptr, wl.d_indices, wl.S))
    u, v = wl.U[0], wl.V[0]
    rhs = np.random.default_rng(15).standard_normal(b)
    x0 = np.linalg.solve(A0, rhs)
    Su = np.linalg.solve(A0, u)
    expect = x0 - Su * np.dot(v, x0) / (1.0 + np.dot(v, Su))
    np.testing.assert_allclose(oracle.bj_apply(oracle.bj_setup(J), rhs), expect, rtol=1e-12)


# ---------------------------------------------------------------- GMRES


def test_gmres_residual_is_krylov_least_squares():
    """At step k the GMRES residual equals min_y ||b - A M K_k y|| over the explicit
    Krylov basis K_k = [b, (AM) b, ..., (AM)^(k-1) b] (numpy lstsq), and never grows."""
    wl = _tiny(Lx=3, Ly=2, N=3, w=1, seed=16, dt=1.0)   # weak diagonal: several iterations
    J = oracle.Jacobian.from_workload(wl)
    F = oracle.bj_setup(J)
    rhs = wl.rhs
    A = _dense_of(J)
    Mop = np.stack([oracle.bj_apply(F, e) for e in np.eye(wl.n)], axis=1)
    x, info = oracle.gmres(J, rhs, restart=40, rtol=1e-13, max_iters=6, factors=F)
    hist = np.array(info["history"])
    assert np.all(np.diff(hist) <= 1e-14)
    AM = A @ Mop
    K = [rhs]
    for k in range(1, len(hist) + 1):
        Kk = np.stack(K, axis=1)
        y, *_ = np.linalg.lstsq(AM @ Kk, rhs, rcond=None)
        res = np.linalg.norm(rhs - AM @ Kk @ y) / np.linalg.norm(rhs)
        assert abs(res - hist[k - 1]) <= 1e-8 * max(res, 1e-14), (k, res, hist[k - 1])
        K.append(AM @ K[-1])


def test_gmres_left_residual_is_krylov_least_squares():
    """Left preconditioning (Section 6, (M A) x = M b): at step k the rotated
    residual is min_y ||M b - M A K_k y|| over the explicit Krylov basis
    K_k = [M b, (MA) M b, ...] (numpy lstsq), scaled by 1 / ||M b||; it never
    grows, and the solution reaches the true residual."""
    wl = _tiny(Lx=3, Ly=2, N=3, w=1, seed=16, dt=1.0)
    J = oracle.Jacobian.from_workload(wl)
    F = oracle.bj_setup(J)
    rhs = wl.rhs
    A = _dense_of(J)
    Mop = np.stack([oracle.bj_apply(F, e) for e in np.eye(wl.n)], axis=1)
    x, info = oracle.gmres(J, rhs, restart=40, rtol=1e-13, max_iters=6, factors=F, left=True)
    hist = np.array(info["history"])
    assert np.all(np.diff(hist) <= 1e-14)
    MA, Mb = Mop @ A, Mop @ rhs
    K = [Mb]
    for k in range(1, len(hist) + 1):
        Kk = np.stack(K, axis=1)
        y, *_ = np.linalg.lstsq(MA @ Kk, Mb, rcond=None)
        res = np.linalg.norm(Mb - MA @ Kk @ y) / np.linalg.norm(Mb)
        assert abs(res - hist[k - 1]) <= 1e-8 * max(res, 1e-14), (k, res, hist[k - 1])
        K.append(MA @ K[-1])
    xs, its = oracle.gmres(J, rhs, restart=4, rtol=1e-12, factors=F, left=True)
    assert its["converged"] and its["restarts"] > 1
    np.testing.assert_allclose(xs, np.linalg.solve(A, rhs), rtol=0, atol=1e-9 * np.abs(xs).max())


def test_gmres_finite_termination_unpreconditioned():
    """m >= n: unpreconditioned GMRES solves exactly in at most n steps."""
    wl = _tiny(Lx=2, Ly=1, N=2, w=1, seed=17, dt=1.0)
    J = oracle.Jacobian.from_workload(wl)
    x, info = oracle.gmres(J, wl.rhs, restart=wl.n, rtol=1e-12, max_iters=wl.n, precond="none")
    assert info["converged"] and info["iterations"] <= wl.n
    np.testing.assert_allclose(x, np.linalg.solve(_dense_of(J), wl.rhs), rtol=1e-10)


def test_gmres_single_cell_bj_one_iteration():
    wl = _tiny(Lx=1, Ly=1, N=8, w=2, seed=18)
    J = oracle.Jacobian.from_workload(wl)
    x, info = oracle.gmres(J, wl.rhs, restart=20, rtol=1e-10)
    assert info["converged"] and info["iterations"] == 1
    np.testing.assert_allclose(oracle.matvec(J, x), wl.rhs, rtol=1e-12)


@pytest.mark.parametrize("restart", [2, 20])
def test_gmres_solution_and_true_residual(restart):
    wl = _tiny(Lx=4, Ly=4, N=4, w=2, seed=19, dt=0.5)
    J = oracle.Jacobian.from_workload(wl)
    x, info = oracle.gmres(J, wl.rhs, restart=restart, rtol=1e-10)
    assert info["converged"]
    r = wl.rhs - oracle.matvec(J, x)
    assert np.linalg.norm(r) / np.linalg.norm(wl.rhs) <= 1e-10
    assert abs(info["true_rel"] - np.linalg.norm(r) / np.linalg.norm(wl.rhs)) < 1e-14
    D = _dense_of(J)
    kappa = np.linalg.cond(D)
    x_np = np.linalg.solve(D, wl.rhs)
    # forward error bound: ||x - x*|| / ||x*|| <= kappa * relative residual
    assert np.linalg.norm(x - x_np) <= 1.01 * kappa * 1e-10 * np.linalg.norm(x_np)
    xt, it = oracle.gmres(J, wl.rhs, restart=restart, rtol=1e-12, trans=True)
    assert it["converged"]
    xt_np = np.linalg.solve(D.T, wl.rhs)
    assert np.linalg.norm(xt - xt_np) <= 1.01 * kappa * 1e-12 * np.linalg.norm(xt_np)


def test_gmres_operator_matches_scipy_solution():
    rng = np.random.default_rng(20)
    A = np.eye(12) * 4 + rng.standard_normal((12, 12))
    b = rng.standard_normal(12)
    x, info = gmres_operator(lambda v: A @ v, lambda v: v, b, restart=12, rtol=1e-13)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10)


def test_gmres_zero_rhs():
    wl = _tiny(Lx=2, Ly=2, N=2, w=1)
    x, info = oracle.gmres(oracle.Jacobian.from_workload(wl), np.zeros(wl.n))
    assert info["converged"] and info["iterations"] == 0 and not x.any()


# ---------------------------------------------------------------- adjoint


def _loss(J, rhs, W):
    x, info = oracle.gmres(J, rhs, restart=30, rtol=1e-15, max_iters=300)
    return 0.5 * float(np.dot(W * x, W * x))


def test_adjoint_matches_dense_solve_and_central_differences():
    wl = _tiny(Lx=2, Ly=2, N=2, w=1, r_diag=2, r_off=1, seed=21, dt=0.2)
    J = oracle.Jacobian.from_workload(wl)
    res = oracle.adjoint(J, wl.rhs, wl.W)
    D = _dense_of(J)
    x_np = np.linalg.solve(D, wl.rhs)
    lam_np = np.linalg.solve(D.T, wl.W ** 2 * x_np)
    np.testing.assert_allclose(res["x"], x_np, rtol=1e-11)
    np.testing.assert_allclose(res["lam"], lam_np, rtol=1e-10)
    rng = np.random.default_rng(22)
    h = 1e-6
    for _ in range(6):
        d = {k: rng.standard_normal(s.shape) for k, s in
             dict(b=wl.rhs, S=wl.S, U=wl.U, V=wl.V).items()}
        tot = np.sqrt(sum(float(np.sum(v * v)) for v in d.values()))
        d = {k: v / tot for k, v in d.items()}
        gd = (np.dot(res["gb"], d["b"]) + np.dot(res["gS"], d["S"]) +
              np.sum(res["gU"] * d["U"]) + np.sum(res["gV"] * d["V"]))

        def L_at(t):
            Jt = oracle.Jacobian.from_workload(wl, S=wl.S + t * d["S"], U=wl.U + t * d["U"],
                                               V=wl.V + t * d["V"])
            return _loss(Jt, wl.rhs + t * d["b"], wl.W)

        fd = (L_at(h) - L_at(-h)) / (2 * h)
        assert abs(gd - fd) <= 1e-6 * max(abs(fd), 1e-12), (gd, fd)
