"""Parity of the HLL-flux Jacobian generator (sts_flow_*) with the FP64 oracle.

The residual and the BR1-BSR blocks of dR/dQ (S in pattern order, the rank-one
pairs U, V in pair order) are compared element by element with
``oracle/flux.py``, itself pinned by complex-step derivatives
(``tests/test_flux_pins.py``).
"""
import numpy as np
import pytest

from oracle import flux
from paper_2403_09198_gb300 import inputs
from paper_2403_09198_gb300.binding import StsFlow
from tests._gpu import dev, host

pytestmark = pytest.mark.gpu

# Tolerance of every residual and Jacobian element, relative to the sum of the
# absolute values of the terms it is formed from (about 1000 ulps of them; the
# observed errors are below 1e-15 of that scale)
TOL_RES = 1e-13


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


CASES = {
    "sub4x3": dict(Lx=4, Ly=3, N=5, w=1, seed=1),
    "super4x3": dict(Lx=4, Ly=3, N=5, w=1, seed=1, mach=2.5),
    "ragged5x3_w2": dict(Lx=5, Ly=3, N=8, w=2, seed=2),
    "one_cell": dict(Lx=1, Ly=1, N=3, w=1, seed=3),
    "column1x7": dict(Lx=1, Ly=7, N=4, w=0, seed=4),
    "row7x1": dict(Lx=7, Ly=1, N=4, w=2, seed=5),
    "grid16_N20": dict(Lx=16, Ly=16, N=20, w=2, seed=6),
    "N40_b43": dict(Lx=3, Ly=2, N=40, w=3, seed=7),
    "N1_single_species": dict(Lx=3, Ly=3, N=1, w=0, seed=8),
    "band_wider_than_levels": dict(Lx=3, Ly=2, N=2, w=3, seed=9),
}


def _res_err(got, m, c, cells=None):
    """Residual error per element, scaled by the sum of the absolute terms that
    make it up (oracle ``residual_rows``): the residual is a cancellation (q^n is
    q within 1%, the face fluxes nearly cancel), so its rounding error is bounded
    by a few ulps of those terms, not of the result."""
    cells = list(range(c.n_cells)) if cells is None else list(cells)
    ref, mag = flux.residual_rows(m, c.Lx, c.Ly, c.Q, c.Qn, cells)
    return float(np.max(np.abs(np.asarray(got) - ref) / mag))


def _scaled_err(got, ref, scale):
    """Largest element error over the oracle's scale of that element: the sum of the
    absolute values of the terms it is formed from (face differences and the
    bound-weighted sums of the Jacobian parts cancel, like the residual)."""
    got, ref, scale = (np.asarray(a, dtype=np.float64).ravel() for a in (got, ref, scale))
    if not ref.size:
        return 0.0
    return float(np.max(np.abs(got - ref) / np.maximum(scale, 1e-300)))


@pytest.mark.parametrize("name", sorted(CASES))
def test_flow_jacobian_and_residual_match_oracle(name):
    c = inputs.make_flow_case(**CASES[name])
    m = flux.model_of(c)
    f = StsFlow(c)
    ref = flux.jacobian_blocks(m, c.Lx, c.Ly, c.Q)
    L = f.layout
    for key in ("block_indptr", "block_indices", "d_indptr", "d_indices", "o_indptr", "o_indices",
                "pair_indptr"):
        assert np.array_equal(getattr(L, key), ref[key]), key
    S, U, V = f.jacobian(dev(c.Q))
    for key, got in (("S", S), ("U", U), ("V", V)):
        assert _scaled_err(host(got), ref[key], ref["scales"][key]) <= TOL_RES, key
    R = host(f.residual(dev(c.Q), dev(c.Qn)))
    assert _res_err(R, m, c) <= TOL_RES
    f.close()


def test_flow_full_size_sampled_rows():
    """128 x 128 cells, N = 60: sampled block rows (corners, edges, interior) and
    their residuals against the oracle one row at a time."""
    c = inputs.make_flow_case(128, 128, N=60, w=2, seed=8)
    m = flux.model_of(c)
    f = StsFlow(c)
    S, U, V = (host(t) for t in f.jacobian(dev(c.Q)))
    L = f.layout
    soff = np.zeros(L.block_indices.shape[0] + 1, dtype=np.int64)
    diag = np.repeat(np.arange(128 * 128), np.diff(L.block_indptr)) == L.block_indices
    np.cumsum(np.where(diag, L.d_indices.shape[0], L.o_indices.shape[0]), out=soff[1:])
    rng = np.random.default_rng(9)
    rows = [0, 127, 128 * 127, 128 * 128 - 1, 64, 128 * 64, 128 * 64 + 127] + list(rng.choice(128 * 128, 24))
    for i in rows:
        for k, Sv, Ur, Vr, Sm, Um, Vm in flux.block_row(m, c.Lx, c.Ly, c.Q, int(i)):
            p0, p1 = L.pair_indptr[k], L.pair_indptr[k + 1]
            assert _scaled_err(S[soff[k]:soff[k + 1]], Sv, Sm) <= TOL_RES, (i, k)
            assert _scaled_err(U[p0:p1], Ur, Um) <= TOL_RES, (i, k)
            assert _scaled_err(V[p0:p1], Vr, Vm) <= TOL_RES, (i, k)
    R = host(f.residual(dev(c.Q), dev(c.Qn)))
    assert _res_err(R[rows], m, c, cells=rows) <= TOL_RES
    f.close()


def test_flow_rejects_bad_constants():
    from paper_2403_09198_gb300.binding import StsError
    c = inputs.make_flow_case(3, 2, N=3, w=1, seed=1)
    c.r[1] = -0.1
    with pytest.raises(StsError) as e:
        StsFlow(c)
    assert e.value.status == 1 and "r[1]" in e.value.message


@pytest.mark.parametrize("variant", ["right", "left", "dense"])
def test_newton_step_matches_oracle_root(variant):
    """sts_flow_newton from Q^0 = Q^n (right or left block-Jacobi GMRES, or the
    dense-BSR storage): converges in as many iterations as the oracle's dense
    Newton (+-1), quadratically at the end, to the same root (1e-9 relative,
    both residuals driven to ~1e-13 of the start)."""
    c = inputs.make_flow_case(6, 5, N=5, w=1, seed=12, dt=2.0)
    m = flux.model_of(c)
    Qo, ho = flux.newton(m, c.Lx, c.Ly, c.Qn, c.Qn, rtol=1e-13)
    f = StsFlow(c)
    jac = f.jacobian_handle(dense=variant == "dense")
    Q = dev(c.Qn.copy())
    info, hist = f.newton(jac, Q, dev(c.Qn), rtol=1e-12, gmres_rtol=1e-13, left=variant == "left")
    assert info["converged"] and info["res"] <= 1e-12 * info["res0"]
    assert abs(info["iterations"] - (len(ho) - 1)) <= 1
    assert abs(hist[0] - ho[0]) <= 1e-12 * ho[0]
    r = hist / hist[0]
    k = int(np.argmax(r < 1e-3))
    assert r[k + 1] <= 10 * r[k] ** 2 or r[k + 1] <= 1e-12, r
    Qg = host(Q)
    assert np.linalg.norm(Qg - Qo) <= 1e-9 * np.linalg.norm(Qo)
    jac.close()
    f.close()


def test_newton_full_size():
    """128 x 128 cells, N = 60, Q^0 = Q^n: the driver converges to 1e-10 in a few
    iterations and the returned state has the residual it reports."""
    c = inputs.make_flow_case(128, 128, N=60, w=2, seed=13, dt=0.5)
    f = StsFlow(c)
    jac = f.jacobian_handle()
    Q, Qn = dev(c.Qn.copy()), dev(c.Qn)
    info, hist = f.newton(jac, Q, Qn, rtol=1e-10)
    assert info["converged"] and info["iterations"] <= 8 and np.all(np.diff(hist) < 0)
    import torch
    R = f.residual(Q, Qn)
    assert abs(float(torch.linalg.norm(R)) - info["res"]) <= 1e-6 * info["res"]
    jac.close()
    f.close()


def test_newton_rejects_a_foreign_handle():
    from paper_2403_09198_gb300.binding import StsError, StsJacobian
    c = inputs.make_flow_case(4, 3, N=4, w=1, seed=1)
    f = StsFlow(c)
    w = inputs.make_workload(4, 3, N=4, w=1, r_diag=1, r_off=2, pairs_per_face=2)
    jac = StsJacobian(w, dev(w.S), dev(w.U), dev(w.V), layout="component")
    with pytest.raises(StsError) as e:
        f.newton(jac, dev(c.Q.copy()), dev(c.Qn))
    assert e.value.status == 1 and "layout" in e.value.message
    jac.close()
    f.close()


def test_newton_inexact_forcing():
    """Inexact Newton (Eisenstat-Walker forcing): the same root as the oracle's
    Newton, in fewer GMRES iterations than solving every step to 1e-13."""
    c = inputs.make_flow_case(6, 5, N=5, w=1, seed=12, dt=2.0)
    m = flux.model_of(c)
    Qo, _ = flux.newton(m, c.Lx, c.Ly, c.Qn, c.Qn, rtol=1e-13)
    f = StsFlow(c)
    jac = f.jacobian_handle()
    runs = {}
    for forcing in (False, True):
        Q = dev(c.Qn.copy())
        info, hist = f.newton(jac, Q, dev(c.Qn), rtol=1e-12, gmres_rtol=1e-13, forcing=forcing)
        assert info["converged"] and info["res"] <= 1e-12 * info["res0"] and np.all(np.diff(hist) < 0)
        assert np.linalg.norm(host(Q) - Qo) <= 1e-9 * np.linalg.norm(Qo)
        runs[forcing] = info
    assert runs[True]["linear_iterations"] < runs[False]["linear_iterations"]
    jac.close()
    f.close()
