"""Planted mistakes in the FP64 oracle (on the CPU, through monkeypatch) must trip
the pins of tests/test_oracle_pins.py: each test repeats the core comparison of
one pin with one mistake planted and checks that it fails clearly.  (The
transposed-operand mistake u v^T -> v u^T is checked inside the Section 5.1
worked-example pin itself.)"""
import sys

import numpy as np

import oracle
from paper_2403_09198_gb300 import inputs


def _tiny(**kw):
    base = dict(Lx=3, Ly=2, N=3, w=1, r_diag=2, r_off=1, seed=7)
    base.update(kw)
    return inputs.make_workload(base.pop("Lx"), base.pop("Ly"), **base)


def _dense_of(J, trans=False):
    return np.stack([oracle.matvec(J, np.eye(J.n)[k], trans=trans) for k in range(J.n)], axis=1)


def test_planted_transposed_solve_mistake_is_caught(monkeypatch):
    """A block-Jacobi apply that ignores trans fails the 1x1-mesh numpy pin."""
    wl = _tiny(Lx=1, Ly=1, N=6, w=2)
    J = oracle.Jacobian.from_workload(wl)
    F = oracle.bj_setup(J)
    x = np.random.default_rng(8).standard_normal(wl.n)
    D = _dense_of(J)
    real = oracle.bj_apply
    monkeypatch.setattr(oracle, "bj_apply", lambda F_, v, trans=False: real(F_, v, trans=False))
    zt = oracle.bj_apply(F, x, trans=True)
    ref = np.linalg.solve(D.T, x)
    assert np.abs(zt - ref).max() > 1e-6 * np.abs(ref).max()


def test_planted_preconditioner_mix_up_is_caught(monkeypatch):
    """GMRES that applies M^T instead of M (a transposed-solve mix-up in the
    preconditioner) still solves the system, but its rotated residuals leave the
    explicit (A M)-Krylov least-squares values the pin compares with."""
    wl = _tiny(Lx=3, Ly=2, N=3, w=1, seed=16, dt=1.0)
    J = oracle.Jacobian.from_workload(wl)
    F = oracle.bj_setup(J)
    A = _dense_of(J)
    Mop = np.stack([oracle.bj_apply(F, e) for e in np.eye(wl.n)], axis=1)
    gm = sys.modules["oracle.gmres"]
    real = gm.bj_apply
    monkeypatch.setattr(gm, "bj_apply", lambda F_, v, trans=False: real(F_, v, trans=not trans))
    _, info = oracle.gmres(J, wl.rhs, restart=40, rtol=1e-13, max_iters=4, factors=F)
    hist = np.array(info["history"])
    AM, K, worst = A @ Mop, [wl.rhs], 0.0
    for k in range(1, len(hist) + 1):
        Kk = np.stack(K, axis=1)
        y, *_ = np.linalg.lstsq(AM @ Kk, wl.rhs, rcond=None)
        res = np.linalg.norm(wl.rhs - AM @ Kk @ y) / np.linalg.norm(wl.rhs)
        worst = max(worst, abs(res - hist[k - 1]) / max(res, 1e-14))
        K.append(AM @ K[-1])
    assert worst > 1e-6


def test_planted_gradient_sign_is_caught(monkeypatch):
    """An S gradient with the wrong sign fails the central-difference pin."""
    wl = _tiny(Lx=2, Ly=2, N=2, w=1, seed=21, dt=0.2)
    J = oracle.Jacobian.from_workload(wl)
    adj = sys.modules["oracle.adjoint"]
    real = adj.grad

    def wrong(J_, lam, x):
        gS, gU, gV = real(J_, lam, x)
        return -gS, gU, gV
    monkeypatch.setattr(adj, "grad", wrong)
    res = oracle.adjoint(J, wl.rhs, wl.W)
    d = np.random.default_rng(22).standard_normal(wl.S.shape)
    d /= np.linalg.norm(d)
    h = 1e-6

    def L_at(t):
        Jt = oracle.Jacobian.from_workload(wl, S=wl.S + t * d)
        x, _ = oracle.gmres(Jt, wl.rhs, restart=30, rtol=1e-15, max_iters=300)
        return 0.5 * float(np.dot(wl.W * x, wl.W * x))

    fd = (L_at(h) - L_at(-h)) / (2 * h)
    gd = float(np.dot(res["gS"], d))
    assert abs(gd - fd) > 1e-3 * abs(fd)
