"""Pins of the HLL-flux oracle (``oracle/flux.py``) against things other than itself.

The derivatives the oracle assembles by hand (Eqs. r1_flux_left / r1_flux_right,
the sound-speed gradient, the source Jacobian, the block assembly of dR/dQ) are
checked against complex-step derivatives of the oracle's own flux, source and
residual functions: Im f(q + i h e_j) / h equals df/dq e_j to rounding for
h = 1e-30, by a route that shares none of the hand-derived formulas.  The flux
itself is checked against textbook HLL properties and a single-species closed
form.
"""
import numpy as np
import pytest

import oracle
from oracle import flux
from paper_2403_09198_gb300 import inputs

H = 1e-30


def _cs_jacobian(f, q):
    """Complex-step Jacobian of f at the real point q."""
    cols = []
    for j in range(q.shape[0]):
        qc = q.astype(np.complex128)
        qc[j] += 1j * H
        cols.append(np.imag(f(qc)) / H)
    return np.stack(cols, axis=1)


def _close(a, b, tol=1e-12):
    scale = max(np.abs(b).max(), 1e-300)
    assert np.abs(a - b).max() <= tol * scale, np.abs(a - b).max() / scale


def _case(mach=0.4, seed=1, N=5, w=1):
    c = inputs.make_flow_case(4, 3, N=N, w=w, seed=seed, mach=mach)
    return c, flux.model_of(c)


FACES = [(0, 1), (1, 0), (0, 4), (5, 1), (6, 7), (10, 6)]


@pytest.mark.parametrize("mach", [0.4, 2.5])
def test_hll_jacobian_parts_equal_complex_step(mach):
    """A_L = A0_L + u1 v1L^T + u2 v2L^T and A_R likewise (Section 4.1) against the
    complex-step Jacobian of Eq. HLL_flux, subsonic and supersonic."""
    c, m = _case(mach=mach)
    seen = set()
    for i, j in FACES:
        n = flux.face_normal(c.Lx, i, j)
        qL, qR = c.Q[i], c.Q[j]
        seen.add(flux.wave_speeds(m, qL, qR, n)[2:])
        A0L, A0R, u1, v1L, v1R, u2, v2L, v2R = flux.hll_parts(m, qL, qR, n)
        JL = _cs_jacobian(lambda q: flux.hll_flux(m, q, qR, n), qL)
        JR = _cs_jacobian(lambda q: flux.hll_flux(m, qL, q, n), qR)
        _close(A0L + np.outer(u1, v1L) + np.outer(u2, v2L), JL)
        _close(A0R + np.outer(u1, v1R) + np.outer(u2, v2R), JR)
    if mach < 1:
        assert {(1, 2), (2, 1)} <= seen or {(1, 1), (2, 2)} <= seen, seen
    else:
        assert any(0 in s for s in seen), seen       # clipped bounds on supersonic faces


def test_sparse_part_has_the_flux_pattern():
    """A0_L and A0_R vanish outside the neighbour-block pattern of Section 4.1
    (level rows: diagonal and the flow columns; flow rows dense), checked on the
    complex-step Jacobian minus the two rank-one pairs."""
    c, m = _case()
    op, oi = inputs.off_pattern(m.N)
    mask = np.zeros((m.b, m.b), dtype=bool)
    for p in range(m.b):
        mask[p, oi[op[p]:op[p + 1]]] = True
    for i, j in FACES[:3]:
        n = flux.face_normal(c.Lx, i, j)
        _, _, u1, v1L, _, u2, v2L, _ = flux.hll_parts(m, c.Q[i], c.Q[j], n)
        JL = _cs_jacobian(lambda q: flux.hll_flux(m, q, c.Q[j], n), c.Q[i])
        rest = JL - np.outer(u1, v1L) - np.outer(u2, v2L)
        assert np.abs(rest[~mask]).max() <= 1e-13 * np.abs(JL).max()


def test_hll_consistency_conservation_and_compact_form():
    """f(q, q, n) = f_n(q); f(qL, qR, n) = -f(qR, qL, -n); Eq. HLL_flux_compact."""
    c, m = _case()
    for i, j in FACES:
        n = flux.face_normal(c.Lx, i, j)
        qL, qR = c.Q[i], c.Q[j]
        _close(flux.hll_flux(m, qL, qL, n), flux.normal_flux(m, qL, n), 1e-14)
        _close(flux.hll_flux(m, qL, qR, n), -flux.hll_flux(m, qR, qL, (-n[0], -n[1])), 1e-14)
        sL, sR, _, _ = flux.wave_speeds(m, qL, qR, n)
        af, cf = 0.5 * (sL + sR) / (sR - sL), sL * sR / (sR - sL)
        fL, fR = flux.normal_flux(m, qL, n), flux.normal_flux(m, qR, n)
        compact = 0.5 * (fL + fR) - af * (fR - fL) + cf * (flux.conserved(m, qR) - flux.conserved(m, qL))
        _close(flux.hll_flux(m, qL, qR, n), compact, 1e-14)


def test_supersonic_face_is_upwind():
    """With both bounds on one side of zero the flux is the upwind flux and the
    rank-one parts vanish (a_f = +-1/2, c_f = 0 and their gradients are zero)."""
    c, m = _case(mach=2.5)
    qL, qR, n = c.Q[0], c.Q[1], (1.0, 0.0)
    sL, sR, iL, _ = flux.wave_speeds(m, qL, qR, n)
    assert iL == 0 and sL == 0.0
    _close(flux.hll_flux(m, qL, qR, n), flux.normal_flux(m, qL, n), 1e-15)
    A0L, A0R, u1, v1L, v1R, u2, v2L, v2R = flux.hll_parts(m, qL, qR, n)
    for v in (v1L, v1R, v2L, v2R):
        assert np.abs(v).max() == 0.0
    _close(A0L, flux.jac_An(m, qL, n), 1e-15)
    assert np.abs(A0R).max() == 0.0


def test_single_species_sound_speed_closed_form():
    """N = 1: a = sqrt(gamma r T) with gamma = (c_v + r) / c_v (Section 2.1)."""
    c, m = _case(N=1, w=0)
    for q in c.Q[:4]:
        gam = (m.cv[0] + m.r[0]) / m.cv[0]
        assert abs(flux.sound_speed(m, q) - np.sqrt(gam * m.r[0] * q[3])) <= 1e-15
        _close(flux.grad_a(m, q), _cs_jacobian(lambda x: np.atleast_1d(flux.sound_speed(m, x)), q)[0])


def test_source_jacobian_is_band_plus_rank_one():
    c, m = _case(w=2)
    for q in c.Q[:3]:
        G0, wse, gw = flux.source_parts(m, q)
        _close(G0 + np.outer(wse, gw), _cs_jacobian(lambda x: flux.source(m, x), q))


def test_residual_jacobian_assembly():
    """The BR1-BSR blocks of dR/dQ (oracle matvec on unit vectors) equal the
    complex-step Jacobian of the whole residual on a 3 x 2 mesh; the pair counts
    are 1 + 2 per face on diagonal blocks and 2 on neighbour blocks."""
    c = inputs.make_flow_case(3, 2, N=3, w=1, seed=4)
    m = flux.model_of(c)
    d = flux.jacobian_blocks(m, c.Lx, c.Ly, c.Q)
    d.pop("scales")
    J = oracle.Jacobian(n_cells=c.n_cells, b=m.b, **d)
    n = c.n_cells * m.b
    D = np.stack([oracle.matvec(J, np.eye(n)[k]) for k in range(n)], axis=1)
    Jcs = _cs_jacobian(lambda x: flux.residual(m, c.Lx, c.Ly, x.reshape(c.n_cells, m.b), c.Qn).ravel(),
                       c.Q.ravel())
    _close(D, Jcs)
    ref = inputs.make_workload(3, 2, N=3, w=1, r_diag=1, r_off=2, pairs_per_face=2)
    assert np.array_equal(d["pair_indptr"], ref.pair_indptr)
    assert d["S"].shape[0] == ref.S.shape[0]


def test_newton_converges_quadratically_to_a_root():
    """The oracle's Newton iteration reaches R(Q) = 0 to rounding from Q^0 = Q^n, and
    its last steps shrink ||R|| quadratically (r_{k+1} <= C r_k^2), the signature of
    an exact Jacobian."""
    c = inputs.make_flow_case(4, 3, N=4, w=1, seed=11, dt=0.5)
    m = flux.model_of(c)
    Q, hist = flux.newton(m, c.Lx, c.Ly, c.Qn, c.Qn, rtol=1e-13)
    assert hist[-1] <= 1e-13 * hist[0] and len(hist) <= 8
    r = np.array(hist) / hist[0]
    k = int(np.argmax(r < 1e-3))
    assert r[k + 1] <= 10 * r[k] ** 2 or r[k + 1] <= 1e-13, r


# ---------------------------------------------------------------- the Euler flux itself
# conserved() and normal_flux() (Section 2.1 model, the f_n that Eq. HLL_flux wraps)
# against forms written here from the textbook statement of the Euler equations,
# not from the oracle: a calorically perfect gas in (rho, u, v, p), with the total
# energy from gamma = (c_v + r) / c_v, and the exact rotational symmetry of the flux.


def _model(N, r, cv, e0):
    z = np.zeros(N)
    return flux.FluxModel(N=N, w=0, r=np.asarray(r, float), cv=np.asarray(cv, float),
                          e0=np.asarray(e0, float), beta=z, ws=z, K=np.zeros((N, 1)), A=0.0,
                          theta=1.0, dt=1.0)


def _euler_textbook(rho, u, v, p, n, gamma, rho_e0):
    """Single-gas Euler state and normal flux from (rho, u, v, p): total energy
    E = p / (gamma - 1) + rho e0 + rho |u|^2 / 2; F.n = (rho u_n, rho u u_n + p n_x,
    rho v u_n + p n_y, (E + p) u_n)."""
    E = p / (gamma - 1.0) + rho_e0 + 0.5 * rho * (u * u + v * v)
    un = u * n[0] + v * n[1]
    U = np.array([rho, rho * u, rho * v, E])
    F = np.array([rho * un, rho * u * un + p * n[0], rho * v * un + p * n[1], (E + p) * un])
    return U, F


NORMALS = [(1.0, 0.0), (0.0, 1.0), (-1.0, 0.0), (0.6, -0.8), (-0.28, 0.96)]
STATES = [(1.3, 0.4, -0.2, 0.9), (0.7, -1.1, 0.5, 2.2), (2.0, 0.0, 0.0, 1.0), (0.9, 2.7, 1.9, 0.6)]


def _textbook_gap(nf, cons, N=1):
    """Largest relative gap of (conserved, normal_flux) against the textbook Euler
    state and flux over single-gas states (N = 1) or a mixture of N species with
    one gas's constants (an effective single species of density sum rho_k)."""
    r, cv, e0 = 0.287, 0.718, 0.05
    m = _model(N, [r] * N, [cv] * N, [e0] * N)
    gamma = (cv + r) / cv
    frac = np.arange(1, N + 1, dtype=float)
    frac /= frac.sum()
    worst = 0.0
    for rho, u, v, T in STATES:
        q = np.concatenate([rho * frac, [u, v, T]])
        p = rho * r * T
        for n in NORMALS:
            U, F = _euler_textbook(rho, u, v, p, n, gamma, rho * e0)
            un = u * n[0] + v * n[1]
            Ug = np.concatenate([rho * frac, U[1:]])
            Fg = np.concatenate([rho * frac * un, F[1:]])
            for got, ref in ((cons(m, q), Ug), (nf(m, q, n), Fg)):
                worst = max(worst, float(np.abs(got - ref).max() / np.abs(ref).max()))
    return worst


@pytest.mark.parametrize("N", [1, 4])
def test_euler_flux_matches_textbook_single_gas(N):
    """N = 1, and N species that share one gas's constants (the mixture collapses
    to one effective species): the oracle's conserved variables and normal flux
    equal the textbook Euler ones to rounding, for normals along and off the axes."""
    assert _textbook_gap(flux.normal_flux, flux.conserved, N) <= 1e-14


def test_euler_flux_rotational_invariance():
    """f(q, n) = R(n)^T f(R(n) q, e_x) for a mixture with distinct species constants:
    rotating the velocity into the face frame, taking the x-direction flux and
    rotating the momentum flux back gives the flux through the face."""
    c, m = _case(N=5, w=1)
    for q in c.Q[:6]:
        N = m.N
        for n in NORMALS:
            u, v = q[N], q[N + 1]
            qr = q.copy()
            qr[N], qr[N + 1] = u * n[0] + v * n[1], -u * n[1] + v * n[0]
            fr = flux.normal_flux(m, qr, (1.0, 0.0))
            back = fr.copy()
            back[N] = n[0] * fr[N] - n[1] * fr[N + 1]
            back[N + 1] = n[1] * fr[N] + n[0] * fr[N + 1]
            _close(flux.normal_flux(m, q, n), back, 1e-14)


def test_mixture_flux_is_additive_over_identical_species():
    """Splitting each species into two copies with the same constants and half
    the density leaves the momentum and energy fluxes and the conserved momentum
    and energy unchanged, and each species flux halves (Dalton's law and the
    mass-weighted energy of Section 2.1)."""
    c, m = _case(N=3, w=1)
    m2 = _model(6, np.repeat(m.r, 2), np.repeat(m.cv, 2), np.repeat(m.e0, 2))
    for q in c.Q[:4]:
        N = m.N
        q2 = np.concatenate([np.repeat(q[:N] / 2, 2), q[N:]])
        for n in NORMALS[:3]:
            f1, f2 = flux.normal_flux(m, q, n), flux.normal_flux(m2, q2, n)
            _close(f2[2 * N:], f1[N:], 1e-14)
            _close(f2[:2 * N].reshape(N, 2).sum(axis=1), f1[:N], 1e-14)
        _close(flux.conserved(m2, q2)[2 * N:], flux.conserved(m, q)[N:], 1e-14)


# ---------------------------------------------------------------- planted mistakes
# Each plants one plausible mistake in the oracle (on the CPU, through monkeypatch)
# and checks that the pin it should trip reports it: the pins above are not
# blind to these.


def _parts_error(m, c):
    """Largest relative gap between the oracle's Jacobian parts and the complex
    step, over the faces of FACES."""
    worst = 0.0
    for i, j in FACES:
        n = flux.face_normal(c.Lx, i, j)
        qL, qR = c.Q[i], c.Q[j]
        A0L, A0R, u1, v1L, v1R, u2, v2L, v2R = flux.hll_parts(m, qL, qR, n)
        JL = _cs_jacobian(lambda q: flux.hll_flux(m, q, qR, n), qL)
        JR = _cs_jacobian(lambda q: flux.hll_flux(m, qL, q, n), qR)
        for got, ref in ((A0L + np.outer(u1, v1L) + np.outer(u2, v2L), JL),
                         (A0R + np.outer(u1, v1R) + np.outer(u2, v2R), JR)):
            worst = max(worst, float(np.abs(got - ref).max() / np.abs(ref).max()))
    return worst


def test_planted_sound_speed_gradient_mistake_is_caught(monkeypatch):
    c, m = _case()
    assert _parts_error(m, c) <= 1e-12
    real = flux.grad_a

    def wrong(m_, q):                       # a 1% error in the species components
        g = real(m_, q)
        g[:m_.N] *= 1.01
        return g
    monkeypatch.setattr(flux, "grad_a", wrong)
    assert _parts_error(m, c) > 1e-6


def test_planted_wave_speed_weight_sign_is_caught(monkeypatch):
    c, m = _case()
    real = flux.jac_H
    monkeypatch.setattr(flux, "jac_H", lambda m_, q: -real(m_, q))   # -c_f H -> +c_f H
    assert _parts_error(m, c) > 1e-6


def test_planted_source_band_sign_is_caught(monkeypatch):
    c, m = _case(w=2)
    real = flux.source_parts

    def wrong(m_, q):
        G0, wse, gw = real(m_, q)
        return -G0, wse, gw
    monkeypatch.setattr(flux, "source_parts", wrong)
    q = c.Q[0]
    G0, wse, gw = flux.source_parts(m, q)
    err = np.abs(G0 + np.outer(wse, gw) - _cs_jacobian(lambda x: flux.source(m, x), q)).max()
    assert err > 1e-6


def test_planted_assembly_mistake_is_caught(monkeypatch):
    """A neighbour block built from the left-state gradients (v1L, v2L) instead of
    the right-state ones fails the whole-residual complex-step pin."""
    c = inputs.make_flow_case(3, 2, N=3, w=1, seed=4)
    m = flux.model_of(c)
    real = flux.hll_parts

    def wrong(m_, qL, qR, n):
        A0L, A0R, u1, v1L, v1R, u2, v2L, v2R = real(m_, qL, qR, n)
        return A0L, A0R, u1, v1L, v1L, u2, v2L, v2L
    monkeypatch.setattr(flux, "hll_parts", wrong)
    d = flux.jacobian_blocks(m, c.Lx, c.Ly, c.Q)
    d.pop("scales")
    J = oracle.Jacobian(n_cells=c.n_cells, b=m.b, **d)
    n = c.n_cells * m.b
    D = np.stack([oracle.matvec(J, np.eye(n)[k]) for k in range(n)], axis=1)
    Jcs = _cs_jacobian(lambda x: flux.residual(m, c.Lx, c.Ly, x.reshape(c.n_cells, m.b), c.Qn).ravel(),
                       c.Q.ravel())
    assert np.abs(D - Jcs).max() > 1e-6 * np.abs(Jcs).max()


def test_planted_pressure_term_mistake_is_caught(monkeypatch):
    """An x-momentum flux without its pressure term p n_x fails the textbook pin."""
    real = flux.normal_flux

    def wrong(m_, q, n):
        f = real(m_, q, n)
        T = q[m_.N + 2]
        f[m_.N] -= (q[:m_.N] * m_.r).sum() * T * n[0]
        return f
    assert _textbook_gap(real, flux.conserved) <= 1e-14
    monkeypatch.setattr(flux, "normal_flux", wrong)
    assert _textbook_gap(flux.normal_flux, flux.conserved) > 1e-3


def test_planted_energy_mistake_is_caught(monkeypatch):
    """A total energy without the kinetic part fails the textbook pin."""
    real = flux.conserved

    def wrong(m_, q):
        U = real(m_, q)
        N = m_.N
        U[N + 2] -= 0.5 * q[:N].sum() * (q[N] ** 2 + q[N + 1] ** 2)
        return U
    monkeypatch.setattr(flux, "conserved", wrong)
    assert _textbook_gap(flux.normal_flux, flux.conserved) > 1e-3
