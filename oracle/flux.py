"""Plain FP64 HLL flux, its r1-sparse Jacobian parts, and the first-order
finite-volume residual of a toy N-species flow model (test infrastructure only).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may use this module.  It shares no code with the CUDA
library.  Every function accepts complex states as well, so that tests can
differentiate it by the complex step (f(q + i h e) has imaginary part h f'(q) e
up to O(h^2), free of cancellation) as an independent check of the derivatives.

Model (Section 2.1, with synthetic constants):
  q = (rho_0 .. rho_{N-1}, u, v, T)          primitive variables, b = N + 3
  rho = sum rho_k,  p = sum rho_k r_k T,      e_k(T) = e0_k + cv_k T
  rho e = sum rho_k e_k,  rho e_tot = rho e + rho (u^2 + v^2) / 2
  c_v = sum Y_k cv_k,  r = sum Y_k r_k,  gamma = (c_v + r) / c_v,  a = sqrt(gamma r T)
  u(q)   = (rho_k, rho u, rho v, rho e_tot)                       conserved variables
  f_n(q) = (rho_k u_n, rho u u_n + p n_x, rho v u_n + p n_y, (rho e_tot + p) u_n)
Flux (Section 3.2, Eq. HLL_flux): f = (s_R f_L - s_L f_R + s_L s_R (u_R - u_L)) / (s_R - s_L)
with the wave-speed bounds s_L = min(0, u_nL - a_L, u_nR - a_R), s_R = max(0, u_nL + a_L,
u_nR + a_R); ties go to the first candidate in that order.
Jacobian parts (Section 4.1, Eqs. r1_flux_left / r1_flux_right):
  A_L = A0_L - (f_R - f_L) (d a_f / d q_L)^T + (u_R - u_L) (d c_f / d q_L)^T
  A_R = A0_R - (f_R - f_L) (d a_f / d q_R)^T + (u_R - u_L) (d c_f / d q_R)^T
  A0_L = (1/2 + a_f) A_n(q_L) - c_f H(q_L),  A0_R = (1/2 - a_f) A_n(q_R) + c_f H(q_R)
  a_f = (s_L + s_R) / (2 (s_R - s_L)),  c_f = s_L s_R / (s_R - s_L)
Source (Section 2.2 shape: level rows only): Omega_k = -sum_{|l-k|<=w} K_kl rho_l + ws_k omega,
omega = A exp(-theta / T) sum beta_k rho_k; its Jacobian is the band -K plus the rank-one
ws (d omega / d q)^T (Section 4.2: source contributions grouped into a rank-one term).
Residual (Section 3.3, Eq. system_residual, unit cells and faces, outward normals):
  R_i = u(q_i) - u(q_i^n) + dt (sum_{faces} f(q_i, q_j, n_ij) - Omega(q_i))
"""
from __future__ import annotations

import dataclasses
import functools

import numpy as np


@dataclasses.dataclass
class FluxModel:
    """Constants of the toy model; arrays are float64 of length N, K is [N][2w+1]."""

    N: int
    w: int
    r: np.ndarray
    cv: np.ndarray
    e0: np.ndarray
    beta: np.ndarray
    ws: np.ndarray
    K: np.ndarray
    A: float
    theta: float
    dt: float

    @property
    def b(self) -> int:
        return self.N + 3


def _mix(m: FluxModel, q):
    N = m.N
    rho_k = q[:N]
    u, v, T = q[N], q[N + 1], q[N + 2]
    rho = rho_k.sum()
    Rt = (rho_k * m.r).sum()
    Ct = (rho_k * m.cv).sum()
    E0 = (rho_k * m.e0).sum()
    ke = 0.5 * (u * u + v * v)
    p = Rt * T
    rhoetot = E0 + Ct * T + rho * ke
    g = (Ct + Rt) * Rt / (rho * Ct)
    a = np.sqrt(g * T)
    return dict(rho_k=rho_k, u=u, v=v, T=T, rho=rho, Rt=Rt, Ct=Ct, E0=E0, ke=ke, p=p,
                rhoetot=rhoetot, g=g, a=a)


def conserved(m: FluxModel, q):
    s = _mix(m, q)
    return np.concatenate([s["rho_k"], [s["rho"] * s["u"], s["rho"] * s["v"], s["rhoetot"]]])


def normal_flux(m: FluxModel, q, n):
    s = _mix(m, q)
    un = n[0] * s["u"] + n[1] * s["v"]
    return np.concatenate([s["rho_k"] * un,
                           [s["rho"] * s["u"] * un + s["p"] * n[0],
                            s["rho"] * s["v"] * un + s["p"] * n[1],
                            (s["rhoetot"] + s["p"]) * un]])


def sound_speed(m: FluxModel, q):
    return _mix(m, q)["a"]


def jac_H(m: FluxModel, q) -> np.ndarray:
    """H = d u / d q (dense b x b)."""
    N, b = m.N, m.b
    s = _mix(m, q)
    H = np.zeros((b, b), dtype=np.result_type(q, np.float64))
    H[:N, :N] = np.eye(N)
    H[N, :N] = s["u"]
    H[N, N] = s["rho"]
    H[N + 1, :N] = s["v"]
    H[N + 1, N + 1] = s["rho"]
    H[N + 2, :N] = m.e0 + m.cv * s["T"] + s["ke"]
    H[N + 2, N] = s["rho"] * s["u"]
    H[N + 2, N + 1] = s["rho"] * s["v"]
    H[N + 2, N + 2] = s["Ct"]
    return H


def jac_An(m: FluxModel, q, n) -> np.ndarray:
    """A_n = d f_n / d q (dense b x b)."""
    N, b = m.N, m.b
    s = _mix(m, q)
    u, v, T, rho = s["u"], s["v"], s["T"], s["rho"]
    un = n[0] * u + n[1] * v
    A = np.zeros((b, b), dtype=np.result_type(q, np.float64))
    for k in range(N):
        A[k, k] = un
        A[k, N] = s["rho_k"][k] * n[0]
        A[k, N + 1] = s["rho_k"][k] * n[1]
    A[N, :N] = u * un + m.r * T * n[0]
    A[N, N] = rho * un + rho * u * n[0]
    A[N, N + 1] = rho * u * n[1]
    A[N, N + 2] = s["Rt"] * n[0]
    A[N + 1, :N] = v * un + m.r * T * n[1]
    A[N + 1, N] = rho * v * n[0]
    A[N + 1, N + 1] = rho * un + rho * v * n[1]
    A[N + 1, N + 2] = s["Rt"] * n[1]
    A[N + 2, :N] = (m.e0 + m.cv * T + s["ke"] + m.r * T) * un
    A[N + 2, N] = rho * u * un + (s["rhoetot"] + s["p"]) * n[0]
    A[N + 2, N + 1] = rho * v * un + (s["rhoetot"] + s["p"]) * n[1]
    A[N + 2, N + 2] = (s["Ct"] + s["Rt"]) * un
    return A


def grad_a(m: FluxModel, q):
    """d a / d q, from a^2 = T g(rho_k), g = (C + R) R / (rho C), C = sum rho_k cv_k, R = sum rho_k r_k."""
    N = m.N
    s = _mix(m, q)
    Rt, Ct, rho, g, a, T = s["Rt"], s["Ct"], s["rho"], s["g"], s["a"], s["T"]
    d = rho * Ct
    dn = (m.cv + m.r) * Rt + (Ct + Rt) * m.r
    dd = Ct + rho * m.cv
    out = np.zeros(m.b, dtype=np.result_type(q, np.float64))
    out[:N] = T / (2 * a) * (dn - g * dd) / d
    out[N + 2] = a / (2 * T)
    return out


def grad_un(m: FluxModel, n):
    out = np.zeros(m.b)
    out[m.N] = n[0]
    out[m.N + 1] = n[1]
    return out


def _pick(cands, smallest: bool):
    """Index and value of the smallest (largest) candidate by real part; ties to the first."""
    best = 0
    for i in range(1, len(cands)):
        if (np.real(cands[i]) < np.real(cands[best])) if smallest else (np.real(cands[i]) > np.real(cands[best])):
            best = i
    return best, cands[best]


def wave_speeds(m: FluxModel, qL, qR, n):
    sl, sr = _mix(m, qL), _mix(m, qR)
    unL = n[0] * sl["u"] + n[1] * sl["v"]
    unR = n[0] * sr["u"] + n[1] * sr["v"]
    iL, sL = _pick([0.0 * unL, unL - sl["a"], unR - sr["a"]], True)
    iR, sR = _pick([0.0 * unL, unL + sl["a"], unR + sr["a"]], False)
    return sL, sR, iL, iR


def hll_flux(m: FluxModel, qL, qR, n):
    """Eq. HLL_flux."""
    sL, sR, _, _ = wave_speeds(m, qL, qR, n)
    fL, fR = normal_flux(m, qL, n), normal_flux(m, qR, n)
    uL, uR = conserved(m, qL), conserved(m, qR)
    return (sR * fL - sL * fR + sL * sR * (uR - uL)) / (sR - sL)


def hll_parts(m: FluxModel, qL, qR, n):
    """Eqs. r1_flux_left / r1_flux_right: (A0_L, A0_R, u1, v1L, v1R, u2, v2L, v2R) with
    A_L = A0_L + u1 v1L^T + u2 v2L^T and A_R = A0_R + u1 v1R^T + u2 v2R^T."""
    sL, sR, iL, iR = wave_speeds(m, qL, qR, n)
    den = sR - sL
    af = 0.5 * (sL + sR) / den
    cf = sL * sR / den
    gun = grad_un(m, n)
    dsL = [np.zeros(m.b), np.zeros(m.b)]          # d s_L / d q_L, d s_L / d q_R
    dsR = [np.zeros(m.b), np.zeros(m.b)]
    if iL == 1:
        dsL[0] = gun - grad_a(m, qL)
    elif iL == 2:
        dsL[1] = gun - grad_a(m, qR)
    if iR == 1:
        dsR[0] = gun + grad_a(m, qL)
    elif iR == 2:
        dsR[1] = gun + grad_a(m, qR)
    daf = [(sR * dsL[x] - sL * dsR[x]) / den ** 2 for x in range(2)]
    dcf = [(sR * sR * dsL[x] - sL * sL * dsR[x]) / den ** 2 for x in range(2)]
    A0L = (0.5 + af) * jac_An(m, qL, n) - cf * jac_H(m, qL)
    A0R = (0.5 - af) * jac_An(m, qR, n) + cf * jac_H(m, qR)
    u1 = -(normal_flux(m, qR, n) - normal_flux(m, qL, n))
    u2 = conserved(m, qR) - conserved(m, qL)
    return A0L, A0R, u1, daf[0], daf[1], u2, dcf[0], dcf[1]


def source(m: FluxModel, q):
    N = m.N
    s = _mix(m, q)
    rho_k = s["rho_k"]
    omega = m.A * np.exp(-m.theta / s["T"]) * (m.beta * rho_k).sum()
    out = np.zeros(m.b, dtype=np.result_type(q, np.float64))
    for k in range(N):
        for l in range(max(0, k - m.w), min(N, k + m.w + 1)):
            out[k] -= m.K[k, l - k + m.w] * rho_k[l]
        out[k] += m.ws[k] * omega
    return out


def source_parts(m: FluxModel, q):
    """(G0, ws_ext, grad_omega) with d Omega / d q = G0 + ws_ext grad_omega^T."""
    N, b = m.N, m.b
    s = _mix(m, q)
    G0 = np.zeros((b, b))
    for k in range(N):
        for l in range(max(0, k - m.w), min(N, k + m.w + 1)):
            G0[k, l] = -m.K[k, l - k + m.w]
    kap = m.A * np.exp(-m.theta / s["T"])
    gw = np.zeros(b, dtype=np.result_type(q, np.float64))
    gw[:N] = kap * m.beta
    gw[N + 2] = kap * m.theta / s["T"] ** 2 * (m.beta * s["rho_k"]).sum()
    return G0, np.concatenate([m.ws, np.zeros(3)]), gw


def face_normal(Lx: int, i: int, j: int):
    """Outward unit normal of cell i towards its face neighbour j on the quad grid."""
    d = j - i
    return {1: (1.0, 0.0), -1: (-1.0, 0.0), Lx: (0.0, 1.0), -Lx: (0.0, -1.0)}[d]


def residual_rows(m: FluxModel, Lx: int, Ly: int, Q, Qn, rows):
    """Eq. system_residual for the cells ``rows``, and per element the sum of the
    absolute values of its terms (|u(q)| + |u(q^n)| + dt (sum |f| + |Omega|)), the
    scale of its rounding error: R cancels (q^n close to q, face fluxes of
    opposite sides), so its error is a few ulps of those terms, not of R."""
    from paper_2403_09198_gb300.inputs import mesh_adjacency
    bptr, bidx = mesh_adjacency(Lx, Ly)
    dtype = np.result_type(Q, np.float64)
    R = np.zeros((len(rows), m.b), dtype=dtype)
    mag = np.zeros((len(rows), m.b))
    for s_, i in enumerate(rows):
        uq, un, src = conserved(m, Q[i]), conserved(m, Qn[i]), source(m, Q[i])
        fsum = np.zeros(m.b, dtype=dtype)
        fabs = np.zeros(m.b)
        for k in range(bptr[i], bptr[i + 1]):
            j = int(bidx[k])
            if j != i:
                fj = hll_flux(m, Q[i], Q[j], face_normal(Lx, i, j))
                fsum = fsum + fj
                fabs = fabs + np.abs(np.real(fj))
        R[s_] = (uq - un) + m.dt * (fsum - src)
        mag[s_] = np.abs(np.real(uq)) + np.abs(np.real(un)) + m.dt * (fabs + np.abs(np.real(src)))
    return R, mag


def residual(m: FluxModel, Lx: int, Ly: int, Q, Qn):
    """Eq. system_residual for every cell; Q, Qn are [nc][b] (Q may be complex)."""
    return residual_rows(m, Lx, Ly, Q, Qn, range(Lx * Ly))[0]


@functools.lru_cache(maxsize=8)
def _layout_of(N: int, w: int, Lx: int, Ly: int):
    from paper_2403_09198_gb300.inputs import diag_pattern, mesh_adjacency, off_pattern
    bptr, bidx = mesh_adjacency(Lx, Ly)
    dp, di = diag_pattern(N, w)
    op, oi = off_pattern(N)
    return bptr, bidx, dp, di, op, oi


def _layout(m: FluxModel, Lx: int, Ly: int):
    """Block CSR of the grid and the two block patterns (shared, read-only arrays)."""
    return _layout_of(m.N, m.w, Lx, Ly)


def _grad_a_mag(m: FluxModel, q):
    """|terms| bound of grad_a: T / (2a) (|dn| + |g dd|) / d for the species, |a / 2T| for T."""
    N = m.N
    s = _mix(m, q)
    d = s["rho"] * s["Ct"]
    dn = (m.cv + m.r) * s["Rt"] + (s["Ct"] + s["Rt"]) * m.r
    dd = s["Ct"] + s["rho"] * m.cv
    out = np.zeros(m.b)
    out[:N] = s["T"] / (2 * s["a"]) * (np.abs(dn) + np.abs(s["g"] * dd)) / d
    out[N + 2] = s["a"] / (2 * s["T"])
    return out


def _parts_mag(m: FluxModel, qL, qR, n):
    """Scales of the rounding error of hll_parts: the absolute values of the terms
    each result combines (the face differences and the bound-weighted sums cancel)."""
    sL, sR, iL, iR = wave_speeds(m, qL, qR, n)
    den2 = (sR - sL) ** 2
    af = 0.5 * (sL + sR) / (sR - sL)
    cf = sL * sR / (sR - sL)
    gun = np.abs(grad_un(m, n))
    gaL, gaR = _grad_a_mag(m, qL), _grad_a_mag(m, qR)
    z = np.zeros(m.b)
    dsL = [gun + gaL if iL == 1 else z, gun + gaR if iL == 2 else z]
    dsR = [gun + gaL if iR == 1 else z, gun + gaR if iR == 2 else z]
    vaf = [(abs(sR) * dsL[x] + abs(sL) * dsR[x]) / den2 for x in range(2)]
    vcf = [(sR * sR * dsL[x] + sL * sL * dsR[x]) / den2 for x in range(2)]
    A0L = abs(0.5 + af) * np.abs(jac_An(m, qL, n)) + abs(cf) * np.abs(jac_H(m, qL))
    A0R = abs(0.5 - af) * np.abs(jac_An(m, qR, n)) + abs(cf) * np.abs(jac_H(m, qR))
    u1 = np.abs(normal_flux(m, qR, n)) + np.abs(normal_flux(m, qL, n))
    u2 = np.abs(conserved(m, qR)) + np.abs(conserved(m, qL))
    return A0L, A0R, u1, vaf[0], vaf[1], u2, vcf[0], vcf[1]


def block_row(m: FluxModel, Lx: int, Ly: int, Q, i: int):
    """Block row i of dR/dQ: per block of the row (block order) a tuple
    (k, S values in pattern order, U rows, V rows, scales of S, U, V).

    The diagonal block is H(q_i) + dt (sum over faces A0_L - G0) with pairs
    [(-dt ws, grad omega), then per face in block order (dt u1, v1L), (dt u2, v2L)];
    the block of neighbour j is dt A0_R with pairs (dt u1, v1R), (dt u2, v2R) of the
    face i -> j.  S values follow the diagonal pattern (band +-w) and the neighbour
    pattern (diagonal plus flow columns, dense flow rows) of the synthetic workloads.
    The scales are the sums of the absolute values of the terms behind each value
    (its rounding error is a few ulps of them)."""
    bptr, bidx, dp, di, op, oi = _layout(m, Lx, Ly)
    b, dt = m.b, m.dt
    faces = [int(j) for j in bidx[bptr[i]:bptr[i + 1]] if j != i]
    parts = {j: hll_parts(m, Q[i], Q[j], face_normal(Lx, i, j)) for j in faces}
    mags = {j: _parts_mag(m, Q[i], Q[j], face_normal(Lx, i, j)) for j in faces}
    out = []
    for k in range(bptr[i], bptr[i + 1]):
        j = int(bidx[k])
        if j == i:
            G0, wse, gw = source_parts(m, Q[i])
            D = jac_H(m, Q[i]) - dt * G0
            Dm = np.abs(jac_H(m, Q[i])) + dt * np.abs(G0)
            for jj in faces:
                D = D + dt * parts[jj][0]
                Dm = Dm + dt * mags[jj][0]
            ent = [(p, di[e]) for p in range(b) for e in range(dp[p], dp[p + 1])]
            Ur, Vr = [-dt * wse], [gw]
            Um, Vm = [dt * np.abs(wse)], [np.abs(gw)]
            for jj in faces:
                _, _, u1, v1L, _, u2, v2L, _ = parts[jj]
                _, _, u1m, v1Lm, _, u2m, v2Lm, _ = mags[jj]
                Ur += [dt * u1, dt * u2]
                Vr += [v1L, v2L]
                Um += [dt * u1m, dt * u2m]
                Vm += [v1Lm, v2Lm]
        else:
            _, A0R, u1, _, v1R, u2, _, v2R = parts[j]
            _, A0Rm, u1m, _, v1Rm, u2m, _, v2Rm = mags[j]
            D, Dm = dt * A0R, dt * A0Rm
            ent = [(p, oi[e]) for p in range(b) for e in range(op[p], op[p + 1])]
            Ur, Vr = [dt * u1, dt * u2], [v1R, v2R]
            Um, Vm = [dt * u1m, dt * u2m], [v1Rm, v2Rm]
        f64 = lambda a: np.asarray(a, dtype=np.float64)
        out.append((k, f64([D[p, c] for p, c in ent]), f64(Ur), f64(Vr),
                    f64([Dm[p, c] for p, c in ent]), f64(Um), f64(Vm)))
    return out


def jacobian_blocks(m: FluxModel, Lx: int, Ly: int, Q):
    """dR/dQ in the BR1-BSR layout (Section 5.1): S, U, V and the index arrays, the
    block rows of ``block_row`` concatenated in block order."""
    bptr, bidx, dp, di, op, oi = _layout(m, Lx, Ly)
    cols = [[] for _ in range(6)]
    pip = [0]
    for i in range(Lx * Ly):
        for row in block_row(m, Lx, Ly, Q, i):
            for c, a in zip(cols, row[1:]):
                c.append(a)
            pip.append(pip[-1] + row[2].shape[0])
    S, U, V, Sm, Um, Vm = (np.concatenate(c) for c in cols)
    return dict(block_indptr=bptr.copy(), block_indices=bidx.copy(), d_indptr=dp.copy(), d_indices=di.copy(),
                o_indptr=op.copy(), o_indices=oi.copy(), pair_indptr=np.asarray(pip, dtype=np.int32),
                S=S, U=U, V=V, scales=dict(S=Sm, U=Um, V=Vm))


def model_of(case) -> FluxModel:
    """The FluxModel of an inputs.FlowCase (field copy)."""
    return FluxModel(N=case.N, w=case.w, r=case.r, cv=case.cv, e0=case.e0, beta=case.beta,
                     ws=case.ws, K=case.K, A=case.A, theta=case.theta, dt=case.dt)


def newton(m: FluxModel, Lx: int, Ly: int, Q0, Qn, rtol: float = 1e-12, max_newton: int = 20,
           max_halvings: int = 8):
    """Newton-Raphson for R(Q) = 0 from Q0 (Section 3.3, Eq. LinearSystem): dQ from a
    dense solve of the assembled dR/dQ (numpy), Q <- Q + alpha dQ with alpha = 1
    halved while ||R|| does not decrease.  Returns (Q, history of ||R||)."""
    from .native import Jacobian, matvec
    nc, b = Lx * Ly, m.b
    Q = np.array(Q0, dtype=np.float64, copy=True)
    R = residual(m, Lx, Ly, Q, Qn)
    hist = [float(np.linalg.norm(R))]
    while hist[-1] > rtol * hist[0] and len(hist) <= max_newton:
        d = jacobian_blocks(m, Lx, Ly, Q)
        d.pop("scales")
        J = Jacobian(n_cells=nc, b=b, **d)
        D = np.stack([matvec(J, e) for e in np.eye(nc * b)], axis=1)
        dQ = np.linalg.solve(D, -R.ravel()).reshape(nc, b)
        alpha = 1.0
        for _ in range(max_halvings + 1):
            Qt = Q + alpha * dQ
            Rt = residual(m, Lx, Ly, Qt, Qn)
            if np.linalg.norm(Rt) < hist[-1]:
                break
            alpha *= 0.5
        else:
            break
        Q, R = Qt, Rt
        hist.append(float(np.linalg.norm(R)))
    return Q, hist
