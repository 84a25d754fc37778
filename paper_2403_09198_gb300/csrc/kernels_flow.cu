// kernels_flow.cu -- residual and r1-sparse Jacobian of a toy HLL-flux flow
// model (Section 2.1 model, Section 3.2 Eq. HLL_flux, Section 3.3 Eq.
// system_residual, Section 4.1 Eqs. r1_flux_left / r1_flux_right).
//
// One warp per cell: the lanes sum the species terms of a state (mixture
// density, gas constant, heat capacity, energy at T = 0) with a fixed
// shuffle tree and broadcast lane 0's result, so every lane holds the same
// scalars and takes the same wave-speed branch.  Per face the warp forms the
// HLL bounds s_L, s_R, the coefficients a_f, c_f and their gradients, writes the
// face's two rank-one pairs into the diagonal block of its cell and into the
// neighbour block, and the neighbour block's sparse part dt A0_R; the diagonal
// block's sparse part H + dt (sum A0_L + K) is written last.  Every face is
// evaluated from both of its cells (once per block row), which keeps the writes
// of a block row in one warp: no atomics, deterministic.
//
// These kernels are bound by the FP64 pipe (a warp-wide FP64 instruction holds
// a sub-partition's pipe for 64 cycles), so the FP64 work per entry is kept
// small.  A_n is linear in the normal, so the diagonal block's face sum
// sum_f (1/2 + a_f) A_{n_f}(q_i) is A_n(q_i) at the summed normal.  Level rows,
// whose entries of A_n and H are u_n, rho_p n and 1, are written from four
// per-face coefficient sums with lanes over rows; only the three dense flow rows
// evaluate A_n and H entry by entry (lanes over columns), once per block;
// reciprocals are formed once per face and per state, not per component.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "sts_internal.h"

namespace sts {
namespace {

constexpr int kFlowWarps = 4;     // cells (warps) per block

struct FlowDev {
    int Lx, nc, N, b, w, nnz_d, nnz_o;
    const double *r, *cv, *e0, *beta, *ws, *K;
    double A, theta, dt;
    const int *bptr, *bidx, *pip;
    const long long *soff;
    const int *d_ptr;       // row starts of the diagonal pattern (the neighbour pattern's are 4p, then 4N + b (p-N))
};

struct Mix {
    double rho, Rt, Ct, E0, u, v, T, ke, p, rhoetot, g, a;
    double cga, gaT;        // T / (2 a rho C) and a / (2 T): the factors of da/dq
};

// Sum over the warp, the same value on every lane (tree to lane 0, then broadcast).
__device__ __forceinline__ double warp_total(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return __shfl_sync(0xffffffffu, x, 0);
}

__device__ Mix mixture(const FlowDev &F, const double *q, int lane) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int k = lane; k < F.N; k += 32) {
        const double rk = q[k];
        s0 += rk;
        s1 += rk * F.r[k];
        s2 += rk * F.cv[k];
        s3 += rk * F.e0[k];
    }
    Mix m;
    m.rho = warp_total(s0);
    m.Rt = warp_total(s1);
    m.Ct = warp_total(s2);
    m.E0 = warp_total(s3);
    m.u = q[F.N];
    m.v = q[F.N + 1];
    m.T = q[F.N + 2];
    m.ke = 0.5 * (m.u * m.u + m.v * m.v);
    m.p = m.Rt * m.T;
    m.rhoetot = m.E0 + m.Ct * m.T + m.rho * m.ke;
    m.g = (m.Ct + m.Rt) * m.Rt / (m.rho * m.Ct);
    m.a = sqrt(m.g * m.T);
    m.cga = m.T / (2.0 * m.a * m.rho * m.Ct);
    m.gaT = m.a / (2.0 * m.T);
    return m;
}

// component c of the conserved variables u(q) and of the normal flux f_n(q)
__device__ __forceinline__ double cons_c(const FlowDev &F, const double *q, const Mix &m, int c) {
    if (c < F.N) return q[c];
    if (c == F.N) return m.rho * m.u;
    if (c == F.N + 1) return m.rho * m.v;
    return m.rhoetot;
}

__device__ __forceinline__ double flux_c(const FlowDev &F, const double *q, const Mix &m, double nx, double ny,
                                         int c) {
    const double un = nx * m.u + ny * m.v;
    if (c < F.N) return q[c] * un;
    if (c == F.N) return m.rho * m.u * un + m.p * nx;
    if (c == F.N + 1) return m.rho * m.v * un + m.p * ny;
    return (m.rhoetot + m.p) * un;
}

// entry (p, c) of H = du/dq
__device__ double H_e(const FlowDev &F, const Mix &m, int p, int c) {
    const int N = F.N;
    if (p < N) return c == p ? 1.0 : 0.0;
    if (p == N) return c < N ? m.u : c == N ? m.rho : 0.0;
    if (p == N + 1) return c < N ? m.v : c == N + 1 ? m.rho : 0.0;
    if (c < N) return F.e0[c] + F.cv[c] * m.T + m.ke;
    if (c == N) return m.rho * m.u;
    if (c == N + 1) return m.rho * m.v;
    return m.Ct;
}

// entry (p, c) of A_n = d f_n / dq
__device__ double An_e(const FlowDev &F, const double *q, const Mix &m, double nx, double ny, int p, int c) {
    const int N = F.N;
    const double un = nx * m.u + ny * m.v;
    if (p < N) {
        if (c == p) return un;
        if (c == N) return q[p] * nx;
        if (c == N + 1) return q[p] * ny;
        return 0.0;
    }
    if (p == N) {
        if (c < N) return m.u * un + F.r[c] * m.T * nx;
        if (c == N) return m.rho * un + m.rho * m.u * nx;
        if (c == N + 1) return m.rho * m.u * ny;
        return m.Rt * nx;
    }
    if (p == N + 1) {
        if (c < N) return m.v * un + F.r[c] * m.T * ny;
        if (c == N) return m.rho * m.v * nx;
        if (c == N + 1) return m.rho * un + m.rho * m.v * ny;
        return m.Rt * ny;
    }
    if (c < N) return (F.e0[c] + F.cv[c] * m.T + m.ke + F.r[c] * m.T) * un;
    if (c == N) return m.rho * m.u * un + (m.rhoetot + m.p) * nx;
    if (c == N + 1) return m.rho * m.v * un + (m.rhoetot + m.p) * ny;
    return (m.Ct + m.Rt) * un;
}

// component c of da/dq: a^2 = T g, g = (C + R) R / (rho C)
__device__ double grad_a_c(const FlowDev &F, const Mix &m, int c) {
    if (c < F.N) {
        const double dn = (F.cv[c] + F.r[c]) * m.Rt + (m.Ct + m.Rt) * F.r[c];
        const double dd = m.Ct + m.rho * F.cv[c];
        return m.cga * (dn - m.g * dd);
    }
    return c == F.N + 2 ? m.gaT : 0.0;
}

struct Face {
    double nx, ny, sL, sR, af, cf, inv_den, inv_den2;
    int iL, iR;
};

// HLL bounds and coefficients of the face from cell L to cell R
__device__ Face face_of(const Mix &mL, const Mix &mR, double nx, double ny) {
    Face f;
    f.nx = nx;
    f.ny = ny;
    const double unL = nx * mL.u + ny * mL.v, unR = nx * mR.u + ny * mR.v;
    f.sL = 0.0;
    f.iL = 0;
    if (unL - mL.a < f.sL) { f.sL = unL - mL.a; f.iL = 1; }
    if (unR - mR.a < f.sL) { f.sL = unR - mR.a; f.iL = 2; }
    f.sR = 0.0;
    f.iR = 0;
    if (unL + mL.a > f.sR) { f.sR = unL + mL.a; f.iR = 1; }
    if (unR + mR.a > f.sR) { f.sR = unR + mR.a; f.iR = 2; }
    // a_f and c_f by division: on a supersonic face a_f is exactly +-1/2 and the
    // upwind side's weight 1/2 -+ a_f exactly zero; the per-component products
    // use the reciprocal
    const double den = f.sR - f.sL;
    f.af = 0.5 * (f.sL + f.sR) / den;
    f.cf = f.sL * f.sR / den;
    f.inv_den = 1.0 / den;
    f.inv_den2 = f.inv_den * f.inv_den;
    return f;
}

__device__ __forceinline__ void normal_of(int Lx, int i, int j, double &nx, double &ny) {
    const int d = j - i;
    nx = d == 1 ? 1.0 : d == -1 ? -1.0 : 0.0;
    ny = d == Lx ? 1.0 : d == -Lx ? -1.0 : 0.0;
    if (Lx == 1) {      // a one-column grid: every neighbour is vertical
        nx = 0.0;
        ny = d > 0 ? 1.0 : -1.0;
    }
}

__global__ void __launch_bounds__(kFlowWarps * 32) k_flow_jac(FlowDev F, const double *Q, double *S, double *U,
                                                               double *V) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kFlowWarps + (threadIdx.x >> 5);
    if (i >= F.nc) return;
    const int b = F.b, N = F.N, w = F.w;
    const double dt = F.dt;
    const double *qi = Q + (size_t)i * b;
    const Mix mi = mixture(F, qi, lane);
    const int k0 = F.bptr[i], k1 = F.bptr[i + 1];
    int kd = k0;
    for (int k = k0; k < k1; ++k)
        if (F.bidx[k] == i) kd = k;
    int nf = 0;
    // sums over the faces for the diagonal block:
    // sum (1/2 + a_f) u_n(q_i), sum c_f, sum (1/2 + a_f) n_x, sum (1/2 + a_f) n_y
    double cun = 0.0, ccf = 0.0, cnx = 0.0, cny = 0.0;
    for (int k = k0; k < k1 && nf < 4; ++k) {
        const int j = F.bidx[k];
        if (j == i) continue;
        const double *qj = Q + (size_t)j * b;
        const Mix mj = mixture(F, qj, lane);
        double nx, ny;
        normal_of(F.Lx, i, j, nx, ny);
        const Face f = face_of(mi, mj, nx, ny);
        const double wL = 0.5 + f.af, wR = 0.5 - f.af;
        cun += wL * (nx * mi.u + ny * mi.v);
        ccf += f.cf;
        cnx += wL * nx;
        cny += wL * ny;
        // neighbour block dt A0_R = dt ((1/2 - a_f) A_n(q_j) + c_f H(q_j)):
        // level row p holds (p, p) = u_n(q_j) and 1, (p, N) = rho_p n_x, (p, N+1) = rho_p n_y, (p, N+2) = 0
        double *Sk = S + F.soff[k];
        const double unj = nx * mj.u + ny * mj.v;
        for (int p = lane; p < N; p += 32) {
            const double wq = wR * qj[p];
            Sk[4 * p] = dt * (wR * unj + f.cf);
            Sk[4 * p + 1] = dt * (wq * nx);
            Sk[4 * p + 2] = dt * (wq * ny);
            Sk[4 * p + 3] = 0.0;
        }
        for (int e = lane; e < 3 * b; e += 32) {
            const int p = N + e / b, c = e - (e / b) * b;
            Sk[4 * N + e] = dt * (wR * An_e(F, qj, mj, nx, ny, p, c) + f.cf * H_e(F, mj, p, c));
        }
        // the face's two pairs: into the diagonal block (d/dq_i) and the neighbour block (d/dq_j)
        const size_t pd = (size_t)(F.pip[kd] + 1 + 2 * nf), po = (size_t)F.pip[k];
        for (int c = lane; c < b; c += 32) {
            const double u1 = -(flux_c(F, qj, mj, nx, ny, c) - flux_c(F, qi, mi, nx, ny, c));
            const double u2 = cons_c(F, qj, mj, c) - cons_c(F, qi, mi, c);
            const double gun = c == N ? nx : c == N + 1 ? ny : 0.0;
            const double gaL = grad_a_c(F, mi, c), gaR = grad_a_c(F, mj, c);
            const double dsLL = f.iL == 1 ? gun - gaL : 0.0, dsLR = f.iL == 2 ? gun - gaR : 0.0;
            const double dsRL = f.iR == 1 ? gun + gaL : 0.0, dsRR = f.iR == 2 ? gun + gaR : 0.0;
            U[pd * b + c] = dt * u1;
            V[pd * b + c] = (f.sR * dsLL - f.sL * dsRL) * f.inv_den2;
            U[(pd + 1) * b + c] = dt * u2;
            V[(pd + 1) * b + c] = (f.sR * f.sR * dsLL - f.sL * f.sL * dsRL) * f.inv_den2;
            U[po * b + c] = dt * u1;
            V[po * b + c] = (f.sR * dsLR - f.sL * dsRR) * f.inv_den2;
            U[(po + 1) * b + c] = dt * u2;
            V[(po + 1) * b + c] = (f.sR * f.sR * dsLR - f.sL * f.sL * dsRR) * f.inv_den2;
        }
        ++nf;
    }
    // diagonal block H(q_i) + dt K + sum over faces dt A0_L: level row p holds the
    // band (K, plus H = 1 and the face terms on the diagonal), then (p, N), (p, N+1), (p, N+2)
    double *Sd = S + F.soff[kd];
    for (int p = lane; p < N; p += 32) {
        double *row = Sd + F.d_ptr[p];
        const int c0 = max(0, p - w), c1 = min(N - 1, p + w);
        const double *Kp = F.K + (size_t)p * (2 * w + 1) - p + w;      // Kp[c] = K[p][c - p + w]
        for (int c = c0; c <= c1; ++c) {
            const double kb = dt * Kp[c];
            row[c - c0] = c == p ? (1.0 + kb) + dt * (cun - ccf) : kb;
        }
        const double qp = dt * qi[p];
        row[c1 - c0 + 1] = qp * cnx;
        row[c1 - c0 + 2] = qp * cny;
        row[c1 - c0 + 3] = 0.0;
    }
    // flow rows: A_n is linear in n, so sum_f (1/2 + a_f) A_{n_f}(q_i) = A_{(cnx, cny)}(q_i)
    // (K is zero on the flow rows)
    double *Sf = Sd + F.d_ptr[N];
    for (int e = lane; e < 3 * b; e += 32) {
        const int p = N + e / b, c = e - (e / b) * b;
        const double h = H_e(F, mi, p, c);
        Sf[e] = h + dt * (An_e(F, qi, mi, cnx, cny, p, c) - ccf * h);
    }
    // source pair (-dt ws, d omega / dq)
    double sb = 0.0;
    for (int k = lane; k < N; k += 32) sb += F.beta[k] * qi[k];
    sb = warp_total(sb);
    const double kap = F.A * exp(-F.theta / mi.T);
    const double kT = kap * F.theta / (mi.T * mi.T) * sb;
    const size_t ps = (size_t)F.pip[kd];
    for (int c = lane; c < b; c += 32) {
        U[ps * b + c] = c < N ? -dt * F.ws[c] : 0.0;
        V[ps * b + c] = c < N ? kap * F.beta[c] : c == N + 2 ? kT : 0.0;
    }
}

__global__ void __launch_bounds__(kFlowWarps * 32) k_flow_res(FlowDev F, const double *Q, const double *Qn,
                                                               double *R) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kFlowWarps + (threadIdx.x >> 5);
    if (i >= F.nc) return;
    const int b = F.b, N = F.N;
    const double *qi = Q + (size_t)i * b, *qn = Qn + (size_t)i * b;
    const Mix mi = mixture(F, qi, lane), mn = mixture(F, qn, lane);
    double sb = 0.0;
    for (int k = lane; k < N; k += 32) sb += F.beta[k] * qi[k];
    sb = warp_total(sb);
    const double omega = F.A * exp(-F.theta / mi.T) * sb;
    // components c = lane + 32 t, at most 8 per lane (b <= 256)
    constexpr int kMaxPerLane = 8;
    double fsum[kMaxPerLane];
#pragma unroll
    for (int t = 0; t < kMaxPerLane; ++t) fsum[t] = 0.0;
    const int k0 = F.bptr[i], k1 = F.bptr[i + 1];
    for (int k = k0; k < k1; ++k) {
        const int j = F.bidx[k];
        if (j == i) continue;
        const double *qj = Q + (size_t)j * b;
        const Mix mj = mixture(F, qj, lane);
        double nx, ny;
        normal_of(F.Lx, i, j, nx, ny);
        const Face f = face_of(mi, mj, nx, ny);
#pragma unroll
        for (int t = 0; t < kMaxPerLane; ++t) {
            const int c = lane + 32 * t;
            if (c < b) {
                const double fL = flux_c(F, qi, mi, nx, ny, c), fR = flux_c(F, qj, mj, nx, ny, c);
                const double uL = cons_c(F, qi, mi, c), uR = cons_c(F, qj, mj, c);
                fsum[t] = fsum[t] + (f.sR * fL - f.sL * fR + f.sL * f.sR * (uR - uL)) * f.inv_den;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < kMaxPerLane; ++t) {
        const int c = lane + 32 * t;
        if (c >= b) break;
        double src = 0.0;
        if (c < N) {
            for (int l = max(0, c - F.w); l < min(N, c + F.w + 1); ++l)
                src -= F.K[(size_t)c * (2 * F.w + 1) + (l - c + F.w)] * qi[l];
            src += F.ws[c] * omega;
        }
        R[(size_t)i * b + c] = (cons_c(F, qi, mi, c) - cons_c(F, qn, mn, c)) + F.dt * (fsum[t] - src);
    }
}

constexpr int kNormBlocks = 304;     // 2 x 152 SMs
constexpr int kNormThreads = 256;

// Per-block sums of squares (block tree in shared memory); the host adds the
// kNormBlocks partials in block order, so the norm is deterministic.
__global__ void __launch_bounds__(kNormThreads) k_flow_sumsq(const double *x, long long n, double *partial) {
    __shared__ double sh[kNormThreads];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * kNormThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kNormThreads)
        s = fma(x[i], x[i], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kNormThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// y = a + alpha * d   (alpha = 0 and a = 0: y = -d when neg is set)
__global__ void k_flow_axpy(double *y, const double *a, double alpha, const double *d, long long n, int neg) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = neg ? -d[i] : fma(alpha, d[i], a[i]);
}

}  // namespace
}  // namespace sts

using namespace sts;

struct sts_flow_s {
    FlowDev dev{};
    cudaStream_t stream = nullptr;
    int Lx = 0, Ly = 0;
    std::vector<int> bptr, bidx, dptr, didx, optr, oidx, pip;
    long long nnz_S = 0;
    std::vector<void *> bufs;
    // Newton workspace, allocated on the first sts_flow_newton
    double *S = nullptr, *U = nullptr, *V = nullptr, *R = nullptr, *Rt = nullptr, *rhs = nullptr,
           *dQ = nullptr, *Qt = nullptr, *partial = nullptr, *h_partial = nullptr;
};

namespace {

void flow_free(sts_flow_s *f) {
    for (void *p : f->bufs) cudaFree(p);
    f->bufs.clear();
    if (f->h_partial) cudaFreeHost(f->h_partial);
    f->h_partial = nullptr;
}

sts_status flow_alloc(sts_flow_s *f, double **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, (n ? n : 1) * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(STS_ERR_ALLOC, "sts_flow_newton: cudaMalloc of %zu doubles failed: %s", n,
                         cudaGetErrorString(e));
    }
    f->bufs.push_back(q);
    *p = static_cast<double *>(q);
    return STS_OK;
}

// ||x||_2 of a device vector of the generator's stream (synchronous)
sts_status flow_norm(sts_flow_s *f, const double *x, long long n, double *out) {
    k_flow_sumsq<<<kNormBlocks, kNormThreads, 0, f->stream>>>(x, n, f->partial);
    STS_LAUNCHED();
    STS_CK(cudaMemcpyAsync(f->h_partial, f->partial, kNormBlocks * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
    STS_CK(cudaStreamSynchronize(f->stream));
    double s = 0.0;
    for (int i = 0; i < kNormBlocks; ++i) s += f->h_partial[i];
    *out = std::sqrt(s);
    return STS_OK;
}

unsigned flow_grid(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16); }

sts_status flow_newton(sts_flow_s *f, sts_jac_t jac, double *Q, const double *Qn, const sts_newton_opts *o,
                       sts_newton_info *info) {
    if (!f || !jac || !Q || !Qn) return set_error(STS_ERR_INVALID_ARG, "sts_flow_newton: NULL argument");
    sts_newton_opts d{};
    if (o) d = *o;
    const int max_newton = d.max_newton > 0 ? d.max_newton : 20;
    const double rtol = d.rtol > 0 ? d.rtol : 1e-10;
    const double atol = d.atol > 0 ? d.atol : 0.0;
    const int max_halvings = d.max_halvings > 0 ? d.max_halvings : 8;
    if (d.gmres.vectors_on_host) return set_error(STS_ERR_INVALID_ARG, "sts_flow_newton: gmres.vectors_on_host must be 0");
    if (d.gmres.trans) return set_error(STS_ERR_INVALID_ARG, "sts_flow_newton: gmres.trans must be 0");
    // the handle must hold this generator's layout
    if (jac->layout != STS_LAYOUT_CELL_MAJOR || jac->nc != f->dev.nc ||
        jac->b != f->dev.b || jac->bidx != f->bidx || jac->bptr != f->bptr || jac->pbase != f->pip ||
        jac->dptr != f->dptr || jac->didx != f->didx || jac->optr != f->optr || jac->oidx != f->oidx)
        return set_error(STS_ERR_INVALID_ARG, "sts_flow_newton: jac is not a cell-major handle of this "
                                              "generator's layout");
    const long long n = (long long)f->dev.nc * f->dev.b;
    if (!f->R) {
        STS_TRY(flow_alloc(f, &f->S, (size_t)f->nnz_S));
        STS_TRY(flow_alloc(f, &f->U, (size_t)f->pip.back() * f->dev.b));
        STS_TRY(flow_alloc(f, &f->V, (size_t)f->pip.back() * f->dev.b));
        STS_TRY(flow_alloc(f, &f->R, n));
        STS_TRY(flow_alloc(f, &f->Rt, n));
        STS_TRY(flow_alloc(f, &f->rhs, n));
        STS_TRY(flow_alloc(f, &f->dQ, n));
        STS_TRY(flow_alloc(f, &f->Qt, n));
        STS_TRY(flow_alloc(f, &f->partial, kNormBlocks));
        STS_CK(cudaMallocHost(&f->h_partial, kNormBlocks * sizeof(double)));
    }
    const unsigned grid = (unsigned)((f->dev.nc + kFlowWarps - 1) / kFlowWarps), eg = flow_grid(n);
    sts_newton_info inf{0, 0, 0, 0, 0.0, 0.0};
    k_flow_res<<<grid, kFlowWarps * 32, 0, f->stream>>>(f->dev, Q, Qn, f->R);
    STS_LAUNCHED();
    double r = 0.0;
    STS_TRY(flow_norm(f, f->R, n, &r));
    inf.res0 = inf.res = r;
    if (d.history) d.history[0] = r;
    if (!std::isfinite(r)) {
        if (info) *info = inf;
        return set_error(STS_ERR_NUMERIC, "sts_flow_newton: the initial residual is NaN or Inf");
    }
    const double tol = std::max(rtol * r, atol);
    sts_status status = STS_OK;
    // inexact Newton forcing (Eisenstat & Walker, choice 2; Kelley's safeguards)
    constexpr double kEtaMax = 0.9, kGamma = 0.9;
    double eta = kEtaMax, r_prev = r;
    while (true) {
        if (r <= tol) {
            inf.converged = 1;
            break;
        }
        if (inf.iterations >= max_newton) break;
        NvtxRange nvtx_it("newton iteration");
        // Jacobian at Q into the handle, block-Jacobi, then J dQ = -R
        k_flow_jac<<<grid, kFlowWarps * 32, 0, f->stream>>>(f->dev, Q, f->S, f->U, f->V);
        STS_LAUNCHED();
        k_flow_axpy<<<eg, 256, 0, f->stream>>>(f->rhs, nullptr, 0.0, f->R, n, 1);
        STS_LAUNCHED();
        STS_CK(cudaMemsetAsync(f->dQ, 0, n * sizeof(double), f->stream));
        STS_CK(cudaStreamSynchronize(f->stream));
        STS_TRY(sts_jac_update_values(jac, f->S, f->U, f->V, 0));
        if (d.gmres.precond != STS_PRECOND_NONE) STS_TRY(sts_jac_bjacobi_setup(jac));
        sts_gmres_info gi{};
        sts_gmres_opts go = d.gmres;
        if (d.forcing) {
            if (inf.iterations > 0) {
                const double ea = kGamma * (r / r_prev) * (r / r_prev);
                const double eb = kGamma * eta * eta > 0.1 ? std::max(ea, kGamma * eta * eta) : ea;
                eta = std::min(kEtaMax, std::max(eb, 0.5 * tol / r));
            }
            go.rtol = eta;
        }
        const sts_status gs = sts_gmres_solve(jac, f->rhs, f->dQ, &go, &gi);
        if (gs != STS_OK && gs != STS_ERR_NOT_CONVERGED) return gs;
        inf.linear_iterations += gi.iterations;
        // line search: alpha = 1, 1/2, ... until ||R|| decreases
        double alpha = 1.0, rt = 0.0;
        bool accepted = false;
        for (int hv = 0; hv <= max_halvings; ++hv) {
            k_flow_axpy<<<eg, 256, 0, f->stream>>>(f->Qt, Q, alpha, f->dQ, n, 0);
            STS_LAUNCHED();
            k_flow_res<<<grid, kFlowWarps * 32, 0, f->stream>>>(f->dev, f->Qt, Qn, f->Rt);
            STS_LAUNCHED();
            STS_TRY(flow_norm(f, f->Rt, n, &rt));
            if (std::isfinite(rt) && rt < r) {
                accepted = true;
                break;
            }
            alpha *= 0.5;
            ++inf.halvings;
        }
        ++inf.iterations;
        if (!accepted) {
            status = set_error(STS_ERR_NOT_CONVERGED, "sts_flow_newton: no decrease of ||R|| = %.3e after %d halvings "
                                                      "(iteration %d)", r, max_halvings, inf.iterations);
            break;
        }
        STS_CK(cudaMemcpyAsync(Q, f->Qt, n * sizeof(double), cudaMemcpyDeviceToDevice, f->stream));
        std::swap(f->R, f->Rt);
        r_prev = r;
        r = rt;
        inf.res = r;
        if (d.history) d.history[inf.iterations] = r;
    }
    STS_CK(cudaStreamSynchronize(f->stream));
    if (info) *info = inf;
    if (status != STS_OK) return status;
    if (!inf.converged)
        return set_error(STS_ERR_NOT_CONVERGED, "sts_flow_newton: %d iterations, ||R|| = %.3e > %.3e", inf.iterations,
                         r, tol);
    return STS_OK;
}

template <typename T>
sts_status flow_upload(sts_flow_s *f, const T **dst, const T *src, size_t n) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(STS_ERR_ALLOC, "sts_flow_create: cudaMalloc failed: %s", cudaGetErrorString(e));
    }
    f->bufs.push_back(p);
    if (n) STS_CK(cudaMemcpyAsync(p, src, n * sizeof(T), cudaMemcpyHostToDevice, f->stream));
    *dst = static_cast<const T *>(p);
    return STS_OK;
}

sts_status flow_create(const sts_flow_desc *d, sts_flow_t *out) {
    if (!out) return set_error(STS_ERR_INVALID_ARG, "sts_flow_create: out is NULL");
    *out = nullptr;
    if (!d) return set_error(STS_ERR_INVALID_ARG, "sts_flow_create: desc is NULL");
    const int N = d->n_species, w = d->band;
    if (d->Lx < 1 || d->Ly < 1 || N < 1 || w < 0)
        return set_error(STS_ERR_INVALID_ARG, "sts_flow_create: need Lx, Ly, n_species >= 1 and band >= 0");
    if (N + 3 > 256) return set_error(STS_ERR_INVALID_ARG, "sts_flow_create: block size N + 3 must be <= 256");
    if ((long long)d->Lx * d->Ly * (N + 3) > (1LL << 31) - 1)
        return set_error(STS_ERR_INVALID_ARG, "sts_flow_create: n_cells * block_size must fit in int32");
    if (!d->r || !d->cv || !d->e0 || !d->beta || !d->ws || !d->K)
        return set_error(STS_ERR_INVALID_ARG, "sts_flow_create: a constant array is NULL");
    for (int k = 0; k < N; ++k) {
        if (!(d->r[k] > 0.0) || !(d->cv[k] > 0.0) || !std::isfinite(d->r[k]) || !std::isfinite(d->cv[k]))
            return set_error(STS_ERR_INVALID_ARG, "sts_flow_create: r[%d] and cv[%d] must be finite and > 0", k, k);
        if (!std::isfinite(d->e0[k]) || !std::isfinite(d->beta[k]) || !std::isfinite(d->ws[k]))
            return set_error(STS_ERR_INVALID_ARG, "sts_flow_create: non-finite constant of species %d", k);
    }
    for (long long e = 0; e < (long long)N * (2 * w + 1); ++e)
        if (!std::isfinite(d->K[e])) return set_error(STS_ERR_INVALID_ARG, "sts_flow_create: non-finite K");
    if (!std::isfinite(d->A) || !std::isfinite(d->theta) || !std::isfinite(d->dt))
        return set_error(STS_ERR_INVALID_ARG, "sts_flow_create: non-finite A, theta or dt");

    sts_flow_s *f = new sts_flow_s();
    f->stream = static_cast<cudaStream_t>(d->stream);
    f->Lx = d->Lx;
    f->Ly = d->Ly;
    const int Lx = d->Lx, Ly = d->Ly, nc = Lx * Ly, b = N + 3;
    // mesh adjacency: i-Lx, i-1, i, i+1, i+Lx where present
    f->bptr.assign(1, 0);
    for (int i = 0; i < nc; ++i) {
        const int ix = i % Lx, iy = i / Lx;
        if (iy > 0) f->bidx.push_back(i - Lx);
        if (ix > 0) f->bidx.push_back(i - 1);
        f->bidx.push_back(i);
        if (ix < Lx - 1) f->bidx.push_back(i + 1);
        if (iy < Ly - 1) f->bidx.push_back(i + Lx);
        f->bptr.push_back((int)f->bidx.size());
    }
    // patterns (the kernels write them in this order)
    f->dptr.assign(1, 0);
    f->optr.assign(1, 0);
    for (int p = 0; p < b; ++p) {
        if (p < N) {
            for (int c = std::max(0, p - w); c <= std::min(N - 1, p + w); ++c) f->didx.push_back(c);
            for (int c = N; c < b; ++c) f->didx.push_back(c);
            f->oidx.push_back(p);
            for (int c = N; c < b; ++c) f->oidx.push_back(c);
        } else {
            for (int c = 0; c < b; ++c) {
                f->didx.push_back(c);
                f->oidx.push_back(c);
            }
        }
        f->dptr.push_back((int)f->didx.size());
        f->optr.push_back((int)f->oidx.size());
    }
    // S offsets and pairs: 1 + 2 per face on the diagonal block, 2 on a neighbour block
    const int nnzb = (int)f->bidx.size();
    std::vector<long long> soff(nnzb + 1, 0);
    f->pip.assign(nnzb + 1, 0);
    for (int i = 0; i < nc; ++i) {
        const int deg = f->bptr[i + 1] - f->bptr[i] - 1;
        for (int k = f->bptr[i]; k < f->bptr[i + 1]; ++k) {
            const bool diag = f->bidx[k] == i;
            soff[k + 1] = soff[k] + (diag ? (long long)f->didx.size() : (long long)f->oidx.size());
            f->pip[k + 1] = f->pip[k] + (diag ? 1 + 2 * deg : 2);
        }
    }
    f->nnz_S = soff[nnzb];
    FlowDev &D = f->dev;
    D.Lx = Lx;
    D.nc = nc;
    D.N = N;
    D.b = b;
    D.w = w;
    D.nnz_d = (int)f->didx.size();
    D.nnz_o = (int)f->oidx.size();
    D.A = d->A;
    D.theta = d->theta;
    D.dt = d->dt;
    sts_status st = STS_OK;
    do {
        if ((st = flow_upload(f, &D.r, d->r, N)) != STS_OK) break;
        if ((st = flow_upload(f, &D.cv, d->cv, N)) != STS_OK) break;
        if ((st = flow_upload(f, &D.e0, d->e0, N)) != STS_OK) break;
        if ((st = flow_upload(f, &D.beta, d->beta, N)) != STS_OK) break;
        if ((st = flow_upload(f, &D.ws, d->ws, N)) != STS_OK) break;
        if ((st = flow_upload(f, &D.K, d->K, (size_t)N * (2 * w + 1))) != STS_OK) break;
        if ((st = flow_upload(f, &D.bptr, f->bptr.data(), f->bptr.size())) != STS_OK) break;
        if ((st = flow_upload(f, &D.bidx, f->bidx.data(), f->bidx.size())) != STS_OK) break;
        if ((st = flow_upload(f, &D.pip, f->pip.data(), f->pip.size())) != STS_OK) break;
        if ((st = flow_upload(f, &D.soff, soff.data(), soff.size())) != STS_OK) break;
        if ((st = flow_upload(f, &D.d_ptr, f->dptr.data(), f->dptr.size())) != STS_OK) break;
        cudaError_t e = cudaStreamSynchronize(f->stream);   // the host vectors above are temporaries
        if (e != cudaSuccess) st = set_error(STS_ERR_CUDA, "sts_flow_create: %s", cudaGetErrorString(e));
    } while (false);
    if (st != STS_OK) {
        cudaStreamSynchronize(f->stream);
        flow_free(f);
        delete f;
        return st;
    }
    *out = f;
    return STS_OK;
}

}  // namespace

#define STS_FLOW_GUARD(body)                                                      \
    try {                                                                         \
        body                                                                      \
    } catch (const std::bad_alloc &) {                                            \
        return set_error(STS_ERR_ALLOC, "host allocation failed");                \
    } catch (...) {                                                               \
        return set_error(STS_ERR_INVALID_ARG, "unexpected exception");            \
    }

extern "C" {

sts_status sts_flow_create(const sts_flow_desc *d, sts_flow_t *out) {
    NvtxRange nvtx_range("sts_flow_create");
    STS_FLOW_GUARD(return flow_create(d, out);)
}

sts_status sts_flow_get_sizes(sts_flow_t f, sts_flow_sizes *s) {
    if (!f || !s) return set_error(STS_ERR_INVALID_ARG, "sts_flow_get_sizes: NULL argument");
    s->n_cells = f->dev.nc;
    s->block_size = f->dev.b;
    s->nnzb = (int)f->bidx.size();
    s->nnz_d = f->dev.nnz_d;
    s->nnz_o = f->dev.nnz_o;
    s->n_pairs = f->pip.back();
    s->nnz_S = f->nnz_S;
    return STS_OK;
}

sts_status sts_flow_get_layout(sts_flow_t f, int *block_indptr, int *block_indices, int *d_indptr, int *d_indices,
                               int *o_indptr, int *o_indices, int *pair_indptr) {
    if (!f || !block_indptr || !block_indices || !d_indptr || !d_indices || !o_indptr || !o_indices || !pair_indptr)
        return set_error(STS_ERR_INVALID_ARG, "sts_flow_get_layout: NULL argument");
    std::copy(f->bptr.begin(), f->bptr.end(), block_indptr);
    std::copy(f->bidx.begin(), f->bidx.end(), block_indices);
    std::copy(f->dptr.begin(), f->dptr.end(), d_indptr);
    std::copy(f->didx.begin(), f->didx.end(), d_indices);
    std::copy(f->optr.begin(), f->optr.end(), o_indptr);
    std::copy(f->oidx.begin(), f->oidx.end(), o_indices);
    std::copy(f->pip.begin(), f->pip.end(), pair_indptr);
    return STS_OK;
}

sts_status sts_flow_residual(sts_flow_t f, const double *Q, const double *Qn, double *R) {
    NvtxRange nvtx_range("sts_flow_residual");
    if (!f || !Q || !Qn || !R) return set_error(STS_ERR_INVALID_ARG, "sts_flow_residual: NULL argument");
    const unsigned grid = (unsigned)((f->dev.nc + kFlowWarps - 1) / kFlowWarps);
    k_flow_res<<<grid, kFlowWarps * 32, 0, f->stream>>>(f->dev, Q, Qn, R);
    STS_LAUNCHED();
    return STS_OK;
}

sts_status sts_flow_jacobian(sts_flow_t f, const double *Q, double *S, double *U, double *V) {
    NvtxRange nvtx_range("sts_flow_jacobian");
    if (!f || !Q || !S || !U || !V) return set_error(STS_ERR_INVALID_ARG, "sts_flow_jacobian: NULL argument");
    const unsigned grid = (unsigned)((f->dev.nc + kFlowWarps - 1) / kFlowWarps);
    k_flow_jac<<<grid, kFlowWarps * 32, 0, f->stream>>>(f->dev, Q, S, U, V);
    STS_LAUNCHED();
    return STS_OK;
}

sts_status sts_flow_newton(sts_flow_t f, sts_jac_t jac, double *Q, const double *Qn, const sts_newton_opts *opts,
                           sts_newton_info *info) {
    NvtxRange nvtx_range("sts_flow_newton");
    STS_FLOW_GUARD(return flow_newton(f, jac, Q, Qn, opts, info);)
}

sts_status sts_flow_destroy(sts_flow_t f) {
    if (!f) return STS_OK;
    cudaStreamSynchronize(f->stream);
    flow_free(f);
    delete f;
    return STS_OK;
}

}  // extern "C"
