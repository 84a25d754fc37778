// kernels_krylov.cu -- restarted right-preconditioned GMRES(m) on the device.
//
// Section 6 (Eq. right_precond_system): solve (A M) y = b, x = M y.  Each
// cycle starts from the true FP64 residual r = b - A x, builds the Krylov basis
// by classical Gram-Schmidt with a second pass (CGS2: two fused multi-dot +
// update sweeps per step, same result as modified Gram-Schmidt in exact
// arithmetic), reduces the Hessenberg matrix with Givens rotations on the host
// in FP64 and updates x += Z y with Z = [M v_0, ..., M v_{k-1}] (for a fixed M
// this equals x += M (V y)).  Convergence is declared on the recomputed true
// residual only.  Mixed mode (flexible GMRES): z_j = M32(v_j) and w = A32 z_j in
// FP32; the basis, the orthogonalisation, x and the residual refresh stay FP64.
// Left preconditioning (Eq. left_precond_system, (M A) x = M b): the cycle's
// first vector is M r / ||M r||, each step forms w = M (A v_j), x += V y, and a
// cycle stops when the preconditioned residual has fallen by the factor the
// true residual still needs.
//
// All reductions are deterministic: a fixed grid writes per-block partial sums
// and the block that finishes last adds them in a fixed order.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "sts_internal.h"

namespace sts {
namespace {

constexpr int kRedBlocks = 304;     // 2 x 152 SMs
constexpr int kRedThreads = 256;
constexpr int kDotChunk = 16;       // vectors per multi-dot sweep

// Per-block sums of the first NV of the values v at once: every warp reduces
// them with shuffles, then thread i < NV adds the warps' results in warp order
// and writes row[i].  One barrier for all NV values.  sh: 8 * NV doubles.
template <int NV, int NA>
__device__ __forceinline__ void block_partials(double (&v)[NA], double *row, double *sh) {
    static_assert(NV <= NA, "values to reduce");
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
        if (lane == 0) sh[w * NV + i] = v[i];
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k * NV + threadIdx.x];
        row[threadIdx.x] = s;
    }
}

// The block that finishes last adds the per-block partial sums of `cnt`
// outputs (partial[b * ld + o], o = o0 .. o0 + cnt - 1) into out[o]: warp w
// takes outputs w, w + 8, ...; lane l adds blocks l, l + 32, ... and the
// shuffle tree adds the lanes, so the order of additions never depends on
// which block is last or on scheduling.  The ticket counts finished blocks
// and is reset for the next launch.
__device__ __forceinline__ void last_block_reduce(double *partial, int ld, int o0, int cnt, double *out,
                                                  unsigned int *ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int o = o0 + w; o < o0 + cnt; o += nw) {
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(partial + (size_t)b * ld + o);
#pragma unroll
        for (int k = 16; k > 0; k >>= 1) s += __shfl_down_sync(0xffffffffu, s, k);
        if (lane == 0) out[o] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) *ticket = 0u;
}

// partial[blk * ld + i0 + i] = sum over this block's elements of V_{i0+i} . w,
// for i < CNT (CNT <= kDotChunk).  With SELF the next slot holds w . w.  The
// count is a template parameter: a predicated-off FP64 FMA still occupies the
// FP64 pipe, so the loop must issue exactly CNT (+ SELF) FMAs per element.
template <int CNT, bool SELF>
__global__ void __launch_bounds__(kRedThreads) k_mdot(const double *V, long long n, int i0,
                                                      const double *w, double *partial, int ld, double *out,
                                                      unsigned int *ticket) {
    // elements per thread and iteration: all their loads are issued before the
    // FMAs, so a thread keeps several memory requests in flight
    constexpr int U = CNT + 1 <= 3 ? 4 : CNT + 1 <= 7 ? 2 : 1;
    constexpr int NO = CNT + (SELF ? 1 : 0);          // outputs
    __shared__ double sh[(kRedThreads / 32) * (CNT + 1)];
    double acc[CNT + 1];
#pragma unroll
    for (int i = 0; i <= CNT; ++i) acc[i] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e + (U - 1) * stride < n; e += U * stride) {
        double we[U], vv[U][CNT > 0 ? CNT : 1];
#pragma unroll
        for (int u = 0; u < U; ++u) we[u] = w[e + u * stride];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int i = 0; i < CNT; ++i) vv[u][i] = V[(size_t)(i0 + i) * n + e + u * stride];
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int i = 0; i < CNT; ++i) acc[i] = fma(vv[u][i], we[u], acc[i]);
            if (SELF) acc[CNT] = fma(we[u], we[u], acc[CNT]);
        }
    }
    for (; e < n; e += stride) {
        const double we = w[e];
#pragma unroll
        for (int i = 0; i < CNT; ++i) acc[i] = fma(V[(size_t)(i0 + i) * n + e], we, acc[i]);
        if (SELF) acc[CNT] = fma(we, we, acc[CNT]);
    }
    block_partials<NO>(acc, partial + (size_t)blockIdx.x * ld + i0, sh);
    last_block_reduce(partial, ld, i0, NO, out, ticket);
}

template <int CNT>
void mdot_launch(const double *V, long long n, int i0, const double *w, double *partial, int ld, bool self,
                 double *out, unsigned int *ticket, cudaStream_t st) {
    if (self) k_mdot<CNT, true><<<kRedBlocks, kRedThreads, 0, st>>>(V, n, i0, w, partial, ld, out, ticket);
    else k_mdot<CNT, false><<<kRedBlocks, kRedThreads, 0, st>>>(V, n, i0, w, partial, ld, out, ticket);
}

// cnt in 0..kDotChunk (cnt = 0 only with self: w . w alone)
void mdot_dispatch(int cnt, const double *V, long long n, int i0, const double *w, double *partial, int ld,
                   bool self, double *out, unsigned int *ticket, cudaStream_t st) {
    static_assert(kDotChunk == 16, "one case per count");
    switch (cnt) {
        case 0: mdot_launch<0>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 1: mdot_launch<1>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 2: mdot_launch<2>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 3: mdot_launch<3>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 4: mdot_launch<4>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 5: mdot_launch<5>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 6: mdot_launch<6>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 7: mdot_launch<7>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 8: mdot_launch<8>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 9: mdot_launch<9>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 10: mdot_launch<10>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 11: mdot_launch<11>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 12: mdot_launch<12>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 13: mdot_launch<13>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 14: mdot_launch<14>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        case 15: mdot_launch<15>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
        default: mdot_launch<16>(V, n, i0, w, partial, ld, self, out, ticket, st); break;
    }
}

// w -= sum_{i<CNT} h_{i0+i} V_{i0+i}; with NORM also out[0] = ||w||^2 after the
// update (accumulated in the same sweep, reduced by the last block).  CNT is a
// template parameter for the same reason as in k_mdot.
template <int CNT, bool NORM>
__global__ void __launch_bounds__(kRedThreads) k_update(double *w, const double *V, long long n,
                                                        const double *hcoef, int i0, double *partial,
                                                        double *out, unsigned int *ticket) {
    constexpr int U = CNT + 1 <= 3 ? 4 : CNT + 1 <= 7 ? 2 : 1;
    __shared__ double sh[kRedThreads / 32];
    double h[CNT > 0 ? CNT : 1];
#pragma unroll
    for (int i = 0; i < CNT; ++i) h[i] = __ldg(hcoef + i0 + i);
    double acc = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e + (U - 1) * stride < n; e += U * stride) {
        double v[U], vv[U][CNT > 0 ? CNT : 1];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = w[e + u * stride];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int i = 0; i < CNT; ++i) vv[u][i] = V[(size_t)(i0 + i) * n + e + u * stride];
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int i = 0; i < CNT; ++i) v[u] = fma(-h[i], vv[u][i], v[u]);
            w[e + u * stride] = v[u];
            if (NORM) acc = fma(v[u], v[u], acc);
        }
    }
    for (; e < n; e += stride) {
        double v = w[e];
#pragma unroll
        for (int i = 0; i < CNT; ++i) v = fma(-h[i], V[(size_t)(i0 + i) * n + e], v);
        w[e] = v;
        if (NORM) acc = fma(v, v, acc);
    }
    if (NORM) {
        double a1[1] = {acc};
        block_partials<1>(a1, partial + blockIdx.x, sh);
        last_block_reduce(partial, 1, 0, 1, out, ticket);
    }
}

template <int CNT>
void update_launch(double *w, const double *V, long long n, const double *hcoef, int i0, bool norm,
                   double *partial, double *out, unsigned int *ticket, cudaStream_t st) {
    if (norm) k_update<CNT, true><<<kRedBlocks, kRedThreads, 0, st>>>(w, V, n, hcoef, i0, partial, out, ticket);
    else k_update<CNT, false><<<kRedBlocks, kRedThreads, 0, st>>>(w, V, n, hcoef, i0, partial, out, ticket);
}

// cnt in 1..kDotChunk
void update_dispatch(int cnt, double *w, const double *V, long long n, const double *hcoef, int i0, bool norm,
                     double *partial, double *out, unsigned int *ticket, cudaStream_t st) {
    switch (cnt) {
        case 1: update_launch<1>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 2: update_launch<2>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 3: update_launch<3>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 4: update_launch<4>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 5: update_launch<5>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 6: update_launch<6>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 7: update_launch<7>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 8: update_launch<8>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 9: update_launch<9>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 10: update_launch<10>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 11: update_launch<11>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 12: update_launch<12>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 13: update_launch<13>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 14: update_launch<14>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        case 15: update_launch<15>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
        default: update_launch<16>(w, V, n, hcoef, i0, norm, partial, out, ticket, st); break;
    }
}

__global__ void __launch_bounds__(kRedThreads) k_norm2(const double *v, long long n, double *partial, double *out,
                                                       unsigned int *ticket) {
    __shared__ double sh[kRedThreads / 32];
    double acc = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        acc = fma(v[e], v[e], acc);
    double a1[1] = {acc};
    block_partials<1>(a1, partial + blockIdx.x, sh);
    last_block_reduce(partial, 1, 0, 1, out, ticket);
}

__global__ void k_sub(double *r, const double *b, const double *y, long long n) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        r[e] = b[e] - y[e];
}

__global__ void k_scale(double *out, const double *in, double s, long long n) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        out[e] = in[e] * s;
}

template <typename T>
__global__ void k_axpy_multi(double *x, const T *Z, long long n, const double *y, int k) {
    __shared__ double ys[64];
    for (int i0 = 0; i0 < k; i0 += 64) {
        const int cnt = min(64, k - i0);
        __syncthreads();
        if (threadIdx.x < cnt) ys[threadIdx.x] = y[i0 + threadIdx.x];
        __syncthreads();
        for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
             e += (long long)gridDim.x * blockDim.x) {
            double v = x[e];
            for (int i = 0; i < cnt; ++i) v = fma(ys[i], (double)Z[(size_t)(i0 + i) * n + e], v);
            x[e] = v;
        }
    }
}

template <typename To, typename Ti>
__global__ void k_convert(To *out, const Ti *in, long long n) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        out[e] = (To)in[e];
}

inline int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152LL * 32) g = 152LL * 32;
    if (g < 1) g = 1;
    return (int)g;
}

// Operators shared with the public entry points.
sts_status opA64(sts_jac_s *h, int dir, const double *x, double *y) {
    if (h->rep == STS_REP_DENSE_BSR) return dense_matvec(h, x, y);
    return mv_apply64(h, dir, x, y, h->c64);
}
sts_status opM64(sts_jac_s *h, int dir, const double *x, double *z) {
    if (h->rep == STS_REP_DENSE_BSR) return dense_apply(h, x, z);
    return smw_apply64(h, dir, x, z);
}

struct Red {
    sts_jac_s *h;
    long long n;
    // device: per-block partials in h->kry.partial, totals written by each
    // kernel's last block (h->kry.ticket)
    sts_status dots(const double *V, int k, const double *w, int self, double *out) {
        Krylov &K = h->kry;
        const int ld = K.m + 2;
        for (int i0 = 0; i0 < k; i0 += kDotChunk) {
            const int cnt = std::min(kDotChunk, k - i0);
            const int sf = self && (i0 + cnt == k);
            mdot_dispatch(cnt, V, n, i0, w, K.partial, ld, sf != 0, out, K.ticket, h->stream);
            STS_LAUNCHED();
        }
        return STS_OK;
    }
    sts_status update(double *w, const double *V, int k, const double *hcoef, int norm, double *out) {
        Krylov &K = h->kry;
        for (int i0 = 0; i0 < k; i0 += kDotChunk) {
            const int cnt = std::min(kDotChunk, k - i0);
            update_dispatch(cnt, w, V, n, hcoef, i0, norm && i0 + cnt == k, K.partial, out, K.ticket, h->stream);
            STS_LAUNCHED();
        }
        return STS_OK;
    }
    sts_status norm2(const double *v, double *out) {
        Krylov &K = h->kry;
        k_norm2<<<kRedBlocks, kRedThreads, 0, h->stream>>>(v, n, K.partial, out, K.ticket);
        STS_LAUNCHED();
        return STS_OK;
    }
};

sts_status ensure_workspace(sts_jac_s *h, int m, bool mixed) {
    Krylov &K = h->kry;
    const size_t n = (size_t)h->b * h->ncp;
    if (K.m < m) {
        // a larger restart replaces the basis buffers (the stream is idle here:
        // every solve ends with a synchronisation)
        STS_CK(cudaStreamSynchronize(h->stream));
        dev_free(h, K.V);
        dev_free(h, K.Z);
        dev_free(h, K.Z32);
        dev_free(h, K.partial);
        dev_free(h, K.red);
        K.V = K.Z = K.partial = K.red = nullptr;
        // the cycle graphs hold the old buffers and sizes
        for (auto &row : K.gexec)
            for (auto &ge : row) {
                if (ge) cudaGraphExecDestroy(ge);
                ge = nullptr;
            }
        for (double **g : {&K.gH, &K.gcs, &K.gsn, &K.gg, &K.ghist, &K.gpar}) {
            dev_free(h, *g);
            *g = nullptr;
        }
        dev_free(h, K.gstate);
        K.gstate = nullptr;
        if (K.g_pinned) cudaFreeHost(K.g_pinned);
        K.g_pinned = nullptr;
        K.Z32 = nullptr;
        K.m = 0;
        STS_TRY(dalloc(h, &K.V, (size_t)(m + 1) * n));
        STS_TRY(dalloc(h, &K.Z, (size_t)m * n));
        STS_TRY(dalloc(h, &K.partial, (size_t)kRedBlocks * (m + 2)));
        STS_TRY(dalloc(h, &K.red, (size_t)3 * (m + 2)));
        if (!K.ticket) {
            STS_TRY(dalloc(h, &K.ticket, 1));
            STS_CK(cudaMemsetAsync(K.ticket, 0, sizeof(unsigned int), h->stream));
        }
        if (!K.w) {
            STS_TRY(dalloc(h, &K.w, n));
            STS_TRY(dalloc(h, &K.r, n));
            STS_TRY(dalloc(h, &K.xb, n));
            STS_TRY(dalloc(h, &K.bb, n));
            STS_TRY(dalloc(h, &K.tmp, n));
        }
        if (K.h_pinned) cudaFreeHost(K.h_pinned);
        K.h_pinned = nullptr;
        STS_CK(cudaMallocHost(&K.h_pinned, sizeof(double) * 3 * (m + 2)));
        K.m = m;
    }
    if (mixed && !K.Z32) {
        STS_TRY(dalloc(h, &K.Z32, (size_t)K.m * n));
        if (!K.t32a) {
            STS_TRY(dalloc(h, &K.t32a, n));
            STS_TRY(dalloc(h, &K.t32b, n));
        }
    }
    return STS_OK;
}

// ---------------------------------------------------------------------------
// One Arnoldi cycle as a CUDA graph.  Step j of the cycle is the body of a
// conditional (IF) node, nested in step j - 1's body: z_j = M v_j, w = A z_j,
// the two Gram-Schmidt passes,
// then k_givens, which folds the new Hessenberg column into the rotations on
// the device (the host loop's arithmetic, in the same order), records the
// rotated residual, and switches step j + 1 on or off, and finally v_{j+1} =
// w / h(j+1, j).  The host launches the graph once per cycle and reads the
// rotated system back once, instead of synchronising after every step.

// Step j's rotations (one thread).  red: h1 at red[0..], h2 at red[ld..], the
// squared norm at red[2 ld]; par: stop threshold, history scale, 1 / h(j+1,j)
// (output), steps allowed; state: steps taken, stop reason (0 none, 1
// criterion met, 2 NaN or Inf).
__global__ void k_givens(int j, int m, const double *red, int ld, double *H, double *cs, double *sn, double *g,
                         double *hist, double *par, int *state, cudaGraphConditionalHandle next, int has_next) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double *h1 = red, *h2 = red + ld;
    const double w0 = sqrt(h1[j + 1]);
    const double hn = sqrt(red[2 * ld]);
    bool bad = !isfinite(w0) || !isfinite(hn);
    for (int i = 0; i <= j; ++i) {
        H[(size_t)i * m + j] = h1[i] + h2[i];
        bad = bad || !isfinite(H[(size_t)i * m + j]);
    }
    int stop = 0;
    if (bad) {
        stop = 2;
    } else {
        H[(size_t)(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {
            const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
            H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
            H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
        }
        const double hjj = H[(size_t)j * m + j];
        const double den = hypot(hjj, hn);
        cs[j] = hjj / den;
        sn[j] = hn / den;
        H[(size_t)j * m + j] = den;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        hist[j] = fabs(g[j + 1]) * par[1];
        const bool happy = hn <= 1e-14 * w0;
        if (happy || fabs(g[j + 1]) <= par[0] || (double)(j + 1) >= par[3]) stop = 1;
        par[2] = 1.0 / hn;
    }
    state[0] = j + 1;
    state[1] = stop;
    if (has_next) cudaGraphSetConditional(next, stop ? 0u : 1u);
}

__global__ void k_scale_dev(double *out, const double *in, const double *s, long long n) {
    const double f = *s;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        out[e] = in[e] * f;
}

// Build (once per restart length, direction, preconditioning and stream) the
// graph of a whole cycle of m steps.  The kernels of a step are recorded by
// capturing the ordinary host code on a private stream into the step's body.
sts_status cycle_graph(sts_jac_s *h, int m, int dir, bool pre) {
    Krylov &K = h->kry;
    cudaGraphExec_t &exec = K.gexec[dir][pre ? 1 : 0];
    if (exec && K.g_m[dir][pre ? 1 : 0] == m && K.g_stream[dir][pre ? 1 : 0] == h->stream) return STS_OK;
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    if (!K.gH) {
        const size_t M = (size_t)K.m;
        STS_TRY(dalloc(h, &K.gH, (M + 1) * M));
        STS_TRY(dalloc(h, &K.gcs, M));
        STS_TRY(dalloc(h, &K.gsn, M));
        STS_TRY(dalloc(h, &K.gg, M + 1));
        STS_TRY(dalloc(h, &K.ghist, M));
        STS_TRY(dalloc(h, &K.gpar, 4));
        STS_TRY(dalloc(h, &K.gstate, 2));
        STS_CK(cudaMallocHost(&K.g_pinned, sizeof(double) * ((M + 1) * M + (M + 1) + M + 8)));
    }
    const long long n = (long long)h->b * h->ncp;
    const int ld = m + 2;
    cudaGraph_t graph = nullptr;
    STS_CK(cudaGraphCreate(&graph, 0));
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_error(STS_ERR_CUDA, "gmres graph: cudaStreamCreate failed: %s", cudaGetErrorString(e));
    }
    std::vector<cudaGraphConditionalHandle> hd(m);
    sts_status st = STS_OK;
    for (int j = 0; j < m && e == cudaSuccess; ++j)
        e = cudaGraphConditionalHandleCreate(&hd[j], graph, j == 0 ? 1u : 0u, cudaGraphCondAssignDefault);
    cudaStream_t saved = h->stream;
    // step j + 1's conditional node sits at the end of step j's body, so once a
    // step switches the next one off nothing further of the cycle is evaluated
    cudaGraph_t parent = graph;
    std::vector<cudaGraphNode_t> deps;
    Red R{h, n};
    for (int j = 0; j < m && e == cudaSuccess && st == STS_OK; ++j) {
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = hd[j];
        p.conditional.type = cudaGraphCondTypeIf;
        p.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        e = cudaGraphAddNode(&node, parent, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p);
        if (e != cudaSuccess) break;
        cudaGraph_t body = p.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) break;
        h->stream = cs;
        auto step = [&]() -> sts_status {
            double *vj = K.V + (size_t)j * n, *zj = K.Z + (size_t)j * n;
            if (pre) STS_TRY(opM64(h, dir, vj, zj));
            else STS_CK(cudaMemcpyAsync(zj, vj, n * sizeof(double), cudaMemcpyDeviceToDevice, cs));
            STS_TRY(opA64(h, dir, zj, K.w));
            double *h1 = K.red, *h2 = K.red + ld, *nr = K.red + 2 * ld;
            STS_TRY(R.dots(K.V, j + 1, K.w, 1, h1));
            STS_TRY(R.update(K.w, K.V, j + 1, h1, 0, nullptr));
            STS_TRY(R.dots(K.V, j + 1, K.w, 0, h2));
            STS_TRY(R.update(K.w, K.V, j + 1, h2, 1, nr));
            const int has_next = j + 1 < m ? 1 : 0;
            k_givens<<<1, 32, 0, cs>>>(j, m, K.red, ld, K.gH, K.gcs, K.gsn, K.gg, K.ghist, K.gpar, K.gstate,
                                       has_next ? hd[j + 1] : hd[j], has_next);
            STS_LAUNCHED();
            if (has_next) {
                k_scale_dev<<<grid_for(n, 256), 256, 0, cs>>>(K.V + (size_t)(j + 1) * n, K.w, K.gpar + 2, n);
                STS_LAUNCHED();
            }
            return STS_OK;
        };
        st = step();
        h->stream = saved;
        if (st == STS_OK) {
            cudaStreamCaptureStatus cst;
            const cudaGraphNode_t *last = nullptr;
            size_t nlast = 0;
            e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &last, nullptr, &nlast);
            if (e == cudaSuccess) deps.assign(last, last + nlast);
        }
        cudaGraph_t captured = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
        if (e == cudaSuccess) e = e2;
        parent = body;
    }
    h->stream = saved;
    if (st == STS_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (st != STS_OK) return st;
    if (e != cudaSuccess) {
        exec = nullptr;
        return set_error(STS_ERR_CUDA, "gmres graph: building the cycle graph failed: %s", cudaGetErrorString(e));
    }
    K.g_m[dir][pre ? 1 : 0] = m;
    K.g_stream[dir][pre ? 1 : 0] = h->stream;
    return STS_OK;
}

}  // namespace

// Krylov building blocks on one handle's internal vectors of n = b * ncp
// entries, for the domain-decomposed driver (kernels_dd.cu).  Reductions leave
// their totals in device memory (out_dev); the caller copies them out.
sts_status kry_reserve(sts_jac_s *h, int m) { return ensure_workspace(h, m, false); }
sts_status kry_dots(sts_jac_s *h, const double *V, int k, const double *w, int self, double *out_dev) {
    Red R{h, (long long)h->b * h->ncp};
    return R.dots(V, k, w, self, out_dev);
}
sts_status kry_update(sts_jac_s *h, double *w, const double *V, int k, const double *hcoef_dev, int norm,
                      double *out_dev) {
    Red R{h, (long long)h->b * h->ncp};
    return R.update(w, V, k, hcoef_dev, norm, out_dev);
}
sts_status kry_norm2(sts_jac_s *h, const double *v, double *out_dev) {
    Red R{h, (long long)h->b * h->ncp};
    return R.norm2(v, out_dev);
}
sts_status kry_sub(sts_jac_s *h, double *r, const double *b, const double *y) {
    const long long n = (long long)h->b * h->ncp;
    k_sub<<<grid_for(n, 256), 256, 0, h->stream>>>(r, b, y, n);
    STS_LAUNCHED();
    return STS_OK;
}
sts_status kry_scale(sts_jac_s *h, double *out, const double *in, double s) {
    const long long n = (long long)h->b * h->ncp;
    k_scale<<<grid_for(n, 256), 256, 0, h->stream>>>(out, in, s, n);
    STS_LAUNCHED();
    return STS_OK;
}
sts_status kry_axpy(sts_jac_s *h, double *x, const double *Z, int k, const double *y_dev) {
    const long long n = (long long)h->b * h->ncp;
    k_axpy_multi<double><<<grid_for(n, 256), 256, 0, h->stream>>>(x, Z, n, y_dev, k);
    STS_LAUNCHED();
    return STS_OK;
}

sts_status op_matvec64(sts_jac_s *h, int dir, const double *x, double *y) { return opA64(h, dir, x, y); }
sts_status op_apply64(sts_jac_s *h, int dir, const double *x, double *z) { return opM64(h, dir, x, z); }

sts_status gmres(sts_jac_s *h, const double *b_pub, double *x_pub, const sts_gmres_opts *o,
                 sts_gmres_info *info) {
    sts_gmres_opts d{};
    if (o) d = *o;
    const int m = d.restart > 0 ? d.restart : 30;
    const int max_iters = d.max_iters > 0 ? d.max_iters : 1000;
    const double rtol = d.rtol > 0 ? d.rtol : 1e-10;
    const double inner = d.inner_rtol > 0 ? d.inner_rtol : 1e-6;
    const bool pre = d.precond != STS_PRECOND_NONE;
    const int dir = d.trans ? 1 : 0;
    const bool mixed = d.mixed != 0;
    const bool left = d.left != 0;
    // graph cycles for right preconditioning in FP64, unless the caller asks for
    // host-driven steps; restart lengths above 64 keep the host loop (a step's
    // conditional node is nested in the previous step's body)
    const bool use_graph = d.arnoldi != STS_ARNOLDI_HOST && !left && !mixed && m <= 64;
    if (left && (!pre || mixed))
        return set_error(STS_ERR_INVALID_ARG, "gmres: left preconditioning needs precond BJ and mixed = 0");
    if (d.precond != STS_PRECOND_BJ && d.precond != STS_PRECOND_NONE)
        return set_error(STS_ERR_INVALID_ARG, "gmres: unknown precond %d", d.precond);
    if (m > 512) return set_error(STS_ERR_INVALID_ARG, "gmres: restart %d exceeds 512", m);
    if (dir == 1 && (!h->has_T || h->rep != STS_REP_FACTORED))
        return set_error(STS_ERR_INVALID_ARG, "gmres: trans = 1 needs a factored handle created with enable_transpose");
    if (mixed && (h->dtype != STS_MIXED || h->rep != STS_REP_FACTORED))
        return set_error(STS_ERR_INVALID_ARG, "gmres: mixed = 1 needs a factored handle created with dtype STS_MIXED");
    if (pre) {
        const bool ready = h->rep == STS_REP_FACTORED ? h->smw.ready : h->dense.ready;
        if (!ready) return set_error(STS_ERR_NOT_SETUP, "gmres: block-Jacobi preconditioner used before sts_jac_bjacobi_setup");
    }
    STS_TRY(ensure_workspace(h, m, mixed));
    Krylov &K = h->kry;
    const long long n = (long long)h->b * h->ncp;
    Red R{h, n};
    const int nb = grid_for(n, 256);
    const size_t vbytes = (size_t)h->nc * h->b * sizeof(double);
    // inputs into the internal layout
    const double *b_src = b_pub;
    const double *x_src = x_pub;
    if (d.vectors_on_host) {
        STS_CK(cudaMemcpyAsync(h->vin, b_pub, vbytes, cudaMemcpyHostToDevice, h->stream));
        STS_TRY(to_internal64(h, h->vin, K.bb));
        STS_CK(cudaMemcpyAsync(h->vin, x_pub, vbytes, cudaMemcpyHostToDevice, h->stream));
        STS_TRY(to_internal64(h, h->vin, K.xb));
    } else {
        STS_TRY(to_internal64(h, b_src, K.bb));
        STS_TRY(to_internal64(h, x_src, K.xb));
    }
    double *hp = K.h_pinned;
    // ||b||^2 and ||x0||^2: a zero guess starts from r = b without a product
    STS_TRY(R.norm2(K.bb, K.red));
    STS_TRY(R.norm2(K.xb, K.red + 1));
    STS_CK(cudaMemcpyAsync(hp, K.red, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    STS_CK(cudaStreamSynchronize(h->stream));
    const double bnorm = std::sqrt(hp[0]);
    bool zero_guess = hp[1] == 0.0;
    if (!std::isfinite(bnorm)) return set_error(STS_ERR_NUMERIC, "gmres: right-hand side has NaN or Inf");
    sts_gmres_info inf{0, 0, 1, 0.0, 0, 0};
    sts_status status = STS_OK;
    if (bnorm == 0.0) {
        STS_CK(cudaMemsetAsync(K.xb, 0, n * sizeof(double), h->stream));
    } else {
        std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
        int its = 0;
        for (;;) {
            NvtxRange nvtx_cycle("gmres cycle");
            // true residual r = b - A x (r = b exactly for the zero guess)
            double beta = bnorm;
            if (zero_guess) {
                STS_CK(cudaMemcpyAsync(K.r, K.bb, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
                zero_guess = false;
            } else {
                STS_TRY(opA64(h, dir, K.xb, K.w));
                ++inf.matvecs;
                k_sub<<<nb, 256, 0, h->stream>>>(K.r, K.bb, K.w, n);
                STS_LAUNCHED();
                STS_TRY(R.norm2(K.r, K.red));
                STS_CK(cudaMemcpyAsync(hp, K.red, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
                STS_CK(cudaStreamSynchronize(h->stream));
                beta = std::sqrt(hp[0]);
            }
            if (!std::isfinite(beta)) {
                status = set_error(STS_ERR_NUMERIC, "gmres: residual norm is NaN or Inf");
                break;
            }
            inf.true_rel_residual = beta / bnorm;
            if (beta / bnorm <= rtol) { inf.converged = 1; break; }
            if (its >= max_iters) { inf.converged = 0; break; }
            double stop_abs = mixed ? std::max(rtol * bnorm, inner * beta) : rtol * bnorm;
            double g0 = beta, hscale = 1.0 / bnorm;
            if (left) {
                // z = M r; the cycle works on the preconditioned residual
                STS_TRY(opM64(h, dir, K.r, K.tmp));
                ++inf.applies;
                STS_TRY(R.norm2(K.tmp, K.red));
                STS_CK(cudaMemcpyAsync(hp, K.red, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
                STS_CK(cudaStreamSynchronize(h->stream));
                g0 = std::sqrt(hp[0]);
                if (!std::isfinite(g0) || g0 == 0.0) {
                    status = set_error(STS_ERR_NUMERIC, "gmres: preconditioned residual norm is %g", g0);
                    break;
                }
                stop_abs = g0 * (rtol * bnorm / beta);
                hscale = beta / (g0 * bnorm);
            }
            k_scale<<<nb, 256, 0, h->stream>>>(K.V, left ? K.tmp : K.r, 1.0 / g0, n);
            STS_LAUNCHED();
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = g0;
            int k = 0;
            if (use_graph) {
                // the whole cycle on the device; one synchronisation to read its rotated system
                NvtxRange nvtx_graph("gmres cycle graph");
                STS_TRY(cycle_graph(h, m, dir, pre));
                double *pp = K.g_pinned;
                const size_t nH = (size_t)(m + 1) * m;
                double *pH = pp + 8, *pg = pH + nH, *ph = pg + (m + 1);
                int *ps = reinterpret_cast<int *>(pp + 4);
                pp[0] = stop_abs;
                pp[1] = hscale;
                pp[2] = 0.0;
                pp[3] = (double)std::min(m, max_iters - its);
                for (int i = 0; i <= m; ++i) pg[i] = g[i];
                STS_CK(cudaMemcpyAsync(K.gpar, pp, sizeof(double) * 4, cudaMemcpyHostToDevice, h->stream));
                STS_CK(cudaMemcpyAsync(K.gg, pg, sizeof(double) * (m + 1), cudaMemcpyHostToDevice, h->stream));
                STS_CK(cudaGraphLaunch(K.gexec[dir][pre ? 1 : 0], h->stream));
                STS_CK(cudaMemcpyAsync(ps, K.gstate, sizeof(int) * 2, cudaMemcpyDeviceToHost, h->stream));
                STS_CK(cudaMemcpyAsync(pH, K.gH, sizeof(double) * nH, cudaMemcpyDeviceToHost, h->stream));
                STS_CK(cudaMemcpyAsync(pg, K.gg, sizeof(double) * (m + 1), cudaMemcpyDeviceToHost, h->stream));
                STS_CK(cudaMemcpyAsync(ph, K.ghist, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream));
                STS_CK(cudaStreamSynchronize(h->stream));
                k = ps[0];
                if (ps[1] == 2) {
                    status = set_error(STS_ERR_NUMERIC, "gmres: NaN or Inf in the Arnoldi process");
                    break;
                }
                std::copy(pH, pH + nH, H.begin());
                std::copy(pg, pg + (m + 1), g.begin());
                for (int i = 0; i < k; ++i)
                    if (d.history && its + i < max_iters) d.history[its + i] = ph[i];
                its += k;
                inf.matvecs += k;
                if (pre) inf.applies += k;
            }
            for (int j = 0; j < m && !use_graph; ++j) {
                NvtxRange nvtx_step("gmres arnoldi step");
                double *vj = K.V + (size_t)j * n;
                // z_j = M v_j, w = A z_j (left: w = M (A v_j))
                if (left) {
                    STS_TRY(opA64(h, dir, vj, K.tmp));
                    STS_TRY(opM64(h, dir, K.tmp, K.w));
                    ++inf.matvecs;
                    ++inf.applies;
                } else if (!mixed) {
                    double *zj = K.Z + (size_t)j * n;
                    if (pre) STS_TRY(opM64(h, dir, vj, zj));
                    else STS_CK(cudaMemcpyAsync(zj, vj, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
                    STS_TRY(opA64(h, dir, zj, K.w));
                    ++inf.matvecs;
                    if (pre) ++inf.applies;
                } else {
                    float *zj = K.Z32 + (size_t)j * n;
                    k_convert<float, double><<<nb, 256, 0, h->stream>>>(pre ? K.t32a : zj, vj, n);
                    STS_LAUNCHED();
                    if (pre) STS_TRY(smw_apply32(h, dir, K.t32a, zj));
                    STS_TRY(mv_apply32(h, dir, zj, K.t32b, h->c32));
                    k_convert<double, float><<<nb, 256, 0, h->stream>>>(K.w, K.t32b, n);
                    STS_LAUNCHED();
                }
                // CGS2: h1 = V^T w (+ w.w), w -= V h1; h2 = V^T w, w -= V h2, ||w||^2
                double *h1 = K.red, *h2 = K.red + (m + 2), *nr = K.red + 2 * (m + 2);
                STS_TRY(R.dots(K.V, j + 1, K.w, 1, h1));
                STS_TRY(R.update(K.w, K.V, j + 1, h1, 0, nullptr));
                STS_TRY(R.dots(K.V, j + 1, K.w, 0, h2));
                STS_TRY(R.update(K.w, K.V, j + 1, h2, 1, nr));
                STS_CK(cudaMemcpyAsync(hp, K.red, sizeof(double) * 3 * (m + 2), cudaMemcpyDeviceToHost, h->stream));
                STS_CK(cudaStreamSynchronize(h->stream));
                const double *H1 = hp, *H2 = hp + (m + 2);
                const double w0 = std::sqrt(H1[j + 1]);
                double hn = std::sqrt(hp[2 * (m + 2)]);
                bool bad = !std::isfinite(w0) || !std::isfinite(hn);
                for (int i = 0; i <= j; ++i) {
                    H[(size_t)i * m + j] = H1[i] + H2[i];
                    bad = bad || !std::isfinite(H[(size_t)i * m + j]);
                }
                if (bad) { status = set_error(STS_ERR_NUMERIC, "gmres: NaN or Inf in the Arnoldi process"); break; }
                H[(size_t)(j + 1) * m + j] = hn;
                for (int i = 0; i < j; ++i) {
                    const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
                    H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
                    H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
                }
                const double hjj = H[(size_t)j * m + j];
                const double den = std::hypot(hjj, hn);
                cs[j] = hjj / den;
                sn[j] = hn / den;
                H[(size_t)j * m + j] = den;
                H[(size_t)(j + 1) * m + j] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                ++its;
                k = j + 1;
                if (d.history && its <= max_iters) d.history[its - 1] = std::fabs(g[j + 1]) * hscale;
                const bool happy = hn <= 1e-14 * w0;
                if (happy || std::fabs(g[j + 1]) <= stop_abs || its >= max_iters) break;
                k_scale<<<nb, 256, 0, h->stream>>>(K.V + (size_t)(j + 1) * n, K.w, 1.0 / hn, n);
                STS_LAUNCHED();
            }
            if (status != STS_OK) break;
            for (int i = k - 1; i >= 0; --i) {
                double s = g[i];
                for (int l = i + 1; l < k; ++l) s -= H[(size_t)i * m + l] * y[l];
                y[i] = s / H[(size_t)i * m + i];
            }
            std::copy(y.begin(), y.begin() + k, hp);
            STS_CK(cudaMemcpyAsync(K.red, hp, sizeof(double) * k, cudaMemcpyHostToDevice, h->stream));
            if (!mixed) k_axpy_multi<double><<<nb, 256, 0, h->stream>>>(K.xb, left ? K.V : K.Z, n, K.red, k);
            else k_axpy_multi<float><<<nb, 256, 0, h->stream>>>(K.xb, K.Z32, n, K.red, k);
            STS_LAUNCHED();
            ++inf.restarts;
        }
        inf.iterations = its;
    }
    if (status == STS_OK || status == STS_ERR_NOT_CONVERGED) {
        if (d.vectors_on_host) {
            STS_TRY(from_internal64(h, K.xb, h->vout));
            STS_CK(cudaMemcpyAsync(x_pub, h->vout, vbytes, cudaMemcpyDeviceToHost, h->stream));
        } else {
            STS_TRY(from_internal64(h, K.xb, x_pub));
        }
        STS_CK(cudaStreamSynchronize(h->stream));
    }
    if (info) *info = inf;
    if (status != STS_OK) return status;
    if (!inf.converged)
        return set_error(STS_ERR_NOT_CONVERGED, "gmres: %d iterations, true relative residual %.3e > rtol %.3e",
                         inf.iterations, inf.true_rel_residual, rtol);
    return STS_OK;
}

}  // namespace sts
