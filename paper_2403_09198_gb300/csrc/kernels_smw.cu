// kernels_smw.cu -- block-Jacobi through the Sherman-Morrison-Woodbury formula
// (Section 6).  Each diagonal block is A_k = A_k^0 + U_k V_k^T with A_k^0 = S_kk
// sparse (Eq. R1_Block_Jacobian).
//
// Setup (all cells share one schedule; thread index = cell, fastest):
//   LU of A_k^0 without pivoting on the symbolic schedule of the shared
//   pattern (natural order; for the paper's arrow pattern there is no fill),
//   one thread per cell;
//   W_k = (A_k^0)^-1 U_k   (SMW-1, r sparse solves), one thread per solve;
//   C_k = I + V_k^T W_k    (FP64), one thread per entry; C_k^-1 by Gauss-Jordan
//   with pivoting, one thread per cell.
// Apply (SMW-1..3): x0 = (A_k^0)^-1 b_k, t = V_k^T x0, z = C_k^-1 t (FP64),
//   x_k = x0 - W_k z.  The paper prints "+ W_k z"; with C_k = I + V^T A0^-1 U the
//   Woodbury identity needs the minus sign, which is what is computed here.
// Transposed apply: (A0 + U V^T)^-T = (A0^T + V U^T)^-1, i.e. the same steps with
//   A0^T (solved from the same LU factors), U and V swapped and C_k^T.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdio>
#include <type_traits>
#include <vector>

#include "ring.cuh"
#include "smw_stream.cuh"
#include "sts_internal.h"

namespace sts {
namespace {

struct SetupArgs {
    const double *Sd, *Ud, *Vd;
    double *lu, *dinv, *W, *Wt, *Cinv;
    const int *lu_diag, *src_slot, *d_ptr;
    const int *colL_ptr, *colL_slot, *upd_ptr, *upd_tgt, *upd_src;
    const int *fwd_ptr0, *fwd_col0, *fwd_slot0, *bwd_ptr0, *bwd_col0, *bwd_slot0;
    const int *fwd_ptr1, *fwd_col1, *fwd_slot1, *bwd_ptr1, *bwd_col1, *bwd_slot1;
    int *err_cell;
    int nc, ncp, b, r, nnz_lu, nnz_d, with_T;
};

// Solve A0 w = rhs in place on w[q * ncp + cell] (column of W), N direction.
__device__ void lu_solve_N(const SetupArgs &a, double *w, int cell) {
    const size_t P = a.ncp;
    for (int i = 0; i < a.b; ++i) {
        double acc = w[i * P + cell];
        for (int e = a.fwd_ptr0[i]; e < a.fwd_ptr0[i + 1]; ++e)
            acc = fma(-a.lu[(size_t)a.fwd_slot0[e] * P + cell], w[(size_t)a.fwd_col0[e] * P + cell], acc);
        w[i * P + cell] = acc;
    }
    for (int r = 0; r < a.b; ++r) {
        const int i = a.b - 1 - r;
        double acc = w[i * P + cell];
        for (int e = a.bwd_ptr0[r]; e < a.bwd_ptr0[r + 1]; ++e)
            acc = fma(-a.lu[(size_t)a.bwd_slot0[e] * P + cell], w[(size_t)a.bwd_col0[e] * P + cell], acc);
        w[i * P + cell] = acc * a.dinv[i * P + cell];
    }
}

// Solve A0^T w = rhs in place: U^T (forward, with the pivots), then L^T (unit).
__device__ void lu_solve_T(const SetupArgs &a, double *w, int cell) {
    const size_t P = a.ncp;
    for (int i = 0; i < a.b; ++i) {
        double acc = w[i * P + cell];
        for (int e = a.fwd_ptr1[i]; e < a.fwd_ptr1[i + 1]; ++e)
            acc = fma(-a.lu[(size_t)a.fwd_slot1[e] * P + cell], w[(size_t)a.fwd_col1[e] * P + cell], acc);
        w[i * P + cell] = acc * a.dinv[i * P + cell];
    }
    for (int r = 0; r < a.b; ++r) {
        const int i = a.b - 1 - r;
        double acc = w[i * P + cell];
        for (int e = a.bwd_ptr1[r]; e < a.bwd_ptr1[r + 1]; ++e)
            acc = fma(-a.lu[(size_t)a.bwd_slot1[e] * P + cell], w[(size_t)a.bwd_col1[e] * P + cell], acc);
        w[i * P + cell] = acc;
    }
}

// Setup step 1, one thread per cell: the static-pivot LU of S_kk on the shared
// schedule.  A padding cell gets the identity, so steps 2 and 3 give it W = 0 and
// C^-1 = I without a special case.
__global__ void k_smw_lu(SetupArgs a) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= a.ncp) return;
    const size_t P = a.ncp;
    for (int s = 0; s < a.nnz_lu; ++s) a.lu[s * P + cell] = 0.0;
    if (cell >= a.nc) {
        for (int i = 0; i < a.b; ++i) {
            a.lu[(size_t)a.lu_diag[i] * P + cell] = 1.0;
            a.dinv[i * P + cell] = 1.0;
        }
        return;
    }
    for (int e = 0; e < a.nnz_d; ++e) a.lu[(size_t)a.src_slot[e] * P + cell] = a.Sd[e * P + cell];
    for (int k = 0; k < a.b; ++k) {
        double rowmax = 0.0;
        for (int e = a.d_ptr[k]; e < a.d_ptr[k + 1]; ++e) rowmax = fmax(rowmax, fabs(a.Sd[e * P + cell]));
        const double piv = a.lu[(size_t)a.lu_diag[k] * P + cell];
        if (!(fabs(piv) > 1e-14 * rowmax)) {
            atomicMin(a.err_cell, cell);
            return;
        }
        const double d = 1.0 / piv;
        a.dinv[k * P + cell] = d;
        for (int e = a.colL_ptr[k]; e < a.colL_ptr[k + 1]; ++e) {
            const size_t sl = (size_t)a.colL_slot[e] * P + cell;
            const double l = a.lu[sl] * d;
            a.lu[sl] = l;
            for (int u = a.upd_ptr[e]; u < a.upd_ptr[e + 1]; ++u)
                a.lu[(size_t)a.upd_tgt[u] * P + cell] =
                    fma(-l, a.lu[(size_t)a.upd_src[u] * P + cell], a.lu[(size_t)a.upd_tgt[u] * P + cell]);
        }
    }
}

// Setup step 2, one thread per (cell, pair k, direction): W_k = A0^-1 U_k (SMW-1)
// and, for the adjoint, Wt_k = A0^-T V_k.  Consecutive threads take consecutive
// cells, so every [slot][cell] access of a warp is one coalesced request.
__global__ void k_smw_w(SetupArgs a) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per_dir = (long long)a.ncp * a.r;
    if (t >= per_dir * (a.with_T ? 2 : 1)) return;
    const int dir = (int)(t / per_dir);
    const long long u = t - dir * per_dir;
    const int k = (int)(u / a.ncp), cell = (int)(u - (long long)k * a.ncp);
    const size_t P = a.ncp;
    double *w = (dir ? a.Wt : a.W) + (size_t)k * a.b * P;
    const double *src = (dir ? a.Vd : a.Ud) + (size_t)k * a.b * P;
    for (int q = 0; q < a.b; ++q) w[q * P + cell] = src[q * P + cell];
    if (dir) lu_solve_T(a, w, cell);
    else lu_solve_N(a, w, cell);
}

// Setup step 3a, one thread per (cell, k, l): C_kl = delta_kl + V_k . W_l (FP64),
// written into the C^-1 array, which step 3b inverts in place.
__global__ void k_smw_cmat(SetupArgs a) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = a.r;
    if (t >= (long long)a.ncp * r * r) return;
    const int kl = (int)(t / a.ncp), cell = (int)(t - (long long)kl * a.ncp);
    const int k = kl / r, l = kl - k * r;
    const size_t P = a.ncp;
    const double *v = a.Vd + (size_t)k * a.b * P + cell, *w = a.W + (size_t)l * a.b * P + cell;
    double acc = k == l ? 1.0 : 0.0;
    for (int q = 0; q < a.b; ++q) acc = fma(v[q * P], w[q * P], acc);
    a.Cinv[(size_t)kl * P + cell] = acc;
}

// Setup step 3b, one thread per cell: C^-1 by Gauss-Jordan with partial pivoting,
// in place in the C^-1 array.
__global__ void k_smw_cinv(SetupArgs a) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= a.ncp) return;
    const size_t P = a.ncp;
    const int r = a.r;
    double C[kMaxPairsDiag][kMaxPairsDiag], X[kMaxPairsDiag][kMaxPairsDiag];
    double cmax = 0.0;
    for (int k = 0; k < r; ++k)
        for (int l = 0; l < r; ++l) {
            C[k][l] = a.Cinv[((size_t)k * r + l) * P + cell];
            X[k][l] = k == l ? 1.0 : 0.0;
            cmax = fmax(cmax, fabs(C[k][l]));
        }
    for (int k = 0; k < r; ++k) {
        int pr = k;
        for (int i = k + 1; i < r; ++i)
            if (fabs(C[i][k]) > fabs(C[pr][k])) pr = i;
        if (!(fabs(C[pr][k]) > 1e-14 * cmax)) {
            atomicMin(a.err_cell, cell);
            return;
        }
        if (pr != k)
            for (int j = 0; j < r; ++j) {
                double t = C[k][j]; C[k][j] = C[pr][j]; C[pr][j] = t;
                t = X[k][j]; X[k][j] = X[pr][j]; X[pr][j] = t;
            }
        const double d = 1.0 / C[k][k];
        for (int j = 0; j < r; ++j) { C[k][j] *= d; X[k][j] *= d; }
        for (int i = 0; i < r; ++i) {
            if (i == k) continue;
            const double f = C[i][k];
            for (int j = 0; j < r; ++j) { C[i][j] -= f * C[k][j]; X[i][j] -= f * X[k][j]; }
        }
    }
    for (int k = 0; k < r; ++k)
        for (int l = 0; l < r; ++l) a.Cinv[((size_t)k * r + l) * P + cell] = X[k][l];
}

// Write the apply streams: forward coefficients, then per backward row its
// pivot inverse followed by its coefficients (scaled by the row's dinv where the
// program asks for it).
template <typename T>
__global__ void k_smw_pack(T *out, const double *lu, const double *dinv, const int *pk_slot,
                           const int *pk_scale, int len, int ncp) {
    const long long total = (long long)len * ncp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int cell = (int)(i % ncp), pos = (int)(i / ncp);
        const int sl = pk_slot[pos], sc = pk_scale[pos];
        double v;
        if (sl >= 0) {
            v = lu[(size_t)sl * ncp + cell];
            if (sc >= 0) v *= dinv[(size_t)sc * ncp + cell];
        } else {
            v = dinv[(size_t)sc * ncp + cell];
        }
        out[i] = (T)v;
    }
}

template <typename T>
__global__ void k_round(T *out, const double *in, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (T)in[i];
}

template <typename T>
struct ApplyArgs {
    const T *st;            // [len][ncp] stream
    const unsigned *desc;   // [len] apply program
    const T *dv;            // [r][b][ncp] dot vectors (V for N, U for T)
    const T *W;             // [r][b][ncp] (W for N, Wt for T)
    const double *Cinv;     // [r][r][ncp]
    const T *x;
    T *y;
    int len, b, r, ncp, trans;
};

constexpr int kApStage = 32;    // stream positions per shared-memory stage
constexpr int kApStages = 3;    // stages in flight (two ahead of the one consumed)

// One warp per 32 cells, one lane per cell.  The tile's apply stream is
// copied into a ring of shared-memory stages with cp.async two stages ahead of
// its use; the working vector lives in shared memory [q][lane]; the triangular
// sweeps run a flat program (one descriptor per stream position).
template <typename T, int RMAX>
__global__ void __launch_bounds__(32) k_smw_apply(ApplyArgs<T> a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *stg = reinterpret_cast<T *>(smem_raw);                  // [kApStages][kApStage][32]
    T *w = stg + kApStages * kApStage * kTile;                  // [b][32]
    const int lane = threadIdx.x;
    const int tile = blockIdx.x;
    const int cell = tile * kTile + lane;
    const size_t P = a.ncp;
    const T *__restrict__ x = a.x;
    Ring<T, kApStage, kApStages> R;
    R.start(stg, a.st + (size_t)tile * kTile, P, a.len, lane);
    for (int i = 0; i < a.b; ++i) w[i * kTile + lane] = __ldg(x + i * P + cell);
    const unsigned *__restrict__ dd = a.desc;
    T acc = T(0);
    for (int i = 0; i < a.len; ++i) {
        const unsigned d = __ldg(dd + i);
        const T v = R.next();
        const int row = (d >> 12) & 0xfffu, col = d & 0xfffu;
        if (d & kApScale) {
            acc = v * w[row * kTile + lane];
        } else {
            if (d & kApBegin) acc = w[row * kTile + lane];
            acc = fma(-v, w[col * kTile + lane], acc);
        }
        if (d & kApEnd) w[row * kTile + lane] = acc;
    }
    R.finish();
    // t = dv^T x0, z = C^-1 t (FP64), x = x0 - W z
    T t[RMAX];
#pragma unroll
    for (int k = 0; k < RMAX; ++k) t[k] = T(0);
    const T *__restrict__ dv = a.dv + cell;
#pragma unroll 4
    for (int q = 0; q < a.b; ++q) {
        const T xq = w[q * kTile + lane];
#pragma unroll
        for (int k = 0; k < RMAX; ++k)
            if (k < a.r) t[k] = fma(__ldg(dv + ((size_t)k * a.b + q) * P), xq, t[k]);
    }
    T z[RMAX];
#pragma unroll
    for (int k = 0; k < RMAX; ++k) {
        double s = 0.0;
        if (k < a.r) {
#pragma unroll
            for (int l = 0; l < RMAX; ++l)
                if (l < a.r) {
                    const double cij = a.trans ? __ldg(a.Cinv + ((size_t)l * a.r + k) * P + cell)
                                               : __ldg(a.Cinv + ((size_t)k * a.r + l) * P + cell);
                    s = fma(cij, (double)t[l], s);
                }
        }
        z[k] = (T)s;
    }
    const T *__restrict__ Wp = a.W + cell;
#pragma unroll 4
    for (int q = 0; q < a.b; ++q) {
        T v = w[q * kTile + lane];
#pragma unroll
        for (int k = 0; k < RMAX; ++k)
            if (k < a.r) v = fma(-__ldg(Wp + ((size_t)k * a.b + q) * P), z[k], v);
        a.y[q * P + cell] = v;
    }
}

// ---------------------------------------------------------------------------
// Structured apply for the paper's pattern family (level band of half-width W
// plus NF = 3 dense flow rows / columns).  Its LU has no fill:
//   L: level row i holds the band (i, i-W..i-1); flow rows are dense.
//   U: level row i holds (i, i..i+W) and the flow columns; the flow block is
//      upper triangular.
// Both directions are "forward unit-lower arrow-band sweep, then backward
// scaled unit-upper arrow-band sweep" over a per-direction coefficient stream:
//   forward level row i:  W band coefficients (oldest first), then the NF
//                          coefficients of the flow rows in column i, which
//                          feed NF independent accumulators;
//   forward flow rows:    the 3 coefficients among the flow unknowns;
//   backward flow rows:   per row its pivot inverse and coefficients, then the
//                          RMAX dot-vector entries of t = V^T x0 for that unknown
//                          (one group, or one group per row where the three
//                          rows are wider than a chunk);
//   backward level row i: pivot inverse, NF flow coefficients, W band
//                          coefficients (farthest first), RMAX dot-vector entries;
//   tail:                 W[a][q] for the correction x = x0 - W C^-1 t, with
//                          C^-1 read per cell (FP64, r x r registers); in the
//                          instances that fold (sap_fold) the capacitance solve
//                          is folded into the tail instead: (W C^-1)[q][a],
//                          formed in FP64 when the stream is packed, and
//                          x = x0 - (W C^-1) t needs neither C^-1 nor its registers.
// A cell with fewer than RMAX pairs has zero dot and tail entries.
// The band recurrences keep their last W values in registers, so the only
// dependency chain is one FMA per row.
//
// Stream layout.  Rows are packed in groups of whole 16-byte vectors (VEC =
// 16 / sizeof(T) positions): a group is a run of consecutive rows of one
// section whose width is a multiple of VEC and at least 16 positions (rows
// past the end of the section are zero; see sap_group_rows), or one single row
// padded with zeros.  Groups never
// straddle a chunk of K positions (8 KB), and each tile's stream is padded to
// whole chunks, so one tile's stream is Lt contiguous positions stored as
// [tile][position / VEC][lane][VEC]: a chunk is one bulk copy and a lane reads
// VEC positions with one 16-byte shared-memory load.
template <typename T>
struct SApplyArgs {
    const T *st;            // [n_tiles][Lt / VEC][32][VEC]
    const double *Cinv;     // [r][r][ncp] (instances that do not fold only)
    const T *x;
    T *y;
    int *err;               // set when a bounded wait gave up
    int Lt, b, N, r, ncp, trans, n_tiles;
    int pre;                // the stream and C^-1 may be read before the grid-dependency wait
    int evict_first;        // the stream of one call is larger than L2
};

constexpr int kApWarps = 4;              // consumer warps per block of the structured apply (one per sub-partition)
constexpr int kSApStages = 5;            // ring stages of the structured apply (three chunks in flight)
constexpr int kSApChunkBytes = 8192;     // bytes per stage (one bulk copy)

// Pair slots RMAX of the structured apply instance for r pairs per diagonal
// block and band half-width w: 2, 4, or nine (one source pair plus two per face
// of a 2D cell, Section 4.3).  Ten for w = 4, whose backward rows are then 18
// positions wide instead of 17 (two 17-wide rows would not fit one chunk), and
// for w = 2, whose 16-wide rows then form one-row groups: the extra zero slot
// costs two FMAs per row but frees the registers a second row would hold.
// 0: more pairs than any structured instance holds.
__host__ __device__ constexpr int sap_rmax_big(int w) { return w == 2 || w == 4 ? 10 : 9; }
__host__ __device__ constexpr int sap_rmax(int r, int w) {
    return r <= 2 ? 2 : r <= 4 ? 4 : r <= sap_rmax_big(w) ? sap_rmax_big(w) : 0;
}
// Whether the instance folds C^-1 into its tail vectors: always above four
// pairs, and wherever the r x r FP64 registers of the unfolded form would spill
// (more than two pairs, or band half-width 1 or 4, by the ptxas register
// reports).  Where both fit, the unfolded form measured faster (band 2, two pairs).
__host__ __device__ constexpr bool sap_fold(int rmax, int w) { return rmax > 2 || w == 1 || w == 4; }

// Rows per group: the fewest rows of whole vectors, repeated up to at least 16
// positions (the per-group bookkeeping is then spread over 16 or more FMAs);
// forward groups hold at most NF + 1 rows, so that their working-vector reads
// past the last level row stay inside the block.
__host__ __device__ constexpr int sap_group_rows(int width, int vec) {
    return sap_rows(width, vec) * ((16 + sap_rows(width, vec) * width - 1) / (sap_rows(width, vec) * width));
}
__host__ __device__ constexpr int sap_fwd_rows(int width, int vec, int nf) {
    return sap_group_rows(width, vec) <= nf + 1 ? sap_group_rows(width, vec)
                                                : (sap_rows(width, vec) > nf + 1 ? sap_rows(width, vec) : nf + 1 -
                                                   (nf + 1) % sap_rows(width, vec));
}
// shared memory of one consumer warp: stages, 128 bytes of mbarriers (full,
// empty, the first tile's x), working vector [b][32]
constexpr int kSApBarBytes = 128;
static_assert((2 * kSApStages + 1) * 8 <= kSApBarBytes, "full, empty and x barriers fit");
__host__ __device__ inline size_t sap_warp_bytes(int b, int elem) {
    const size_t raw = (size_t)kSApStages * kSApChunkBytes + kSApBarBytes + (size_t)b * kTile * elem;
    return (raw + 127) / 128 * 128;
}


// Consumer warp w of block k takes tiles w * gridDim.x + k, + nc * gridDim.x,
// ... so that tiles are dealt to SMs round-robin and no sub-partition runs two
// tiles while another idles; the block's last warp is the producer, whose
// lane 0 issues every bulk copy of the block's rings.  A consumer's tiles form
// one continuous stream for its ring, so the next tile's first chunks arrive
// during the current tail; the next tile's x is copied into the working vector
// one group of rows at a time as the tail frees it.  Within a section the next group
// (coefficients and working-vector entries) is loaded into registers before
// the current one is used, so the shared-memory latency overlaps the FMAs.
//
// GW: the working vector lives in y instead of shared memory (the forward
// sweep reads x from global memory and writes its rows into y; the backward
// sweep and the tail read and rewrite them in place, loaded a group ahead so
// the L2 latency overlaps the FMAs).  Chosen where b rows per warp would leave
// fewer than four consumers per SM (b > 65 in FP64, b > 131 in FP32): the ring
// alone then fits four.  Plain (coherent) loads throughout, since the kernel
// rewrites the rows it reads and x may be y.  wl is then not used.
template <typename T, int W, int RMAX, bool GW>
__global__ void __launch_bounds__((kApWarps + 1) * 32) k_smw_sapply(SApplyArgs<T> a) {
    constexpr int NF = kStructNF, VEC = 16 / (int)sizeof(T);
    constexpr int K = kSApChunkBytes / (kTile * (int)sizeof(T));
    constexpr int FW = W + NF, UF = sap_fwd_rows(FW, VEC, NF), GF = UF * FW;
    constexpr int GFF = sap_round(3, VEC), GBF = sap_round(6 + 3 * RMAX, VEC);
    // the three backward flow rows form one group, or one group each where that is wider than a chunk
    constexpr bool FSPLIT = GBF > K;
    constexpr int G2 = sap_round(1 + RMAX, VEC), G1 = sap_round(2 + RMAX, VEC), G0 = sap_round(3 + RMAX, VEC);
    constexpr int BW = 1 + NF + W + RMAX, UB = sap_group_rows(BW, VEC), GB = UB * BW;
    constexpr int UT = sap_group_rows(RMAX, VEC), GT = UT * RMAX;
    static_assert(GF % VEC == 0 && GB % VEC == 0 && GT % VEC == 0, "groups are whole vectors");
    static_assert(GF <= K && G0 <= K && GB <= K && GT <= K, "groups fit a chunk");
    constexpr bool FOLD = sap_fold(RMAX, W);
    static_assert(UF <= NF + 1, "forward rows read past N stay inside the block");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nc = (int)(blockDim.x >> 5) - 1;                  // consumer warps
    const size_t wbytes = sap_warp_bytes(GW ? 0 : a.b, (int)sizeof(T));
    const int nw = nc * gridDim.x;
    const int nch = a.Lt / K;
    if (threadIdx.x == 0) {
        for (int w = 0; w < nc; ++w) {
            const uint32_t full = smem_addr(smem_raw + (size_t)w * wbytes + (size_t)kSApStages * kSApChunkBytes);
#pragma unroll
            for (int st = 0; st < kSApStages; ++st) {
                mbar_init(full + 8u * st, 1);
                mbar_init(full + 8u * (kSApStages + st), 32);
            }
            mbar_init(full + 8u * (2 * kSApStages), 1);     // the first tile's x
        }
        mbar_init_fence();
    }
    __syncthreads();
    if (warp == nc) {
        // ---- producer
        if (lane == 0) {
            // the L2 policy of the copies is a template argument: a test in the
            // issue loop slowed the FP32 apply (about 1 us at 128 x 128 cells)
            auto produce = [&](auto evict_first) {
                RingProducer<T, K, kSApStages, kApWarps, decltype(evict_first)::value> pr;
                pr.src = a.st;
                pr.seg_elems = (size_t)a.Lt * kTile;
                pr.nc = nc;
                pr.seg_step = nw;
                pr.nch = nch;
                pr.maxc = 0;
#pragma unroll
                for (int w = 0; w < kApWarps; ++w) {
                    unsigned char *reg = smem_raw + (size_t)min(w, nc - 1) * wbytes;
                    pr.stg[w] = reinterpret_cast<T *>(reg);
                    pr.full[w] = smem_addr(reg + (size_t)kSApStages * kSApChunkBytes);
                    pr.empty[w] = pr.full[w] + 8u * kSApStages;
                    pr.seg0[w] = w * gridDim.x + blockIdx.x;
                    pr.nseg[w] = (w < nc && pr.seg0[w] < a.n_tiles) ? (a.n_tiles - 1 - pr.seg0[w]) / nw + 1 : 0;
                    pr.issued[w] = 0;
                    pr.pk[w] = 0;
                    pr.pl[w] = 0;
                    pr.maxc = max(pr.maxc, pr.nseg[w] * nch);
                }
                bool ok = a.pre ? pr.issue_upto(kSApStages) : true;
                pdl_wait();
                pdl_trigger();
                if (ok) ok = pr.run();
                if (!ok) atomicExch(a.err, 1);
                pr.drain();
            };
            if (a.evict_first) produce(std::true_type{});
            else produce(std::false_type{});
        } else {
            pdl_wait();
            pdl_trigger();
        }
        return;
    }
    // ---- consumers
    const int gw = warp * gridDim.x + blockIdx.x;
    if (gw >= a.n_tiles) return;
    const int my = (a.n_tiles - 1 - gw) / nw + 1;
    const size_t P = a.ncp;
    const int N = a.N, b = a.b, r = a.r;
    unsigned char *mine = smem_raw + (size_t)warp * wbytes;
    const uint32_t full = smem_addr(mine + (size_t)kSApStages * kSApChunkBytes);
    T *wl = reinterpret_cast<T *>(mine + (size_t)kSApStages * kSApChunkBytes + kSApBarBytes) + lane;  // row i at wl[i * 32]
    RingConsumer<T, K, kSApStages> R;
    R.start(reinterpret_cast<T *>(mine), full, full + 8u * kSApStages, lane);
    pdl_wait();
    pdl_trigger();
    // The first tile's x.  FP64: one bulk copy per row (rows lane, lane + 32,
    // ...), completed on the warp's x barrier; per-lane cp.async of the b rows
    // measured slower (their issue stalls once the SM's outstanding loads
    // fill).  FP32 (128-byte rows): per-lane cp.async measured faster (11.5
    // against 12.9 us on 128 x 128 cells, N = 60).
    constexpr bool XBULK = !GW && sizeof(T) == 8;
    const uint32_t xbar = full + 8u * (2 * kSApStages);
    if constexpr (XBULK) {
        if (lane == 0) mbar_expect_tx(xbar, (uint32_t)((size_t)b * kTile * sizeof(T)));
        __syncwarp();
        for (int i = lane; i < b; i += kTile)
            bulk_copy_g2s(smem_addr(wl - lane + (size_t)i * kTile), a.x + (size_t)i * P + (size_t)gw * kTile,
                          (uint32_t)(kTile * sizeof(T)), xbar);
    } else if constexpr (!GW) {
        for (int i = 0; i < b; ++i) cp_async_elem(wl + i * kTile, a.x + (size_t)i * P + (size_t)gw * kTile + lane);
        cp_async_commit();
    }
    for (int k = 0; k < my; ++k) {
        const int cell = (gw + k * nw) * kTile + lane;
        // row j of the working vector, and row j of this tile's x
        auto wv = [&](int j) -> T & {
            if constexpr (GW) return a.y[(size_t)j * P + cell];
            else return wl[j * kTile];
        };
        auto xin = [&](int j) -> T {
            if constexpr (GW) return a.x[(size_t)j * P + cell];
            else return wl[j * kTile];
        };
        double cz[FOLD ? 1 : RMAX * RMAX];      // C^-1 (transposed for A^T), zero outside r x r
        if constexpr (!FOLD) {
#pragma unroll
            for (int i = 0; i < RMAX; ++i)
#pragma unroll
                for (int l = 0; l < RMAX; ++l)
                    cz[i * RMAX + l] =
                        (i < r && l < r) ? __ldg(a.Cinv + (a.trans ? (size_t)l * r + i : (size_t)i * r + l) * P + cell)
                                         : 0.0;
        }
        if constexpr (!GW) {
            if (XBULK && k == 0) {
                if (!mbar_wait_bounded(xbar, 0)) goto fail;
            } else {
                cp_async_wait<0>();             // copied in by the previous tile's tail (or, FP32, before it)
            }
            __syncwarp();
        }
        // ---- forward sweep over the level rows: row i = [W band, oldest first | NF flow]
        T win[W > 0 ? W : 1];
#pragma unroll
        for (int q = 0; q < W; ++q) win[q] = T(0);
        T accf[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) accf[f] = T(0);
        sap_section<T, GF, UF>(
            R, N, [&](int j) { return xin(min(j, b - 1)); },
            [&](const Group<T, GF> &g, T acc, int u, int) {
#pragma unroll
                for (int q = 0; q < W; ++q) acc = fma(-g[u * FW + q], win[q], acc);
#pragma unroll
                for (int f = 0; f < NF; ++f) accf[f] = fma(g[u * FW + W + f], acc, accf[f]);
#pragma unroll
                for (int q = 0; q + 1 < W; ++q) win[q] = win[q + 1];
                if (W > 0) win[W > 0 ? W - 1 : 0] = acc;
                return acc;
            },
            [&](int j, T v) { wv(j) = v; });
        // ---- forward flow rows: (N+1,N), (N+2,N), (N+2,N+1)
        T wf[NF];
        {
            Group<T, GFF> g;
            g.load(R.take(GFF));
            wf[0] = xin(N) - accf[0];
            wf[1] = fma(-g[0], wf[0], xin(N + 1) - accf[1]);
            wf[2] = fma(-g[2], wf[1], fma(-g[1], wf[0], xin(N + 2) - accf[2]));
        }
        // ---- backward flow rows, with t = V^T x0 accumulated on the way
        T t[RMAX];
#pragma unroll
        for (int q = 0; q < RMAX; ++q) t[q] = T(0);
        T xf[NF];
        {
            // rows [d2, V(N+2) | d1, u(N+1,N+2), V(N+1) | d0, u(N,N+1), u(N,N+2), V(N)], V padded to RMAX
            auto flow = [&](auto e2, auto e1, auto e0) {
                xf[2] = e2(0) * wf[2];
#pragma unroll
                for (int q = 0; q < RMAX; ++q) t[q] = fma(e2(1 + q), xf[2], t[q]);
                xf[1] = fma(-e1(1), xf[2], e1(0) * wf[1]);
#pragma unroll
                for (int q = 0; q < RMAX; ++q) t[q] = fma(e1(2 + q), xf[1], t[q]);
                xf[0] = fma(-e0(2), xf[2], fma(-e0(1), xf[1], e0(0) * wf[0]));
#pragma unroll
                for (int q = 0; q < RMAX; ++q) t[q] = fma(e0(3 + q), xf[0], t[q]);
            };
            if constexpr (FSPLIT) {
                Group<T, G2> g2;
                Group<T, G1> g1;
                Group<T, G0> g0;
                g2.load(R.take(G2));
                g1.load(R.take(G1));
                g0.load(R.take(G0));
                flow([&](int e) { return g2[e]; }, [&](int e) { return g1[e]; }, [&](int e) { return g0[e]; });
            } else {
                constexpr int o1 = 1 + RMAX, o0 = o1 + 2 + RMAX;
                Group<T, GBF> g;
                g.load(R.take(GBF));
                flow([&](int e) { return g[e]; }, [&](int e) { return g[o1 + e]; }, [&](int e) { return g[o0 + e]; });
            }
        }
        if (R.failed) goto fail;
        // ---- backward level rows i = N-1-j: [pivot inverse | NF flow | W band, farthest first | V (RMAX)]
        {
            T xw[W > 0 ? W : 1];
#pragma unroll
            for (int q = 0; q < W; ++q) xw[q] = T(0);
            sap_section<T, GB, UB>(
                R, N, [&](int j) { return wv(max(N - 1 - j, 0)); },
                [&](const Group<T, GB> &g, T wi, int u, int) {
                    T acc = g[u * BW] * wi;
#pragma unroll
                    for (int f = 0; f < NF; ++f) acc = fma(-g[u * BW + 1 + f], xf[f], acc);
#pragma unroll
                    for (int q = 0; q < W; ++q) acc = fma(-g[u * BW + 1 + NF + q], xw[W - 1 - q], acc);
#pragma unroll
                    for (int q = 0; q < RMAX; ++q) t[q] = fma(g[u * BW + 1 + NF + W + q], acc, t[q]);
#pragma unroll
                    for (int q = W - 1; q > 0; --q) xw[q] = xw[q - 1];
                    if (W > 0) xw[0] = acc;
                    return acc;
                },
                [&](int j, T v) { wv(N - 1 - j) = v; });
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) wv(N + f) = xf[f];
        // ---- z = C^-1 t in FP64, then x = x0 - W z (tail row q = W[0..RMAX)[q]);
        //      folded: z = t and tail row q = (W C^-1)[q][0..RMAX)
        {
            T z[RMAX];
#pragma unroll
            for (int i = 0; i < RMAX; ++i) {
                if constexpr (FOLD) {
                    z[i] = t[i];
                } else {
                    double sacc = 0.0;
#pragma unroll
                    for (int l = 0; l < RMAX; ++l) sacc = fma(cz[i * RMAX + l], (double)t[l], sacc);
                    z[i] = (T)sacc;
                }
            }
            const T *xn = a.x + (size_t)cell + (size_t)nw * kTile;
            T *y = a.y + cell;
            // the next tile's x is copied in one group of rows at a time, at
            // the group's last row (all its rows have been read by then): a
            // test of the runtime flag on every row measured about 25 cycles
            // a row even when never taken
            const bool more = k + 1 < my;
            sap_section<T, GT, UT>(
                R, b, [&](int j) { return wv(min(j, b - 1)); },
                [&](const Group<T, GT> &g, T val, int u, int j) {
#pragma unroll
                    for (int l = 0; l < RMAX; ++l) val = fma(-g[u * RMAX + l], z[l], val);
                    if constexpr (!GW) {
                        if (u == UT - 1 && more) {
#pragma unroll
                            for (int q = 0; q < UT; ++q)
                                cp_async_elem(wl + (j - q) * kTile, xn + (size_t)(j - q) * P);
                        }
                    }
                    return val;
                },
                [&](int j, T v) { y[(size_t)j * P] = v; });
            if constexpr (!GW) {
                if (more) {
                    for (int j = b / UT * UT; j < b; ++j) cp_async_elem(wl + j * kTile, xn + (size_t)j * P);  // ragged last group
                    cp_async_commit();
                }
            }
        }
        if (R.failed) goto fail;
        R.end_segment();
    }
    return;
fail:
    // the producer waits (bounded) for every copy it issued before it exits;
    // this warp waits (bounded) for its own copies of the first tile's x
    if (lane == 0) atomicExch(a.err, 1);
    if constexpr (XBULK) mbar_wait_bounded(xbar, 0);
    cp_async_wait<0>();
}

// Structured stream packing: per position a source code and argument
//   src >= 0: LU slot (times the pivot inverse of row arg if arg >= 0)
//   src = -1: pivot inverse of row arg      src = -2: dot vector entry arg
//   src = -3: W entry arg                   src = -4: zero
//   src = -5: folded tail entry arg = a * b + q: (W C^-1)[q][a] =
//             sum_l W[l][q] C^-1[l][a], or for the transposed operator
//             sum_l W'[l][q] C^-1[a][l] (C^-T), in FP64
// Output element i is (tile, vector, lane, element) of the layout above.
template <typename T>
__global__ void k_smw_spack(T *out, const double *lu, const double *dinv, const double *DV, const double *WW,
                            const double *Cinv, const int *src, const int *arg, int Lt, int ncp, int b, int r,
                            int trans) {
    constexpr int VEC = 16 / (int)sizeof(T);
    const long long per_tile = (long long)Lt * kTile;
    const long long total = per_tile * (ncp / kTile);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long tile = i / per_tile;
        const int e = (int)(i - tile * per_tile);
        const int pv = e / (kTile * VEC), rem = e - pv * kTile * VEC;
        const int lane = rem / VEC, pos = pv * VEC + rem % VEC;
        const int cell = (int)tile * kTile + lane;
        const int sv = src[pos], ag = arg[pos];
        double v = 0.0;
        if (sv >= 0) {
            v = lu[(size_t)sv * ncp + cell];
            if (ag >= 0) v *= dinv[(size_t)ag * ncp + cell];
        } else if (sv == -1) {
            v = dinv[(size_t)ag * ncp + cell];
        } else if (sv == -2) {
            v = DV[(size_t)ag * ncp + cell];
        } else if (sv == -3) {
            v = WW[(size_t)ag * ncp + cell];
        } else if (sv == -5) {
            const int aa = ag / b, q = ag - aa * b;
            for (int l = 0; l < r; ++l) {
                const double c = Cinv[(size_t)(trans ? aa * r + l : l * r + aa) * ncp + cell];
                v = fma(WW[((size_t)l * b + q) * ncp + cell], c, v);
            }
        }
        out[i] = (T)v;
    }
}

// Repack diagonal-block values into [entry][cell] and the diagonal pairs into
// [k][q][cell]; a cell with fewer than r pairs gets zero pairs (u = v = 0 leaves
// A_k unchanged and adds an identity row and column to C_k).
__global__ void k_smw_repack(double *Sd, double *Ud, double *Vd, const double *S, const double *U,
                             const double *V, const int *diag_blk, const long long *soff,
                             const int *pbase, int nc, int ncp, int nnz_d, int b, int r) {
    const long long nS = (long long)nnz_d * ncp, nP = (long long)r * b * ncp;
    const long long total = nS + nP;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < nS) {
            const int cell = (int)(i % ncp), e = (int)(i / ncp);
            Sd[i] = cell < nc ? S[soff[diag_blk[cell]] + e] : 0.0;
        } else {
            const long long j = i - nS;
            const int cell = (int)(j % ncp);
            const long long kq = j / ncp;
            const int q = (int)(kq % b), k = (int)(kq / b);
            double u = 0.0, v = 0.0;
            if (cell < nc && k < pbase[diag_blk[cell] + 1] - pbase[diag_blk[cell]]) {
                const size_t src = (size_t)(pbase[diag_blk[cell]] + k) * b + q;
                u = U[src];
                v = V[src];
            }
            Ud[j] = u;
            Vd[j] = v;
        }
    }
}

inline int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152LL * 64) g = 152LL * 64;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

// Host: symbolic factorisation of the shared diagonal pattern and the programs
// of the two apply directions.
sts_status smw_build(sts_jac_s *h) {
    SmwPlan &M = h->smw;
    const int b = h->b;
    if (b > 4095) return set_error(STS_ERR_INVALID_ARG, "block_size above 4095 is not supported by the SMW apply");
    if (h->r_diag > kMaxPairsDiag)
        return set_error(STS_ERR_INVALID_ARG, "r_diag = %d exceeds the supported %d pairs per diagonal block",
                         h->r_diag, kMaxPairsDiag);
    std::vector<char> nz((size_t)b * b, 0);
    for (int p = 0; p < b; ++p)
        for (int e = h->dptr[p]; e < h->dptr[p + 1]; ++e) nz[(size_t)p * b + h->didx[e]] = 1;
    for (int k = 0; k < b; ++k)               // symbolic elimination, natural order
        for (int i = k + 1; i < b; ++i)
            if (nz[(size_t)i * b + k])
                for (int j = k + 1; j < b; ++j)
                    if (nz[(size_t)k * b + j]) nz[(size_t)i * b + j] = 1;
    std::vector<int> slot((size_t)b * b, -1);
    M.h_lu_ptr.assign(b + 1, 0);
    M.h_lu_idx.clear();
    M.h_lu_diag.assign(b, -1);
    for (int i = 0; i < b; ++i) {
        for (int j = 0; j < b; ++j)
            if (nz[(size_t)i * b + j]) {
                slot[(size_t)i * b + j] = (int)M.h_lu_idx.size();
                if (i == j) M.h_lu_diag[i] = (int)M.h_lu_idx.size();
                M.h_lu_idx.push_back(j);
            }
        M.h_lu_ptr[i + 1] = (int)M.h_lu_idx.size();
    }
    M.nnz_lu = (int)M.h_lu_idx.size();
    M.h_src_slot.assign(h->nnz_d, 0);
    for (int p = 0; p < b; ++p)
        for (int e = h->dptr[p]; e < h->dptr[p + 1]; ++e) M.h_src_slot[e] = slot[(size_t)p * b + h->didx[e]];
    // factorisation schedule
    std::vector<int> colL_ptr(b + 1, 0), colL_slot, upd_ptr(1, 0), upd_tgt, upd_src;
    for (int k = 0; k < b; ++k) {
        for (int i = k + 1; i < b; ++i) {
            if (slot[(size_t)i * b + k] < 0) continue;
            colL_slot.push_back(slot[(size_t)i * b + k]);
            for (int j = k + 1; j < b; ++j)
                if (slot[(size_t)k * b + j] >= 0) {
                    upd_tgt.push_back(slot[(size_t)i * b + j]);
                    upd_src.push_back(slot[(size_t)k * b + j]);
                }
            upd_ptr.push_back((int)upd_tgt.size());
        }
        colL_ptr[k + 1] = (int)colL_slot.size();
    }
    // apply programs.  dir 0 (A0):  forward  L rows   (i, j<i), coefficient L_ij
    //                               backward U rows   (i, j>i), coefficient U_ij * dinv_i
    //                  dir 1 (A0^T): forward  U cols   (j<i, i), coefficient U_ji * dinv_j
    //                               backward L cols   (j>i, i), coefficient L_ji
    // Setup solves use the unscaled LU slots with the same row lists.
    for (int dir = 0; dir < 2; ++dir) {
        std::vector<int> fptr(b + 1, 0), fcol, fslot, fscale, bptr(b + 1, 0), bcol, bslot, bscale;
        // the setup's unscaled solves use (fcol, fslot) and (bcol, bslot); the
        // apply streams carry the scaled coefficients described by (fscale, bscale)
        for (int i = 0; i < b; ++i) {
            for (int j = 0; j < i; ++j) {
                const int sl = dir == 0 ? slot[(size_t)i * b + j] : slot[(size_t)j * b + i];
                if (sl < 0) continue;
                fcol.push_back(j);
                fslot.push_back(sl);
                fscale.push_back(dir == 0 ? -1 : j);
            }
            fptr[i + 1] = (int)fcol.size();
        }
        for (int r = 0; r < b; ++r) {
            const int i = b - 1 - r;
            for (int j = i + 1; j < b; ++j) {
                const int sl = dir == 0 ? slot[(size_t)i * b + j] : slot[(size_t)j * b + i];
                if (sl < 0) continue;
                bcol.push_back(j);
                bslot.push_back(sl);
                bscale.push_back(dir == 0 ? i : -1);
            }
            bptr[r + 1] = (int)bcol.size();
        }
        M.n_fwd[dir] = (int)fcol.size();
        M.n_bwd[dir] = (int)bcol.size();
        // pack tables: stream = forward entries, then per backward row [dinv_i, entries...]
        std::vector<int> pk_slot, pk_scale;
        for (size_t e = 0; e < fcol.size(); ++e) {
            pk_slot.push_back(fslot[e]);
            pk_scale.push_back(fscale[e]);
        }
        for (int r = 0; r < b; ++r) {
            const int i = b - 1 - r;
            pk_slot.push_back(-1);
            pk_scale.push_back(i);
            for (int e = bptr[r]; e < bptr[r + 1]; ++e) {
                pk_slot.push_back(bslot[e]);
                pk_scale.push_back(bscale[e]);
            }
        }
        STS_TRY(upload(h, &M.ap_fwd_ptr[dir], fptr));
        STS_TRY(upload(h, &M.ap_fwd_col[dir], fcol));
        STS_TRY(upload(h, &M.ap_fwd_slot[dir], fslot));
        STS_TRY(upload(h, &M.ap_bwd_ptr[dir], bptr));
        STS_TRY(upload(h, &M.ap_bwd_col[dir], bcol));
        STS_TRY(upload(h, &M.ap_bwd_slot[dir], bslot));
        STS_TRY(upload(h, &M.pk_slot[dir], pk_slot));
        STS_TRY(upload(h, &M.pk_scale[dir], pk_scale));
        // apply program, same position order as the pack tables
        std::vector<unsigned> desc;
        for (int i = 0; i < b; ++i)
            for (int e = fptr[i]; e < fptr[i + 1]; ++e) {
                unsigned d = (unsigned)fcol[e] | ((unsigned)i << 12);
                if (e == fptr[i]) d |= kApBegin;
                if (e == fptr[i + 1] - 1) d |= kApEnd;
                desc.push_back(d);
            }
        for (int r = 0; r < b; ++r) {
            const int i = b - 1 - r;
            desc.push_back(((unsigned)i << 12) | kApScale | (bptr[r + 1] == bptr[r] ? kApEnd : 0u));
            for (int e = bptr[r]; e < bptr[r + 1]; ++e) {
                unsigned d = (unsigned)bcol[e] | ((unsigned)i << 12);
                if (e == bptr[r + 1] - 1) d |= kApEnd;
                desc.push_back(d);
            }
        }
        if (desc.size() != pk_slot.size()) return set_error(STS_ERR_INVALID_ARG, "internal: apply program size");
        STS_TRY(upload(h, &M.ap_desc[dir], desc));
    }
    // structured apply tables (both directions; FP64 and, for mixed handles, FP32)
    const int sw = struct_band(b, h->dptr, h->didx);
    M.structured = sw >= 0 && sap_rmax(h->r_diag, sw) > 0 && M.nnz_lu == h->nnz_d;
    if (M.structured) {
        const int NF = kStructNF, N = b - NF, r = h->r_diag;
        M.s_w = sw;
        auto sl = [&](int i, int j) { return slot[(size_t)i * b + j]; };
        const int RMAX = sap_rmax(r, sw);      // the kernel instance chosen at apply time
        for (int prec = 0; prec < 2; ++prec) {
            if (prec == 1 && h->dtype != STS_MIXED) continue;
            const int elem = prec == 0 ? 8 : 4, vec = 16 / elem, K = kSApChunkBytes / (kTile * elem);
            for (int dir = 0; dir < 2; ++dir) {
                std::vector<int> src, arg, gsrc, garg;
                auto put = [&](int s_, int a_) { gsrc.push_back(s_); garg.push_back(a_); };
                auto zero = [&](int n) { for (int k = 0; k < n; ++k) put(-4, 0); };
                // close one group: whole vectors, never straddling a chunk (zero padding)
                bool fits = true;
                auto group = [&]() {
                    while (gsrc.size() % vec) put(-4, 0);
                    const int G = (int)gsrc.size(), off = (int)(src.size() % K);
                    if (G > K) fits = false;
                    if (off + G > K)
                        for (int k = off; k < K; ++k) { src.push_back(-4); arg.push_back(0); }
                    src.insert(src.end(), gsrc.begin(), gsrc.end());
                    arg.insert(arg.end(), garg.begin(), garg.end());
                    gsrc.clear();
                    garg.clear();
                };
                auto vd = [&](int q) {              // dot-vector entries of unknown q, padded to RMAX
                    for (int k = 0; k < RMAX; ++k) put(k < r ? -2 : -4, k < r ? k * b + q : 0);
                };
                // lower factor of this direction: dir 0 L, dir 1 U'^T (U scaled by the row pivot inverse)
                auto lo = [&](int i, int j) {       // coefficient (i, j), i > j
                    if (dir == 0) put(sl(i, j), -1);
                    else put(sl(j, i), j);
                };
                // upper factor after the pivot scaling: dir 0 U' = D^-1 U, dir 1 L^T
                auto up = [&](int i, int j) {       // coefficient (i, j), i < j
                    if (dir == 0) put(sl(i, j), i);
                    else put(sl(j, i), -1);
                };
                const int FW = sw + NF, UF = sap_fwd_rows(FW, vec, NF);
                for (int i0 = 0; i0 < N; i0 += UF) {
                    for (int i = i0; i < i0 + UF; ++i) {
                        if (i >= N) {
                            zero(FW);
                            continue;
                        }
                        for (int k = 0; k < sw; ++k) {
                            const int j = i - sw + k;
                            if (j >= 0) lo(i, j);
                            else put(-4, 0);
                        }
                        for (int f = 0; f < NF; ++f) lo(N + f, i);
                    }
                    group();
                }
                lo(N + 1, N);
                lo(N + 2, N);
                lo(N + 2, N + 1);
                group();
                const bool fsplit = sap_round(6 + 3 * RMAX, vec) > K;   // as FSPLIT in the kernel
                put(-1, N + 2);
                vd(N + 2);
                if (fsplit) group();
                put(-1, N + 1);
                up(N + 1, N + 2);
                vd(N + 1);
                if (fsplit) group();
                put(-1, N);
                up(N, N + 1);
                up(N, N + 2);
                vd(N);
                group();
                const int BW = 1 + NF + sw + RMAX, UB = sap_group_rows(BW, vec);
                for (int j0 = 0; j0 < N; j0 += UB) {
                    for (int j = j0; j < j0 + UB; ++j) {
                        const int i = N - 1 - j;
                        if (i < 0) {
                            zero(BW);
                            continue;
                        }
                        put(-1, i);
                        for (int f = 0; f < NF; ++f) up(i, N + f);
                        for (int k = sw - 1; k >= 0; --k) {
                            const int jj = i + 1 + k;
                            if (jj < N) up(i, jj);
                            else put(-4, 0);
                        }
                        vd(i);
                    }
                    group();
                }
                const int UT = sap_group_rows(RMAX, vec);
                const int tail_src = sap_fold(RMAX, sw) ? -5 : -3;
                for (int q0 = 0; q0 < b; q0 += UT) {
                    for (int q = q0; q < q0 + UT; ++q) {
                        if (q >= b) {
                            zero(RMAX);
                            continue;
                        }
                        for (int k = 0; k < RMAX; ++k) put(k < r ? tail_src : -4, k < r ? k * b + q : 0);
                    }
                    group();
                }
                while (src.size() % K) {
                    src.push_back(-4);
                    arg.push_back(0);
                }
                if (!fits) return set_error(STS_ERR_INVALID_ARG, "internal: structured apply group wider than a chunk");
                for (size_t e = 0; e < src.size(); ++e)
                    if (src[e] < -5 || (src[e] >= 0 && src[e] >= M.nnz_lu))
                        return set_error(STS_ERR_INVALID_ARG, "internal: structured apply table");
                M.s_lt[prec] = (int)src.size();
                STS_TRY(upload(h, &M.spk_src[prec][dir], src));
                STS_TRY(upload(h, &M.spk_arg[prec][dir], arg));
            }
        }
    }
    STS_TRY(upload(h, &M.lu_diag, M.h_lu_diag));
    STS_TRY(upload(h, &M.src_slot, M.h_src_slot));
    STS_TRY(upload(h, &M.d_ptr, h->dptr));
    STS_TRY(upload(h, &M.f_colL_ptr, colL_ptr));
    STS_TRY(upload(h, &M.f_colL_slot, colL_slot));
    STS_TRY(upload(h, &M.f_upd_ptr, upd_ptr));
    STS_TRY(upload(h, &M.f_upd_tgt, upd_tgt));
    STS_TRY(upload(h, &M.f_upd_src, upd_src));
    const size_t P = h->ncp;
    const int r = h->r_diag;
    STS_TRY(dalloc(h, &M.Sd, (size_t)h->nnz_d * P));
    STS_TRY(dalloc(h, &M.Ud, (size_t)std::max(r, 1) * b * P));
    STS_TRY(dalloc(h, &M.Vd, (size_t)std::max(r, 1) * b * P));
    STS_TRY(dalloc(h, &M.lu, (size_t)M.nnz_lu * P));
    STS_TRY(dalloc(h, &M.dinv, (size_t)b * P));
    STS_TRY(dalloc(h, &M.W, (size_t)std::max(r, 1) * b * P));
    if (h->has_T) STS_TRY(dalloc(h, &M.Wt, (size_t)std::max(r, 1) * b * P));
    STS_TRY(dalloc(h, &M.Cinv, (size_t)std::max(r * r, 1) * P));
    for (int dir = 0; dir < 2; ++dir) {
        if (dir == 1 && !h->has_T) continue;
        const size_t len = M.structured ? (size_t)M.s_lt[0] : (size_t)M.n_fwd[dir] + M.n_bwd[dir] + b;
        const size_t len32 = M.structured ? (size_t)M.s_lt[1] : len;
        STS_TRY(dalloc(h, &M.ap64[dir], len * P));
        if (h->dtype == STS_MIXED) {
            STS_TRY(dalloc(h, &M.ap32[dir], len32 * P));
            STS_TRY(dalloc(h, &M.W32[dir], (size_t)std::max(r, 1) * b * P));
            STS_TRY(dalloc(h, &M.DV32[dir], (size_t)std::max(r, 1) * b * P));
        }
    }
    STS_TRY(dalloc(h, &M.err_cell, 1));
    std::vector<int> diag_blk(h->nc);
    for (int c = 0; c < h->nc; ++c)
        for (int k = h->bptr[c]; k < h->bptr[c + 1]; ++k)
            if (h->bidx[k] == c) diag_blk[c] = k;
    STS_TRY(upload(h, &M.diag_blk, diag_blk));
    return STS_OK;
}

sts_status smw_repack(sts_jac_s *h, const double *S, const double *U, const double *V) {
    SmwPlan &M = h->smw;
    M.ready = false;
    const long long total = (long long)h->nnz_d * h->ncp + (long long)h->r_diag * h->b * h->ncp;
    k_smw_repack<<<grid_for(total, 256), 256, 0, h->stream>>>(
        M.Sd, M.Ud, M.Vd, S, U, V, M.diag_blk, h->d_soff, h->d_pbase, h->nc, h->ncp, h->nnz_d,
        h->b, h->r_diag);
    STS_LAUNCHED();
    return STS_OK;
}

sts_status smw_setup(sts_jac_s *h) {
    SmwPlan &M = h->smw;
    M.ready = false;
    SetupArgs a;
    a.Sd = M.Sd; a.Ud = M.Ud; a.Vd = M.Vd;
    a.lu = M.lu; a.dinv = M.dinv; a.W = M.W; a.Wt = M.Wt; a.Cinv = M.Cinv;
    a.lu_diag = M.lu_diag; a.src_slot = M.src_slot; a.d_ptr = M.d_ptr;
    a.colL_ptr = M.f_colL_ptr; a.colL_slot = M.f_colL_slot;
    a.upd_ptr = M.f_upd_ptr; a.upd_tgt = M.f_upd_tgt; a.upd_src = M.f_upd_src;
    a.fwd_ptr0 = M.ap_fwd_ptr[0]; a.fwd_col0 = M.ap_fwd_col[0]; a.fwd_slot0 = M.ap_fwd_slot[0];
    a.bwd_ptr0 = M.ap_bwd_ptr[0]; a.bwd_col0 = M.ap_bwd_col[0]; a.bwd_slot0 = M.ap_bwd_slot[0];
    a.fwd_ptr1 = M.ap_fwd_ptr[1]; a.fwd_col1 = M.ap_fwd_col[1]; a.fwd_slot1 = M.ap_fwd_slot[1];
    a.bwd_ptr1 = M.ap_bwd_ptr[1]; a.bwd_col1 = M.ap_bwd_col[1]; a.bwd_slot1 = M.ap_bwd_slot[1];
    a.err_cell = M.err_cell;
    a.nc = h->nc; a.ncp = h->ncp; a.b = h->b; a.r = h->r_diag; a.nnz_lu = M.nnz_lu;
    a.nnz_d = h->nnz_d; a.with_T = h->has_T ? 1 : 0;
    const int big = INT_MAX;
    STS_CK(cudaMemcpyAsync(M.err_cell, &big, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    k_smw_lu<<<(h->ncp + 63) / 64, 64, 0, h->stream>>>(a);
    STS_LAUNCHED();
    const long long nw = (long long)h->ncp * a.r * (a.with_T ? 2 : 1);
    if (nw > 0) {
        k_smw_w<<<(unsigned)((nw + 63) / 64), 64, 0, h->stream>>>(a);
        STS_LAUNCHED();
        const long long nc2 = (long long)h->ncp * a.r * a.r;
        k_smw_cmat<<<(unsigned)((nc2 + 255) / 256), 256, 0, h->stream>>>(a);
        STS_LAUNCHED();
        k_smw_cinv<<<(h->ncp + 63) / 64, 64, 0, h->stream>>>(a);
        STS_LAUNCHED();
    }
    int bad = INT_MAX;
    STS_CK(cudaMemcpyAsync(&bad, M.err_cell, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    STS_CK(cudaStreamSynchronize(h->stream));
    if (bad != INT_MAX)
        return set_error(STS_ERR_SINGULAR,
                         "block-Jacobi setup: cell %d has a pivot below 1e-14 x its row maximum "
                         "(static pivot order) or a singular capacitance matrix C_k", bad);
    const size_t P = h->ncp;
    const int b = h->b, r = h->r_diag;
    for (int dir = 0; dir < 2; ++dir) {
        if (dir == 1 && !h->has_T) continue;
        const double *DV = dir == 0 ? M.Vd : M.Ud;
        const double *WW = dir == 0 ? M.W : M.Wt;
        if (M.structured) {
            const long long n64 = (long long)M.s_lt[0] * P;
            k_smw_spack<double><<<grid_for(n64, 256), 256, 0, h->stream>>>(
                M.ap64[dir], M.lu, M.dinv, DV, WW, M.Cinv, M.spk_src[0][dir], M.spk_arg[0][dir], M.s_lt[0],
                h->ncp, b, r, dir);
            STS_LAUNCHED();
            if (M.ap32[dir]) {
                const long long n32 = (long long)M.s_lt[1] * P;
                k_smw_spack<float><<<grid_for(n32, 256), 256, 0, h->stream>>>(
                    M.ap32[dir], M.lu, M.dinv, DV, WW, M.Cinv, M.spk_src[1][dir], M.spk_arg[1][dir], M.s_lt[1],
                    h->ncp, b, r, dir);
                STS_LAUNCHED();
            }
            continue;
        }
        const int len = M.n_fwd[dir] + M.n_bwd[dir] + b;
        const long long n = (long long)len * P;
        k_smw_pack<double><<<grid_for(n, 256), 256, 0, h->stream>>>(M.ap64[dir], M.lu, M.dinv, M.pk_slot[dir],
                                                                     M.pk_scale[dir], len, h->ncp);
        STS_LAUNCHED();
        if (M.ap32[dir]) {
            k_smw_pack<float><<<grid_for(n, 256), 256, 0, h->stream>>>(M.ap32[dir], M.lu, M.dinv, M.pk_slot[dir],
                                                                       M.pk_scale[dir], len, h->ncp);
            STS_LAUNCHED();
            const long long nw = (long long)r * b * P;
            if (nw > 0) {
                k_round<float><<<grid_for(nw, 256), 256, 0, h->stream>>>(M.W32[dir], WW, nw);
                STS_LAUNCHED();
                k_round<float><<<grid_for(nw, 256), 256, 0, h->stream>>>(M.DV32[dir], DV, nw);
                STS_LAUNCHED();
            }
        }
    }
    M.ready = true;
    h->streams_dirty = true;
    return STS_OK;
}

template <typename T>
static sts_status smw_apply_t(sts_jac_s *h, int dir, const T *st, const T *dv, const T *W, const T *x,
                              T *z) {
    const SmwPlan &M = h->smw;
    ApplyArgs<T> a;
    a.st = st; a.desc = M.ap_desc[dir]; a.dv = dv; a.W = W; a.Cinv = M.Cinv; a.x = x; a.y = z;
    a.len = M.n_fwd[dir] + M.n_bwd[dir] + h->b; a.b = h->b; a.r = h->r_diag; a.ncp = h->ncp; a.trans = dir;
    const size_t smem = ((size_t)kApStages * kApStage + h->b) * kTile * sizeof(T);
    auto kern = a.r <= 2 ? k_smw_apply<T, 2> : a.r <= 4 ? k_smw_apply<T, 4> : k_smw_apply<T, kMaxPairsDiag>;
    if (smem > 48 * 1024)
        STS_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<h->n_tiles, kTile, smem, h->stream>>>(a);
    STS_LAUNCHED();
    return STS_OK;
}

template <typename T, int W, bool GW>
static void (*sap_kernel_gw(int rmax))(SApplyArgs<T>) {
    return rmax == 2 ? k_smw_sapply<T, W, 2, GW> : rmax == 4 ? k_smw_sapply<T, W, 4, GW>
                                                              : k_smw_sapply<T, W, sap_rmax_big(W), GW>;
}
template <typename T, int W>
static void (*sap_kernel(int rmax, bool gw))(SApplyArgs<T>) {
    return gw ? sap_kernel_gw<T, W, true>(rmax) : sap_kernel_gw<T, W, false>(rmax);
}

template <typename T>
static sts_status smw_sapply_t(sts_jac_s *h, int dir, const T *st, const T *x, T *z) {
    const SmwPlan &M = h->smw;
    SApplyArgs<T> a;
    a.st = st; a.Cinv = M.Cinv; a.x = x; a.y = z; a.err = h->d_err;
    a.Lt = M.s_lt[sizeof(T) == 8 ? 0 : 1]; a.b = h->b; a.N = h->b - kStructNF; a.r = h->r_diag; a.ncp = h->ncp;
    a.trans = dir; a.n_tiles = h->n_tiles;
    a.pre = h->streams_dirty ? 0 : 1;
    a.evict_first = (double)a.n_tiles * a.Lt * kTile * sizeof(T) > (double)h->l2_bytes ? 1 : 0;
    // the working vector moves to y where b rows per warp would leave fewer
    // than kApWarps consumers per SM
    const bool gw = (size_t)(227 * 1024) / sap_warp_bytes(h->b, (int)sizeof(T)) < (size_t)kApWarps;
    const size_t per_warp = sap_warp_bytes(gw ? 0 : h->b, (int)sizeof(T));
    const int wpb = (int)std::min<size_t>(kApWarps, (size_t)(227 * 1024) / per_warp);
    if (wpb < 1)
        return set_error(STS_ERR_INVALID_ARG, "block size %d needs %zu bytes of shared memory per warp", h->b, per_warp);
    const size_t smem = (size_t)wpb * per_warp;
    void (*kern)(SApplyArgs<T>) = nullptr;
    const int rm = sap_rmax(h->r_diag, M.s_w);
    switch (M.s_w) {
        case 0: kern = sap_kernel<T, 0>(rm, gw); break;
        case 1: kern = sap_kernel<T, 1>(rm, gw); break;
        case 2: kern = sap_kernel<T, 2>(rm, gw); break;
        case 3: kern = sap_kernel<T, 3>(rm, gw); break;
        default: kern = sap_kernel<T, 4>(rm, gw); break;
    }
    bool &attr = h->sap_attr[sizeof(T) == 8 ? 0 : 1];
    if (!attr && smem > 48 * 1024)
        STS_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
    const int blocks = std::max(1, std::min(h->nsm, (h->n_tiles + wpb - 1) / wpb));
    STS_CK(launch_pdl(kern, dim3(blocks), dim3((wpb + 1) * kTile), smem, h->stream, a));
    STS_LAUNCHED();
    h->streams_dirty = false;
    return STS_OK;
}

sts_status smw_apply64(sts_jac_s *h, int dir, const double *x, double *z) {
    const SmwPlan &M = h->smw;
    if (M.structured) return smw_sapply_t<double>(h, dir, M.ap64[dir], x, z);
    return smw_apply_t<double>(h, dir, M.ap64[dir], dir == 0 ? M.Vd : M.Ud, dir == 0 ? M.W : M.Wt, x, z);
}

sts_status smw_apply32(sts_jac_s *h, int dir, const float *x, float *z) {
    const SmwPlan &M = h->smw;
    if (M.structured) return smw_sapply_t<float>(h, dir, M.ap32[dir], x, z);
    return smw_apply_t<float>(h, dir, M.ap32[dir], M.DV32[dir], M.W32[dir], x, z);
}

}  // namespace sts
