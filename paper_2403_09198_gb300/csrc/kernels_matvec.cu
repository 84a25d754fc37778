// kernels_matvec.cu -- the factored Jacobian-vector product (Section 5.2).
//
//   c_p = v_p . x_col(p)                      for every rank-one pair p   (pass 1)
//   y_i = sum_j S_ij x_j + sum_{p in row i} c_p u_p                       (pass 2)
//
// The paper's CPU listing computes pass 1 for one block row and then
// accumulates that row; here pass 1 runs for all pairs first (one warp per
// tile and dot task; for the paper's pattern family the dense flow rows of S
// are dot tasks too) and pass 2 runs one warp per (tile, row group).  In both
// passes lane = cell, each lane accumulates its own sums serially (one FMA per
// multiply-add, no cross-lane reduction), and every stream value is read once
// with a coalesced 32-lane request.  The transposed product J^T x uses the
// same kernels on the transposed plan (S^T patterns, roles of u and v swapped).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include <mutex>
#include <type_traits>

#include "ring.cuh"
#include "sts_internal.h"

namespace sts {
namespace {

template <typename T>
struct MvArgs {
    const T *main;          // [n_tiles][tile_len][32]
    const T *dotv;          // [n_tiles][n_dtasks][Lp][32]
    const T *x;             // [b][ncp]
    T *y;                   // [b][ncp]
    T *c;                   // [n_tiles][n_dtasks][32]
    int *err;               // set when a bounded wait gave up
    unsigned *sched;        // [2] pass-2 item counter and finished warps, zero between launches
    int pre;                // the coefficient streams may be read before the grid-dependency wait
    const int *nbr;         // [n_tiles][n_slots][32]
    const unsigned *slot_mask;
    const int *grp_rows;
    const long long *row_off;
    const int *dtask_slot;  // [n_dtasks]
    const int *pat_ptr;     // [2][b+1]
    const int *pat_idx;
    const unsigned *desc;   // [tile_len] program of the generic main pass
    long long tile_len;
    int n_tiles, n_slots, n_pslots, n_dtasks, Lp, n_groups, b, ncp, nnz_d;
    int sN, s_rl, s_gl, n_lgroups, wd, structured;   // structured layout (see MvPlan)
};

// Chunk of stream positions held in registers (two chunks in flight per lane).
// FP64: 4 positions measured faster than 8 (100.6 against 102.2 us per matvec
// on 128 x 128 cells, N = 60): pass 1 then needs 48 registers instead of 80,
// and about 10 warps per sub-partition hide the load latency better than 6
// warps with twice the loads in flight each; 16 took 110.3 us.
template <typename T> struct Chunk { static constexpr int CH = 4; };
template <> struct Chunk<float> { static constexpr int CH = 16; };


// Pass 1: one warp per (tile, dot task); lane = cell.  A dot task is one
// length-b dot product  c = d . x_j  with j the neighbour of the task's slot:
// the pair dots v . x_j of every rank-one pair and, for the paper's pattern
// family, the dense flow rows of S.  Two register buffers alternate so the
// loads of the next chunk are in flight while the current one is multiplied;
// the stream is padded to Lp (a multiple of the chunk) with zero coefficients.
// Pass-1 stream loads: FP32 positions in 16-byte vectors of 4 (the FP32
// kernel is bound by memory instructions), FP64 one position per load (the
// FP64 kernel is bound by the FP64 pipe, and measured faster so).
// The stream is read with evict-first (streaming) loads: each call reads it
// once and it is larger than L2, so the x values the tasks share stay there.
template <typename T> struct DotVec;
template <> struct DotVec<double> {
    using type = double;
    static constexpr int n = 1;
};
template <> struct DotVec<float> {
    using type = float4;
    static constexpr int n = 4;
};
__device__ __forceinline__ double dot_el(double v, int) { return v; }
__device__ __forceinline__ float dot_el(const float4 &v, int i) { return vel(v, i); }

template <typename T>
__global__ void __launch_bounds__(128) k_dots(MvArgs<T> a) {
    using V = typename DotVec<T>::type;
    constexpr int CH = Chunk<T>::CH;
    constexpr int VEC = DotVec<T>::n, NV = CH / VEC;
    static_assert(CH % VEC == 0, "a chunk is whole vectors");
    const int lane = threadIdx.x & 31;
    const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= (long long)a.n_tiles * a.n_dtasks) return;
    const int t = (int)(wid / a.n_dtasks), k = (int)(wid % a.n_dtasks);
    const int s = a.dtask_slot[k];
    const bool present = (a.slot_mask[t] >> s) & 1u;
    const int j = present ? a.nbr[((size_t)t * a.n_slots + s) * kTile + lane] : -1;
    // the task's stream as [Lp / VEC][lane][VEC]: vector p of this lane at dv[p * 32]
    const V *__restrict__ dv =
        reinterpret_cast<const V *>(a.dotv + ((size_t)t * a.n_dtasks + k) * a.Lp * kTile) + lane;
    V va[NV], vb[NV];
    T xa[CH], xb[CH];
    if (present && a.pre) {
#pragma unroll
        for (int i = 0; i < NV; ++i) va[i] = __ldcs(dv + i * kTile);
    }
    pdl_wait();
    pdl_trigger();
    T acc = T(0);
    if (present) {
        // an absent neighbour reads the lane's own cell: its coefficients are zero
        const T *__restrict__ xj = a.x + (j >= 0 ? j : t * kTile + lane);
        const int bm1 = a.b - 1;
        const size_t ncp = a.ncp;
        if (!a.pre) {
#pragma unroll
            for (int i = 0; i < NV; ++i) va[i] = __ldcs(dv + i * kTile);
        }
#pragma unroll
        for (int i = 0; i < CH; ++i) xa[i] = __ldg(xj + (size_t)min(i, bm1) * ncp);
        for (int base = 0; base < a.Lp; base += 2 * CH) {
            if (base + CH < a.Lp) {
#pragma unroll
                for (int i = 0; i < NV; ++i) vb[i] = __ldcs(dv + ((base + CH) / VEC + i) * kTile);
#pragma unroll
                for (int i = 0; i < CH; ++i) xb[i] = __ldg(xj + (size_t)min(base + CH + i, bm1) * ncp);
            }
#pragma unroll
            for (int i = 0; i < CH; ++i) acc = fma(dot_el(va[i / VEC], i % VEC), xa[i], acc);
            if (base + CH >= a.Lp) break;
            if (base + 2 * CH < a.Lp) {
#pragma unroll
                for (int i = 0; i < NV; ++i) va[i] = __ldcs(dv + ((base + 2 * CH) / VEC + i) * kTile);
#pragma unroll
                for (int i = 0; i < CH; ++i) xa[i] = __ldg(xj + (size_t)min(base + 2 * CH + i, bm1) * ncp);
            }
#pragma unroll
            for (int i = 0; i < CH; ++i) acc = fma(dot_el(vb[i / VEC], i % VEC), xb[i], acc);
        }
    }
    a.c[((size_t)t * a.n_dtasks + k) * kTile + lane] = acc;
}

// Pass 2, generic patterns: one warp per (tile, row group); lane = cell.  The
// group's stream positions are consumed in order under a flat program (one
// descriptor per position: column and block slot of an S entry, or the pair
// slot of a pair term, plus an end-of-row flag); each row is accumulated
// serially.  Stream values are double-buffered in registers one chunk ahead.
template <typename T>
__global__ void __launch_bounds__(128) k_mv_main(MvArgs<T> a) {
    constexpr int CH = Chunk<T>::CH;
    __shared__ int snb[4][kMaxSlots][kTile];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
    if (wid >= (long long)a.n_tiles * a.n_groups) return;
    const int t = (int)(wid / a.n_groups), g = (int)(wid % a.n_groups);
    for (int s = 0; s < a.n_slots; ++s) snb[wib][s][lane] = a.nbr[((size_t)t * a.n_slots + s) * kTile + lane];
    __syncwarp();
    const int p0 = a.grp_rows[g], p1 = a.grp_rows[g + 1];
    const long long q0 = a.row_off[p0];
    const int L = (int)(a.row_off[p1] - q0);
    const T *__restrict__ sv = a.main + ((size_t)t * a.tile_len + q0) * kTile + lane;
    const unsigned *__restrict__ dd = a.desc + q0;
    const T *__restrict__ xp = a.x;
    const T *__restrict__ cc = a.c + (size_t)t * a.n_dtasks * kTile + lane;
    T *__restrict__ yp = a.y + (size_t)p0 * a.ncp + (size_t)t * kTile + lane;
    T cur[CH], nxt[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) cur[i] = i < L ? __ldg(sv + (size_t)i * kTile) : T(0);
    T acc = T(0);
    for (int base = 0; base < L; base += CH) {
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int pp = base + CH + i;
            nxt[i] = pp < L ? __ldg(sv + (size_t)pp * kTile) : T(0);
        }
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int pp = base + i;
            if (pp < L) {
                const unsigned d = __ldg(dd + pp);
                T opnd;
                if (d & kDescPair) {
                    opnd = __ldg(cc + (size_t)(d & 0xffffu) * kTile);
                } else {
                    const int j = snb[wib][(d >> 16) & 0x1fu][lane];
                    opnd = j >= 0 ? __ldg(xp + (size_t)(d & 0xffffu) * a.ncp + j) : T(0);
                }
                acc = fma(cur[i], opnd, acc);
                if (d & kDescEnd) {
                    *yp = acc;
                    yp += a.ncp;
                    acc = T(0);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < CH; ++i) cur[i] = nxt[i];
    }
}

// Pass 2, the paper's pattern family (arrow + level band, see MvPlan): column
// indices are arithmetic, so no program is read.  Warps of a tile are groups
// of s_gl level rows, plus one warp for the dense flow rows, whose products
// with x came out of pass 1:
//   level row p: diagonal-slot band q = p-WD..p+WD and the NF flow columns,
//                every neighbour slot's entry q = p and its flow columns, then
//                the pair terms u_k[p] c_k.
//   flow row N+f: sum over slots of the pass-1 flow dots, then the pair terms.
// Held in registers for the whole group: the flow-column x values of every
// slot, the pass-1 pair dots c_k (NREG = 8: up to 8 of them; NREG = 32: up to
// 32; NREG = 0: read per row), and a sliding window of the 2 WD + 1 own-cell x
// values of the band; the x values of the next row are loaded one row ahead.
// Each row's coefficients (s_rl positions, contiguous) are staged in shared
// memory by one bulk copy, two rows per warp in flight.
//
// Pair terms in registers run as fall-through switches (Duff's device), so
// register indices stay static and no FP64 FMA is issued for a missing term (a
// predicated-off FMA still takes its pipe slot).  NREG = 8: term k sits in
// cq[8 - nps + k] and the switch enters at case 8 - nps.  NREG = 32: with more
// than 16 terms the first 16 sit in cq[0..16) and run as one block; the other
// m <= 16 terms sit at the end of cq[16..32) and the switch enters at 16 - m.
constexpr int kStructDuff = 16;

__host__ __device__ inline size_t mv_struct_warp_bytes(int rl, int elem) {
    return 128 + 2 * (size_t)rl * kTile * elem;     // two mbarriers (padded), two row stages
}

template <typename T, int WD, int NREG>
__global__ void __launch_bounds__(64) k_mv_struct(MvArgs<T> a) {
    static_assert(NREG == 0 || NREG == 8 || NREG == 2 * kStructDuff, "register pair slots");
    constexpr int NF = kStructNF;
    constexpr int NS = kStructMaxSlots;
    constexpr int BANDW = 2 * WD + 1;
    const int lane = threadIdx.x & 31;
    const int ns = a.n_slots, nps = a.n_pslots, N = a.sN;
    const size_t ncp = a.ncp;
    const int RL = a.s_rl;
    const uint32_t row_bytes = (uint32_t)RL * kTile * (uint32_t)sizeof(T);
    extern __shared__ __align__(128) unsigned char mv_smem[];
    unsigned char *mine = mv_smem + (size_t)(threadIdx.x >> 5) * mv_struct_warp_bytes(RL, (int)sizeof(T));
    const uint32_t bar = smem_addr(mine);
    T *stage0 = reinterpret_cast<T *>(mine + 128);
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 8, 1);
        mbar_init_fence();
    }
    __syncwarp();
    uint32_t parity = 0;        // bit sg: parity of the next phase of stage sg to wait for
    // persistent: warp items (tile, group), the first round dealt by warp id
    const long long n_items = (long long)a.n_tiles * a.n_groups;
    const long long wstep = (long long)gridDim.x * (blockDim.x >> 5);
    const long long wid0 = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    // the first item's first two rows are copied before the grid-dependency
    // wait when the streams are not being written by the previous grid
    bool primed = false;
    if (a.pre && wid0 < n_items && (int)(wid0 % a.n_groups) != a.n_lgroups) {
        const int t0 = (int)(wid0 / a.n_groups), q0 = (int)(wid0 % a.n_groups) * a.s_gl;
        const int q1 = min(N, q0 + a.s_gl);
        const T *src = a.main + ((size_t)t0 * a.tile_len + (size_t)q0 * RL) * kTile;
        for (int r = q0; r < min(q0 + 2, q1); ++r)
            if (lane == 0) {
                const int sg = (r - q0) & 1;
                mbar_expect_tx(bar + 8u * sg, row_bytes);
                bulk_copy_g2s_stream(smem_addr(stage0 + (size_t)sg * RL * kTile), src + (size_t)(r - q0) * RL * kTile,
                              row_bytes, bar + 8u * sg);
            }
        primed = true;
    }
    pdl_wait();
    pdl_trigger();
    // Each warp's first item is wid0; later items come from a counter, so
    // that sub-partitions running more warps, or lighter items, take more
    // (static round-robin dealing left the sub-partitions with four warps
    // finishing last).  The next ticket is taken at the start of an item and
    // read at its end, so the atomic's latency is hidden.
    unsigned ticket = 0;
    for (long long wid = wid0; wid < n_items; wid = wstep + (long long)__shfl_sync(0xffffffffu, ticket, 0)) {
    if (lane == 0) ticket = atomicAdd(a.sched, 1u);
    const int t = (int)(wid / a.n_groups), g = (int)(wid % a.n_groups);
    const size_t cell = (size_t)t * kTile + lane;
    const T *__restrict__ cc = a.c + (size_t)t * a.n_dtasks * kTile + lane;
    if (g == a.n_lgroups) {
        const T *__restrict__ su = a.main + ((size_t)t * a.tile_len + (size_t)N * RL) * kTile + lane;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T acc = T(0);
            for (int s = 0; s < ns; ++s) acc += __ldg(cc + (size_t)(nps + f * ns + s) * kTile);
            for (int k = 0; k < nps; ++k)
                acc = fma(__ldg(su + (size_t)(f * nps + k) * kTile), __ldg(cc + (size_t)k * kTile), acc);
            a.y[(size_t)(N + f) * ncp + cell] = acc;
        }
        continue;
    }
    const int p0 = g * a.s_gl, p1 = min(N, p0 + a.s_gl);
    const T *__restrict__ src0 = a.main + ((size_t)t * a.tile_len + (size_t)p0 * RL) * kTile;
    auto issue = [&](int row) {             // bulk copy of one row into stage (row - p0) & 1
        const int sg = (row - p0) & 1;
        if (lane == 0) {
            mbar_expect_tx(bar + 8u * sg, row_bytes);
            bulk_copy_g2s_stream(smem_addr(stage0 + (size_t)sg * RL * kTile), src0 + (size_t)(row - p0) * RL * kTile,
                          row_bytes, bar + 8u * sg);
        }
    };
    if (!primed) {
        issue(p0);
        if (p0 + 1 < p1) issue(p0 + 1);
    }
    primed = false;
    const T *xs[NS];
    T xf[NS][NF];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int j = s < ns ? a.nbr[((size_t)t * ns + s) * kTile + lane] : -1;
        // an absent neighbour reads the lane's own cell: its coefficients are zero
        xs[s] = a.x + (j >= 0 ? (size_t)j : cell);
#pragma unroll
        for (int f = 0; f < NF; ++f) xf[s][f] = s < ns ? __ldg(xs[s] + (size_t)(N + f) * ncp) : T(0);
    }
    // pair dots in registers (see above): an optional block of RB = 16, then the
    // last m terms aligned to the end of the D switch slots
    constexpr int D = NREG == 8 ? 8 : kStructDuff, RB = NREG > D ? D : 0;
    const bool blk = RB > 0 && nps > D;
    const int m = blk ? nps - D : nps, poff = D - m;
    T cq[NREG > 0 ? NREG : 1];
#pragma unroll
    for (int i = 0; i < RB; ++i) cq[i] = blk ? __ldg(cc + (size_t)i * kTile) : T(0);
#pragma unroll
    for (int i = 0; i < (NREG > 0 ? D : 0); ++i)
        cq[RB + i] = i >= poff ? __ldg(cc + (size_t)((blk ? D : 0) + i - poff) * kTile) : T(0);
    // band window: xb[k] = x_own[p - WD + k] (clipped; clipped entries carry zero coefficients)
    T xb[BANDW];
#pragma unroll
    for (int k = 0; k + 1 < BANDW; ++k) xb[k + 1] = __ldg(xs[0] + (size_t)min(max(p0 - WD + k, 0), N - 1) * ncp);
    T xbn = __ldg(xs[0] + (size_t)min(p0 + WD, N - 1) * ncp);
    T xn[NS];
#pragma unroll
    for (int s = 1; s < NS; ++s) xn[s] = s < ns ? __ldg(xs[s] + (size_t)p0 * ncp) : T(0);
    T *yp = a.y + (size_t)p0 * ncp + cell;
    T ylag = T(0);          // row p-1's result, stored during row p (its FMA has long completed)
    for (int p = p0; p < p1; ++p) {
        const int sg = (p - p0) & 1;
        if (!mbar_wait_bounded(bar + 8u * sg, (parity >> sg) & 1u)) {
            if (lane == 0) atomicExch(a.err, 1);
            for (int q = p; q < min(p + 2, p1); ++q) {            // copies still in flight
                const int sq = (q - p0) & 1;
                if (!mbar_wait_bounded(bar + 8u * sq, (parity >> sq) & 1u)) break;
                parity ^= 1u << sq;
            }
            goto done;
        }
        parity ^= 1u << sg;
#pragma unroll
        for (int k = 0; k + 1 < BANDW; ++k) xb[k] = xb[k + 1];
        xb[BANDW - 1] = xbn;
        T xc[NS];
#pragma unroll
        for (int s = 1; s < NS; ++s) xc[s] = xn[s];
        if (p + 1 < p1) {
            xbn = __ldg(xs[0] + (size_t)min(p + 1 + WD, N - 1) * ncp);
#pragma unroll
            for (int s = 1; s < NS; ++s)
                if (s < ns) xn[s] = __ldg(xs[s] + (size_t)(p + 1) * ncp);
        }
        const T *v = stage0 + (size_t)sg * RL * kTile + lane;
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < BANDW; ++k) acc = fma(v[k * kTile], xb[k], acc);
#pragma unroll
        for (int f = 0; f < NF; ++f) acc = fma(v[(BANDW + f) * kTile], xf[0][f], acc);
#pragma unroll
        for (int s = 1; s < NS; ++s) {
            if (s < ns) {
                const T *vs = v + (BANDW + NF + (s - 1) * (1 + NF)) * kTile;
                acc = fma(vs[0], xc[s], acc);
#pragma unroll
                for (int f = 0; f < NF; ++f) acc = fma(vs[(1 + f) * kTile], xf[s][f], acc);
            }
        }
        const T *vu = v + (BANDW + NF + (ns - 1) * (1 + NF)) * kTile;
        if constexpr (NREG == 8) {
            const T *vo = vu - poff * kTile;
            switch (poff) {
                case 0: acc = fma(vo[0 * kTile], cq[0], acc); [[fallthrough]];
                case 1: acc = fma(vo[1 * kTile], cq[1], acc); [[fallthrough]];
                case 2: acc = fma(vo[2 * kTile], cq[2], acc); [[fallthrough]];
                case 3: acc = fma(vo[3 * kTile], cq[3], acc); [[fallthrough]];
                case 4: acc = fma(vo[4 * kTile], cq[4], acc); [[fallthrough]];
                case 5: acc = fma(vo[5 * kTile], cq[5], acc); [[fallthrough]];
                case 6: acc = fma(vo[6 * kTile], cq[6], acc); [[fallthrough]];
                case 7: acc = fma(vo[7 * kTile], cq[7], acc); [[fallthrough]];
                default: break;
            }
        } else if constexpr (NREG > 0) {
            static_assert(kStructDuff == 16, "one case per slot");
            if (blk) {
#pragma unroll
                for (int i = 0; i < RB; ++i) acc = fma(vu[i * kTile], cq[i], acc);
            }
            const T *vo = vu + ((blk ? D : 0) - poff) * kTile;
            const T *c = cq + RB;
            switch (poff) {
                case 0: acc = fma(vo[0 * kTile], c[0], acc); [[fallthrough]];
                case 1: acc = fma(vo[1 * kTile], c[1], acc); [[fallthrough]];
                case 2: acc = fma(vo[2 * kTile], c[2], acc); [[fallthrough]];
                case 3: acc = fma(vo[3 * kTile], c[3], acc); [[fallthrough]];
                case 4: acc = fma(vo[4 * kTile], c[4], acc); [[fallthrough]];
                case 5: acc = fma(vo[5 * kTile], c[5], acc); [[fallthrough]];
                case 6: acc = fma(vo[6 * kTile], c[6], acc); [[fallthrough]];
                case 7: acc = fma(vo[7 * kTile], c[7], acc); [[fallthrough]];
                case 8: acc = fma(vo[8 * kTile], c[8], acc); [[fallthrough]];
                case 9: acc = fma(vo[9 * kTile], c[9], acc); [[fallthrough]];
                case 10: acc = fma(vo[10 * kTile], c[10], acc); [[fallthrough]];
                case 11: acc = fma(vo[11 * kTile], c[11], acc); [[fallthrough]];
                case 12: acc = fma(vo[12 * kTile], c[12], acc); [[fallthrough]];
                case 13: acc = fma(vo[13 * kTile], c[13], acc); [[fallthrough]];
                case 14: acc = fma(vo[14 * kTile], c[14], acc); [[fallthrough]];
                case 15: acc = fma(vo[15 * kTile], c[15], acc); [[fallthrough]];
                default: break;
            }
        } else {
            for (int k = 0; k < nps; ++k) acc = fma(vu[k * kTile], __ldg(cc + (size_t)k * kTile), acc);
        }
        if (p > p0) {
            *yp = ylag;
            yp += ncp;
        }
        ylag = acc;
        __syncwarp();     // every lane is done with the stage before it is refilled
        if (p + 2 < p1) issue(p + 2);
    }
    if (p1 > p0) *yp = ylag;
    }
done:
    // The last warp to finish resets the counters for the next launch.  A
    // warp counts itself out only after it has used the value its last ticket
    // returned, so every ticket has been taken when the count completes; no
    // fence is needed (one measured as a membar stall: it waits for the
    // warp's output stores).
    __syncwarp();
    if (lane == 0) {
        if (atomicAdd(a.sched + 1, 1u) == (unsigned)(wstep - 1)) {
            atomicExch(a.sched, 0u);
            atomicExch(a.sched + 1, 0u);
        }
    }
}

// Repack the public values into one stream of one direction.  Each stream
// position (per tile and lane) is an S entry of a block slot, an entry of a
// pair vector (the axpy vectors in the main stream, the dot vectors in the
// pass-1 stream), or a zero.  A block with fewer pairs than its kind's
// largest count gets zero vectors in the remaining pair slots.  With vec > 1 each run of vec positions of a
// lane is contiguous ([tile][position / vec][lane][vec]), for 16-byte loads.
template <typename T>
__global__ void k_repack(T *out, const double *S, const double *AX, const int *blk,
                              const long long *soff, const int *pbase, const int *pos_kind,
                              const int *pos_arg, const int *pat_src, const int *pslot_slot,
                              const int *pslot_local, long long tile_len, int n_tiles, int n_slots,
                              int b, int vec) {
    const long long per_tile = tile_len * kTile;
    const long long total = (long long)n_tiles * per_tile;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        // element i is (tile, position / vec, lane, position % vec)
        const int t = (int)(i / per_tile);
        const long long e = i - (long long)t * per_tile;
        const long long vb = e / (kTile * vec);
        const int rem = (int)(e - vb * kTile * vec);
        const int lane = rem / vec;
        const long long pos = vb * vec + rem % vec;
        const int kind = pos_kind[pos], arg = pos_arg[pos];
        double v = 0.0;
        if (kind == kPosZero) {
            v = 0.0;
        } else if (kind >= 0) {
            const int k = blk[((size_t)t * n_slots + kind) * kTile + lane];
            if (k >= 0) v = S[soff[k] + pat_src[arg]];
        } else {
            const int ps = -1 - kind;
            const int k = blk[((size_t)t * n_slots + pslot_slot[ps]) * kTile + lane];
            const int l = pslot_local[ps];
            if (k >= 0 && l < pbase[k + 1] - pbase[k]) v = AX[(size_t)(pbase[k] + l) * b + arg];
        }
        out[i] = (T)v;
    }
}

// Public vector -> internal [b][ncp].  Cell-major input is transposed through
// shared memory in 32 x 32 tiles so that both sides are coalesced.
template <typename T>
__global__ void k_cell_to_comp(const T *__restrict__ x, T *__restrict__ xi, int nc, int b, int ncp) {
    __shared__ T tile[32][33];
    const int c0 = blockIdx.x * 32, q0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r, q = q0 + threadIdx.x;
        tile[r][threadIdx.x] = (c < nc && q < b) ? x[(size_t)c * b + q] : T(0);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int q = q0 + r, c = c0 + threadIdx.x;
        if (q < b && c < ncp) xi[(size_t)q * ncp + c] = tile[threadIdx.x][r];
    }
}

template <typename T>
__global__ void k_comp_to_cell(const T *__restrict__ xi, T *__restrict__ x, int nc, int b, int ncp) {
    __shared__ T tile[32][33];
    const int c0 = blockIdx.x * 32, q0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int q = q0 + r, c = c0 + threadIdx.x;
        tile[r][threadIdx.x] = (q < b && c < ncp) ? xi[(size_t)q * ncp + c] : T(0);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r, q = q0 + threadIdx.x;
        if (c < nc && q < b) x[(size_t)c * b + q] = tile[threadIdx.x][r];
    }
}

template <typename T>
__global__ void k_comp_pad(const T *__restrict__ x, T *__restrict__ xi, int nc, int b, int ncp) {
    const long long total = (long long)b * ncp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % ncp), q = (int)(i / ncp);
        xi[i] = c < nc ? x[(size_t)q * nc + c] : T(0);
    }
}

template <typename T>
__global__ void k_comp_unpad(const T *__restrict__ xi, T *__restrict__ x, int nc, int b, int ncp) {
    const long long total = (long long)b * nc;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % nc), q = (int)(i / nc);
        x[i] = xi[(size_t)q * ncp + c];
    }
}

inline int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152LL * 64) g = 152LL * 64;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename T>
MvArgs<T> make_args(sts_jac_s *h, int dir, const T *main, const T *dotv, const T *x, T *y, T *c) {
    const MvPlan &P = h->mv[dir];
    MvArgs<T> a;
    a.main = main;
    a.dotv = dotv;
    a.x = x;
    a.y = y;
    a.c = c;
    a.err = h->d_err;
    a.sched = h->d_sched;
    a.pre = h->streams_dirty ? 0 : 1;
    a.nbr = P.nbr;
    a.slot_mask = P.slot_mask;
    a.grp_rows = P.grp_rows;
    a.row_off = P.row_off;
    a.dtask_slot = P.dtask_slot;
    a.pat_ptr = P.pat_ptr;
    a.pat_idx = P.pat_idx;
    a.desc = P.desc;
    a.tile_len = P.tile_len;
    a.n_tiles = h->n_tiles;
    a.n_slots = P.n_slots;
    a.n_pslots = P.n_pslots;
    a.n_dtasks = P.n_dtasks;
    a.Lp = P.Lp;
    a.n_groups = P.n_groups;
    a.b = h->b;
    a.ncp = h->ncp;
    a.nnz_d = h->nnz_d;
    a.sN = P.sN;
    a.s_rl = P.s_rl;
    a.s_gl = P.s_gl;
    a.n_lgroups = P.n_lgroups;
    a.wd = P.s_wd;
    a.structured = P.structured ? 1 : 0;
    return a;
}

template <typename T>
sts_status dots_launch(sts_jac_s *h, const MvArgs<T> &a) {
    if (a.n_dtasks == 0) return STS_OK;
    const long long warps = (long long)a.n_tiles * a.n_dtasks;
    k_dots<T><<<(unsigned)((warps + 3) / 4), 128, 0, h->stream>>>(a);
    STS_LAUNCHED();
    h->streams_dirty = false;
    return STS_OK;
}

template <typename T, int WD>
void (*mv_struct_kernel(int nreg))(MvArgs<T>) {
    return nreg == 8 ? k_mv_struct<T, WD, 8> : nreg ? k_mv_struct<T, WD, 2 * kStructDuff> : k_mv_struct<T, WD, 0>;
}

// Level rows per pass-2 item.  The persistent grid runs n_tiles x (groups + 1)
// items on W resident warps: the first round by warp id, the rest from a
// counter.  With many items per warp the plan's size stands.  With few, the
// size trades the per-item work (loading the neighbour x values and pair dots
// and priming the copies: fewer, larger items) against the tail of the last
// items (smaller items): the best size grows as sqrt(N / s_rl).  Measured at
// N = 60 (us per FP64 matvec, items of 4 / 5 / 6 / 7 / 8 rows): 128 x 128 cells
// with s_rl = 30, 102.7 / 102.0 / 106.5 / - / -; with the paper's pair counts
// (s_rl = 41), 145.0 / 144.8 / 147.5 / 148.5 / 148.2.  The constant puts both
// at 5 rows.
inline int pass2_group_rows(int N, int n_tiles, long long W, int s_plan, int s_rl) {
    const long long items = (long long)n_tiles * ((N + s_plan - 1) / s_plan + 1);
    if (W <= 0 || items >= 8 * W) return s_plan;
    const int s = (int)std::lround(3.8 * std::sqrt((double)N / std::max(s_rl, 1)));
    return std::max(1, std::min({N, 8, std::max(4, s)}));
}

template <typename T>
sts_status mv_launch(sts_jac_s *h, const MvArgs<T> &args) {
    STS_TRY(dots_launch<T>(h, args));
    MvArgs<T> a = args;
    long long warps = (long long)a.n_tiles * a.n_groups;
    const unsigned grid = (unsigned)((warps + 3) / 4);
    if (a.structured) {
        constexpr int kWarpsPerBlock = 2;      // two row stages per warp; small blocks pack the SM finely
        const size_t smem = (size_t)kWarpsPerBlock * mv_struct_warp_bytes(a.s_rl, (int)sizeof(T));
        void (*kern)(MvArgs<T>) = nullptr;
        const int nreg = a.n_pslots <= 8 ? 8 : a.n_pslots <= 2 * kStructDuff ? 2 * kStructDuff : 0;
        switch (a.wd) {
            case 0: kern = mv_struct_kernel<T, 0>(nreg); break;
            case 1: kern = mv_struct_kernel<T, 1>(nreg); break;
            case 2: kern = mv_struct_kernel<T, 2>(nreg); break;
            case 3: kern = mv_struct_kernel<T, 3>(nreg); break;
            default: kern = mv_struct_kernel<T, 4>(nreg); break;
        }
        // blocks resident at once, found once per kernel instance and shared-memory
        // size: the instance (pair slots) and the row length differ between the
        // forward and transposed plans
        int resident = 0;
        for (const auto &e : h->mvs_resident)
            if (e.kern == reinterpret_cast<const void *>(kern) && e.smem == smem) resident = e.blocks;
        if (!resident) {
            if (smem > 48 * 1024)
                STS_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int per_sm = 0;
            STS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpsPerBlock * kTile, smem));
            resident = std::max(per_sm, 1) * h->nsm;
            h->mvs_resident.push_back({reinterpret_cast<const void *>(kern), smem, resident});
        }
        a.s_gl = pass2_group_rows(a.sN, a.n_tiles, (long long)resident * kWarpsPerBlock, a.s_gl, a.s_rl);
        a.n_lgroups = (a.sN + a.s_gl - 1) / a.s_gl;
        a.n_groups = a.n_lgroups + 1;
        warps = (long long)a.n_tiles * a.n_groups;
        const long long need = (warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
        const long long blocks = std::max(1LL, std::min(need, (long long)resident));
        // programmatic dependent launch: the blocks start, and copy their first
        // rows, while pass 1 finishes; items are taken from a counter, so
        // blocks that start late do not finish late
        STS_CK(launch_pdl(kern, dim3((unsigned)blocks), dim3(kWarpsPerBlock * kTile), smem, h->stream, a));
    } else {
        k_mv_main<T><<<grid, 128, 0, h->stream>>>(a);
    }
    STS_LAUNCHED();
    return STS_OK;
}

}  // namespace

sts_status mv_repack(sts_jac_s *h, int dir, const double *S, const double *U, const double *V) {
    MvPlan &P = h->mv[dir];
    const double *AX = dir == 0 ? U : V;   // axpy vectors (main stream)
    const double *DV = dir == 0 ? V : U;   // dot vectors (pass-1 stream)
    const long long nm = (long long)h->n_tiles * P.tile_len * kTile;
    const long long nd = (long long)h->n_tiles * P.n_dtasks * P.Lp * kTile;
    auto rp = [&](auto *out, const double *vec, const int *pk, const int *pa, long long len, long long total,
                  int vw) {
        using T = std::remove_pointer_t<decltype(out)>;
        k_repack<T><<<grid_for(total, 256), 256, 0, h->stream>>>(out, S, vec, P.blk, h->d_soff, h->d_pbase, pk, pa,
                                                                 P.pat_src, P.pslot_slot, P.pslot_local, len,
                                                                 h->n_tiles, P.n_slots, h->b, vw);
    };
    // the pass-1 stream is read with loads of DotVec<T>::n positions per lane
    const long long dlen = (long long)P.n_dtasks * P.Lp;
    if (P.main64) { rp(P.main64, AX, P.pos_kind, P.pos_arg, P.tile_len, nm, 1); STS_LAUNCHED(); }
    if (P.main32) { rp(P.main32, AX, P.pos_kind, P.pos_arg, P.tile_len, nm, 1); STS_LAUNCHED(); }
    if (nd > 0 && P.dotv64) { rp(P.dotv64, DV, P.dpos_kind, P.dpos_arg, dlen, nd, DotVec<double>::n); STS_LAUNCHED(); }
    if (nd > 0 && P.dotv32) { rp(P.dotv32, DV, P.dpos_kind, P.dpos_arg, dlen, nd, DotVec<float>::n); STS_LAUNCHED(); }
    return STS_OK;
}

sts_status mv_apply64(sts_jac_s *h, int dir, const double *x, double *y, double *c) {
    const MvPlan &P = h->mv[dir];
    return mv_launch<double>(h, make_args<double>(h, dir, P.main64, P.dotv64, x, y, c));
}

sts_status mv_dots64(sts_jac_s *h, int dir, const double *x, double *c) {
    const MvPlan &P = h->mv[dir];
    return dots_launch<double>(h, make_args<double>(h, dir, P.main64, P.dotv64, x, nullptr, c));
}

// ---------------------------------------------------------------------------
// Matvec without any device allocation: the pass-1 dot products go to a
// library-owned, file-scope device array instead of a handle buffer.  The
// array (kNoAllocScratch doubles, 4 MiB) exists on every GPU that loads the
// library, for the life of the process.  Its device address is looked up with
// cudaGetSymbolAddress once per device, on the first call for a handle of that
// device (which must be the current device during the call).  Every call shares the array, so calls that overlap on the
// GPU (several streams, several threads) race on it; each call writes every
// entry it later reads, so nothing has to be cleared between calls.
constexpr size_t kNoAllocScratch = size_t(1) << 19;
static __device__ __align__(256) double g_noalloc_dots[kNoAllocScratch];

namespace {
std::mutex g_noalloc_mu;
constexpr int kNoAllocMaxDevices = 64;
double *g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace

sts_status mv_apply64_noalloc(sts_jac_s *h, int dir, const double *x, double *y) {
    const MvPlan &P = h->mv[dir];
    const size_t need = (size_t)h->n_tiles * P.n_dtasks * kTile;
    if (need > kNoAllocScratch)
        return set_error(STS_ERR_INVALID_ARG,
                         "sts_jac_matvec_noalloc: this Jacobian needs %zu scratch values (tiles x dot tasks x 32), "
                         "more than the %zu of the static buffer; use sts_jac_matvec",
                         need, kNoAllocScratch);
    // the scratch address belongs to the handle's device, which must be current
    const int dev = h->device;
    int cur = -1;
    STS_CK(cudaGetDevice(&cur));
    if (cur != dev)
        return set_error(STS_ERR_INVALID_ARG,
                         "sts_jac_matvec_noalloc: the handle lives on device %d but device %d is current", dev, cur);
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return set_error(STS_ERR_INVALID_ARG, "sts_jac_matvec_noalloc: device %d out of range", dev);
    double *c = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_dots);
            if (e != cudaSuccess || !p)
                return set_error(STS_ERR_CUDA, "sts_jac_matvec_noalloc: cudaGetSymbolAddress failed: %s",
                                 cudaGetErrorString(e));
            g_noalloc_ptr[dev] = static_cast<double *>(p);
        }
        c = g_noalloc_ptr[dev];
    }
    return mv_launch<double>(h, make_args<double>(h, dir, P.main64, P.dotv64, x, y, c));
}

sts_status mv_apply32(sts_jac_s *h, int dir, const float *x, float *y, float *c) {
    const MvPlan &P = h->mv[dir];
    return mv_launch<float>(h, make_args<float>(h, dir, P.main32, P.dotv32, x, y, c));
}

template <typename T>
static sts_status to_internal(sts_jac_s *h, const T *x, T *xi) {
    if (h->layout == STS_LAYOUT_CELL_MAJOR) {
        dim3 grid((h->ncp + 31) / 32, (h->b + 31) / 32), block(32, 8);
        k_cell_to_comp<T><<<grid, block, 0, h->stream>>>(x, xi, h->nc, h->b, h->ncp);
        STS_LAUNCHED();
    } else {
        const long long n = (long long)h->b * h->ncp;
        k_comp_pad<T><<<grid_for(n, 256), 256, 0, h->stream>>>(x, xi, h->nc, h->b, h->ncp);
        STS_LAUNCHED();
    }
    return STS_OK;
}

template <typename T>
static sts_status from_internal(sts_jac_s *h, const T *xi, T *x) {
    if (h->layout == STS_LAYOUT_CELL_MAJOR) {
        dim3 grid((h->nc + 31) / 32, (h->b + 31) / 32), block(32, 8);
        k_comp_to_cell<T><<<grid, block, 0, h->stream>>>(xi, x, h->nc, h->b, h->ncp);
        STS_LAUNCHED();
    } else {
        const long long n = (long long)h->b * h->nc;
        k_comp_unpad<T><<<grid_for(n, 256), 256, 0, h->stream>>>(xi, x, h->nc, h->b, h->ncp);
        STS_LAUNCHED();
    }
    return STS_OK;
}

sts_status to_internal64(sts_jac_s *h, const double *x, double *xi) { return to_internal<double>(h, x, xi); }
sts_status from_internal64(sts_jac_s *h, const double *xi, double *x) { return from_internal<double>(h, xi, x); }
sts_status to_internal32(sts_jac_s *h, const float *x, float *xi) { return to_internal<float>(h, x, xi); }
sts_status from_internal32(sts_jac_s *h, const float *xi, float *x) { return from_internal<float>(h, xi, x); }

}  // namespace sts
