// ring.cuh -- shared-memory rings that stream coefficient positions (32 lanes
// x sizeof(T) bytes each) from global memory ahead of the consumer, and the
// device helpers they use.
//
// Ring:         one warp, strided positions copied with cp.async (16 bytes per
//               lane and instruction); waits are cp.async.wait_group, no spin
//               loop.  Used by the generic block-Jacobi apply.
// RingConsumer / RingProducer: contiguous 8 KB chunks copied by the bulk-copy
//               (TMA) engine, issued by one producer thread for all the rings
//               of a block and completed on a "full" mbarrier per stage; the
//               consumer warp releases a stage through an "empty" mbarrier;
//               every wait is bounded in time.  Used by the structured apply.
// In all of them chunk c lives in stage c % S and a stage is refilled only
// after every lane has finished reading it.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace sts {

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
// One element (4 or 8 bytes) per lane.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem_dst, const T *gmem_src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async element of 4 or 8 bytes");
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gmem_src), "n"((int)sizeof(T)) : "memory");
}

// K positions per chunk, S stages.  stg points at this warp's S*K*32 elements
// (16-byte aligned); src at the first position of this warp's sequence for
// lane 0; stride is the element distance between consecutive positions.
template <typename T, int K, int S>
struct Ring {
    static constexpr int PIECES = 32 * (int)sizeof(T) / 16;    // 16-byte pieces per position
    static constexpr int PER_ITER = 32 / PIECES;                // positions per warp-wide copy
    T *stg;
    const T *src;
    size_t stride;
    int L, nch, ch, off, lane;
    const T *cur;

    __device__ __forceinline__ void issue(int c) {
        T *dst0 = stg + (c % S) * K * 32;
        const int piece = lane % PIECES;
#pragma unroll
        for (int it = 0; it < K / PER_ITER; ++it) {
            const int pos = it * PER_ITER + lane / PIECES;
            const int gp = c * K + pos;
            if (gp < L)
                cp_async16(dst0 + pos * 32 + piece * (16 / (int)sizeof(T)),
                           src + (size_t)gp * stride + piece * (16 / (int)sizeof(T)));
        }
        cp_async_commit();
    }
    __device__ __forceinline__ void enter(int c) {
        cp_async_wait<S - 2>();
        __syncwarp();
        if (c + S - 1 < nch) issue(c + S - 1);
        else cp_async_commit();
        cur = stg + (c % S) * K * 32 + lane;
    }
    // Start streaming positions [0, L); the first chunk is ready on return.
    __device__ __forceinline__ void start(T *stg_, const T *src_, size_t stride_, int L_, int lane_) {
        stg = stg_;
        src = src_;
        stride = stride_;
        L = L_;
        lane = lane_;
        nch = (L + K - 1) / K;
        ch = 0;
        off = 0;
#pragma unroll
        for (int c = 0; c < S - 1; ++c) {
            if (c < nch) issue(c);
            else cp_async_commit();
        }
        enter(0);
    }
    __device__ __forceinline__ T next() {
        if (off == K) {
            ++ch;
            off = 0;
            enter(ch);
        }
        return cur[(off++) * 32];
    }
    __device__ __forceinline__ void finish() { cp_async_wait<0>(); }
};

// Programmatic dependent launch.  pdl_wait returns once the grids this one
// depends on have completed and their writes are visible (immediately when
// the launch had no such dependency); pdl_trigger lets the next grid on the
// stream start.  Kernels of this library trigger only after their own wait,
// so a kernel that starts early knows every grid before its predecessor has
// completed.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// 16-byte vector of T (2 doubles or 4 floats) and its element i (constant i
// after unrolling, so no data moves).
template <typename T>
struct Vec16;
template <>
struct Vec16<double> {
    using type = double2;
};
template <>
struct Vec16<float> {
    using type = float4;
};
__device__ __forceinline__ double vel(const double2 &v, int i) { return i == 0 ? v.x : v.y; }
__device__ __forceinline__ float vel(const float4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// ---------------------------------------------------------------------------
// Bulk copies completed on mbarriers.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// The same copy with an L2 evict-first policy, for coefficient streams that a
// call reads once and that are larger than L2: the vectors the call re-reads
// (x, the pair dots) then stay in L2.  Measured on 128 x 128 cells, N = 60
// together with streaming loads of the pass-1 coefficients: FP64 matvec 107.0
// -> 102.6 us, apply 45.7 -> 45.5 us.  A stream smaller than L2 (the FP32
// apply's 68.5 MB there) is better copied with the default policy: part of it
// is still in L2 at the next call.
__device__ __forceinline__ void bulk_copy_g2s_stream(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Wait for the phase of the given parity to complete; give up after about a
// second (false).
constexpr unsigned long long kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitLimitNs) return false;
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// Warp-specialised bulk-copy rings.  Each consumer warp owns a ring of S
// stages of K positions (one 8 KB chunk each) in shared memory, with a "full"
// mbarrier per stage (completed by the bulk copy's byte count) and an "empty"
// mbarrier per stage (32 arrivals: every lane of the consumer).  One producer
// thread issues the copies of all the block's rings, so the consumers never
// execute a copy instruction.  A ring streams a sequence of equal-length
// segments (one per tile its consumer processes): segment k starts at
// src + (seg0 + k * seg_step) * seg_elems and holds nch chunks.  Positions are
// laid out as [position / VEC][lane][VEC], so a lane reads VEC consecutive
// positions with one 16-byte load.
//
// Entering chunk c releases chunk c - 2 (never c - 1), so a consumer may load
// its next group, possibly from chunk c, before it has used the values it
// loaded from chunk c - 1; S - 2 chunks are thus in flight ahead of the
// current one.  All waits are bounded.
template <typename T, int K, int S>
struct RingConsumer {
    static constexpr int VEC = 16 / (int)sizeof(T);
    static_assert(K % VEC == 0, "chunk must hold whole vectors");
    static_assert(S >= 3, "two stages plus at least one in flight");
    T *stg;
    uint32_t full, empty;
    int ch, off, lane;
    bool failed;                  // a wait gave up; later takes return stale data
    const T *cur;

    __device__ __forceinline__ void start(T *stg_, uint32_t full_, uint32_t empty_, int lane_) {
        stg = stg_;
        full = full_;
        empty = empty_;
        lane = lane_;
        ch = -1;
        off = K;
        failed = false;
        cur = stg + lane * VEC;
    }
    __device__ __forceinline__ void enter(int c) {
        if (failed) return;
        const int s = c % S;
        if (!mbar_wait_bounded(full + 8u * s, (uint32_t)(c / S) & 1u)) {
            failed = true;
            return;
        }
        if (c >= 2) mbar_arrive(empty + 8u * ((c - 2) % S));
        cur = stg + (size_t)s * K * 32 + lane * VEC;
    }
    // The next G positions (G a multiple of VEC, G <= K) as one group; groups
    // never straddle a chunk (the packer pads).  Lane pointer to the group's
    // first vector, vector j at + j * 32 * VEC.  After a failed wait the
    // pointer still addresses the ring, with stale values.
    __device__ __forceinline__ const T *take(int G) {
        if (off + G > K) {
            enter(++ch);
            off = 0;
        }
        const T *p = cur + off * 32;
        off += G;
        return p;
    }
    // The current segment is done: the next take starts the next chunk.
    __device__ __forceinline__ void end_segment() { off = K; }
};

// Producer side, one thread, for up to NC rings of one block.  stg[w], full[w],
// empty[w]: ring w's stages and barriers; seg0[w] / nseg[w]: its first segment
// and number of segments.  Issues chunk c of every ring in turn once the
// ring's consumer has released chunk c - S.  The first `first` chunks of each
// ring may be issued before the caller's grid-dependency wait (issue_upto),
// the rest after (run).  At the end it waits for every copy it issued, so none
// is in flight when its block exits.  Returns false if a wait gave up.
// EVICT_FIRST: copy with the L2 evict-first hint (streams larger than L2).
template <typename T, int K, int S, int NC, bool EVICT_FIRST = false>
struct RingProducer {
    static constexpr uint32_t CB = (uint32_t)K * 32u * (uint32_t)sizeof(T);
    T *stg[NC];
    uint32_t full[NC], empty[NC];
    const T *src;
    size_t seg_elems;
    int seg0[NC], nseg[NC], issued[NC], pk[NC], pl[NC];
    int nc, seg_step, nch, maxc;

    __device__ __forceinline__ bool issue_upto(int cmax) {
        for (int c = issued_min(); c < cmax; ++c) {
#pragma unroll
            for (int w = 0; w < NC; ++w) {
                if (w >= nc || c >= nseg[w] * nch || c < issued[w]) continue;
                const int s = c % S;
                if (c >= S && !mbar_wait_bounded(empty[w] + 8u * s, (uint32_t)(c / S - 1) & 1u)) return false;
                const T *g = src + (size_t)(seg0[w] + pk[w] * seg_step) * seg_elems + (size_t)pl[w] * K * 32;
                mbar_expect_tx(full[w] + 8u * s, CB);
                if constexpr (EVICT_FIRST) bulk_copy_g2s_stream(smem_addr(stg[w] + (size_t)s * K * 32), g, CB, full[w] + 8u * s);
                else bulk_copy_g2s(smem_addr(stg[w] + (size_t)s * K * 32), g, CB, full[w] + 8u * s);
                if (++pl[w] == nch) {
                    pl[w] = 0;
                    ++pk[w];
                }
                issued[w] = c + 1;
            }
        }
        return true;
    }
    __device__ __forceinline__ int issued_min() const {
        int m = 1 << 30;
#pragma unroll
        for (int w = 0; w < NC; ++w)
            if (w < nc && issued[w] < nseg[w] * nch) m = min(m, issued[w]);
        return m == (1 << 30) ? maxc : m;
    }
    __device__ __forceinline__ bool run() { return issue_upto(maxc); }
    __device__ __forceinline__ void drain() {
#pragma unroll
        for (int w = 0; w < NC; ++w) {
            if (w >= nc) continue;
            for (int c = max(0, issued[w] - S); c < issued[w]; ++c)
                if (!mbar_wait_bounded(full[w] + 8u * (c % S), (uint32_t)(c / S) & 1u)) return;
        }
    }
};

}  // namespace sts
