// ring.cuh -- per-warp shared-memory rings that stream coefficient positions
// (32 lanes x sizeof(T) bytes each) from global memory ahead of the consumer.
//
// Ring:     strided positions, copied with cp.async (16 bytes per lane and
//           instruction); waits are cp.async.wait_group, no spin loop.
// BulkRing: contiguous chunks copied by the bulk-copy (TMA) engine, one
//           cp.async.bulk per chunk issued by lane 0 and completed on one
//           mbarrier per stage; waits are bounded in time.
// In both, chunk c lives in stage c % S and the warp synchronises before a
// stage is refilled, so every lane has finished reading it.
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
    // The next `width` positions as one row (width <= K): rows never straddle
    // a chunk, the producer pads a chunk with zeros where the next row would
    // not fit.  Returns the lane's pointer to the row's first value.
    __device__ __forceinline__ const T *take(int width) {
        if (off + width > K) {
            ++ch;
            off = 0;
            enter(ch);
        }
        const T *p = cur + off * 32;
        off += width;
        return p;
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

// Per-warp ring over a sequence of equal-length segments (one per tile the
// warp processes): segment k starts at src + (seg0 + k * seg_step) * seg_elems
// and holds nch chunks of K positions.  Positions are laid out as
// [position / VEC][lane][VEC], so a lane reads VEC consecutive positions with
// one 16-byte load.  stg: S * K * 32 elements (16-byte aligned); bars: S
// mbarriers (8-byte aligned).
//
// S - 2 chunks are in flight ahead of the current one: entering chunk c
// refills the stage of chunk c - 2, never that of c - 1, so a consumer may
// load its next group (possibly from chunk c) before it has used the values
// it loaded from chunk c - 1.
template <typename T, int K, int S>
struct BulkRing {
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr uint32_t CB = (uint32_t)K * 32u * (uint32_t)sizeof(T);   // bytes per chunk
    static_assert(K % VEC == 0, "chunk must hold whole vectors");
    static_assert(S >= 3, "two stages plus at least one in flight");
    T *stg;
    uint32_t bar;
    const T *src;
    size_t seg_elems;
    int seg0, seg_step, nch;
    int total, issued, pk, pl;    // producer: chunks issued, next (segment, chunk)
    int ch, off, lane;            // consumer: current chunk and position in it
    int waited;                   // chunks [0, waited) have completed
    bool failed;                  // a wait gave up; later takes return stale data
    const T *cur;

    __device__ __forceinline__ void issue() {
        const int s = issued % S;
        if (lane == 0) {
            const T *g = src + (size_t)(seg0 + pk * seg_step) * seg_elems + (size_t)pl * K * 32;
            mbar_expect_tx(bar + 8u * s, CB);
            bulk_copy_g2s(smem_addr(stg + (size_t)s * K * 32), g, CB, bar + 8u * s);
        }
        if (++pl == nch) {
            pl = 0;
            ++pk;
        }
        ++issued;
    }
    // Barriers are initialised by lane 0; the first S-2 chunks are issued
    // (now, or by prime() when the source may not be read yet).
    __device__ __forceinline__ void start(T *stg_, uint64_t *bars, const T *src_, size_t seg_elems_, int seg0_,
                                          int seg_step_, int nseg, int nch_, int lane_, bool issue_now = true) {
        stg = stg_;
        bar = smem_addr(bars);
        src = src_;
        seg_elems = seg_elems_;
        seg0 = seg0_;
        seg_step = seg_step_;
        nch = nch_;
        total = nseg * nch_;
        issued = 0;
        pk = 0;
        pl = 0;
        ch = -1;
        off = K;
        lane = lane_;
        waited = 0;
        failed = false;
        cur = stg + lane * VEC;
        if (lane == 0) {
#pragma unroll
            for (int s = 0; s < S; ++s) mbar_init(bar + 8u * s, 1);
            mbar_init_fence();
        }
        __syncwarp();
        if (issue_now) prime();
    }
    __device__ __forceinline__ void prime() {
        for (int c = 0; c < S - 2 && issued < total; ++c) issue();
    }
    // Make chunk c current (waiting for it) and refill the stage of c - 2.
    __device__ __forceinline__ void enter(int c) {
        if (failed) return;
        const int s = c % S;
        if (!mbar_wait_bounded(bar + 8u * s, (uint32_t)(c / S) & 1u)) {
            failed = true;
            return;
        }
        waited = c + 1;
        __syncwarp();
        if (issued < total) issue();
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
    // After a failed wait: wait (bounded) for the copies still in flight, so
    // that none lands after the kernel has returned.
    __device__ __forceinline__ void drain() {
        for (int c = waited; c < issued; ++c)
            if (!mbar_wait_bounded(bar + 8u * (c % S), (uint32_t)(c / S) & 1u)) return;
    }
};

}  // namespace sts
