// ring.cuh -- per-warp shared-memory ring that streams a sequence of
// positions (32 lanes x sizeof(T) contiguous bytes each) from global memory
// with cp.async, kept S-1 chunks ahead of the consumer.
//
// The waits are cp.async.wait_group (hardware group completion), so there is
// no spin loop.  Chunk c lives in stage c % S; before stage s is refilled the
// warp synchronises, so every lane has finished reading it.
#pragma once

#include <cuda_runtime.h>

namespace sts {

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

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

}  // namespace sts
