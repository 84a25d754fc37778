// fp64_probe.cu -- throughput and dependent-issue cost of FP64 and FP32 FMA on
// the current GPU, and streaming read bandwidth.  Used to derive the FP64
// roofline the benchmark reports: a warp-wide FP64 FMA occupies one SM
// sub-partition's FP64 pipe for (32 / FMAs-per-clock-per-sub-partition) cycles.
#include <cstdio>
#include <cuda_runtime.h>

#define CK(x)                                                                            \
    do {                                                                                 \
        cudaError_t e = (x);                                                             \
        if (e != cudaSuccess) {                                                          \
            printf("CUDA error %s at line %d: %s\n", #x, __LINE__, cudaGetErrorString(e)); \
            return 1;                                                                    \
        }                                                                                \
    } while (0)

template <typename T>
__global__ void fma_throughput(T *out, int iters, T a, T b) {
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
      x7 = x0 + 7;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// One dependent chain per thread; cycles per warp-wide instruction.
__global__ void fma_chain(double *out, int iters, double a, double b, long long *cyc, int active) {
    if ((int)(threadIdx.x & 31) >= active) return;
    double x = threadIdx.x;
    const long long t0 = clock64();
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 16; k++) x = fma(x, a, b);
    }
    const long long t1 = clock64();
    out[threadIdx.x] = x;
    if ((threadIdx.x & 31) == 0) cyc[threadIdx.x / 32] = t1 - t0;
}

// Same as fma_throughput<double> with only the first `active` lanes of each
// warp working: does a warp instruction with fewer active lanes take less of
// the FP64 pipe?
__global__ void fma_partial(double *out, int iters, double a, double b, int active) {
    if ((int)(threadIdx.x & 31) >= active) return;
    double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
           x7 = x0 + 7;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// One warp: a dependent FP64 FMA chain with NOPS independent FP32 FMAs (four
// chains) after each FP64 FMA.  Cycles per (1 + NOPS) group tell whether the
// warp can issue other work while its FP64 FMA occupies the pipe.
template <int NOPS>
__global__ void fma_mix(double *out, float *fout, int iters, double a, double b, long long *cyc) {
    double x = threadIdx.x;
    float f0 = threadIdx.x, f1 = f0 + 1.f, f2 = f0 + 2.f, f3 = f0 + 3.f;
    const long long t0 = clock64();
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            x = fma(x, a, b);
#pragma unroll
            for (int j = 0; j < NOPS; j += 4) {
                f0 = fmaf(f0, 0.999f, 1e-3f); f1 = fmaf(f1, 0.999f, 1e-3f);
                f2 = fmaf(f2, 0.999f, 1e-3f); f3 = fmaf(f3, 0.999f, 1e-3f);
            }
        }
    }
    const long long t1 = clock64();
    out[threadIdx.x] = x;
    fout[threadIdx.x] = f0 + f1 + f2 + f3;
    if (threadIdx.x == 0) cyc[0] = t1 - t0;
}

template <int NOPS>
static int run_mix(double *dout, float *fout, long long *cyc) {
    fma_mix<NOPS><<<1, 32>>>(dout, fout, 64, 0.999, 1e-3, cyc);
    CK(cudaDeviceSynchronize());
    fma_mix<NOPS><<<1, 32>>>(dout, fout, 64, 0.999, 1e-3, cyc);
    long long h;
    CK(cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost));
    printf("one warp, FP64 FMA chain + %2d FP32 FMAs after each: %.1f cycles per group\n", NOPS,
           (double)h / (64 * 8));
    return 0;
}

// One warp, dependent FP64 FMA chain of 512 steps; per step the multiplier
// comes from shared memory (mode 1: loaded just before use, mode 2: loaded one
// step ahead) and/or the result is stored to shared memory (mode 3), or the
// result also feeds an FP32 accumulator (mode 4).  Cycles per step.
__global__ void fma_smem(double *out, int mode, long long *cyc) {
    __shared__ double sm[512 + 32];
    __shared__ double so[64 * 32];
    const int lane = threadIdx.x;
    for (int i = lane; i < 512 + 32; i += 32) sm[i] = 0.999 + 1e-6 * (i & 7);
    __syncwarp();
    double x = lane;
    float f = 0.f;
    long long t0 = 0, t1 = 0;
    for (int rep = 0; rep < 2; ++rep) {
        t0 = clock64();
        if (mode == 0) {
#pragma unroll 16
            for (int i = 0; i < 512; ++i) x = fma(x, 0.999, 1e-3);
        } else if (mode == 1) {
#pragma unroll 16
            for (int i = 0; i < 512; ++i) x = fma(x, sm[i], 1e-3);
        } else if (mode == 2) {
            double m = sm[0];
#pragma unroll 16
            for (int i = 0; i < 512; ++i) {
                const double mn = sm[i + 1];
                x = fma(x, m, 1e-3);
                m = mn;
            }
        } else if (mode == 3) {
#pragma unroll 16
            for (int i = 0; i < 512; ++i) {
                x = fma(x, 0.999, 1e-3);
                so[(i & 63) * 32 + lane] = x;
            }
        } else {
#pragma unroll 16
            for (int i = 0; i < 512; ++i) {
                x = fma(x, 0.999, 1e-3);
                f += (float)x;
            }
        }
        t1 = clock64();
    }
    out[lane] = x + f + so[lane * 7];
    if (lane == 0) cyc[0] = t1 - t0;
}

__global__ void read_stream(const float4 *__restrict__ p, size_t n, float *out) {
    float s = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = __ldg(p + i);
        s += v.x + v.y + v.z + v.w;
    }
    if (s == 12345.678f) out[0] = s;
}

int main() {
    cudaDeviceProp pr;
    CK(cudaGetDeviceProperties(&pr, 0));
    int clk_khz = 0;
    CK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0));
    const int nsm = pr.multiProcessorCount;
    printf("device %s sm_%d%d SMs %d L2 %d bytes max clock %.0f MHz\n", pr.name, pr.major, pr.minor, nsm,
           pr.l2CacheSize, clk_khz / 1e3);
    double *dout;
    float *fout;
    long long *cyc;
    CK(cudaMalloc(&dout, 1 << 24));
    CK(cudaMalloc(&fout, 1 << 24));
    CK(cudaMalloc(&cyc, 64 * sizeof(long long)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = nsm * 8, bs = 512;     // grid * bs * 8 bytes < 1 << 24
    for (int pass = 0; pass < 2; pass++) {
        const int it64 = 64, it32 = 1024;
        fma_throughput<double><<<grid, bs>>>(dout, it64, 0.999, 1e-3);
        CK(cudaEventRecord(e0));
        fma_throughput<double><<<grid, bs>>>(dout, it64, 0.999, 1e-3);
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        const double f64 = (double)grid * bs * it64 * 64 / (ms * 1e-3);
        fma_throughput<float><<<grid, bs>>>(fout, it32, 0.999f, 1e-3f);
        CK(cudaEventRecord(e0));
        fma_throughput<float><<<grid, bs>>>(fout, it32, 0.999f, 1e-3f);
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        cudaEventElapsedTime(&ms, e0, e1);
        const double f32 = (double)grid * bs * it32 * 64 / (ms * 1e-3);
        if (pass == 1)
            printf("FP64 FMA %.4f T/s (%.3f per SM per clock at max clock); FP32 FMA %.3f T/s\n", f64 / 1e12,
                   f64 / nsm / (clk_khz * 1e3), f32 / 1e12);
    }
    for (int active : {1, 32}) {
        fma_chain<<<1, 32>>>(dout, 256, 0.999, 1e-3, cyc, active);
        CK(cudaDeviceSynchronize());
        fma_chain<<<1, 32>>>(dout, 256, 0.999, 1e-3, cyc, active);
        long long h;
        CK(cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost));
        printf("dependent FP64 FMA, one warp, %2d active lanes: %.1f cycles per instruction\n", active,
               (double)h / (256 * 16));
    }
    for (int active : {32, 16, 8}) {
        const int it64 = 64;
        fma_partial<<<grid, bs>>>(dout, it64, 0.999, 1e-3, active);
        CK(cudaEventRecord(e0));
        fma_partial<<<grid, bs>>>(dout, it64, 0.999, 1e-3, active);
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        const double winst = (double)grid * (bs / 32) * it64 * 64 / (ms * 1e-3);
        printf("FP64 FMA, %2d active lanes per warp: %.4f T lane-FMA/s, %.3f warp instructions per SM per clock\n",
               active, winst * active / 1e12, winst / nsm / (clk_khz * 1e3));
    }
    if (run_mix<0>(dout, fout, cyc) || run_mix<8>(dout, fout, cyc) || run_mix<16>(dout, fout, cyc) ||
        run_mix<32>(dout, fout, cyc) || run_mix<48>(dout, fout, cyc) || run_mix<64>(dout, fout, cyc) ||
        run_mix<96>(dout, fout, cyc))
        return 1;
    {
        const char *what[5] = {"constant multiplier", "multiplier loaded from shared memory just before use",
                               "multiplier loaded from shared memory one step ahead",
                               "result stored to shared memory each step", "result also added to an FP32 sum"};
        for (int mode = 0; mode < 5; ++mode) {
            fma_smem<<<1, 32>>>(dout, mode, cyc);
            CK(cudaDeviceSynchronize());
            long long h;
            CK(cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost));
            printf("one warp, dependent FP64 FMA chain, %s: %.1f cycles per step\n", what[mode], (double)h / 512);
        }
    }
    const size_t bytes = (size_t)4 << 30;
    void *buf;
    CK(cudaMalloc(&buf, bytes));
    CK(cudaMemset(buf, 0, bytes));
    const size_t n = bytes / 16;
    read_stream<<<nsm * 8, 256>>>((const float4 *)buf, n, fout);
    CK(cudaEventRecord(e0));
    for (int r = 0; r < 5; r++) read_stream<<<nsm * 8, 256>>>((const float4 *)buf, n, fout);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms;
    cudaEventElapsedTime(&ms, e0, e1);
    printf("streaming read %.1f GB/s\n", 5.0 * bytes / (ms * 1e-3) / 1e9);
    CK(cudaGetLastError());
    return 0;
}
