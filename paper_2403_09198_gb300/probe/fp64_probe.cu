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
