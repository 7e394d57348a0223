// Arithmetic-rate probe for the roofline denominators the benchmark uses on
// this part: FP64 FMA (DFMA), FP64 tensor-core MMA (mma.sync m8n8k4 f64) and
// FP32 FMA (FFMA).  Every thread runs independent dependency chains so that
// the pipes, not latency, bound the rate; a grid of 8 CTAs per SM covers the
// whole GPU.  Times with CUDA events, best of several runs, after a warm-up.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 peaks.cu -o peaks && ./peaks
#include <cstdio>
#include <cuda_runtime.h>

constexpr int ITERS = 4096;
constexpr int CHAINS = 8;

__global__ void dfma_kernel(double *out, double a, double b) {
    double x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == 12345.678) out[0] = s;  // keeps the chains live
}

__global__ void ffma_kernel(float *out, float a, float b) {
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == 12345.678f) out[0] = s;
}

// one m8n8k4 FP64 MMA: D (8x8) += A (8x4) B (4x8); per thread 1 A, 1 B, 2 C/D values
__global__ void dmma_kernel(double *out, double a0, double b0) {
    double c[CHAINS][2];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) { c[k][0] = 0.0; c[k][1] = 0.0; }
    const double a = a0 + threadIdx.x * 1e-6, b = b0;
    for (int i = 0; i < ITERS / 4; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c[k][0]), "+d"(c[k][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += c[k][0] + c[k][1];
    if (s == 12345.678) out[0] = s;
}

template <typename F>
static double best_ms(F launch) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();
    cudaDeviceSynchronize();
    double best = 1e30;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

int main() {
    int dev = 0, nsm = 0, clk = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    double *dout = nullptr;
    if (cudaMalloc(&dout, 64) != cudaSuccess) return 1;
    const int blocks = nsm * 8, threads = 256;
    const double nthr = (double)blocks * threads;
    const double t_dfma = best_ms([&] { dfma_kernel<<<blocks, threads>>>(dout, 0.999, 1e-3); });
    const double t_ffma = best_ms([&] { ffma_kernel<<<blocks, threads>>>((float *)dout, 0.999f, 1e-3f); });
    const double t_dmma = best_ms([&] { dmma_kernel<<<blocks, threads>>>(dout, 1e-3, 0.5); });
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { printf("{\"error\": \"%s\"}\n", cudaGetErrorString(e)); return 1; }
    // flops: 2 per FMA; an m8n8k4 MMA is 2*8*8*4 = 512 flops per warp
    const double dfma = nthr * ITERS * CHAINS * 2.0 / (t_dfma * 1e-3) / 1e12;
    const double ffma = nthr * ITERS * CHAINS * 2.0 / (t_ffma * 1e-3) / 1e12;
    const double dmma = (nthr / 32.0) * (ITERS / 4) * CHAINS * 512.0 / (t_dmma * 1e-3) / 1e12;
    printf("{\"sms\": %d, \"clock_mhz_attr\": %.0f, \"fp64_fma_tflops\": %.4f, \"fp64_mma_tflops\": %.4f, "
           "\"fp32_fma_tflops\": %.3f, \"ms\": [%.3f, %.3f, %.3f]}\n",
           nsm, clk / 1e3, dfma, dmma, ffma, t_dfma, t_dmma, t_ffma);
    cudaFree(dout);
    return 0;
}
