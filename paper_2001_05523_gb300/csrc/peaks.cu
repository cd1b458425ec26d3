// Arithmetic peaks of the GPU for the units the H^2 kernels are bound by:
// FP32 FMA, FP64 FMA, FP32 reciprocal square root (MUFU), FP64 reciprocal
// square root approximation, FP64 tensor MMA (mma.sync m8n8k4).  Each kernel
// runs a fixed number of iterations of independent dependency chains on every
// SM (no waits, no memory traffic in the loop); the rate is operations divided
// by the CUDA-event time of the launch.  Prints one JSON object.
//
// Build and run: nvcc -O3 -gencode arch=compute_103a,code=sm_103a peaks.cu -o peaks && ./peaks
#include <cuda_runtime.h>

#include <cstdio>

namespace {
constexpr int kChains = 8;

__global__ void k_ffma(int iters, float* out) {
    float a[kChains];
    const float b = 0.999999f, c = 1e-7f * (threadIdx.x + 1);
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.0f + j;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
    float s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 12345.678f) out[0] = s;  // keeps the chains alive
}

__global__ void k_dfma(int iters, double* out) {
    double a[kChains];
    const double b = 0.999999, c = 1e-7 * (threadIdx.x + 1);
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.0 + j;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    double s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 12345.678) out[0] = s;
}

__global__ void k_rsqrt32(int iters, float* out) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.0f + 0.1f * j + 1e-6f * threadIdx.x;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            float y;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[j]));
            a[j] = y;  // the map y -> 1/sqrt(y) stays in [1/sqrt(2), sqrt(2)]
        }
    float s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 12345.678f) out[0] = s;
}

__global__ void k_rsqrt64(int iters, double* out) {
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.0 + 0.1 * j + 1e-6 * threadIdx.x;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            double y;
            asm volatile("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a[j]));
            a[j] = y;
        }
    double s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 12345.678) out[0] = s;
}

// FP64 tensor MMA: D(8x8) = A(8x4) B(4x8) + C per warp, 4 independent accumulators
__global__ void k_dmma(int iters, double* out) {
    const double a = 1.0 + 1e-9 * threadIdx.x, b = 0.5;
    double d[4][2];
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j][0] = d[j][1] = 0.0;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(d[j][0]), "+d"(d[j][1])
                         : "d"(a), "d"(b));
    double s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) s += d[j][0] + d[j][1];
    if (s == 12345.678) out[0] = s;
}

template <typename F>
float time_ms(F launch) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();  // warm-up
    cudaDeviceSynchronize();
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}
}  // namespace

int main() {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, 0) != cudaSuccess) {
        std::printf("{\"error\": \"no device\"}\n");
        return 1;
    }
    const int sms = prop.multiProcessorCount;
    const int blocks = sms * 8, threads = 256;
    const double nthr = (double)blocks * threads;
    float* f = nullptr;
    double* d = nullptr;
    cudaMalloc(&f, 16);
    cudaMalloc(&d, 16);
    const int it = 1 << 16;
    const float t_ffma = time_ms([&] { k_ffma<<<blocks, threads>>>(it, f); });
    const float t_dfma = time_ms([&] { k_dfma<<<blocks, threads>>>(it / 16, d); });
    const float t_rs32 = time_ms([&] { k_rsqrt32<<<blocks, threads>>>(it / 4, f); });
    const float t_rs64 = time_ms([&] { k_rsqrt64<<<blocks, threads>>>(it / 16, d); });
    const float t_dmma = time_ms([&] { k_dmma<<<blocks, threads>>>(it / 16, d); });
    const cudaError_t err = cudaDeviceSynchronize();
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    const double ffma = nthr * it * kChains * 2 / (t_ffma * 1e-3) / 1e12;
    const double dfma = nthr * (it / 16) * kChains * 2 / (t_dfma * 1e-3) / 1e12;
    const double rs32 = nthr * (it / 4) * kChains / (t_rs32 * 1e-3) / 1e12;
    const double rs64 = nthr * (it / 16) * kChains / (t_rs64 * 1e-3) / 1e12;
    const double dmma = (nthr / 32) * (it / 16) * 4 * (2.0 * 8 * 8 * 4) / (t_dmma * 1e-3) / 1e12;
    std::printf(
        "{\"device\": \"%s\", \"sms\": %d, \"clock_mhz_attr\": %.0f, \"fp32_fma_tflops\": %.3f, "
        "\"fp64_fma_tflops\": %.4f, \"rsqrt_f32_tops\": %.4f, \"rsqrt_f64_approx_tops\": %.5f, "
        "\"fp64_mma_tflops\": %.4f, \"status\": \"%s\"}\n",
        prop.name, sms, clk_khz / 1e3, ffma, dfma, rs32, rs64, dmma, cudaGetErrorString(err));
    cudaFree(f);
    cudaFree(d);
    return err == cudaSuccess ? 0 : 1;
}
