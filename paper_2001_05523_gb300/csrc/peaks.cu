// Arithmetic peaks of the GPU for the units the H^2 kernels are bound by:
// FP32 FMA (scalar and packed f32x2), FP64 FMA, FP32 reciprocal square root
// (MUFU), FP64 reciprocal square root approximation, FP64 tensor MMA
// (mma.sync m8n8k4), and tcgen05.mma throughput for TF32 and BF16 operands at
// several tile shapes (one CTA per SM, one thread issuing back-to-back MMAs
// into rotating tensor-memory accumulators; every wait is bounded).  Each
// arithmetic kernel runs a fixed number of iterations of independent
// dependency chains on every SM; the rate is operations divided by the
// CUDA-event time of the launch.  Prints one JSON object.
//
// Build and run: nvcc -O3 -gencode arch=compute_103a,code=sm_103a peaks.cu -o peaks && ./peaks
#include <cuda_runtime.h>

#include <cstdint>
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

__global__ void k_ffma2(int iters, float* out) {
    unsigned long long a[kChains];
    const float2 bb = make_float2(0.999999f, 0.999998f), cc = make_float2(1e-7f * (threadIdx.x + 1), 2e-7f);
    const unsigned long long b = *reinterpret_cast<const unsigned long long*>(&bb);
    const unsigned long long c = *reinterpret_cast<const unsigned long long*>(&cc);
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        const float2 v = make_float2(1.0f + j, 2.0f + j);
        a[j] = *reinterpret_cast<const unsigned long long*>(&v);
    }
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[j]) : "l"(b), "l"(c));
    float s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        const float2 v = *reinterpret_cast<const float2*>(&a[j]);
        s += v.x + v.y;
    }
    if (s == 12345.678f) out[0] = s;
}

// tcgen05.mma throughput: KIND 0 TF32 (K = 8), 1 BF16 (K = 16); A: M x 128 B,
// B: N x 128 B, both K-major with 128-byte swizzle (zero-filled); the issuing
// thread rotates over NACC accumulators of N columns (NACC * N <= 512).
__device__ int g_mma_timeout;

template <int KIND, int M, int N>
__global__ void __launch_bounds__(128) k_tc_mma(int iters) {
    constexpr int NACC = 512 / N < 4 ? 512 / N : 4;
    extern __shared__ __align__(16) unsigned char smraw[];
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smraw);
    unsigned char* base = smraw + ((1024 - (s0 & 1023)) & 1023);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    for (int e = threadIdx.x; e < (M + N) * 128 / 16; e += blockDim.x)
        reinterpret_cast<uint4*>(base)[e] = make_uint4(0, 0, 0, 0);
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot;
    if (threadIdx.x == 0) {
        const uint32_t sa = (uint32_t)__cvta_generic_to_shared(base), sb = sa + M * 128;
        auto desc = [](uint32_t addr) {
            return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
                   ((uint64_t)2 << 61);
        };
        const uint64_t ad = desc(sa), bd = desc(sb);
        constexpr uint32_t fmt = KIND == 0 ? 2u : 1u;
        constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
        for (int i = 0; i < iters; ++i) {
            const uint32_t d = tmem + (uint32_t)((i % NACC) * N);
            const uint32_t acc = i >= NACC;
            if (KIND == 0)
                asm volatile("{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}" ::"r"(d),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            else
                asm volatile("{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}" ::"r"(d),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
    }
    const long long t0 = clock64();
    uint32_t done = 0;
    while (!done) {
        asm volatile("{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.b32 %0, 1, 0, P;\n}"
                     : "=r"(done)
                     : "r"(mb), "r"(0)
                     : "memory");
        if (!done && clock64() - t0 > 4000000000LL) {
            atomicExch(&g_mma_timeout, 1);
            break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
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
    const float t_ffma2 = time_ms([&] { k_ffma2<<<blocks, threads>>>(it / 2, f); });
    // tcgen05: one CTA per SM
    const int tci = 2048;
    auto tc = [&](auto kern, int M, int N, int K) {
        const int smem = 1024 + (M + N) * 128;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        const float ms = time_ms([&] { kern<<<sms, 128, smem>>>(tci); });
        return (double)sms * tci * 2.0 * M * N * K / (ms * 1e-3) / 1e12;
    };
    const double tf32_128_256 = tc(k_tc_mma<0, 128, 256>, 128, 256, 8);
    const double tf32_128_16 = tc(k_tc_mma<0, 128, 16>, 128, 16, 8);
    const double tf32_64_8 = tc(k_tc_mma<0, 64, 8>, 64, 8, 8);
    const double tf32_64_64 = tc(k_tc_mma<0, 64, 64>, 64, 64, 8);
    const double bf16_128_256 = tc(k_tc_mma<1, 128, 256>, 128, 256, 16);
    const double bf16_64_8 = tc(k_tc_mma<1, 64, 8>, 64, 8, 16);
    int mma_timeout = 0;
    cudaMemcpyFromSymbol(&mma_timeout, g_mma_timeout, sizeof(int));
    const cudaError_t err = cudaDeviceSynchronize();
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    const double ffma = nthr * it * kChains * 2 / (t_ffma * 1e-3) / 1e12;
    const double dfma = nthr * (it / 16) * kChains * 2 / (t_dfma * 1e-3) / 1e12;
    const double rs32 = nthr * (it / 4) * kChains / (t_rs32 * 1e-3) / 1e12;
    const double rs64 = nthr * (it / 16) * kChains / (t_rs64 * 1e-3) / 1e12;
    const double dmma = (nthr / 32) * (it / 16) * 4 * (2.0 * 8 * 8 * 4) / (t_dmma * 1e-3) / 1e12;
    const double ffma2 = nthr * (it / 2) * kChains * 4 / (t_ffma2 * 1e-3) / 1e12;
    std::printf(
        "{\"device\": \"%s\", \"sms\": %d, \"clock_mhz_attr\": %.0f, \"fp32_fma_tflops\": %.3f, "
        "\"fp64_fma_tflops\": %.4f, \"rsqrt_f32_tops\": %.4f, \"rsqrt_f64_approx_tops\": %.5f, "
        "\"fp64_mma_tflops\": %.4f, \"fp32x2_fma_tflops\": %.3f, \"tc_tf32_m128n256_tflops\": %.1f, "
        "\"tc_tf32_m128n16_tflops\": %.2f, \"tc_tf32_m64n8_tflops\": %.3f, \"tc_tf32_m64n64_tflops\": %.2f, "
        "\"tc_bf16_m128n256_tflops\": %.1f, \"tc_bf16_m64n8_tflops\": %.3f, \"tc_timeout\": %d, \"status\": \"%s\"}\n",
        prop.name, sms, clk_khz / 1e3, ffma, dfma, rs32, rs64, dmma, ffma2, tf32_128_256, tf32_128_16, tf32_64_8,
        tf32_64_64, bf16_128_256, bf16_64_8, mma_timeout, cudaGetErrorString(err));
    cudaFree(f);
    cudaFree(d);
    return err == cudaSuccess ? 0 : 1;
}
