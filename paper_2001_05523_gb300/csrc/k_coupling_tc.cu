// Coupling stage on the tensor cores (tcgen05), section 2 eq. (vsw):
//   yh_t = 1/(4 pi) sum_{(t,s) farfield} S_ts xh_s,   S_ts[nu, mu] = 1 / |xi_{t,nu} - xi_{s,mu}|,
// with the interpolation points xi of section 3.
//
// One CTA (4 warps) per row cluster t.  For every farfield block (t, s) the
// CTA generates S_ts in FP32 from the per-axis squared node differences (one
// reciprocal square root per entry, the same values as the SIMT kernel),
// rounds it to the operand type and stores it in shared memory in the
// K-major layout with 128-byte swizzle (row nu, 128-byte rows of mu, 16-byte
// chunk c of row r at chunk c ^ (r mod 8) of its 1024-byte group of 8 rows);
// x-hat_s is staged the same way with the right-hand sides as rows.  One
// thread issues tcgen05.mma with M = 64 rows of nu per tile, N = 8 or 16
// right-hand sides and K = 8 (TF32) or 16 (BF16) values of mu per
// instruction; the accumulator D (FP32) stays in tensor memory over all blocks
// of the row (one accumulator per row tile: rotating consecutive MMAs over
// several accumulators measured slower) and the epilogue adds it to y-hat in
// FP64.  Two stages of shared memory let the CTA generate block b+1
// while the tensor core consumes block b (an mbarrier per stage, signalled by
// tcgen05.commit).  Accumulator layout for M = 64: row i of a tile is tensor
// memory lane 32 (i / 16) + i % 16, so warp w reads rows 16w .. 16w+15.
//
// Operand kinds: TF32 (round to nearest), BF16, and TF32x3, the error-
// compensated split of Ootomo and Yokota (2022): S = S_hi + S_lo and x = x_hi +
// x_lo in TF32, D += S_hi x_hi + S_hi x_lo + S_lo x_hi, which recovers about
// FP32 accuracy of the products (the dropped S_lo x_lo is ~2^-22 relative).
//
// Every wait on an mbarrier gives up after about a second: the CTA then
// records H2BEM_ERR_TIMEOUT in a device flag, stops issuing, waits (bounded)
// for what it issued, frees its tensor memory and returns.
#include <cstdint>
#include <type_traits>

#include "dmath.cuh"
#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;
constexpr int kThreads = 128;
constexpr long long kWaitCycles = 2000000000LL;  // about a second at the SM clock
constexpr long long kTestWaitCycles = 100000LL;   // the test wait on a barrier nothing signals (~50 us)

__device__ int g_tc_status;  // 0, or H2BEM_ERR_TIMEOUT's value after an expired wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float rsqrt_f32(float a) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}

__device__ __forceinline__ uint32_t to_tf32(float v) {
    uint32_t b;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(v));
    return b;
}

__device__ __forceinline__ uint32_t to_bf16x2(float lo, float hi) {
    uint32_t b;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(b) : "f"(hi), "f"(lo));
    return b;
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
           ((uint64_t)2 << 61);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, long long limit = kWaitCycles) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.b32 %0, 1, 0, P;\n}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// compile-time shape of one configuration
template <int M, int NR, int KIND>  // KIND: 0 TF32, 1 TF32x3, 2 BF16
struct TcShape {
    static constexpr int K = M * M * M;
    static constexpr int EB = KIND == 2 ? 2 : 4;                 // bytes per operand element
    static constexpr int KBLK = 128 / EB;                        // elements per 128-byte row
    static constexpr int KPAD = (K + KBLK - 1) / KBLK * KBLK;
    static constexpr int NKB = KPAD / KBLK;
    static constexpr int MT = (K + 63) / 64;                     // 64-row tiles of nu
    static constexpr int N = NR < 8 ? 8 : NR;                    // MMA N
    static constexpr int KSTEP = KIND == 2 ? 16 : 8;             // K per instruction
    static constexpr int SPK = KBLK / KSTEP;                     // instructions per 128-byte row
    static constexpr int NSPLIT = KIND == 1 ? 2 : 1;
    static constexpr int ATILE = NKB * MT * 8192;                // bytes of one A operand
    static constexpr int BTILE = NKB * (N / 8) * 1024;           // bytes of one B operand
    static constexpr int STAGE = NSPLIT * (ATILE + BTILE);
    static constexpr int TPR = M == 4 ? 2 : 1;                   // threads per row of S
    static constexpr int ROWS = kThreads / TPR;                  // rows generated per pass
    static constexpr int QPT = KPAD / TPR;                       // entries per thread and row
    static constexpr int CH = 16 / EB;                           // entries per 16-byte chunk
    static constexpr int PASSES = KIND == 1 ? 3 : 1;
    static constexpr int STEPS = NKB * SPK * PASSES;             // MMAs per block and row tile
    static constexpr int NACC = 1;                               // accumulators per row tile
    static constexpr int COLS = MT * NACC * N;
    static constexpr int TMEM_COLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : 256;
    static constexpr size_t SMEM = 1024 + 2 * (size_t)STAGE;     // + alignment slack
    static_assert(COLS <= 256, "tensor memory columns");
    static_assert(ROWS * TPR == kThreads && ROWS >= MT * 64 || M == 4, "row mapping");
};

// byte offset of element (row r, column e) in a K-major swizzled operand whose
// 128-byte-row blocks (of KBLK columns) are `blk` bytes apart
template <int EB>
__device__ __forceinline__ int sw_off(int r, int e, int blk) {
    constexpr int KBLK = 128 / EB;
    const int kb = e / KBLK, w = (e % KBLK) * EB;
    return kb * blk + (r >> 3) * 1024 + (r & 7) * 128 + ((((w >> 4) ^ (r & 7))) << 4) + (w & 15);
}

// generate row nu of S_ts (columns P*QPT .. P*QPT+QPT-1) into the stage
template <int M, int NR, int KIND, int P>
__device__ __forceinline__ void gen_row(unsigned char* stage, int nu, const float* X, const float* Y,
                                        const float* Z) {
    using S = TcShape<M, NR, KIND>;
    const int mt = nu >> 6, rr = nu & 63;
    unsigned char* rowbase = stage + mt * 8192 + (rr >> 3) * 1024 + (rr & 7) * 128;
#pragma unroll
    for (int cq = 0; cq < S::QPT / S::CH; ++cq) {
        float v[S::CH];
#pragma unroll
        for (int i = 0; i < S::CH; ++i) {
            const int mu = P * S::QPT + cq * S::CH + i;
            if (mu < S::K) {
                const float r2 = X[mu % M] + Y[(mu / M) % M] + Z[mu / (M * M)];
                v[i] = rsqrt_f32(r2);
            } else {
                v[i] = 0.0f;
            }
        }
        const int mu0 = P * S::QPT + cq * S::CH;
        const int kb = mu0 / S::KBLK, ch = (mu0 % S::KBLK) / S::CH;
        const int off = kb * (S::MT * 8192) + ((ch ^ (rr & 7)) << 4);
        uint4 hi, lo = make_uint4(0, 0, 0, 0);
        if constexpr (KIND == 2) {
            hi.x = to_bf16x2(v[0], v[1]);
            hi.y = to_bf16x2(v[2], v[3]);
            hi.z = to_bf16x2(v[4], v[5]);
            hi.w = to_bf16x2(v[6], v[7]);
        } else {
            hi.x = to_tf32(v[0]);
            hi.y = to_tf32(v[1]);
            hi.z = to_tf32(v[2]);
            hi.w = to_tf32(v[3]);
            if constexpr (KIND == 1) {
                lo.x = to_tf32(v[0] - __uint_as_float(hi.x));
                lo.y = to_tf32(v[1] - __uint_as_float(hi.y));
                lo.z = to_tf32(v[2] - __uint_as_float(hi.z));
                lo.w = to_tf32(v[3] - __uint_as_float(hi.w));
            }
        }
        *reinterpret_cast<uint4*>(rowbase + off) = hi;
        if constexpr (KIND == 1) *reinterpret_cast<uint4*>(rowbase + S::ATILE + S::BTILE + off) = lo;
    }
}
}  // namespace

template <int M, int NR, int KIND>
__global__ void __launch_bounds__(kThreads) k_coupling_tc(Tree t, Consts c, const int* __restrict__ rows,
                                                          const int* __restrict__ ptr, const int* __restrict__ col,
                                                          const float* __restrict__ xh, float* __restrict__ yh,
                                                          int stall_test) {
    using S = TcShape<M, NR, KIND>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    __shared__ float2 zt[3 * M];  // nodes of t as FP32 (hi, lo)
    __shared__ float D2[3 * M * M];
    __shared__ __align__(8) uint64_t mbar[3];  // two pipeline stages; [2] is never signalled (stall_test)
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = rows[blockIdx.x];
    const int b0 = ptr[blockIdx.x], nb = ptr[blockIdx.x + 1] - b0;

    // zero both stages (padding rows and columns stay zero), nodes of t
    for (int e = tid; e < 2 * S::STAGE / 16; e += kThreads) reinterpret_cast<uint4*>(base)[e] = make_uint4(0, 0, 0, 0);
    for (int e = tid; e < 3 * M; e += kThreads) zt[e] = t.zhl[(int64_t)row * 3 * M + e];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "r"(S::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[2])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot;

    // instruction descriptor: D FP32, A/B TF32 (2) or BF16 (1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
    constexpr uint32_t fmt = KIND == 2 ? 1u : 2u;
    constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(S::N >> 3) << 17) | (4u << 24);

    // this thread's row of S and column range
    const int nu = tid % S::ROWS, part = tid / S::ROWS;
    const bool gen = nu < S::K;
    const int ia = nu % M, ib = (nu / M) % M, ic = nu / (M * M);
    bool ok = true;
    int issued = 0;  // commits issued (by thread 0)
    // register prefetch of the next block's x-hat values and box (centre, half-width)
    constexpr int PF = (S::K * NR + kThreads - 1) / kThreads;
    float xpre[PF];
    float2 zpre = make_float2(0.0f, 0.0f);  // node (d, a2) of the column cluster, (hi, lo)
    static_assert(3 * M * M <= kThreads, "one D2 entry per thread");
    auto prefetch = [&](int b) {
        const int s = col[b0 + b];
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int e = tid + j * kThreads;
            xpre[j] = e < S::K * NR ? xh[(int64_t)s * S::K * NR + e] : 0.0f;
        }
        if (tid < 3 * M * M) {
            const int d = tid / (M * M), a2 = tid % M;
            zpre = t.zhl[(int64_t)s * 3 * M + d * M + a2];
        }
    };
    if (nb > 0) prefetch(0);
    for (int b = 0; b < nb; ++b) {
        const int st = b & 1;
        unsigned char* stage = base + st * S::STAGE;
        if (b >= 2) {
            // stall_test: the first of these waits is on mbar[2], which nothing
            // signals, with a short bound, so that it expires (the issued MMAs
            // are still drained below with the normal bound)
            const bool stall = stall_test && b == 2;
            bool w = stall ? mbar_wait(smem_u32(&mbar[2]), 0, kTestWaitCycles)
                           : mbar_wait(smem_u32(&mbar[st]), ((b - 2) >> 1) & 1);
            ok = __syncthreads_and(w) != 0;
            if (!ok) break;
        }
        if (tid < 3 * M * M) {
            const int d = tid / (M * M), a = (tid / M) % M;
            const float2 u = zt[d * M + a];
            const float df = (u.x - zpre.x) + (u.y - zpre.y);
            D2[tid] = df * df;
        }
        // x-hat_s staged transposed: row r, column mu
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int e = tid + j * kThreads;
            if (e >= S::K * NR) break;
            const int mu = e / NR, r = e % NR;
            const float v = xpre[j];
            unsigned char* bt = stage + S::ATILE;
            const int off = sw_off<S::EB>(r, mu, (S::N / 8) * 1024);
            if (KIND == 2) {
                unsigned short h;
                asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(v));
                *reinterpret_cast<unsigned short*>(bt + off) = h;
            } else {
                const uint32_t hb = to_tf32(v);
                *reinterpret_cast<uint32_t*>(bt + off) = hb;
                if (KIND == 1)
                    *reinterpret_cast<uint32_t*>(bt + S::ATILE + S::BTILE + off) = to_tf32(v - __uint_as_float(hb));
            }
        }
        if (b + 1 < nb) prefetch(b + 1);  // in flight while block b is generated
        __syncthreads();
        if (gen) {
            float X[M], Y[M], Z[M];
#pragma unroll
            for (int q = 0; q < M; ++q) {
                X[q] = D2[(0 * M + ia) * M + q];
                Y[q] = D2[(1 * M + ib) * M + q];
                Z[q] = D2[(2 * M + ic) * M + q];
            }
            if (S::TPR == 1 || part == 0) gen_row<M, NR, KIND, 0>(stage, nu, X, Y, Z);
            else gen_row<M, NR, KIND, (S::TPR > 1 ? 1 : 0)>(stage, nu, X, Y, Z);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = smem_u32(stage);
            // consecutive MMAs go to NACC independent accumulators (step % NACC), so
            // that they do not wait on one another; the epilogue sums them
#pragma unroll
            for (int mt = 0; mt < S::MT; ++mt)
#pragma unroll
                for (int kb = 0; kb < S::NKB; ++kb)
#pragma unroll
                    for (int j = 0; j < S::SPK; ++j) {
                        const uint32_t aoff = kb * (S::MT * 8192) + mt * 8192 + j * 32;
                        const uint32_t boff = S::ATILE + kb * ((S::N / 8) * 1024) + j * 32;
#pragma unroll
                        for (int p = 0; p < S::PASSES; ++p) {
                            // TF32x3 passes: (hi, hi), (hi, lo), (lo, hi)
                            const int step = (kb * S::SPK + j) * S::PASSES + p;
                            const uint32_t asel = p == 2 ? S::ATILE + S::BTILE : 0u;
                            const uint32_t bsel = p == 1 ? S::ATILE + S::BTILE : 0u;
                            const uint64_t ad = desc_sw128(sa + asel + aoff);
                            const uint64_t bd = desc_sw128(sa + bsel + boff);
                            const uint32_t acc = (b == 0 && step < S::NACC) ? 0u : 1u;
                            const uint32_t dcol = tmem + (mt * S::NACC + step % S::NACC) * S::N;
                            if (KIND == 2)
                                asm volatile(
                                    "{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n"
                                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}" ::"r"(dcol),
                                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                            else
                                asm volatile(
                                    "{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n"
                                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}" ::"r"(dcol),
                                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                        }
                    }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[st])));
        }
        issued = b + 1;
    }
    // wait for the last block's products (they complete in issue order)
    if (issued > 0) {
        const int lb = issued - 1;
        const bool w = mbar_wait(smem_u32(&mbar[lb & 1]), (lb >> 1) & 1);
        ok = __syncthreads_and(ok && w) != 0;
    }
    if (!ok && tid == 0) atomicExch(&g_tc_status, 5);  // H2BEM_ERR_TIMEOUT
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && nb > 0) {
#pragma unroll
        for (int mt = 0; mt < S::MT; ++mt) {
#pragma unroll
            for (int c0 = 0; c0 < S::N; c0 += 8) {
                float sum[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
                for (int a = 0; a < S::NACC; ++a) {
                    uint32_t v[8];
                    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (mt * S::NACC + a) * S::N + c0;
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                                   "=r"(v[7])
                                 : "r"(ta));
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                    for (int q = 0; q < 8; ++q) sum[q] += __uint_as_float(v[q]);
                }
                const int nu_out = mt * 64 + warp * 16 + lane;
                if (lane < 16 && nu_out < S::K) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (c0 + q < NR) yh[((int64_t)row * S::K + nu_out) * NR + c0 + q] = (float)sum[q] * (float)kInv4Pi;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TMEM_COLS));
}

template <int M, int NR, int KIND>
static void tc_go(int nrows, const Tree& t, const Consts& c, const int* rows, const int* ptr, const int* col,
                  const float* xh, float* yh, int stall_test, cudaStream_t s) {
    constexpr size_t smem = TcShape<M, NR, KIND>::SMEM;
    cudaFuncSetAttribute(k_coupling_tc<M, NR, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_coupling_tc<M, NR, KIND><<<nrows, kThreads, smem, s>>>(t, c, rows, ptr, col, xh, yh, stall_test);
}

template <int M, int KIND>
static void tc_nr(int NR, int nrows, const Tree& t, const Consts& c, const int* rows, const int* ptr, const int* col,
                  const float* xh, float* yh, int st, cudaStream_t s) {
    switch (NR) {
        case 1: tc_go<M, 1, KIND>(nrows, t, c, rows, ptr, col, xh, yh, st, s); break;
        case 4: tc_go<M, 4, KIND>(nrows, t, c, rows, ptr, col, xh, yh, st, s); break;
        case 8: tc_go<M, 8, KIND>(nrows, t, c, rows, ptr, col, xh, yh, st, s); break;
        default: tc_go<M, 16, KIND>(nrows, t, c, rows, ptr, col, xh, yh, st, s); break;
    }
}

bool coupling_tc_supported(int m, int kind) { return m >= 1 && m <= (kind == 1 ? 4 : 5); }

void launch_coupling_tc(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                        int kind, int NR, const float* xh, float* yh, int stall_test, cudaStream_t s) {
    if (nrows <= 0) return;
    auto go = [&](auto mk) {
        constexpr int M = decltype(mk)::value;
        if (kind == 0) tc_nr<M, 0>(NR, nrows, t, c, rows, ptr, col, xh, yh, stall_test, s);
        else if (kind == 1) tc_nr<(M <= 4 ? M : 4), 1>(NR, nrows, t, c, rows, ptr, col, xh, yh, stall_test, s);
        else tc_nr<M, 2>(NR, nrows, t, c, rows, ptr, col, xh, yh, stall_test, s);
    };
    switch (c.m) {
        case 1: go(std::integral_constant<int, 1>{}); break;
        case 2: go(std::integral_constant<int, 2>{}); break;
        case 3: go(std::integral_constant<int, 3>{}); break;
        case 4: go(std::integral_constant<int, 4>{}); break;
        default: go(std::integral_constant<int, 5>{}); break;
    }
}

int coupling_tc_status(bool reset) {
    int v = 0;
    cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int));
    if (reset && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tc_status, &z, sizeof(int));
    }
    return v;
}

}  // namespace h2
