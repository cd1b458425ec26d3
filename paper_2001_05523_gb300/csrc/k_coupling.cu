// Coupling stage of the H^2 product (section 2, eq. (vsw); section 3,
// S_ts[nu,mu] = g(xi_{t,nu}, xi_{s,mu}) of the tensor Chebyshev interpolant):
//   yh_t[nu] = sum_{(t,s) farfield} sum_mu S_ts[nu,mu] xh_s[mu],
// with S_ts generated on the fly; SIMT kernels in FP64 or FP32.
#include <algorithm>
#include <type_traits>

#include "dmath.cuh"
#include "f32x2.cuh"
#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;

template <typename T>
__device__ __forceinline__ T rsq(T x);
template <>
__device__ __forceinline__ double rsq<double>(double x) { return rsqrt_nr(x); }
// FP32: the hardware reciprocal square root alone (PTX rsqrt.approx.ftz.f32,
// ~2^-22.9 relative error); the squared distances between interpolation nodes
// of admissible clusters are far from the subnormal range, so flushing them
// changes nothing, and the range handling of a non-flushing rsqrt would add
// instructions to every entry
template <>
__device__ __forceinline__ float rsq<float>(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// nodes of cluster cl along every axis: z[d*m + a]
__device__ __forceinline__ void cluster_nodes(const Tree& t, const Consts& c, int cl, double* z) {
    for (int e = threadIdx.x; e < 3 * c.m; e += blockDim.x) {
        const int d = e / c.m, a = e % c.m;
        z[e] = t.box[d * t.nc + cl] + t.box[(3 + d) * t.nc + cl] * c.cheb[a];
    }
}
}  // namespace

#define H2_NR_SWITCH(NR, CALL)                         \
    switch (NR) {                                      \
        case 1: { constexpr int R_ = 1; CALL; } break;  \
        case 4: { constexpr int R_ = 4; CALL; } break;  \
        case 8: { constexpr int R_ = 8; CALL; } break;  \
        default: { constexpr int R_ = 16; CALL; } break; \
    }

// ---------------------------------------------------------------------------
// Coupling, SIMT: one CTA per row cluster, S_ts generated on the fly from
// per-axis squared node differences.  Thread (nu, slice) sums over the mu of
// its slice; slices are reduced in shared memory at the end.
// TS: precision of the S entries; TA: accumulation (and staged x-hat);
// TX / TY: storage of x-hat / y-hat.
// ---------------------------------------------------------------------------
template <typename TS, typename TA, typename TX, typename TY, int NR, int M>
__global__ void __launch_bounds__(256) k_coupling_simt(Tree t, Consts c, const int* __restrict__ rows,
                                                       const int* __restrict__ ptr, const int* __restrict__ col,
                                                       const TX* __restrict__ xh, TY* __restrict__ yh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA* xs = reinterpret_cast<TA*>(smem_raw);  // [k][NR], reused for the reduction [256][NR]
    __shared__ double zt[3 * kMaxM], zs[3 * kMaxM];
    __shared__ TS D2[3 * kMaxM * kMaxM];       // D2[d][a][a2] = (z_t,d[a] - z_s,d[a2])^2
    const int row = rows[blockIdx.x];
    const int m = M > 0 ? M : c.m, k = m * m * m;
    const int nslice = blockDim.x / k;
    const int nu = threadIdx.x % k, sl = threadIdx.x / k;
    const bool active = sl < nslice;
    const int ia = nu % m, ib = (nu / m) % m, ic = nu / (m * m);
    cluster_nodes(t, c, row, zt);
    TA acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0;
    for (int b = ptr[blockIdx.x]; b < ptr[blockIdx.x + 1]; ++b) {
        const int s = col[b];
        __syncthreads();
        cluster_nodes(t, c, s, zs);
        for (int e = threadIdx.x; e < k * NR; e += blockDim.x) xs[e] = (TA)xh[(int64_t)s * k * NR + e];
        __syncthreads();
        for (int e = threadIdx.x; e < 3 * m * m; e += blockDim.x) {
            const int d = e / (m * m), a = (e / m) % m, a2 = e % m;
            const double df = zt[d * m + a] - zs[d * m + a2];
            D2[e] = (TS)(df * df);
        }
        __syncthreads();
        if (active) {
            const TS* Dx = D2 + ia * m;
            const TS* Dy = D2 + m * m + ib * m;
            const TS* Dz = D2 + 2 * m * m + ic * m;
            TS dxr[M > 0 ? M : kMaxM];
#pragma unroll
            for (int ja = 0; ja < (M > 0 ? M : kMaxM); ++ja) dxr[ja] = (M > 0 || ja < m) ? Dx[ja] : (TS)0;
            for (int jc = sl; jc < m; jc += nslice) {
                const TS szc = Dz[jc];
#pragma unroll(M > 0 ? M : 1)
                for (int jb = 0; jb < m; ++jb) {
                    const TS sbc = Dy[jb] + szc;
                    const TA* xrow = xs + ((jc * m + jb) * m) * NR;
#pragma unroll
                    for (int ja = 0; ja < (M > 0 ? M : kMaxM); ++ja) {
                        if (M == 0 && ja >= m) break;
                        const TA sv = (TA)rsq<TS>(dxr[ja] + sbc);
#pragma unroll
                        for (int r = 0; r < NR; ++r) acc[r] += sv * xrow[ja * NR + r];
                    }
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; ++r) xs[threadIdx.x * NR + r] = active ? acc[r] : (TA)0;
    __syncthreads();
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) {
        const int v = e / NR, r = e % NR;
        TA s = 0;
        for (int q = 0; q < nslice; ++q) s += xs[(q * k + v) * NR + r];
        yh[(int64_t)row * k * NR + e] = (TY)(s * (TA)kInv4Pi);
    }
}

// Register-blocked variant for compile-time m: thread (row, slice) owns the
// m target nodes nu = (a, b, c), a = 0..m-1, of one (b, c) row and the mu-rows
// (jc, jb) of its slice; every x-hat value loaded from shared memory feeds m
// entries.  Slices are reduced in shared memory at the end.  NSL slices per
// CTA (blockDim = NSL m^2): a tile shape the autotuner chooses.
template <typename TS, typename TA, typename TX, typename TY, int NR, int M, int NSL>
__device__ __forceinline__ void coupling_row(const Tree& t, const Consts& c, const int* __restrict__ rows,
                                             const int* __restrict__ ptr, const int* __restrict__ col,
                                             const TX* __restrict__ xh, TY* __restrict__ yh, int bi) {
    constexpr int K = M * M * M, M2 = M * M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA* xs = reinterpret_cast<TA*>(smem_raw);  // [K][NR]; reused for the reduction [NSL][K][NR]
    // node coordinates: FP64, or for FP32 entries (hi, lo) splits whose
    // differences keep ~1e-7 relative accuracy without the FP64 pipe
    constexpr bool F32N = std::is_same<TS, float>::value;
    __shared__ double zt[3 * M], zs[3 * M];
    __shared__ float2 zt2[3 * M], zs2[3 * M];
    __shared__ TS D2[3 * M2];
    const int row = rows[bi];
    const int rg = threadIdx.x % M2, sl = threadIdx.x / M2;
    const bool active = sl < NSL;
    const int ib = rg % M, ic = rg / M;
    if constexpr (F32N) {
        for (int e = threadIdx.x; e < 3 * M; e += blockDim.x) zt2[e] = t.zhl[(int64_t)row * 3 * M + e];
    } else {
        cluster_nodes(t, c, row, zt);
    }
    // FP32 entries and sums with an even number of right-hand sides: the sums
    // as packed pairs (one f32x2 multiply-add for two right-hand sides)
    constexpr bool PK = std::is_same<TA, float>::value && std::is_same<TS, float>::value && NR % 2 == 0;
    constexpr int NA = PK ? 1 : NR, NP = PK ? NR / 2 : 1;
    TA acc[M][NA];
    f2 acc2[M][NP];
#pragma unroll
    for (int a = 0; a < M; ++a) {
#pragma unroll
        for (int r = 0; r < NA; ++r) acc[a][r] = 0;
#pragma unroll
        for (int q = 0; q < NP; ++q) acc2[a][q] = 0;
    }
    // register prefetch of the next block's x-hat values and column nodes, so
    // that their global-memory latency overlaps the current block's work
    constexpr int NT = M2 * NSL;
    static_assert(3 * M <= NT, "one column node per thread");
    // x-hat of the next block: asynchronous 16-byte copies into the other half
    // of a double buffer (same type in global and shared memory), else a
    // register prefetch with conversion
    constexpr bool ASYNC = std::is_same<TX, TA>::value && (K * NR * sizeof(TA)) % 16 == 0;
    constexpr int PF = ASYNC ? 1 : (K * NR + NT - 1) / NT;
    TX xpre[PF];
    double zpre = 0.0;
    float2 zpre2 = make_float2(0.0f, 0.0f);
    auto prefetch = [&](int b, TA* dst) {
        const int s = col[b];
        if constexpr (ASYNC) {
            const char* src = reinterpret_cast<const char*>(xh + (int64_t)s * K * NR);
            const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(dst);
            for (int e = threadIdx.x; e < (int)(K * NR * sizeof(TA) / 16); e += NT)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + 16 * e), "l"(src + 16 * e)
                             : "memory");
            asm volatile("cp.async.commit_group;" ::: "memory");
        } else {
#pragma unroll
            for (int j = 0; j < PF; ++j) {
                const int e = threadIdx.x + j * NT;
                xpre[j] = e < K * NR ? xh[(int64_t)s * K * NR + e] : (TX)0;
            }
        }
        if (threadIdx.x < 3 * M) {
            if constexpr (F32N) {
                zpre2 = t.zhl[(int64_t)s * 3 * M + threadIdx.x];
            } else {
                const int d = threadIdx.x / M, a = threadIdx.x % M;
                zpre = t.box[d * t.nc + s] + t.box[(3 + d) * t.nc + s] * c.cheb[a];
            }
        }
    };
    const int bbeg = ptr[bi], bend = ptr[bi + 1];
    if (bbeg < bend) prefetch(bbeg, xs);
    for (int b = bbeg; b < bend; ++b) {
        TA* xcur = xs + (ASYNC ? ((b - bbeg) & 1) * K * NR : 0);
        __syncthreads();  // the previous block is done with shared memory
        if constexpr (!ASYNC) {
#pragma unroll
            for (int j = 0; j < PF; ++j) {
                const int e = threadIdx.x + j * NT;
                if (e < K * NR) xcur[e] = (TA)xpre[j];
            }
        }
        if (threadIdx.x < 3 * M) {
            if constexpr (F32N) zs2[threadIdx.x] = zpre2;
            else zs[threadIdx.x] = zpre;
        }
        if (b + 1 < bend) prefetch(b + 1, xs + (ASYNC ? ((b + 1 - bbeg) & 1) * K * NR : 0));
        if constexpr (ASYNC) {
            if (b + 1 < bend) asm volatile("cp.async.wait_group 1;" ::: "memory");
            else asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 3 * M2; e += blockDim.x) {
            const int d = e / M2, a = (e / M) % M, a2 = e % M;
            if constexpr (F32N) {
                const float2 u = zt2[d * M + a], v = zs2[d * M + a2];
                const float df = (u.x - v.x) + (u.y - v.y);
                D2[e] = df * df;
            } else {
                const double df = zt[d * M + a] - zs[d * M + a2];
                D2[e] = (TS)(df * df);
            }
        }
        __syncthreads();
        if (!active) continue;
        TS dx[M][M];
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int ja = 0; ja < M; ++ja) dx[a][ja] = D2[a * M + ja];
        for (int r2 = sl; r2 < M2; r2 += NSL) {
            const int jc = r2 / M, jb = r2 % M;
            const TS sbc = D2[M2 + ib * M + jb] + D2[2 * M2 + ic * M + jc];
            const TA* xrow = xcur + (r2 * M) * NR;
#pragma unroll
            for (int ja = 0; ja < M; ++ja) {
                if constexpr (PK) {
                    f2 xv2[NP];
                    const f2* xr2 = reinterpret_cast<const f2*>(xrow + ja * NR);
#pragma unroll
                    for (int q = 0; q < NP; ++q) xv2[q] = xr2[q];
#pragma unroll
                    for (int a = 0; a < M; ++a) {
                        const float sv = rsq<float>(dx[a][ja] + sbc);
                        const f2 s2 = pk(sv, sv);
#pragma unroll
                        for (int q = 0; q < NP; ++q) acc2[a][q] = fma2(s2, xv2[q], acc2[a][q]);
                    }
                } else {
                    TA xv[NR];
#pragma unroll
                    for (int r = 0; r < NR; ++r) xv[r] = xrow[ja * NR + r];
#pragma unroll
                    for (int a = 0; a < M; ++a) {
                        const TA sv = (TA)rsq<TS>(dx[a][ja] + sbc);
#pragma unroll
                        for (int r = 0; r < NR; ++r) acc[a][r] += sv * xv[r];
                    }
                }
            }
        }
    }
    __syncthreads();
    // reduction over slices: slot [sl][nu][r], nu = a + M * rg
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            TA v;
            if constexpr (PK) {
                float lo, hi;
                upk(acc2[a][r / 2], lo, hi);
                v = (r & 1) ? hi : lo;
            } else {
                v = acc[a][r];
            }
            if (active) xs[((size_t)sl * K + a + M * rg) * NR + r] = v;
        }
    __syncthreads();
    for (int e = threadIdx.x; e < K * NR; e += blockDim.x) {
        TA s = 0;
        for (int q = 0; q < NSL; ++q) s += xs[(size_t)q * K * NR + e];
        yh[(int64_t)row * K * NR + e] = (TY)(s * (TA)kInv4Pi);
    }
}

// One CTA per row cluster (work == nullptr), or persistent CTAs that take the
// next row from the counter *work (zero before the launch) until none is left.
template <typename TS, typename TA, typename TX, typename TY, int NR, int M, int NSL, bool PERSIST>
__global__ void __launch_bounds__(M * M * NSL)
    k_coupling_rows(Tree t, Consts c, int nrows, const int* __restrict__ rows, const int* __restrict__ ptr,
                    const int* __restrict__ col, const TX* __restrict__ xh, TY* __restrict__ yh, int* __restrict__ work) {
    if constexpr (!PERSIST) {
        coupling_row<TS, TA, TX, TY, NR, M, NSL>(t, c, rows, ptr, col, xh, yh, blockIdx.x);
        return;
    }
    __shared__ int s_bi;
    while (true) {
        __syncthreads();  // the previous row is done with shared memory and s_bi
        if (threadIdx.x == 0) s_bi = atomicAdd(work, 1);
        __syncthreads();
        const int bi = s_bi;
        if (bi >= nrows) break;
        coupling_row<TS, TA, TX, TY, NR, M, NSL>(t, c, rows, ptr, col, xh, yh, bi);
    }
}

template <typename TS, typename TA, typename TX, typename TY, int NR, int M, int NSL>
static void coupling_rows_nsl(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                              const int* col, const void* xh, void* yh, int* work, cudaStream_t s) {
    constexpr int K = M * M * M;
    const size_t smem = sizeof(TA) * (size_t)(NSL > 2 ? NSL : 2) * K * NR;  // reduction area, or two x-hat tiles
    if (!work) {
        auto kern = k_coupling_rows<TS, TA, TX, TY, NR, M, NSL, false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<nrows, M * M * NSL, smem, s>>>(t, c, nrows, rows, ptr, col, (const TX*)xh, (TY*)yh, nullptr);
        return;
    }
    auto kern = k_coupling_rows<TS, TA, TX, TY, NR, M, NSL, true>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = std::min(nrows, resident_ctas((const void*)kern, M * M * NSL, smem));
    cudaMemsetAsync(work, 0, sizeof(int), s);
    kern<<<grid, M * M * NSL, smem, s>>>(t, c, nrows, rows, ptr, col, (const TX*)xh, (TY*)yh, work);
}

template <typename TS, typename TA, typename TX, typename TY, int NR, int M>
static void coupling_rows(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                          const void* xh, void* yh, const LaunchCfg& cfg, cudaStream_t s) {
    if (cfg.nsl == 2) coupling_rows_nsl<TS, TA, TX, TY, NR, M, 2>(t, c, nrows, rows, ptr, col, xh, yh, cfg.work, s);
    else if (cfg.nsl == 8) coupling_rows_nsl<TS, TA, TX, TY, NR, M, 8>(t, c, nrows, rows, ptr, col, xh, yh, cfg.work, s);
    else coupling_rows_nsl<TS, TA, TX, TY, NR, M, 4>(t, c, nrows, rows, ptr, col, xh, yh, cfg.work, s);
}

template <typename TS, typename TA, typename TX, typename TY, int NR, int M>
static void coupling_m(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                       const void* xh, void* yh, cudaStream_t s) {
    const size_t smem = sizeof(TA) * (size_t)(256 > c.k ? 256 : c.k) * NR;
    cudaFuncSetAttribute(k_coupling_simt<TS, TA, TX, TY, NR, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_coupling_simt<TS, TA, TX, TY, NR, M><<<nrows, 256, smem, s>>>(t, c, rows, ptr, col, (const TX*)xh, (TY*)yh);
}

template <typename TS, typename TA, typename TX, typename TY, int NR>
static void coupling_simt(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                          const void* xh, void* yh, const LaunchCfg& cfg, cudaStream_t s) {
    if (c.m == 4) coupling_rows<TS, TA, TX, TY, NR, 4>(t, c, nrows, rows, ptr, col, xh, yh, cfg, s);
    else if (c.m == 5) coupling_rows<TS, TA, TX, TY, NR, 5>(t, c, nrows, rows, ptr, col, xh, yh, cfg, s);
    else coupling_m<TS, TA, TX, TY, NR, 0>(t, c, nrows, rows, ptr, col, xh, yh, s);
}

void launch_coupling(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                     int precision, bool xh64, bool yh64, int NR, const void* xh, void* yh, const LaunchCfg& cfg,
                     cudaStream_t s) {
    if (nrows <= 0) return;
    if (precision == 0) {
        H2_NR_SWITCH(NR, (coupling_simt<double, double, double, double, R_>(t, c, nrows, rows, ptr, col, xh, yh, cfg, s)))
    } else if (xh64) {
        // input side in double (double layer, K x): the differentiated basis makes
        // S x-hat cancel strongly, so S and its sums are FP64; y-hat is stored float
        H2_NR_SWITCH(NR, (coupling_simt<double, double, double, float, R_>(t, c, nrows, rows, ptr, col, xh, yh, cfg, s)))
    } else if (yh64) {
        // output side in double (double layer, K^T x): W_t y-hat_t is the normal
        // derivative of a potential that varies along the surface, so on flat
        // faces it cancels to a small fraction of its terms and amplifies the
        // ~1e-7 error of FP32 entries; S and its sums are FP64 as for K x
        H2_NR_SWITCH(NR, (coupling_simt<double, double, float, double, R_>(t, c, nrows, rows, ptr, col, xh, yh, cfg, s)))
    } else {
        H2_NR_SWITCH(NR, (coupling_simt<float, float, float, float, R_>(t, c, nrows, rows, ptr, col, xh, yh, cfg, s)))
    }
}

}  // namespace h2
