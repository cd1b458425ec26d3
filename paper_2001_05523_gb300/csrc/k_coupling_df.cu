// Coupling stage of the FP64 tier's single layer, and of the double layer's
// FP64 side in the mixed tiers (section 2, eq. (vsw); section 3,
// S_ts[nu,mu] = g(xi_{t,nu}, xi_{s,mu})), by double-float arithmetic on the
// FP32 pipe:
//   yh_t[nu] = sum_{(t,s) farfield} sum_mu S_ts[nu,mu] xh_s[mu].
// GB300 issues FP64 at about 1/74 of its FP32 rate, and the FP64 generation
// and products (about 14 FP64 operations per entry at 8 right-hand sides)
// bound this stage.  Here, per block, the squared node differences along each
// axis (FP64) and the staged x-hat values are split into float pairs hi + lo;
// per entry the squared distance is a float-pair sum, 1/r the hardware
// reciprocal square root with one Newton step formed from the pairs (relative
// error about (3/8) e^2 with e < 2^-22), and every product S x-hat is a float
// pair (FMA residuals) accumulated with Knuth's TwoSum.  The per-thread sums
// are converted to FP64 once per row cluster.  Work layout as the SIMT
// kernel's register-blocked variant: thread (row, slice) owns the m target
// nodes nu = (a, b, c), a = 0..m-1, of one (b, c) row and the mu-rows
// (jc, jb) of its slice; slices are reduced in shared memory (FP64).  TX / TY:
// storage of x-hat / y-hat (double, or float on the side of a mixed-tier
// double layer that is not FP64).
#include <algorithm>

#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4PiC = 0.07957747154594766788;

__device__ __forceinline__ void tsum2(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
}  // namespace

template <typename TX, typename TY, int NR, int M, int NSL>
__global__ void __launch_bounds__(M * M * NSL) k_coupling_df(Tree t, Consts c, const int* __restrict__ rows,
                                                             const int* __restrict__ ptr, const int* __restrict__ col,
                                                             const TX* __restrict__ xh, TY* __restrict__ yh) {
    constexpr int K = M * M * M, M2 = M * M, NT = M2 * NSL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* xd = reinterpret_cast<double*>(smem_raw);                    // [K][NR] x-hat of the block; reduction [NSL][K][NR]
    float* xsh = reinterpret_cast<float*>(smem_raw + 8 * (size_t)K * NR);  // [K][NR] hi
    float* xsl = xsh + K * NR;                                             // [K][NR] lo
    __shared__ double zt[3 * M], zs[3 * M];
    __shared__ float D2h[3 * M2], D2l[3 * M2];
    const int row = rows[blockIdx.x];
    const int rg = threadIdx.x % M2, sl = threadIdx.x / M2;
    const int ib = rg % M, ic = rg / M;
    for (int e = threadIdx.x; e < 3 * M; e += NT) {
        const int d = e / M, a = e % M;
        zt[e] = t.box[d * t.nc + row] + t.box[(3 + d) * t.nc + row] * c.cheb[a];
    }
    float ah[M][NR], al[M][NR];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int r = 0; r < NR; ++r) ah[a][r] = al[a][r] = 0.0f;

    for (int b = ptr[blockIdx.x]; b < ptr[blockIdx.x + 1]; ++b) {
        const int s = col[b];
        __syncthreads();  // the previous block is done with shared memory
        for (int e = threadIdx.x; e < 3 * M; e += NT) {
            const int d = e / M, a = e % M;
            zs[e] = t.box[d * t.nc + s] + t.box[(3 + d) * t.nc + s] * c.cheb[a];
        }
        for (int e = threadIdx.x; e < K * NR; e += NT) {
            const double v = (double)xh[(int64_t)s * K * NR + e];
            const float h = (float)v;
            xsh[e] = h;
            xsl[e] = (float)(v - (double)h);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 3 * M2; e += NT) {
            const int d = e / M2, a = (e / M) % M, a2 = e % M;
            const double df = zt[d * M + a] - zs[d * M + a2];
            const double q = df * df;
            const float h = (float)q;
            D2h[e] = h;
            D2l[e] = (float)(q - (double)h);
        }
        __syncthreads();
        float dxh[M][M], dxl[M][M];
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int ja = 0; ja < M; ++ja) {
                dxh[a][ja] = D2h[a * M + ja];
                dxl[a][ja] = D2l[a * M + ja];
            }
        for (int r2 = sl; r2 < M2; r2 += NSL) {
            const int jc = r2 / M, jb = r2 % M;
            // the y and z parts of the squared distance for this (b, c) row and (jb, jc)
            float sbh, sbe;
            tsum2(D2h[M2 + ib * M + jb], D2h[2 * M2 + ic * M + jc], sbh, sbe);
            const float sbl = __fadd_rn(__fadd_rn(D2l[M2 + ib * M + jb], D2l[2 * M2 + ic * M + jc]), sbe);
#pragma unroll
            for (int ja = 0; ja < M; ++ja) {
                const int mu = ja + M * r2;
                float xvh[NR], xvl[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    xvh[r] = xsh[mu * NR + r];
                    xvl[r] = xsl[mu * NR + r];
                }
#pragma unroll
                for (int a = 0; a < M; ++a) {
                    float Rh, e0;
                    tsum2(dxh[a][ja], sbh, Rh, e0);
                    const float Rl = __fadd_rn(__fadd_rn(dxl[a][ja], sbl), e0);
                    float y0;
                    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(Rh));
                    const float y2 = __fmul_rn(y0, y0);
                    const float y2e = __fmaf_rn(y0, y0, -y2);
                    const float tq = __fmaf_rn(-Rh, y2, 1.0f);
                    const float ep = __fsub_rn(tq, __fmaf_rn(Rh, y2e, __fmul_rn(Rl, y2)));
                    const float yc = __fmul_rn(__fmul_rn(0.5f, y0), ep);  // S = y0 + yc
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const float ph = __fmul_rn(y0, xvh[r]);
                        const float pl = __fmaf_rn(y0, xvl[r], __fmaf_rn(yc, xvh[r], __fmaf_rn(y0, xvh[r], -ph)));
                        float e1;
                        tsum2(ah[a][r], ph, ah[a][r], e1);
                        al[a][r] = __fadd_rn(al[a][r], __fadd_rn(e1, pl));
                    }
                }
            }
        }
    }
    __syncthreads();
    // reduction over slices in FP64: slot [sl][nu][r], nu = a + M * rg
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int r = 0; r < NR; ++r) xd[((size_t)sl * K + a + M * rg) * NR + r] = (double)ah[a][r] + (double)al[a][r];
    __syncthreads();
    for (int e = threadIdx.x; e < K * NR; e += NT) {
        double sum = 0.0;
        for (int q = 0; q < NSL; ++q) sum += xd[(size_t)q * K * NR + e];
        yh[(int64_t)row * K * NR + e] = (TY)(sum * kInv4PiC);
    }
}

bool coupling_df_supported(int m, int NR) { return (m == 4 || m == 5) && NR <= 8; }

template <typename TX, typename TY>
static void coupling_df_go(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                           int NR, const void* xh, void* yh, cudaStream_t s) {
    auto go = [&](auto kern, int M, int nsl) {
        const int K = M * M * M;
        // x-hat as float pairs behind the reduction area [NSL][K][NR] (double), which reuses the front
        const size_t smem = std::max((size_t)(8 + 8) * K * NR, (size_t)8 * nsl * K * NR);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<nrows, M * M * nsl, smem, s>>>(t, c, rows, ptr, col, (const TX*)xh, (TY*)yh);
    };
    if (c.m == 4) {
        if (NR == 1) go(k_coupling_df<TX, TY, 1, 4, 4>, 4, 4);
        else if (NR == 4) go(k_coupling_df<TX, TY, 4, 4, 4>, 4, 4);
        else go(k_coupling_df<TX, TY, 8, 4, 4>, 4, 4);
    } else {
        if (NR == 1) go(k_coupling_df<TX, TY, 1, 5, 4>, 5, 4);
        else if (NR == 4) go(k_coupling_df<TX, TY, 4, 5, 4>, 5, 4);
        else go(k_coupling_df<TX, TY, 8, 5, 4>, 5, 4);
    }
}

void launch_coupling_df(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                        int NR, bool xh64, bool yh64, const void* xh, void* yh, cudaStream_t s) {
    if (nrows <= 0) return;
    if (xh64 && yh64) coupling_df_go<double, double>(t, c, nrows, rows, ptr, col, NR, xh, yh, s);
    else if (xh64) coupling_df_go<double, float>(t, c, nrows, rows, ptr, col, NR, xh, yh, s);
    else if (yh64) coupling_df_go<float, double>(t, c, nrows, rows, ptr, col, NR, xh, yh, s);
    else coupling_df_go<float, float>(t, c, nrows, rows, ptr, col, NR, xh, yh, s);
}

}  // namespace h2
