// Nearfield blocks, regular pairs (section 2: nearfield leaves L^-; entries
// of section 1, eq. (slp) / eq. (dlp) by the 7-point rule on each triangle).
//
// One CTA per row leaf t.  Thread (i, kk) owns row i of t and every kk-th
// column of each nearfield column leaf s; columns are staged in shared memory
// one leaf at a time (quadrature points, areas, normals, vertex ids, x).
// Pairs that share a vertex are skipped here (singular kernel).  Partial row
// sums are reduced over kk in shared memory at the end and added to yp.
//
// FP32 variant: points are stored as offsets from their triangle's centroid
// and each pair's centroid difference is formed in FP64 before rounding, so
// x_p - y_q keeps ~1e-7 relative accuracy even for touching neighbours; the
// 49-point sum runs in FP32, the entry times x is accumulated in FP64.
//
// Double layer: y_q lies in the plane of tau_j, so (x_p - y_q).n_j equals the
// height (x_p - c_j).n_j of x_p above that plane, which depends on p only.  It
// is formed once per point and pair, with the centroid part in FP64; this
// avoids the cancellation of (x_p - y_q).n_j for nearly coplanar neighbours.
// The transposed double layer uses the height (y_q - c_i).n_i of y_q above the
// plane of the row triangle in the same way.
#include <type_traits>

#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;
constexpr int kThreads = 256;
constexpr int kSbuf = 4096;  // doubles: >= staging area and >= kThreads * 16

template <typename T>
__device__ __forceinline__ T rsq(T x);
template <>
__device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }
template <>
__device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
}  // namespace

template <int NR, int KER, bool F32>
__global__ void __launch_bounds__(kThreads) k_near_regular(Geom g, Tree t, Consts c, const int* __restrict__ rows,
                                                           const int* __restrict__ ptr, const int* __restrict__ col,
                                                           const double* __restrict__ xp, double* __restrict__ yp) {
    using T = typename std::conditional<F32, float, double>::type;
    __shared__ double sbuf[kSbuf];
    __shared__ int svid[3 * kMaxLeaf];
    T* sq = reinterpret_cast<T*>(sbuf);                      // [3][kMaxLeaf * 7]
    constexpr int kQ = 3 * kMaxLeaf * 7 * sizeof(T) / sizeof(double);
    double* sctr = sbuf + kQ;                                // [3][kMaxLeaf]
    double* sarea = sctr + 3 * kMaxLeaf;                     // [kMaxLeaf]
    double* snrm = sarea + kMaxLeaf;                         // [3][kMaxLeaf]
    double* sx = snrm + 3 * kMaxLeaf;                        // [kMaxLeaf][NR]

    const int row = rows[blockIdx.x];
    const int rb = t.begin[row], R = t.end[row] - rb;
    const int K = kThreads / R;
    const int tid = threadIdx.x;
    const int il = tid % R, kk = tid / R;
    const bool active = kk < K;
    const int n = g.n;

    // row triangle i = rb + il: quadrature points (absolute or centroid offsets)
    T px[7], py[7], pz[7];
    double ci[3] = {0, 0, 0}, rn[3] = {0, 0, 0}, ai = 0;
    int vi[3] = {-1, -1, -1};
    if (active) {
        const int i = rb + il;
        double V[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) V[q] = g.v[q * n + i];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ci[d] = g.ctr[d * n + i];
            rn[d] = g.nrm[d * n + i];
            vi[d] = g.vid[d * n + i];
        }
        ai = g.area[i];
#pragma unroll
        for (int p = 0; p < 7; ++p) {
            double x0 = V[0] + c.ru[p] * (V[3] - V[0]) + c.rv[p] * (V[6] - V[0]);
            double x1 = V[1] + c.ru[p] * (V[4] - V[1]) + c.rv[p] * (V[7] - V[1]);
            double x2 = V[2] + c.ru[p] * (V[5] - V[2]) + c.rv[p] * (V[8] - V[2]);
            if (F32) {
                px[p] = (T)(x0 - ci[0]);
                py[p] = (T)(x1 - ci[1]);
                pz[p] = (T)(x2 - ci[2]);
            } else {
                px[p] = (T)x0;
                py[p] = (T)x1;
                pz[p] = (T)x2;
            }
        }
    }
    double acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0;

    for (int b = ptr[blockIdx.x]; b < ptr[blockIdx.x + 1]; ++b) {
        const int s = col[b];
        const int cb = t.begin[s], C = t.end[s] - cb;
        __syncthreads();
        for (int e = tid; e < C * 7; e += kThreads) {
            const int j = cb + e / 7, q = e % 7;
            double y[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                double v0 = g.v[d * n + j], v1 = g.v[(3 + d) * n + j], v2 = g.v[(6 + d) * n + j];
                y[d] = v0 + c.ru[q] * (v1 - v0) + c.rv[q] * (v2 - v0);
                if (F32) y[d] -= g.ctr[d * n + j];
                sq[d * (kMaxLeaf * 7) + e] = (T)y[d];
            }
        }
        for (int e = tid; e < C; e += kThreads) {
            const int j = cb + e;
            sarea[e] = g.area[j];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                sctr[d * kMaxLeaf + e] = g.ctr[d * n + j];
                snrm[d * kMaxLeaf + e] = g.nrm[d * n + j];
                svid[d * kMaxLeaf + e] = g.vid[d * n + j];
            }
        }
        for (int e = tid; e < C * NR; e += kThreads) sx[e] = xp[(int64_t)cb * NR + e];
        __syncthreads();
        if (!active) continue;
        for (int jl = kk; jl < C; jl += K) {
            bool sing = false;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int bb = 0; bb < 3; ++bb) sing |= (vi[a] == svid[bb * kMaxLeaf + jl]);
            if (sing) continue;
            T Dx = 0, Dy = 0, Dz = 0;
            if (F32) {
                Dx = (T)(ci[0] - sctr[jl]);
                Dy = (T)(ci[1] - sctr[kMaxLeaf + jl]);
                Dz = (T)(ci[2] - sctr[2 * kMaxLeaf + jl]);
            }
            // double layer: heights above the plane carrying the normal
            T hp[7];
            if (KER == DLP) {
                const double nx = snrm[jl], ny = snrm[kMaxLeaf + jl], nz = snrm[2 * kMaxLeaf + jl];
                const double cx = sctr[jl], cy = sctr[kMaxLeaf + jl], cz = sctr[2 * kMaxLeaf + jl];
                if (F32) {
                    const T H0 = (T)((ci[0] - cx) * nx + (ci[1] - cy) * ny + (ci[2] - cz) * nz);
#pragma unroll
                    for (int p = 0; p < 7; ++p) hp[p] = H0 + (px[p] * (T)nx + py[p] * (T)ny + pz[p] * (T)nz);
                } else {
#pragma unroll
                    for (int p = 0; p < 7; ++p)
                        hp[p] = ((double)px[p] - cx) * nx + ((double)py[p] - cy) * ny + ((double)pz[p] - cz) * nz;
                }
            }
            T sum = 0;
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                const T ex = sq[jl * 7 + q], ey = sq[kMaxLeaf * 7 + jl * 7 + q], ez = sq[2 * kMaxLeaf * 7 + jl * 7 + q];
                const T yx = F32 ? Dx - ex : ex, yy = F32 ? Dy - ey : ey, yz = F32 ? Dz - ez : ez;
                T hq = 0;
                if (KER == DLP_T) {
                    if (F32) {
                        const T H0 = (T)((sctr[jl] - ci[0]) * rn[0] + (sctr[kMaxLeaf + jl] - ci[1]) * rn[1] +
                                         (sctr[2 * kMaxLeaf + jl] - ci[2]) * rn[2]);
                        hq = H0 + (ex * (T)rn[0] + ey * (T)rn[1] + ez * (T)rn[2]);
                    } else {
                        hq = ((double)ex - ci[0]) * rn[0] + ((double)ey - ci[1]) * rn[1] + ((double)ez - ci[2]) * rn[2];
                    }
                }
                T sp = 0;
#pragma unroll
                for (int p = 0; p < 7; ++p) {
                    // F32: d = (x_p - c_i) + (c_i - c_j) - (y_q - c_j);  F64: d = x_p - y_q
                    const T dx = F32 ? px[p] + yx : px[p] - yx;
                    const T dy = F32 ? py[p] + yy : py[p] - yy;
                    const T dz = F32 ? pz[p] + yz : pz[p] - yz;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    const T ri = rsq<T>(r2);
                    if (KER == SLP) {
                        sp += (T)c.rw[p] * ri;
                    } else {
                        const T h = KER == DLP ? hp[p] : hq;
                        sp += (T)c.rw[p] * h * (ri * ri * ri);
                    }
                }
                sum += (T)c.rw[q] * sp;
            }
            const double a = ai * sarea[jl] * (double)sum * kInv4Pi;
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] += a * sx[jl * NR + r];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; ++r) sbuf[tid * NR + r] = active ? acc[r] : 0.0;
    __syncthreads();
    for (int e = tid; e < R * NR; e += kThreads) {
        const int i = e / NR, r = e % NR;
        double s = 0.0;
        for (int q = 0; q < K; ++q) s += sbuf[(q * R + i) * NR + r];
        yp[(int64_t)(rb + i) * NR + r] += s;
    }
}

template <int NR, bool F32>
static void near_dispatch_ker(int ker, dim3 grid, cudaStream_t s, const Geom& g, const Tree& t, const Consts& c,
                              const int* rows, const int* ptr, const int* col, const double* xp, double* yp) {
    if (ker == SLP) k_near_regular<NR, SLP, F32><<<grid, kThreads, 0, s>>>(g, t, c, rows, ptr, col, xp, yp);
    else if (ker == DLP) k_near_regular<NR, DLP, F32><<<grid, kThreads, 0, s>>>(g, t, c, rows, ptr, col, xp, yp);
    else k_near_regular<NR, DLP_T, F32><<<grid, kThreads, 0, s>>>(g, t, c, rows, ptr, col, xp, yp);
}

template <bool F32>
static void near_dispatch(int NR, int ker, dim3 grid, cudaStream_t s, const Geom& g, const Tree& t,
                          const Consts& c, const int* rows, const int* ptr, const int* col, const double* xp,
                          double* yp) {
    switch (NR) {
        case 1: near_dispatch_ker<1, F32>(ker, grid, s, g, t, c, rows, ptr, col, xp, yp); break;
        case 4: near_dispatch_ker<4, F32>(ker, grid, s, g, t, c, rows, ptr, col, xp, yp); break;
        case 8: near_dispatch_ker<8, F32>(ker, grid, s, g, t, c, rows, ptr, col, xp, yp); break;
        default: near_dispatch_ker<16, F32>(ker, grid, s, g, t, c, rows, ptr, col, xp, yp); break;
    }
}

void launch_near_regular(const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                         const int* col, int ker, bool fp32, int NR, const double* xp, double* yp, cudaStream_t s) {
    if (nrows <= 0) return;
    dim3 grid(nrows);
    if (fp32) near_dispatch<true>(NR, ker, grid, s, g, t, c, rows, ptr, col, xp, yp);
    else near_dispatch<false>(NR, ker, grid, s, g, t, c, rows, ptr, col, xp, yp);
}

}  // namespace h2
