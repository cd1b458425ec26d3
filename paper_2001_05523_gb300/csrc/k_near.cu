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
// 49-point sum, the entry and the thread's row sums run in FP32; the
// partial row sums of a CTA are combined in FP64.
//
// Double layer: y_q lies in the plane of tau_j, so (x_p - y_q).n_j equals the
// height (x_p - c_j).n_j of x_p above that plane, which depends on p only.  It
// is formed once per point and pair, with the centroid part in FP64; this
// avoids the cancellation of (x_p - y_q).n_j for nearly coplanar neighbours.
// The transposed double layer uses the height (y_q - c_i).n_i of y_q above the
// plane of the row triangle in the same way.
#include <type_traits>

#include "dmath.cuh"
#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;
constexpr int kThreads = 256;
constexpr int kSbuf = 4096;  // doubles: >= staging area and >= kThreads * 16

template <typename T>
__device__ __forceinline__ T rsq(T x);
template <>
__device__ __forceinline__ double rsq<double>(double x) { return rsqrt_nr(x); }
template <>
__device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
}  // namespace

// FP32 tier: no FP64 work per single-layer pair.  Centroids are kept as
// float pairs hi + lo (hi = fl(c), lo = fl(c - hi)); c_i - c_j is formed as
// (hi_i - hi_j) + (lo_i - lo_j), where the first difference is exact for
// nearby points (Sterbenz) and the result keeps ~1e-7 relative accuracy.
// Entries and row sums run in FP32 per thread; the slices of a row are
// reduced in FP64.  The double layer forms the plane height of the row
// centroid and the edge projections in FP64 once per pair (see below).
//
// Double-layer heights: with x_p = c_i + (u_p - 1/3) E1 + (v_p - 1/3) E2
// (E1, E2 the edge vectors of tau_i from its first corner),
//   (x_p - y_q) . n_j = (c_i - c_j) . n_j + (u_p - 1/3) E1 . n_j + (v_p - 1/3) E2 . n_j.
// For nearly coplanar neighbours every term is small against |E|, so the
// three dot products are formed in FP64 (a rounded FP32 normal alone would
// tilt the plane by 6e-8 and spoil heights of size |c_i - c_j|^2 curvature);
// only their combination per point runs in FP32.
template <int NR, int KER, bool F32>
__global__ void __launch_bounds__(kThreads) k_near_regular(Geom g, Tree t, Consts c, const int* __restrict__ rows,
                                                           const int* __restrict__ ptr, const int* __restrict__ col,
                                                           const double* __restrict__ xp, double* __restrict__ yp) {
    using T = typename std::conditional<F32, float, double>::type;
    __shared__ double sbuf[kSbuf];
    __shared__ int svid[3 * kMaxLeaf];
    __shared__ double splane[kMaxLeaf];                    // c_j . n_j (double layer)
    __shared__ double sn64[KER == SLP ? 1 : 3 * kMaxLeaf];   // n_j in FP64 (double layer)
    __shared__ double sedge[KER == DLP_T ? 6 * kMaxLeaf : 1];  // E1_j, E2_j in FP64 (transposed double layer)
    T* sq = reinterpret_cast<T*>(sbuf);                    // [3][kMaxLeaf*7]: F32 y_q - c_j, F64 y_q
    T* sch = sq + 3 * kMaxLeaf * 7;                        // [3][kMaxLeaf] centroid hi (F32) or centroid (F64)
    T* scl = sch + 3 * kMaxLeaf;                           // [3][kMaxLeaf] centroid lo (F32)
    T* sarea = scl + 3 * kMaxLeaf;                         // [kMaxLeaf]
    T* snrm = sarea + kMaxLeaf;                            // [3][kMaxLeaf]
    T* sx = snrm + 3 * kMaxLeaf;                           // [kMaxLeaf][NR]

    const int row = rows[blockIdx.x];
    const int rb = t.begin[row], R = t.end[row] - rb;
    const int K = kThreads / R;
    const int tid = threadIdx.x;
    const int il = tid % R, kk = tid / R;
    const bool active = kk < K;
    const int n = g.n;

    // row triangle i = rb + il: quadrature points (absolute or centroid offsets)
    T px[7], py[7], pz[7];
    double ci[3] = {0, 0, 0}, rn[3] = {0, 0, 0}, rplane = 0.0, E1[3] = {0, 0, 0}, E2[3] = {0, 0, 0};
    T chi[3] = {0, 0, 0}, clo[3] = {0, 0, 0}, ai = 0;
    int vi[3] = {-1, -1, -1};
    if (active) {
        const int i = rb + il;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ci[d] = g.ctr[d * n + i];
            rn[d] = g.nrm[d * n + i];
            vi[d] = g.vid[d * n + i];
            chi[d] = (T)g.chl[d * n + i];
            clo[d] = (T)g.chl[(3 + d) * n + i];
            const double w0 = g.v[d * n + i];
            E1[d] = g.v[(3 + d) * n + i] - w0;
            E2[d] = g.v[(6 + d) * n + i] - w0;
        }
        rplane = g.plane[i];
        ai = (T)g.area[i];
#pragma unroll
        for (int p = 0; p < 7; ++p) {
            if (F32) {
                px[p] = (T)g.qo[((int64_t)0 * n + i) * 7 + p];
                py[p] = (T)g.qo[((int64_t)1 * n + i) * 7 + p];
                pz[p] = (T)g.qo[((int64_t)2 * n + i) * 7 + p];
            } else {
                px[p] = (T)g.qa[((int64_t)0 * n + i) * 7 + p];
                py[p] = (T)g.qa[((int64_t)1 * n + i) * 7 + p];
                pz[p] = (T)g.qa[((int64_t)2 * n + i) * 7 + p];
            }
        }
    }
    T acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0;

    for (int b = ptr[blockIdx.x]; b < ptr[blockIdx.x + 1]; ++b) {
        const int s = col[b];
        const int cb = t.begin[s], C = t.end[s] - cb;
        __syncthreads();
        for (int e = tid; e < C * 7; e += kThreads) {
#pragma unroll
            for (int d = 0; d < 3; ++d)
                sq[d * (kMaxLeaf * 7) + e] = F32 ? (T)g.qo[((int64_t)d * n + cb) * 7 + e]
                                                 : (T)g.qa[((int64_t)d * n + cb) * 7 + e];
        }
        for (int e = tid; e < C; e += kThreads) {
            const int j = cb + e;
            sarea[e] = (T)g.area[j];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (F32) {
                    sch[d * kMaxLeaf + e] = (T)g.chl[d * n + j];
                    scl[d * kMaxLeaf + e] = (T)g.chl[(3 + d) * n + j];
                }
                svid[d * kMaxLeaf + e] = g.vid[d * n + j];
                if (KER != SLP) {
                    const double nd = g.nrm[d * n + j];
                    snrm[d * kMaxLeaf + e] = (T)nd;
                    sn64[d * kMaxLeaf + e] = nd;
                }
                if (KER == DLP_T) {
                    const double w0 = g.v[d * n + j];
                    sedge[d * kMaxLeaf + e] = g.v[(3 + d) * n + j] - w0;
                    sedge[(3 + d) * kMaxLeaf + e] = g.v[(6 + d) * n + j] - w0;
                }
            }
            if (KER != SLP) splane[e] = g.plane[j];
        }
        for (int e = tid; e < C * NR; e += kThreads) sx[e] = (T)xp[(int64_t)cb * NR + e];
        __syncthreads();
        if (!active) continue;
        for (int jl = kk; jl < C; jl += K) {
            bool sing = false;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int bb = 0; bb < 3; ++bb) sing |= (vi[a] == svid[bb * kMaxLeaf + jl]);
            if (sing) continue;
            // F32: D = c_i - c_j from the hi/lo splits
            T Dx = 0, Dy = 0, Dz = 0;
            if (F32) {
                Dx = (chi[0] - sch[jl]) + (clo[0] - scl[jl]);
                Dy = (chi[1] - sch[kMaxLeaf + jl]) + (clo[1] - scl[kMaxLeaf + jl]);
                Dz = (chi[2] - sch[2 * kMaxLeaf + jl]) + (clo[2] - scl[2 * kMaxLeaf + jl]);
            }
            // double layer: heights above the plane that carries the normal
            T hp[7];
            if (KER == DLP) {
                const double nx = sn64[jl], ny = sn64[kMaxLeaf + jl], nz = sn64[2 * kMaxLeaf + jl];
                if (F32) {
                    const T H0 = (T)(ci[0] * nx + ci[1] * ny + ci[2] * nz - splane[jl]);
                    const T e1 = (T)(E1[0] * nx + E1[1] * ny + E1[2] * nz);
                    const T e2 = (T)(E2[0] * nx + E2[1] * ny + E2[2] * nz);
#pragma unroll
                    for (int p = 0; p < 7; ++p)
                        hp[p] = H0 + (T)(c.ru[p] - 1.0 / 3.0) * e1 + (T)(c.rv[p] - 1.0 / 3.0) * e2;
                } else {
#pragma unroll
                    for (int p = 0; p < 7; ++p) hp[p] = (T)(px[p] * nx + py[p] * ny + pz[p] * nz - splane[jl]);
                }
            }
            T H0t = 0, f1 = 0, f2 = 0;
            if (KER == DLP_T && F32) {
                // (y_q - c_i) . n_i = (c_j . n_i - c_i . n_i) + (u_q - 1/3) F1 . n_i + (v_q - 1/3) F2 . n_i
                double cj[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) cj[d] = (double)sch[d * kMaxLeaf + jl] + (double)scl[d * kMaxLeaf + jl];
                H0t = (T)(cj[0] * rn[0] + cj[1] * rn[1] + cj[2] * rn[2] - rplane);
                f1 = (T)(sedge[jl] * rn[0] + sedge[kMaxLeaf + jl] * rn[1] + sedge[2 * kMaxLeaf + jl] * rn[2]);
                f2 = (T)(sedge[3 * kMaxLeaf + jl] * rn[0] + sedge[4 * kMaxLeaf + jl] * rn[1] +
                         sedge[5 * kMaxLeaf + jl] * rn[2]);
            }
            T sum = 0;
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                const T ex = sq[jl * 7 + q], ey = sq[kMaxLeaf * 7 + jl * 7 + q], ez = sq[2 * kMaxLeaf * 7 + jl * 7 + q];
                const T yx = F32 ? Dx - ex : ex, yy = F32 ? Dy - ey : ey, yz = F32 ? Dz - ez : ez;
                T hq = 0;
                if (KER == DLP_T) {
                    if (F32) hq = H0t + (T)(c.ru[q] - 1.0 / 3.0) * f1 + (T)(c.rv[q] - 1.0 / 3.0) * f2;
                    else hq = (T)(ex * rn[0] + ey * rn[1] + ez * rn[2] - rplane);
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
            const T a = ai * sarea[jl] * sum;
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] += a * sx[jl * NR + r];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; ++r) sbuf[tid * NR + r] = active ? (double)acc[r] : 0.0;
    __syncthreads();
    for (int e = tid; e < R * NR; e += kThreads) {
        const int i = e / NR, r = e % NR;
        double s = 0.0;
        for (int q = 0; q < K; ++q) s += sbuf[(q * R + i) * NR + r];
        yp[(int64_t)(rb + i) * NR + r] += s * kInv4Pi;
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
