// Farfield of the H^2 product (section 2, eq. (vsw) and eq. (transfer);
// section 3, tensor Chebyshev interpolation), SIMT kernels in FP64 or FP32.
//
// Interpolation nodes of cluster t along axis d: z_d[a] = ctr_d + half_d *
// cos((2a+1) pi / (2m)); tensor index nu = a + m (b + m c).  1-D Lagrange
// polynomials L_a(y) = prod_{kappa != a} (y - z[kappa]) / (z[a] - z[kappa]).
//
//   leaf forward   xh_s[mu]  = sum_{j in s} B_s[j,mu] x_j,
//                  B = V (int_tau L_mu) or W (int_tau n . grad L_mu)
//   upward         xh_t      = sum_{t'} E_{t'}^T xh_{t'}
//   coupling       yh_t[nu]  = sum_{(t,s) in L+} sum_mu g(xi_{t,nu}, xi_{s,mu}) xh_s[mu]
//   downward       yh_{t'}  += E_{t'} yh_t
//   leaf backward  y_i      += sum_nu B_t[i,nu] yh_t[nu]
// with E_{t'}[nu',nu] = L_{t,nu}(xi_{t',nu'}) applied as a Kronecker product of
// three m x m matrices.  Vectors xh, yh: [cluster][nu][r] with NR columns.
#include <algorithm>
#include <type_traits>
#include <utility>

#include "dmath.cuh"
#include "internal.h"

namespace h2 {

// ---------------------------------------------------------------------------
// Leaf transforms.  rule: nb points (u, v, w) on the unit simplex, exact for
// total degree 3(m-1), weights summing to 1.  One CTA per leaf; the leaf's
// triangles are processed in chunks of CT.  For every point of a chunk the
// scaled node differences d_b = (y - z_b) / half of each axis (exact form
// described in tabulate_chunk) and the m Lagrange values L_a = bary[a] prod_{b != a} d_b
// (and, for the double layer, dL_a/dy = bary[a] sum_{b != a} prod_{c != a,b} d_c / half)
// are tabulated in shared memory in the basis precision TB; thread nu then
// forms B[j,nu] = |tau_j| sum_p w_p L_a L_b L_c (or n_j . grad) and accumulates
// in TA.  No divisions on the device.
// Shared layout (TB unless noted): LT[CT*nb][3][m], dLT (double layer),
// wq[CT*nb] = |tau_j| w_p, nr[CT][3]; then TA xs[CT][NR] (forward) or
// TB prod[CT][k] (backward).
// ---------------------------------------------------------------------------
template <typename TB, bool DLPB>
__device__ void tabulate_chunk(const Geom& g, const Tree& t, const Consts& c, const double* rule, int cl, int j0,
                               int cnt, TB* LT, TB* dLT, TB* wq, TB* nr, double* sABC) {
    const int m = c.m, nb = c.nb, n = g.n;
    // per triangle and axis, in reference units of the cluster box:
    // A = (v0 - ctr) / half, B = (v1 - v0) / half, C = (v2 - v0) / half
    for (int e = threadIdx.x; e < cnt * 3; e += blockDim.x) {
        const int jl = e / 3, d = e % 3, j = j0 + jl;
        const double ih = t.box[(6 + d) * t.nc + cl];
        const double v0 = g.v[d * n + j];
        sABC[3 * e] = (v0 - t.box[d * t.nc + cl]) * ih;
        sABC[3 * e + 1] = (g.v[(3 + d) * n + j] - v0) * ih;
        sABC[3 * e + 2] = (g.v[(6 + d) * n + j] - v0) * ih;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * nb * 3; e += blockDim.x) {
        const int jp = e / 3, d = e % 3, jl = jp / nb, p = jp % nb;
        const double* abc = sABC + 3 * (jl * 3 + d);
        const double tr = fma(rule[3 * p + 1], abc[2], fma(rule[3 * p], abc[1], abc[0]));
        // node differences d_b = t - cheb[b]: FP64 tier directly; FP32 tier as
        // (t_hi - cheb_hi) + (t_lo - cheb_lo) with float splits of both terms,
        // the first difference exact near the node (Sterbenz)
        TB diff[kMaxM];
        if (sizeof(TB) == sizeof(double)) {
            for (int b = 0; b < m; ++b) diff[b] = (TB)(tr - c.cheb[b]);
        } else {
            const float th = (float)tr, tl = (float)(tr - (double)th);
            for (int b = 0; b < m; ++b) diff[b] = (TB)((th - c.cheb_hi[b]) + (tl - c.cheb_lo[b]));
        }
        for (int a = 0; a < m; ++a) {
            TB pr = (TB)c.bary[a];
            for (int b = 0; b < m; ++b)
                if (b != a) pr *= diff[b];
            LT[(jp * 3 + d) * m + a] = pr;
            if (DLPB) {
                TB sd = 0;
                for (int b = 0; b < m; ++b) {
                    if (b == a) continue;
                    TB qv = 1;
                    for (int cc = 0; cc < m; ++cc)
                        if (cc != a && cc != b) qv *= diff[cc];
                    sd += qv;
                }
                dLT[(jp * 3 + d) * m + a] = sd * (TB)c.bary[a] * (TB)t.box[(6 + d) * t.nc + cl];
            }
        }
    }
    for (int e = threadIdx.x; e < cnt * nb; e += blockDim.x)
        wq[e] = (TB)(g.area[j0 + e / nb] * rule[3 * (e % nb) + 2]);
    if (DLPB)
        for (int e = threadIdx.x; e < cnt * 3; e += blockDim.x) nr[e] = (TB)g.nrm[(e % 3) * n + j0 + e / 3];
}

// B[j, nu] for one triangle of the chunk from the tabulated values
template <typename TB, bool DLPB>
__device__ __forceinline__ TB basis_value(const TB* LT, const TB* dLT, const TB* wq, const TB* nr, int jl, int nb,
                                          int m, int ia, int ib, int ic) {
    TB sum = 0;
    const TB* Lj = LT + jl * nb * 3 * m;
    const TB* wj = wq + jl * nb;
    if (DLPB) {
        const TB* dLj = dLT + jl * nb * 3 * m;
        const TB nx = nr[3 * jl], ny = nr[3 * jl + 1], nz = nr[3 * jl + 2];
        for (int p = 0; p < nb; ++p) {
            const TB* L = Lj + p * 3 * m;
            const TB* dL = dLj + p * 3 * m;
            const TB lx = L[ia], ly = L[m + ib], lz = L[2 * m + ic];
            sum += wj[p] * (nx * dL[ia] * ly * lz + ny * lx * dL[m + ib] * lz + nz * lx * ly * dL[2 * m + ic]);
        }
    } else {
        for (int p = 0; p < nb; ++p) {
            const TB* L = Lj + p * 3 * m;
            sum += wj[p] * (L[ia] * L[m + ib] * L[2 * m + ic]);
        }
    }
    return sum;
}

template <typename TB>
__host__ __device__ constexpr size_t chunk_tab_elems(int ct, int nb, int m, bool dlp) {
    return (size_t)ct * nb * 3 * m * (dlp ? 2 : 1) + (size_t)ct * nb + (size_t)ct * 3;
}

template <typename TB, typename TA, int NR, bool DLPB>
__global__ void __launch_bounds__(256) k_leaf_forward(Geom g, Tree t, Consts c, const double* __restrict__ rule,
                                                      const int* __restrict__ leaves, int CT,
                                                      const double* __restrict__ xp, TA* __restrict__ xh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = c.m, k = c.k, nb = c.nb;
    TB* LT = reinterpret_cast<TB*>(smem_raw);
    TB* dLT = LT + (size_t)CT * nb * 3 * m;
    TB* wq = dLT + (DLPB ? (size_t)CT * nb * 3 * m : 0);
    TB* nr = wq + (size_t)CT * nb;
    TA* xs = reinterpret_cast<TA*>(smem_raw + ((chunk_tab_elems<TB>(CT, nb, m, DLPB) * sizeof(TB) + 15) / 16) * 16);
    __shared__ double sABC[kMaxLeaf * 9];
    const int s = leaves[blockIdx.x];
    const int b = t.begin[s], R = t.end[s] - b;
    constexpr int kPer = (kMaxK + 63) / 64;
    TA acc[kPer][NR];
#pragma unroll
    for (int q = 0; q < kPer; ++q)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[q][r] = 0;
    for (int j0 = 0; j0 < R; j0 += CT) {
        const int cnt = min(CT, R - j0);
        __syncthreads();
        tabulate_chunk<TB, DLPB>(g, t, c, rule, s, b + j0, cnt, LT, dLT, wq, nr, sABC);
        for (int e = threadIdx.x; e < cnt * NR; e += blockDim.x) xs[e] = (TA)xp[(int64_t)(b + j0) * NR + e];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int nu = threadIdx.x + q * blockDim.x;
            if (nu >= k) break;
            const int ia = nu % m, ib = (nu / m) % m, ic = nu / (m * m);
            for (int jl = 0; jl < cnt; ++jl) {
                const TA w = (TA)basis_value<TB, DLPB>(LT, dLT, wq, nr, jl, nb, m, ia, ib, ic);
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[q][r] += w * xs[jl * NR + r];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int nu = threadIdx.x + q * blockDim.x;
        if (nu >= k) break;
#pragma unroll
        for (int r = 0; r < NR; ++r) xh[((int64_t)s * k + nu) * NR + r] = acc[q][r];
    }
}

template <typename TB, typename TA, int NR, bool DLPB>
__global__ void __launch_bounds__(256) k_leaf_backward(Geom g, Tree t, Consts c, const double* __restrict__ rule,
                                                       const int* __restrict__ leaves, int CT,
                                                       const TA* __restrict__ yh, double* __restrict__ yp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = c.m, k = c.k, nb = c.nb;
    TB* LT = reinterpret_cast<TB*>(smem_raw);
    TB* dLT = LT + (size_t)CT * nb * 3 * m;
    TB* wq = dLT + (DLPB ? (size_t)CT * nb * 3 * m : 0);
    TB* nr = wq + (size_t)CT * nb;
    TB* prod = reinterpret_cast<TB*>(smem_raw + ((chunk_tab_elems<TB>(CT, nb, m, DLPB) * sizeof(TB) + 15) / 16) * 16);
    TA* ys = reinterpret_cast<TA*>(prod + (((size_t)CT * k * sizeof(TB) + 15) / 16) * 16 / sizeof(TB));
    __shared__ double sABC[kMaxLeaf * 9];
    const int s = leaves[blockIdx.x];
    const int b = t.begin[s], R = t.end[s] - b;
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) ys[e] = yh[(int64_t)s * k * NR + e];
    for (int j0 = 0; j0 < R; j0 += CT) {
        const int cnt = min(CT, R - j0);
        __syncthreads();
        tabulate_chunk<TB, DLPB>(g, t, c, rule, s, b + j0, cnt, LT, dLT, wq, nr, sABC);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt * k; e += blockDim.x) {
            const int jl = e / k, nu = e % k;
            prod[e] = basis_value<TB, DLPB>(LT, dLT, wq, nr, jl, nb, m, nu % m, (nu / m) % m, nu / (m * m));
        }
        __syncthreads();
        for (int e = threadIdx.x; e < cnt * NR; e += blockDim.x) {
            const int jl = e / NR, r = e % NR;
            TA v = 0;
            for (int nu = 0; nu < k; ++nu) v += (TA)prod[jl * k + nu] * ys[nu * NR + r];
            yp[(int64_t)(b + j0 + jl) * NR + r] += (double)v;
        }
    }
}

// ---------------------------------------------------------------------------
// Stored leaf bases.  The basis B_s[j, nu] of a leaf does not depend on x, so
// it is evaluated once (k_leaf_basis, the same tabulation as above) and kept
// in tree order, B[pos * k + nu]: the rows of one leaf are contiguous.  The
// leaf transforms of an apply are then small products over staged tiles:
//   forward   xh_s[nu][r] = sum_{j in s} B[j, nu] x_j[r]
//   backward  y_j[r]     += sum_nu B[j, nu] yh_t[nu][r]
// ---------------------------------------------------------------------------
template <typename TB, bool DLPB>
__global__ void __launch_bounds__(256) k_leaf_basis(Geom g, Tree t, Consts c, const double* __restrict__ rule,
                                                    const int* __restrict__ leaves, int CT, TB* __restrict__ B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = c.m, k = c.k, nb = c.nb;
    TB* LT = reinterpret_cast<TB*>(smem_raw);
    TB* dLT = LT + (size_t)CT * nb * 3 * m;
    TB* wq = dLT + (DLPB ? (size_t)CT * nb * 3 * m : 0);
    TB* nr = wq + (size_t)CT * nb;
    __shared__ double sABC[kMaxLeaf * 9];
    const int s = leaves[blockIdx.x];
    const int b = t.begin[s], R = t.end[s] - b;
    for (int j0 = 0; j0 < R; j0 += CT) {
        const int cnt = min(CT, R - j0);
        __syncthreads();
        tabulate_chunk<TB, DLPB>(g, t, c, rule, s, b + j0, cnt, LT, dLT, wq, nr, sABC);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt * k; e += blockDim.x) {
            const int jl = e / k, nu = e % k;
            B[(int64_t)(b + j0) * k + e] =
                basis_value<TB, DLPB>(LT, dLT, wq, nr, jl, nb, m, nu % m, (nu / m) % m, nu / (m * m));
        }
    }
}

// copy `bytes` bytes of a contiguous tile from global to shared memory:
// 16-byte loads where source and size allow, else 4-byte loads
template <typename T>
__device__ __forceinline__ void stage_tile(T* dst, const T* src, size_t bytes) {
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0 && (bytes & 15) == 0) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        for (size_t e = threadIdx.x; e < bytes / 16; e += blockDim.x) d4[e] = s4[e];
    } else {
        const unsigned* s1 = reinterpret_cast<const unsigned*>(src);
        unsigned* d1 = reinterpret_cast<unsigned*>(dst);
        for (size_t e = threadIdx.x; e < bytes / 4; e += blockDim.x) d1[e] = s1[e];
    }
}

template <typename TB, typename TA, int NR, bool ACC = false>
__global__ void __launch_bounds__(128) k_leaf_fwd_st(Tree t, int k, const int* __restrict__ leaves,
                                                     const TB* __restrict__ B, const double* __restrict__ xp,
                                                     TA* __restrict__ xh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int s = leaves[blockIdx.x];
    const int b = t.begin[s], R = t.end[s] - b;
    TB* sB = reinterpret_cast<TB*>(smem_raw);                                        // [R][k]
    TA* sx = reinterpret_cast<TA*>(smem_raw + (((size_t)R * k * sizeof(TB) + 15) & ~size_t(15)));  // [R][NR]
    const TB* Bs = B + (int64_t)b * k;
    stage_tile(sB, Bs, (size_t)R * k * sizeof(TB));
    if (NR % 2 == 0) {  // x rows of the leaf: 16-byte loads of two doubles
        const double2* x2 = reinterpret_cast<const double2*>(xp + (int64_t)b * NR);
        for (int e = threadIdx.x; e < R * NR / 2; e += blockDim.x) {
            const double2 v = x2[e];
            sx[2 * e] = (TA)v.x;
            sx[2 * e + 1] = (TA)v.y;
        }
    } else {
        for (int e = threadIdx.x; e < R * NR; e += blockDim.x) sx[e] = (TA)xp[(int64_t)b * NR + e];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) {
        const int nu = e / NR, r = e % NR;
        TA acc = 0;
        for (int j = 0; j < R; ++j) acc += (TA)sB[j * k + nu] * sx[j * NR + r];
        if (ACC) xh[((int64_t)s * k + nu) * NR + r] += acc;
        else xh[((int64_t)s * k + nu) * NR + r] = acc;
    }
}

template <typename TB, typename TA, int NR>
__global__ void __launch_bounds__(128) k_leaf_bwd_st(Tree t, int k, const int* __restrict__ leaves,
                                                     const TB* __restrict__ B, const TA* __restrict__ yh,
                                                     double* __restrict__ yp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int s = leaves[blockIdx.x];
    const int b = t.begin[s], R = t.end[s] - b;
    const int kp = k + 1;  // padded row stride: rows of one warp fall in different banks
    TB* sB = reinterpret_cast<TB*>(smem_raw);                                         // [R][kp]
    TA* sy = reinterpret_cast<TA*>(smem_raw + (((size_t)R * kp * sizeof(TB) + 15) & ~size_t(15)));  // [k][NR]
    const TB* Bs = B + (int64_t)b * k;
    if (sizeof(TB) == 4 && (k % 4) == 0) {  // 16-byte loads of four basis values, spread to the padded rows
        const uint4* b4 = reinterpret_cast<const uint4*>(Bs);
        for (int e = threadIdx.x; e < R * k / 4; e += blockDim.x) {
            const uint4 v = b4[e];
            const int j = (4 * e) / k, nu = (4 * e) % k;
            TB* dst = sB + j * kp + nu;
            dst[0] = __uint_as_float(v.x);
            dst[1] = __uint_as_float(v.y);
            dst[2] = __uint_as_float(v.z);
            dst[3] = __uint_as_float(v.w);
        }
    } else {
        for (int e = threadIdx.x; e < R * k; e += blockDim.x) sB[(e / k) * kp + e % k] = Bs[e];
    }
    stage_tile(sy, yh + (int64_t)s * k * NR, (size_t)k * NR * sizeof(TA));
    __syncthreads();
    for (int e = threadIdx.x; e < R * NR; e += blockDim.x) {
        const int j = e / NR, r = e % NR;
        TA acc = 0;
        for (int nu = 0; nu < k; ++nu) acc += (TA)sB[j * kp + nu] * sy[nu * NR + r];
        yp[(int64_t)(b + j) * NR + r] += (double)acc;
    }
}

// Register-tiled leaf transformations for an FP32 basis and FP32 cluster
// vectors, NR a multiple of 4: each thread owns 2 x 4 outputs, so a step of
// the sum takes one 8-byte basis pair and one 16-byte x (or y-hat) quad from
// shared memory for 8 multiply-adds (the kernels above load both operands of
// every multiply-add).  Same products and summation order per output.
// Forward: thread (vp, g) owns x-hat_s[2 vp + (0, 1)][4 g + (0..3)], threads
// ceil(k/2) x NR/4 rounded up to a warp.
template <int NR>
__global__ void __launch_bounds__(256) k_leaf_fwd_t4(Tree t, int k, const int* __restrict__ leaves,
                                                     const float* __restrict__ B, const double* __restrict__ xp,
                                                     float* __restrict__ xh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int s = leaves[blockIdx.x];
    const int b = t.begin[s], R = t.end[s] - b;
    float* sB = reinterpret_cast<float*>(smem_raw);                                         // [R][k]
    float* sx = reinterpret_cast<float*>(smem_raw + (((size_t)R * k * 4 + 15) & ~size_t(15)));  // [R][NR]
    stage_tile(sB, B + (int64_t)b * k, (size_t)R * k * sizeof(float));
    const double2* x2 = reinterpret_cast<const double2*>(xp + (int64_t)b * NR);
    for (int e = threadIdx.x; e < R * NR / 2; e += blockDim.x) {
        const double2 v = x2[e];
        sx[2 * e] = (float)v.x;
        sx[2 * e + 1] = (float)v.y;
    }
    __syncthreads();
    const int KP = (k + 1) / 2;
    const int vp = threadIdx.x % KP, g = threadIdx.x / KP;
    if (g >= NR / 4) return;
    const int nu = 2 * vp;
    const bool two = nu + 1 < k;
    float a0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, a1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int j = 0; j < R; ++j) {
        float b0, b1;
        if ((k & 1) == 0) {
            const float2 bb = *reinterpret_cast<const float2*>(sB + j * k + nu);
            b0 = bb.x;
            b1 = bb.y;
        } else {
            b0 = sB[j * k + nu];
            b1 = two ? sB[j * k + nu + 1] : 0.0f;
        }
        const float4 xv = *reinterpret_cast<const float4*>(sx + j * NR + 4 * g);
        a0[0] += b0 * xv.x;
        a0[1] += b0 * xv.y;
        a0[2] += b0 * xv.z;
        a0[3] += b0 * xv.w;
        a1[0] += b1 * xv.x;
        a1[1] += b1 * xv.y;
        a1[2] += b1 * xv.z;
        a1[3] += b1 * xv.w;
    }
    float4* o = reinterpret_cast<float4*>(xh + ((int64_t)s * k + nu) * NR + 4 * g);
    o[0] = make_float4(a0[0], a0[1], a0[2], a0[3]);
    if (two) o[NR / 4] = make_float4(a1[0], a1[1], a1[2], a1[3]);
}

// Backward: y_{b+j} += sum_nu B[j][nu] y-hat_s[nu]; thread (j, g) owns row j
// and right-hand sides 4 g + (0..3) (threads R x NR/4 rounded up to a warp):
// per step one basis value and one 16-byte y-hat quad for 4 multiply-adds.
// The basis block is staged transposed, [nu][j], by 16-byte loads of
// four consecutive nu of a row, so that the threads of a warp (consecutive
// rows) read consecutive words.
template <int NR>
__global__ void __launch_bounds__(256) k_leaf_bwd_t4(Tree t, int k, const int* __restrict__ leaves,
                                                     const float* __restrict__ B, const float* __restrict__ yh,
                                                     double* __restrict__ yp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int s = leaves[blockIdx.x];
    const int b = t.begin[s], R = t.end[s] - b;
    float* sBt = reinterpret_cast<float*>(smem_raw);                                         // [k][R]
    float* sy = reinterpret_cast<float*>(smem_raw + (((size_t)k * R * 4 + 15) & ~size_t(15)));  // [k][NR]
    const float* Bs = B + (int64_t)b * k;
    if ((k & 3) == 0 && ((reinterpret_cast<uintptr_t>(Bs) & 15) == 0)) {
        const int k4 = k / 4;
        for (int e = threadIdx.x; e < R * k4; e += blockDim.x) {
            const int j = e / k4, nu = 4 * (e - j * k4);
            const float4 v = reinterpret_cast<const float4*>(Bs)[e];
            sBt[nu * R + j] = v.x;
            sBt[(nu + 1) * R + j] = v.y;
            sBt[(nu + 2) * R + j] = v.z;
            sBt[(nu + 3) * R + j] = v.w;
        }
    } else {
        for (int e = threadIdx.x; e < R * k; e += blockDim.x) sBt[(e % k) * R + e / k] = Bs[e];
    }
    stage_tile(sy, yh + (int64_t)s * k * NR, (size_t)k * NR * sizeof(float));
    __syncthreads();
    const int j = threadIdx.x % R, g = threadIdx.x / R;
    if (g >= NR / 4) return;
    float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int nu = 0; nu < k; ++nu) {
        const float bv = sBt[nu * R + j];
        const float4 yv = *reinterpret_cast<const float4*>(sy + nu * NR + 4 * g);
        a[0] += bv * yv.x;
        a[1] += bv * yv.y;
        a[2] += bv * yv.z;
        a[3] += bv * yv.w;
    }
    double* y0 = yp + (int64_t)(b + j) * NR + 4 * g;
#pragma unroll
    for (int r = 0; r < 4; ++r) y0[r] += (double)a[r];
}

// ---------------------------------------------------------------------------
// Transfers between a parent t and its children (Kronecker form).
// E1[ch][d][a'][a] = L_{t,a}^{(d)}(z_{ch,d}[a']).
// ---------------------------------------------------------------------------
template <typename T, int MM>
__device__ void transfer_1d(const Tree& t, const Consts& c, int parent, const int* ch, T* E1) {
    // E1[q][d][a'][a] = L_{p,a}(yhat), yhat = (z_{ch_q}[a'] - c_p) / h_p: FP32
    // vectors take the factors evaluated at set-up (FP64, rounded once); FP64
    // vectors evaluate L_a(yhat) = bary[a] prod_{b != a} (yhat - cheb[b]) here
    const int m = MM > 0 ? MM : c.m;
    for (int e = threadIdx.x; e < 2 * 3 * m * m; e += blockDim.x) {
        const int q = e / (3 * m * m), r = e % (3 * m * m);
        if constexpr (sizeof(T) == sizeof(float)) {
            E1[e] = t.etr[(int64_t)ch[q] * 3 * m * m + r];
        } else {
            const int d = r / (m * m), ap = (r / m) % m, a = r % m;
            const int cl = ch[q];
            const double yd = (t.box[d * t.nc + cl] - t.box[d * t.nc + parent] + t.box[(3 + d) * t.nc + cl] * c.cheb[ap]) *
                              t.box[(6 + d) * t.nc + parent];
            double pr = c.bary[a];
            for (int b = 0; b < m; ++b)
                if (b != a) pr *= yd - c.cheb[b];
            E1[e] = (T)pr;
        }
    }
    __syncthreads();
}

// up: X[a',b',c'] -> out[a,b,c] = sum E_x[a'][a] E_y[b'][b] E_z[c'][c] X
// down: Y[a,b,c] -> out[a',b',c'] = sum E_x[a'][a] E_y[b'][b] E_z[c'][c] Y
// MM: compile-time m (0: runtime m)
template <typename T, int NR, bool UP, int MM>
__device__ void kron_apply(const T* E1, int mrt, const T* in, T* tmp1, T* tmp2, T* out, bool accumulate) {
    const int m = MM > 0 ? MM : mrt;
    const int k = m * m * m;
    const T* Ex = E1;
    const T* Ey = E1 + m * m;
    const T* Ez = E1 + 2 * m * m;
    // contract x
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) {
        const int r = e % NR, nu = e / NR, a = nu % m, rest = nu / m;
        T s = 0;
#pragma unroll
        for (int q = 0; q < (MM > 0 ? MM : kMaxM); ++q) {
            if (MM == 0 && q >= m) break;
            s += (UP ? Ex[q * m + a] : Ex[a * m + q]) * in[((rest * m) + q) * NR + r];
        }
        tmp1[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) {
        const int r = e % NR, nu = e / NR, a = nu % m, b = (nu / m) % m, cc = nu / (m * m);
        T s = 0;
#pragma unroll
        for (int q = 0; q < (MM > 0 ? MM : kMaxM); ++q) {
            if (MM == 0 && q >= m) break;
            s += (UP ? Ey[q * m + b] : Ey[b * m + q]) * tmp1[((cc * m + q) * m + a) * NR + r];
        }
        tmp2[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) {
        const int r = e % NR, nu = e / NR, ab = nu % (m * m), cc = nu / (m * m);
        T s = 0;
#pragma unroll
        for (int q = 0; q < (MM > 0 ? MM : kMaxM); ++q) {
            if (MM == 0 && q >= m) break;
            s += (UP ? Ez[q * m + cc] : Ez[cc * m + q]) * tmp2[((q * m * m) + ab) * NR + r];
        }
        if (accumulate) out[e] += s;
        else out[e] = s;
    }
    __syncthreads();
}

template <typename T, int NR, int MM>
__global__ void __launch_bounds__(256) k_upward(Tree t, Consts c, const int* __restrict__ parents, T* __restrict__ xh) {
    extern __shared__ unsigned char smem_raw[];
    T* E1 = reinterpret_cast<T*>(smem_raw);
    T* buf = E1 + 2 * 3 * kMaxM * kMaxM;
    const int m = MM > 0 ? MM : c.m, k = m * m * m;
    T* in = buf;
    T* tmp1 = in + k * NR;
    T* tmp2 = tmp1 + k * NR;
    T* out = tmp2 + k * NR;
    const int p = parents[blockIdx.x];
    const int ch[2] = {t.child0[p], t.child1[p]};
    transfer_1d<T, MM>(t, c, p, ch, E1);
    for (int q = 0; q < 2; ++q) {
        for (int e = threadIdx.x; e < k * NR; e += blockDim.x) in[e] = xh[(int64_t)ch[q] * k * NR + e];
        __syncthreads();
        kron_apply<T, NR, true, MM>(E1 + q * 3 * m * m, m, in, tmp1, tmp2, out, q == 1);
    }
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) xh[(int64_t)p * k * NR + e] = out[e];
}

template <typename T, int NR, int MM>
__global__ void __launch_bounds__(256) k_downward(Tree t, Consts c, const int* __restrict__ parents,
                                                  T* __restrict__ yh) {
    extern __shared__ unsigned char smem_raw[];
    T* E1 = reinterpret_cast<T*>(smem_raw);
    T* buf = E1 + 2 * 3 * kMaxM * kMaxM;
    const int m = MM > 0 ? MM : c.m, k = m * m * m;
    T* in = buf;
    T* tmp1 = in + k * NR;
    T* tmp2 = tmp1 + k * NR;
    T* out = tmp2 + k * NR;
    const int p = parents[blockIdx.x];
    const int ch[2] = {t.child0[p], t.child1[p]};
    transfer_1d<T, MM>(t, c, p, ch, E1);
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) in[e] = yh[(int64_t)p * k * NR + e];
    __syncthreads();
    for (int q = 0; q < 2; ++q) {
        kron_apply<T, NR, false, MM>(E1 + q * 3 * m * m, m, in, tmp1, tmp2, out, false);
        for (int e = threadIdx.x; e < k * NR; e += blockDim.x) yh[(int64_t)ch[q] * k * NR + e] += out[e];
        __syncthreads();
    }
}

// Warp-per-parent transfers for compile-time m: warp w of a CTA takes parent
// blockIdx.x * W + w; the factors and the three one-dimensional contractions
// of each child run on warp-private shared memory with warp barriers only
// (the CTA-per-parent kernels above synchronise the whole CTA around every
// contraction, ~2 multiply-adds per thread each).  Up: the parent's sums are
// kept in a fourth warp-private array over both children; down: each child's
// block is added to its y-hat in place.  Same factors and summation order per
// element as above.  CG: read the cluster vectors through L2 (ld.global.cg),
// for the whole-tree kernels below, where another SM wrote them during the
// same launch.
template <typename T>
__device__ __forceinline__ T ld_v(const T* p, bool cg) {
    return cg ? __ldcg(p) : *p;
}

template <typename T, int NR, bool UP, int M, bool CG>
__device__ __forceinline__ void updown_parent(const Tree& t, const Consts& c, int p, T* __restrict__ v, T* E1,
                                              int lane) {
    constexpr int K = M * M * M, KN = K * NR, PER = (KN + 31) / 32, F = 3 * M * M;
    T* in = E1 + 2 * F;
    T* tmp1 = in + KN;
    T* tmp2 = tmp1 + KN;
    T* out = tmp2 + KN;  // parent's sums (up)
    const int ch[2] = {t.child0[p], t.child1[p]};
    // E1[q][d][a'][a] = L_{p,a}(z_{ch_q,d}[a']) as in transfer_1d
    for (int e = lane; e < 2 * F; e += 32) {
        const int q = e / F, r = e % F;
        if constexpr (sizeof(T) == sizeof(float)) {
            E1[e] = t.etr[(int64_t)ch[q] * F + r];
        } else {
            const int d = r / (M * M), ap = (r / M) % M, a = r % M;
            const int cl = ch[q];
            const double yd = (t.box[d * t.nc + cl] - t.box[d * t.nc + p] + t.box[(3 + d) * t.nc + cl] * c.cheb[ap]) *
                              t.box[(6 + d) * t.nc + p];
            double pr = c.bary[a];
            for (int b = 0; b < M; ++b)
                if (b != a) pr *= yd - c.cheb[b];
            E1[e] = (T)pr;
        }
    }
    if (!UP)
        for (int e = lane; e < KN; e += 32) in[e] = ld_v(v + (int64_t)p * KN + e, CG);
    for (int q = 0; q < 2; ++q) {
        if (UP)
            for (int e = lane; e < KN; e += 32) in[e] = ld_v(v + (int64_t)ch[q] * KN + e, CG);
        __syncwarp();
        const T* Ex = E1 + q * F;
        const T* Ey = Ex + M * M;
        const T* Ez = Ey + M * M;
#pragma unroll 4
        for (int j = 0; j < PER; ++j) {  // contract x
            const int e = lane + 32 * j;
            if (e < KN) {
                const int r = e % NR, nu = e / NR, a = nu % M, rest = nu / M;
                T sum = 0;
#pragma unroll
                for (int w = 0; w < M; ++w) sum += (UP ? Ex[w * M + a] : Ex[a * M + w]) * in[((rest * M) + w) * NR + r];
                tmp1[e] = sum;
            }
        }
        __syncwarp();
#pragma unroll 4
        for (int j = 0; j < PER; ++j) {  // contract y
            const int e = lane + 32 * j;
            if (e < KN) {
                const int r = e % NR, nu = e / NR, a = nu % M, b = (nu / M) % M, cc = nu / (M * M);
                T sum = 0;
#pragma unroll
                for (int w = 0; w < M; ++w)
                    sum += (UP ? Ey[w * M + b] : Ey[b * M + w]) * tmp1[((cc * M + w) * M + a) * NR + r];
                tmp2[e] = sum;
            }
        }
        __syncwarp();
#pragma unroll 4
        for (int j = 0; j < PER; ++j) {  // contract z
            const int e = lane + 32 * j;
            if (e < KN) {
                const int r = e % NR, nu = e / NR, ab = nu % (M * M), cc = nu / (M * M);
                T sum = 0;
#pragma unroll
                for (int w = 0; w < M; ++w)
                    sum += (UP ? Ez[w * M + cc] : Ez[cc * M + w]) * tmp2[((w * M * M) + ab) * NR + r];
                if (UP) out[e] = q == 0 ? sum : out[e] + sum;
                else v[(int64_t)ch[q] * KN + e] = ld_v(v + (int64_t)ch[q] * KN + e, CG) + sum;
            }
        }
        __syncwarp();  // the next child overwrites in / tmp1 / tmp2
    }
    if (UP)
        for (int e = lane; e < KN; e += 32) v[(int64_t)p * KN + e] = out[e];
}

template <typename T, int NR, bool UP, int M>
__global__ void __launch_bounds__(256) k_updown_w(Tree t, Consts c, int np, const int* __restrict__ parents,
                                                  T* __restrict__ v) {
    constexpr int KN = M * M * M * NR, F = 3 * M * M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* E1 = reinterpret_cast<T*>(smem_raw) + (size_t)warp * (2 * F + 4 * KN);
    const int pi = blockIdx.x * W + warp;
    if (pi >= np) return;  // no CTA-wide barrier in this kernel
    updown_parent<T, NR, UP, M, false>(t, c, parents[pi], v, E1, lane);
}

// Warp-per-parent transfers for FP32, m = 4, 8 right-hand sides, in
// registers: lane (c, r) = (lane / 8, lane % 8) holds the 4 x 4 plane
// v[a + 4 b + 16 c][r] of a cluster vector, so the contractions in x and y
// are lane-local and the one in z takes the other planes by warp shuffles.
// The same factors (etr) and per-element summation order as k_updown_w, with
// no shared memory.  Up: x-hat_p = sum_q E_q x-hat_{ch_q}; down: y-hat_{ch_q}
// += E_q^T y-hat_p.
template <bool UP>
__global__ void __launch_bounds__(256) k_updown_r8(Tree t, int np, const int* __restrict__ parents,
                                                   float* __restrict__ v) {
    constexpr int KN = 64 * 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pi = blockIdx.x * (blockDim.x >> 5) + warp;
    if (pi >= np) return;
    const int p = parents[pi];
    const int r = lane & 7, cz = lane >> 3;
    float pv[16];  // up: the parent's sums; down: the parent's y-hat
    if (UP) {
#pragma unroll
        for (int ab = 0; ab < 16; ++ab) pv[ab] = 0.0f;
    } else {
#pragma unroll
        for (int ab = 0; ab < 16; ++ab) pv[ab] = v[(int64_t)p * KN + (cz * 16 + ab) * 8 + r];
    }
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
        const int ch = q == 0 ? t.child0[p] : t.child1[p];
        // E[d][a'][a] = L_{p,a}(z_{ch,d}[a']): the x and y factors (32 values,
        // the same for every lane) in registers, the lane's z factors below
        const float* Eg = t.etr + (int64_t)ch * 48;
        float E[32];
        const float4* E4 = reinterpret_cast<const float4*>(Eg);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 e = E4[i];
            E[4 * i] = e.x;
            E[4 * i + 1] = e.y;
            E[4 * i + 2] = e.z;
            E[4 * i + 3] = e.w;
        }
        float in[16], t1[16], t2[16];
        if (UP) {
#pragma unroll
            for (int ab = 0; ab < 16; ++ab) in[ab] = v[(int64_t)ch * KN + (cz * 16 + ab) * 8 + r];
        } else {
#pragma unroll
            for (int ab = 0; ab < 16; ++ab) in[ab] = pv[ab];
        }
#pragma unroll
        for (int b = 0; b < 4; ++b)  // contract x
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                float sum = 0.0f;
#pragma unroll
                for (int w = 0; w < 4; ++w) sum += (UP ? E[w * 4 + a] : E[a * 4 + w]) * in[w + 4 * b];
                t1[a + 4 * b] = sum;
            }
#pragma unroll
        for (int b = 0; b < 4; ++b)  // contract y
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                float sum = 0.0f;
#pragma unroll
                for (int w = 0; w < 4; ++w) sum += (UP ? E[16 + w * 4 + b] : E[16 + b * 4 + w]) * t1[a + 4 * w];
                t2[a + 4 * b] = sum;
            }
        // contract z: the planes of the other lanes with the same r
        float zc[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) zc[w] = UP ? Eg[32 + w * 4 + cz] : Eg[32 + cz * 4 + w];
#pragma unroll
        for (int ab = 0; ab < 16; ++ab) {
            float sum = 0.0f;
#pragma unroll
            for (int w = 0; w < 4; ++w) sum += zc[w] * __shfl_sync(0xffffffffu, t2[ab], w * 8 + r);
            if (UP) pv[ab] = q == 0 ? sum : pv[ab] + sum;
            else v[(int64_t)ch * KN + (cz * 16 + ab) * 8 + r] += sum;
        }
    }
    if (UP) {
#pragma unroll
        for (int ab = 0; ab < 16; ++ab) v[(int64_t)p * KN + (cz * 16 + ab) * 8 + r] = pv[ab];
    }
}

// Upward pass over the top of the tree in one launch (section 2, eq.
// (transfer): x-hat_p = sum over the children c of E_c x-hat_c).  Warp w
// starts at cluster start[blockIdx.x * W + w], whose x-hat is complete (a
// leaf's from the leaf transformation, the others' from the per-level
// launches below), and climbs: it counts its arrival at the parent (cnt[p],
// atomically; the count
// keeps running over applies, so arrival a of an apply is the last one when
// (a + 1) is a multiple of the number of children), and only the warp that
// arrives last computes x-hat_p, from both children, and climbs on.  Nothing
// waits: every other warp stops.  The children's vectors are written before a
// fence that precedes the arrival, and read through L2 after it.
template <typename T, int NR, int M>
__global__ void __launch_bounds__(256) k_up_tree(Tree t, Consts c, int nstart, const int* __restrict__ start,
                                                 const int* __restrict__ parent, unsigned* __restrict__ cnt,
                                                 T* __restrict__ v) {
    constexpr int KN = M * M * M * NR, F = 3 * M * M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* E1 = reinterpret_cast<T*>(smem_raw) + (size_t)warp * (2 * F + 4 * KN);
    const int li = blockIdx.x * W + warp;
    if (li >= nstart) return;  // no CTA-wide barrier in this kernel
    int node = start[li];
    for (;;) {
        const int p = parent[node];
        if (p < 0) break;
        __threadfence();  // this warp's x-hat of node (when it computed it) is visible before the arrival
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            const unsigned nch = (t.child0[p] >= 0 ? 1u : 0u) + (t.child1[p] >= 0 ? 1u : 0u);
            const unsigned a = atomicAdd(&cnt[p], 1u);
            last = (a + 1u) % nch == 0u;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) break;
        __threadfence();
        updown_parent<T, NR, true, M, true>(t, c, p, v, E1, lane);
        node = p;
    }
}

// Downward pass over the top of the tree in one launch (section 2: y-hat_c +=
// E_c^T y-hat_p, parents before children), without waits: warp w takes
// cluster v = start[blockIdx.x * W + w] (a cluster of the first per-level
// launch's level, or a leaf above it) and walks from its root down the path
// to v, forming in shared memory z_0 = y-hat_root, z_i = y-hat_{a_i} +
// E_{a_i}^T z_{i-1} for the ancestors a_1 .. a_k of v (their coupling sums,
// which the coupling wrote, plus what their parents pass down), and adds
// E_v^T z_k to y-hat_v.  Only y-hat_v is written; the ancestors' sums are
// formed again by every cluster below them (the top levels hold few clusters:
// a few transfers more per cluster, no launch per level and no inter-warp
// dependence).  The factors are those of the per-level kernels.
constexpr int kMaxDepth = 64;

template <typename T, int NR, int M>
__device__ __forceinline__ void down_one(const Tree& t, const Consts& c, int p, int ch, T* E1, const T* in, T* tmp1,
                                         T* tmp2, T* out, int lane) {
    constexpr int K = M * M * M, KN = K * NR, PER = (KN + 31) / 32, F = 3 * M * M;
    for (int e = lane; e < F; e += 32) {
        if constexpr (sizeof(T) == sizeof(float)) {
            E1[e] = t.etr[(int64_t)ch * F + e];
        } else {
            const int d = e / (M * M), ap = (e / M) % M, a = e % M;
            const double yd = (t.box[d * t.nc + ch] - t.box[d * t.nc + p] + t.box[(3 + d) * t.nc + ch] * c.cheb[ap]) *
                              t.box[(6 + d) * t.nc + p];
            double pr = c.bary[a];
            for (int b = 0; b < M; ++b)
                if (b != a) pr *= yd - c.cheb[b];
            E1[e] = (T)pr;
        }
    }
    __syncwarp();
    const T* Ex = E1;
    const T* Ey = Ex + M * M;
    const T* Ez = Ey + M * M;
#pragma unroll 4
    for (int j = 0; j < PER; ++j) {  // contract x
        const int e = lane + 32 * j;
        if (e < KN) {
            const int r = e % NR, nu = e / NR, a = nu % M, rest = nu / M;
            T sum = 0;
#pragma unroll
            for (int w = 0; w < M; ++w) sum += Ex[a * M + w] * in[((rest * M) + w) * NR + r];
            tmp1[e] = sum;
        }
    }
    __syncwarp();
#pragma unroll 4
    for (int j = 0; j < PER; ++j) {  // contract y
        const int e = lane + 32 * j;
        if (e < KN) {
            const int r = e % NR, nu = e / NR, a = nu % M, b = (nu / M) % M, cc = nu / (M * M);
            T sum = 0;
#pragma unroll
            for (int w = 0; w < M; ++w) sum += Ey[b * M + w] * tmp1[((cc * M + w) * M + a) * NR + r];
            tmp2[e] = sum;
        }
    }
    __syncwarp();
#pragma unroll 4
    for (int j = 0; j < PER; ++j) {  // contract z
        const int e = lane + 32 * j;
        if (e < KN) {
            const int r = e % NR, nu = e / NR, ab = nu % (M * M), cc = nu / (M * M);
            T sum = 0;
#pragma unroll
            for (int w = 0; w < M; ++w) sum += Ez[cc * M + w] * tmp2[((w * M * M) + ab) * NR + r];
            out[e] = sum;
        }
    }
    __syncwarp();
}

template <typename T, int NR, int M>
__global__ void __launch_bounds__(256) k_down_top(Tree t, Consts c, int nstart, const int* __restrict__ start,
                                                  const int* __restrict__ parent, T* __restrict__ v) {
    constexpr int KN = M * M * M * NR, F = 3 * M * M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* E1 = reinterpret_cast<T*>(smem_raw) + (size_t)warp * (2 * F + 4 * KN);
    T* z = E1 + 2 * F;
    T* tmp1 = z + KN;
    T* tmp2 = tmp1 + KN;
    T* out = tmp2 + KN;
    __shared__ int path[8][kMaxDepth];
    const int li = blockIdx.x * W + warp;
    if (li >= nstart || W > 8) return;  // no CTA-wide barrier in this kernel
    const int node = start[li];
    // the ancestors of node, root first (path[0]) to the parent (path[k - 1])
    int k = 0;
    if (lane == 0) {
        for (int a = parent[node]; a >= 0 && k < kMaxDepth; a = parent[a]) path[warp][k++] = a;
        for (int i = 0; i < k / 2; ++i) {
            const int tmp = path[warp][i];
            path[warp][i] = path[warp][k - 1 - i];
            path[warp][k - 1 - i] = tmp;
        }
    }
    k = __shfl_sync(0xffffffffu, k, 0);
    __syncwarp();
    if (k == 0) return;  // a root: its sums are final
    for (int e = lane; e < KN; e += 32) z[e] = v[(int64_t)path[warp][0] * KN + e];
    __syncwarp();
    for (int i = 1; i <= k; ++i) {
        const int p = path[warp][i - 1], ch = i < k ? path[warp][i] : node;
        down_one<T, NR, M>(t, c, p, ch, E1, z, tmp1, tmp2, out, lane);
        if (i < k) {
            for (int e = lane; e < KN; e += 32) z[e] = v[(int64_t)ch * KN + e] + out[e];
        } else {
            for (int e = lane; e < KN; e += 32) v[(int64_t)ch * KN + e] += out[e];
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int far_threads(int k) {
    int th = ((k + 31) / 32) * 32;
    if (th < 64) th = 64;
    if (th > 256) th = 256;
    return th;
}

#define H2_NR_SWITCH(NR, CALL)          \
    switch (NR) {                       \
        case 1: { constexpr int R_ = 1; CALL; } break;  \
        case 4: { constexpr int R_ = 4; CALL; } break;  \
        case 8: { constexpr int R_ = 8; CALL; } break;  \
        default: { constexpr int R_ = 16; CALL; } break; \
    }

// chunk size: tabulated values of one chunk within about 16 KB of shared
// memory, so that many CTAs (of 64-256 threads) fit on an SM
static int leaf_chunk(const Consts& c, size_t tb, bool dlp) {
    const size_t per = ((size_t)c.nb * 3 * c.m * (dlp ? 2 : 1) + c.nb + 3) * tb;
    int ct = (int)(16384 / per);
    return ct < 1 ? 1 : ct > kMaxLeaf ? kMaxLeaf : ct;
}

template <typename TB, typename TA, int NR, bool DLPB>
static void leaf_fwd(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nl, const int* leaves,
                     const double* xp, void* xh, cudaStream_t s) {
    const int ct = leaf_chunk(c, sizeof(TB), DLPB);
    const size_t smem = ((chunk_tab_elems<TB>(ct, c.nb, c.m, DLPB) * sizeof(TB) + 15) / 16) * 16 + (size_t)ct * NR * sizeof(TA);
    cudaFuncSetAttribute(k_leaf_forward<TB, TA, NR, DLPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_leaf_forward<TB, TA, NR, DLPB><<<nl, far_threads(c.k), smem, s>>>(g, t, c, rule, leaves, ct, xp, (TA*)xh);
}

template <typename TB, typename TA, int NR, bool DLPB>
static void leaf_bwd(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nl, const int* leaves,
                     const void* yh, double* yp, cudaStream_t s) {
    const int ct = leaf_chunk(c, sizeof(TB), DLPB);
    const size_t smem = ((chunk_tab_elems<TB>(ct, c.nb, c.m, DLPB) * sizeof(TB) + 15) / 16) * 16 +
                        (((size_t)ct * c.k * sizeof(TB) + 15) / 16) * 16 + (size_t)c.k * NR * sizeof(TA);
    cudaFuncSetAttribute(k_leaf_backward<TB, TA, NR, DLPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_leaf_backward<TB, TA, NR, DLPB><<<nl, far_threads(c.k), smem, s>>>(g, t, c, rule, leaves, ct, (const TA*)yh, yp);
}

template <int NR, bool DLPB>
static void leaf_fwd_prec(bool basis32, bool xh64, const Geom& g, const Tree& t, const Consts& c, const double* rule,
                          int nl, const int* leaves, const double* xp, void* xh, cudaStream_t s) {
    // TB = basis precision, TA = precision of the accumulation and of xh
    if (!basis32 && xh64) leaf_fwd<double, double, NR, DLPB>(g, t, c, rule, nl, leaves, xp, xh, s);
    else if (!basis32) leaf_fwd<double, float, NR, DLPB>(g, t, c, rule, nl, leaves, xp, xh, s);
    else if (xh64) leaf_fwd<float, double, NR, DLPB>(g, t, c, rule, nl, leaves, xp, xh, s);
    else leaf_fwd<float, float, NR, DLPB>(g, t, c, rule, nl, leaves, xp, xh, s);
}

template <int NR, bool DLPB>
static void leaf_bwd_prec(bool basis32, bool yh64, const Geom& g, const Tree& t, const Consts& c, const double* rule,
                          int nl, const int* leaves, const void* yh, double* yp, cudaStream_t s) {
    // TB = basis precision, TA = precision of yh and of the accumulation
    if (!basis32 && yh64) leaf_bwd<double, double, NR, DLPB>(g, t, c, rule, nl, leaves, yh, yp, s);
    else if (!basis32) leaf_bwd<double, float, NR, DLPB>(g, t, c, rule, nl, leaves, yh, yp, s);
    else if (yh64) leaf_bwd<float, double, NR, DLPB>(g, t, c, rule, nl, leaves, yh, yp, s);
    else leaf_bwd<float, float, NR, DLPB>(g, t, c, rule, nl, leaves, yh, yp, s);
}

void launch_leaf_forward(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nleaves,
                         const int* leaves, bool dlp_basis, bool basis32, bool xh64, int NR, const double* xp,
                         void* xh, cudaStream_t s) {
    if (nleaves <= 0) return;
    if (dlp_basis) { H2_NR_SWITCH(NR, (leaf_fwd_prec<R_, true>(basis32, xh64, g, t, c, rule, nleaves, leaves, xp, xh, s))) }
    else { H2_NR_SWITCH(NR, (leaf_fwd_prec<R_, false>(basis32, xh64, g, t, c, rule, nleaves, leaves, xp, xh, s))) }
}

void launch_leaf_backward(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nleaves,
                          const int* leaves, bool dlp_basis, bool basis32, bool yh64, int NR, const void* yh,
                          double* yp, cudaStream_t s) {
    if (nleaves <= 0) return;
    if (dlp_basis) { H2_NR_SWITCH(NR, (leaf_bwd_prec<R_, true>(basis32, yh64, g, t, c, rule, nleaves, leaves, yh, yp, s))) }
    else { H2_NR_SWITCH(NR, (leaf_bwd_prec<R_, false>(basis32, yh64, g, t, c, rule, nleaves, leaves, yh, yp, s))) }
}

void launch_leaf_basis(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nleaves,
                       const int* leaves, bool dlp_basis, bool basis32, void* B, cudaStream_t s) {
    if (nleaves <= 0) return;
    auto go = [&](auto kern, size_t tb) {
        const int ct = leaf_chunk(c, tb, dlp_basis);
        const size_t smem = ((chunk_tab_elems<double>(ct, c.nb, c.m, dlp_basis) * tb + 15) / 16) * 16;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return std::make_pair(ct, smem);
    };
    if (basis32) {
        if (dlp_basis) {
            auto [ct, sm] = go(k_leaf_basis<float, true>, sizeof(float));
            k_leaf_basis<float, true><<<nleaves, far_threads(c.k), sm, s>>>(g, t, c, rule, leaves, ct, (float*)B);
        } else {
            auto [ct, sm] = go(k_leaf_basis<float, false>, sizeof(float));
            k_leaf_basis<float, false><<<nleaves, far_threads(c.k), sm, s>>>(g, t, c, rule, leaves, ct, (float*)B);
        }
    } else {
        if (dlp_basis) {
            auto [ct, sm] = go(k_leaf_basis<double, true>, sizeof(double));
            k_leaf_basis<double, true><<<nleaves, far_threads(c.k), sm, s>>>(g, t, c, rule, leaves, ct, (double*)B);
        } else {
            auto [ct, sm] = go(k_leaf_basis<double, false>, sizeof(double));
            k_leaf_basis<double, false><<<nleaves, far_threads(c.k), sm, s>>>(g, t, c, rule, leaves, ct, (double*)B);
        }
    }
}

template <typename TB, typename TA, int NR>
static void leaf_st(bool fwd, const Tree& t, int k, int maxR, int nl, const int* leaves, const void* B,
                    const double* xp, void* xh, const void* yh, double* yp, cudaStream_t s) {
    if constexpr (std::is_same_v<TB, float> && std::is_same_v<TA, float> && NR % 4 == 0) {
        auto warps = [](int th) { return ((th + 31) / 32) * 32; };
        if (fwd) {
            const int th = warps(((k + 1) / 2) * (NR / 4));
            const size_t smem = (((size_t)maxR * k * 4 + 15) & ~size_t(15)) + (size_t)maxR * NR * 4;
            if (th <= 256) {
                cudaFuncSetAttribute(k_leaf_fwd_t4<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                k_leaf_fwd_t4<NR><<<nl, th, smem, s>>>(t, k, leaves, (const float*)B, xp, (float*)xh);
                return;
            }
        } else {
            const int th = warps(maxR * (NR / 4));
            const size_t smem = (((size_t)k * maxR * 4 + 15) & ~size_t(15)) + (size_t)k * NR * 4;
            if (th <= 256) {
                cudaFuncSetAttribute(k_leaf_bwd_t4<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                k_leaf_bwd_t4<NR><<<nl, th, smem, s>>>(t, k, leaves, (const float*)B, (const float*)yh, yp);
                return;
            }
        }
    }
    if (fwd) {
        const size_t smem = (((size_t)maxR * k * sizeof(TB) + 15) & ~size_t(15)) + (size_t)maxR * NR * sizeof(TA);
        cudaFuncSetAttribute(k_leaf_fwd_st<TB, TA, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_leaf_fwd_st<TB, TA, NR><<<nl, 128, smem, s>>>(t, k, leaves, (const TB*)B, xp, (TA*)xh);
    } else {
        const size_t smem = (((size_t)maxR * (k + 1) * sizeof(TB) + 15) & ~size_t(15)) + (size_t)k * NR * sizeof(TA);
        cudaFuncSetAttribute(k_leaf_bwd_st<TB, TA, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_leaf_bwd_st<TB, TA, NR><<<nl, 128, smem, s>>>(t, k, leaves, (const TB*)B, (const TA*)yh, yp);
    }
}

template <int NR>
static void leaf_st_prec(bool fwd, bool basis32, bool v64, const Tree& t, int k, int maxR, int nl, const int* leaves,
                         const void* B, const double* xp, void* xh, const void* yh, double* yp, cudaStream_t s) {
    if (!basis32 && v64) leaf_st<double, double, NR>(fwd, t, k, maxR, nl, leaves, B, xp, xh, yh, yp, s);
    else if (!basis32) leaf_st<double, float, NR>(fwd, t, k, maxR, nl, leaves, B, xp, xh, yh, yp, s);
    else if (v64) leaf_st<float, double, NR>(fwd, t, k, maxR, nl, leaves, B, xp, xh, yh, yp, s);
    else leaf_st<float, float, NR>(fwd, t, k, maxR, nl, leaves, B, xp, xh, yh, yp, s);
}

void launch_leaf_forward_stored(const Tree& t, int k, int max_leaf, int nleaves, const int* leaves, bool basis32,
                                bool xh64, int NR, const void* B, const double* xp, void* xh, cudaStream_t s) {
    if (nleaves <= 0) return;
    H2_NR_SWITCH(NR, (leaf_st_prec<R_>(true, basis32, xh64, t, k, max_leaf, nleaves, leaves, B, xp, xh, nullptr,
                                       nullptr, s)))
}

// x-hat_s += W^T x|_s with an FP64 basis (the per-corner bases of the
// piecewise-linear double layer are summed this way, one corner at a time)
void launch_leaf_forward_stored_acc(const Tree& t, int k, int max_leaf, int nleaves, const int* leaves, bool xh64,
                                    int NR, const double* B, const double* xp, void* xh, cudaStream_t s) {
    if (nleaves <= 0) return;
    auto pick = [&](auto nr) {
        constexpr int R_ = decltype(nr)::value;
        const size_t sb = ((size_t)max_leaf * k * sizeof(double) + 15) & ~size_t(15);
        if (xh64) {
            const size_t smem = sb + (size_t)max_leaf * R_ * sizeof(double);
            cudaFuncSetAttribute(k_leaf_fwd_st<double, double, R_, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            k_leaf_fwd_st<double, double, R_, true><<<nleaves, 128, smem, s>>>(t, k, leaves, B, xp, (double*)xh);
        } else {
            const size_t smem = sb + (size_t)max_leaf * R_ * sizeof(float);
            cudaFuncSetAttribute(k_leaf_fwd_st<double, float, R_, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            k_leaf_fwd_st<double, float, R_, true><<<nleaves, 128, smem, s>>>(t, k, leaves, B, xp, (float*)xh);
        }
    };
    switch (NR) {
        case 1: pick(std::integral_constant<int, 1>{}); break;
        case 4: pick(std::integral_constant<int, 4>{}); break;
        case 8: pick(std::integral_constant<int, 8>{}); break;
        default: pick(std::integral_constant<int, 16>{}); break;
    }
}

void launch_leaf_backward_stored(const Tree& t, int k, int max_leaf, int nleaves, const int* leaves, bool basis32,
                                 bool yh64, int NR, const void* B, const void* yh, double* yp, cudaStream_t s) {
    if (nleaves <= 0) return;
    H2_NR_SWITCH(NR, (leaf_st_prec<R_>(false, basis32, yh64, t, k, max_leaf, nleaves, leaves, B, nullptr, nullptr,
                                       yh, yp, s)))
}

template <typename T, int NR, bool UP, int MM>
static void updown_m(const Tree& t, const Consts& c, int np, const int* parents, void* v, cudaStream_t s) {
    // warp per parent where a warp's arrays are small (8 warps per CTA, at
    // least 3 CTAs per SM); larger blocks (FP64, m = 5, 16 right-hand sides)
    // would leave too few warps per SM and keep the CTA per parent
    constexpr size_t per_warp = sizeof(T) * (2 * 3 * MM * MM + 4 * (size_t)MM * MM * MM * NR);
    if constexpr (std::is_same_v<T, float> && MM == 4 && NR == 8) {
        constexpr int W = 8;
        k_updown_r8<UP><<<(np + W - 1) / W, 32 * W, 0, s>>>(t, np, parents, (float*)v);
        return;
    }
    if constexpr (MM > 0 && per_warp <= 9 * 1024) {
        constexpr int W = 8;
        auto kern = k_updown_w<T, NR, UP, MM>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(W * per_warp));
        kern<<<(np + W - 1) / W, 32 * W, W * per_warp, s>>>(t, c, np, parents, (T*)v);
        return;
    }
    const size_t smem = sizeof(T) * (2 * 3 * kMaxM * kMaxM + 4 * (size_t)c.k * NR);
    if (UP) {
        cudaFuncSetAttribute(k_upward<T, NR, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_upward<T, NR, MM><<<np, 256, smem, s>>>(t, c, parents, (T*)v);
    } else {
        cudaFuncSetAttribute(k_downward<T, NR, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_downward<T, NR, MM><<<np, 256, smem, s>>>(t, c, parents, (T*)v);
    }
}

template <typename T, int NR, bool UP>
static void updown(const Tree& t, const Consts& c, int np, const int* parents, void* v, cudaStream_t s) {
    if (c.m == 4) updown_m<T, NR, UP, 4>(t, c, np, parents, v, s);
    else if (c.m == 5) updown_m<T, NR, UP, 5>(t, c, np, parents, v, s);
    else updown_m<T, NR, UP, 0>(t, c, np, parents, v, s);
}

// Top-of-tree transfer launches (k_up_tree, k_down_top) where a warp's
// arrays are small (as for k_updown_w: 8 warps per CTA within ~72 KB; FP32,
// m = 4, up to 8 right-hand sides).  Larger blocks keep the per-level launches,
// whose CTA-per-parent kernels finish one parent sooner, and the top levels
// are a chain of single parents.
template <typename T, int NR, int MM>
constexpr size_t tree_per_warp() {
    return sizeof(T) * (2 * 3 * MM * MM + 4 * (size_t)MM * MM * MM * NR);
}

template <typename T, int NR, int MM>
static void tree_updown(bool up, const Tree& t, const Consts& c, int n, const int* start, const int* parent,
                        unsigned* cnt, void* v, cudaStream_t s) {
    constexpr int W = 8;
    const size_t smem = W * tree_per_warp<T, NR, MM>();
    if (up) {
        auto kern = k_up_tree<T, NR, MM>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<(n + W - 1) / W, 32 * W, smem, s>>>(t, c, n, start, parent, cnt, (T*)v);
    } else {
        auto kern = k_down_top<T, NR, MM>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<(n + W - 1) / W, 32 * W, smem, s>>>(t, c, n, start, parent, (T*)v);
    }
}

bool launch_tree_updown(bool up, const Tree& t, const Consts& c, int n, const int* start, const int* parent,
                        unsigned* cnt, bool v64, int NR, void* v, cudaStream_t s) {
    if (c.m != 4 || v64 || NR > 8) return false;
    if (n <= 0) return true;
    switch (NR) {
        case 1: tree_updown<float, 1, 4>(up, t, c, n, start, parent, cnt, v, s); break;
        case 4: tree_updown<float, 4, 4>(up, t, c, n, start, parent, cnt, v, s); break;
        default: tree_updown<float, 8, 4>(up, t, c, n, start, parent, cnt, v, s); break;
    }
    return true;
}

void launch_upward(const Tree& t, const Consts& c, int nparents, const int* parents, bool xh64, int NR, void* xh,
                   cudaStream_t s) {
    if (nparents <= 0) return;
    if (!xh64) { H2_NR_SWITCH(NR, (updown<float, R_, true>(t, c, nparents, parents, xh, s))) }
    else { H2_NR_SWITCH(NR, (updown<double, R_, true>(t, c, nparents, parents, xh, s))) }
}

void launch_downward(const Tree& t, const Consts& c, int nparents, const int* parents, bool yh64, int NR, void* yh,
                     cudaStream_t s) {
    if (nparents <= 0) return;
    if (!yh64) { H2_NR_SWITCH(NR, (updown<float, R_, false>(t, c, nparents, parents, yh, s))) }
    else { H2_NR_SWITCH(NR, (updown<double, R_, false>(t, c, nparents, parents, yh, s))) }
}

}  // namespace h2
