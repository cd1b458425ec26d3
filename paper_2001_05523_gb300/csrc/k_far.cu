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
#include <type_traits>

#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;

template <typename T>
__device__ __forceinline__ T rsq(T x);
template <>
__device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }
template <>
__device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }

// nodes of cluster c along every axis: z[d*m + a]
__device__ __forceinline__ void cluster_nodes(const Tree& t, const Consts& c, int cl, double* z) {
    for (int e = threadIdx.x; e < 3 * c.m; e += blockDim.x) {
        const int d = e / c.m, a = e % c.m;
        z[e] = t.box[d * t.nc + cl] + t.box[(3 + d) * t.nc + cl] * c.cheb[a];
    }
}

__device__ __forceinline__ double lagrange(const double* z, int m, int a, double y) {
    double p = 1.0;
    for (int k = 0; k < m; ++k)
        if (k != a) p *= (y - z[k]) / (z[a] - z[k]);
    return p;
}
__device__ __forceinline__ double lagrange_d(const double* z, int m, int a, double y) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) {
        if (k == a) continue;
        double p = 1.0 / (z[a] - z[k]);
        for (int l = 0; l < m; ++l)
            if (l != a && l != k) p *= (y - z[l]) / (z[a] - z[l]);
        s += p;
    }
    return s;
}
}  // namespace

// ---------------------------------------------------------------------------
// Leaf transforms.  rule: nb points (u, v, w) on the unit simplex, exact for
// total degree 3(m-1), weights summing to 1.  One CTA per leaf.
// Shared: L[p][d][a] (and dL) for the current triangle's points.
// ---------------------------------------------------------------------------
template <typename T, int NR, bool DLPB>
__global__ void __launch_bounds__(256) k_leaf_forward(Geom g, Tree t, Consts c, const double* __restrict__ rule,
                                                      const int* __restrict__ leaves, const double* __restrict__ xp,
                                                      T* __restrict__ xh) {
    __shared__ double z[3 * kMaxM];
    __shared__ T L[kMaxBasisPts * 3 * kMaxM];
    __shared__ T dL[DLPB ? kMaxBasisPts * 3 * kMaxM : 1];
    const int s = leaves[blockIdx.x];
    const int b = t.begin[s], R = t.end[s] - b;
    const int m = c.m, k = c.k, nb = c.nb, n = g.n;
    cluster_nodes(t, c, s, z);
    constexpr int kPer = (kMaxK + 63) / 64;  // nu per thread at blockDim >= 64
    T acc[kPer][NR];
#pragma unroll
    for (int q = 0; q < kPer; ++q)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[q][r] = 0;
    for (int jl = 0; jl < R; ++jl) {
        const int j = b + jl;
        __syncthreads();
        for (int e = threadIdx.x; e < nb * 3 * m; e += blockDim.x) {
            const int p = e / (3 * m), d = (e / m) % 3, a = e % m;
            const double v0 = g.v[d * n + j], v1 = g.v[(3 + d) * n + j], v2 = g.v[(6 + d) * n + j];
            const double y = v0 + rule[3 * p] * (v1 - v0) + rule[3 * p + 1] * (v2 - v0);
            L[e] = (T)lagrange(z + d * m, m, a, y);
            if (DLPB) dL[e] = (T)lagrange_d(z + d * m, m, a, y);
        }
        __syncthreads();
        const double aj = g.area[j];
        T nx = 0, ny = 0, nz = 0;
        if (DLPB) {
            nx = (T)g.nrm[j];
            ny = (T)g.nrm[n + j];
            nz = (T)g.nrm[2 * n + j];
        }
        T xj[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) xj[r] = (T)xp[(int64_t)j * NR + r];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int nu = threadIdx.x + q * blockDim.x;
            if (nu >= k) break;
            const int ia = nu % m, ib = (nu / m) % m, ic = nu / (m * m);
            T sum = 0;
            for (int p = 0; p < nb; ++p) {
                const T* Lp = L + p * 3 * m;
                const T w = (T)rule[3 * p + 2];
                if (DLPB) {
                    const T* dLp = dL + p * 3 * m;
                    const T lx = Lp[ia], ly = Lp[m + ib], lz = Lp[2 * m + ic];
                    sum += w * (nx * dLp[ia] * ly * lz + ny * lx * dLp[m + ib] * lz + nz * lx * ly * dLp[2 * m + ic]);
                } else {
                    sum += w * Lp[ia] * Lp[m + ib] * Lp[2 * m + ic];
                }
            }
            sum *= (T)aj;
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[q][r] += sum * xj[r];
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

template <typename T, int NR, bool DLPB>
__global__ void __launch_bounds__(256) k_leaf_backward(Geom g, Tree t, Consts c, const double* __restrict__ rule,
                                                       const int* __restrict__ leaves, const T* __restrict__ yh,
                                                       double* __restrict__ yp) {
    __shared__ double z[3 * kMaxM];
    __shared__ T L[kMaxBasisPts * 3 * kMaxM];
    __shared__ T dL[DLPB ? kMaxBasisPts * 3 * kMaxM : 1];
    __shared__ T red[8][NR];
    const int s = leaves[blockIdx.x];
    const int b = t.begin[s], R = t.end[s] - b;
    const int m = c.m, k = c.k, nb = c.nb, n = g.n;
    cluster_nodes(t, c, s, z);
    constexpr int kPer = (kMaxK + 63) / 64;
    T yv[kPer][NR];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int nu = threadIdx.x + q * blockDim.x;
#pragma unroll
        for (int r = 0; r < NR; ++r) yv[q][r] = nu < k ? yh[((int64_t)s * k + nu) * NR + r] : (T)0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int il = 0; il < R; ++il) {
        const int i = b + il;
        __syncthreads();
        for (int e = threadIdx.x; e < nb * 3 * m; e += blockDim.x) {
            const int p = e / (3 * m), d = (e / m) % 3, a = e % m;
            const double v0 = g.v[d * n + i], v1 = g.v[(3 + d) * n + i], v2 = g.v[(6 + d) * n + i];
            const double y = v0 + rule[3 * p] * (v1 - v0) + rule[3 * p + 1] * (v2 - v0);
            L[e] = (T)lagrange(z + d * m, m, a, y);
            if (DLPB) dL[e] = (T)lagrange_d(z + d * m, m, a, y);
        }
        __syncthreads();
        T nx = 0, ny = 0, nz = 0;
        if (DLPB) {
            nx = (T)g.nrm[i];
            ny = (T)g.nrm[n + i];
            nz = (T)g.nrm[2 * n + i];
        }
        T part[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) part[r] = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int nu = threadIdx.x + q * blockDim.x;
            if (nu >= k) break;
            const int ia = nu % m, ib = (nu / m) % m, ic = nu / (m * m);
            T sum = 0;
            for (int p = 0; p < nb; ++p) {
                const T* Lp = L + p * 3 * m;
                const T w = (T)rule[3 * p + 2];
                if (DLPB) {
                    const T* dLp = dL + p * 3 * m;
                    const T lx = Lp[ia], ly = Lp[m + ib], lz = Lp[2 * m + ic];
                    sum += w * (nx * dLp[ia] * ly * lz + ny * lx * dLp[m + ib] * lz + nz * lx * ly * dLp[2 * m + ic]);
                } else {
                    sum += w * Lp[ia] * Lp[m + ib] * Lp[2 * m + ic];
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) part[r] += sum * yv[q][r];
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            T v = part[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][r] = v;
        }
        __syncthreads();
        if (threadIdx.x < NR) {
            T v = 0;
            for (int w = 0; w < nwarps; ++w) v += red[w][threadIdx.x];
            yp[(int64_t)i * NR + threadIdx.x] += g.area[i] * (double)v;
        }
    }
}

// ---------------------------------------------------------------------------
// Transfers between a parent t and its children (Kronecker form).
// E1[ch][d][a'][a] = L_{t,a}^{(d)}(z_{ch,d}[a']).
// ---------------------------------------------------------------------------
template <typename T>
__device__ void transfer_1d(const Tree& t, const Consts& c, int parent, const int* ch, T* E1, double* zp,
                            double* zc) {
    const int m = c.m;
    cluster_nodes(t, c, parent, zp);
    for (int q = 0; q < 2; ++q) cluster_nodes(t, c, ch[q], zc + q * 3 * m);
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * 3 * m * m; e += blockDim.x) {
        const int q = e / (3 * m * m), d = (e / (m * m)) % 3, ap = (e / m) % m, a = e % m;
        E1[e] = (T)lagrange(zp + d * m, m, a, zc[q * 3 * m + d * m + ap]);
    }
    __syncthreads();
}

// up: X[a',b',c'] -> out[a,b,c] = sum E_x[a'][a] E_y[b'][b] E_z[c'][c] X
// down: Y[a,b,c] -> out[a',b',c'] = sum E_x[a'][a] E_y[b'][b] E_z[c'][c] Y
template <typename T, int NR, bool UP>
__device__ void kron_apply(const T* E1, int m, const T* in, T* tmp1, T* tmp2, T* out, bool accumulate) {
    const int k = m * m * m;
    const T* Ex = E1;
    const T* Ey = E1 + m * m;
    const T* Ez = E1 + 2 * m * m;
    // contract x
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) {
        const int r = e % NR, nu = e / NR, a = nu % m, rest = nu / m;
        T s = 0;
        for (int q = 0; q < m; ++q) s += (UP ? Ex[q * m + a] : Ex[a * m + q]) * in[((rest * m) + q) * NR + r];
        tmp1[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) {
        const int r = e % NR, nu = e / NR, a = nu % m, b = (nu / m) % m, cc = nu / (m * m);
        T s = 0;
        for (int q = 0; q < m; ++q)
            s += (UP ? Ey[q * m + b] : Ey[b * m + q]) * tmp1[((cc * m + q) * m + a) * NR + r];
        tmp2[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) {
        const int r = e % NR, nu = e / NR, ab = nu % (m * m), cc = nu / (m * m);
        T s = 0;
        for (int q = 0; q < m; ++q) s += (UP ? Ez[q * m + cc] : Ez[cc * m + q]) * tmp2[((q * m * m) + ab) * NR + r];
        if (accumulate) out[e] += s;
        else out[e] = s;
    }
    __syncthreads();
}

template <typename T, int NR>
__global__ void __launch_bounds__(256) k_upward(Tree t, Consts c, const int* __restrict__ parents, T* __restrict__ xh) {
    extern __shared__ unsigned char smem_raw[];
    T* E1 = reinterpret_cast<T*>(smem_raw);
    T* buf = E1 + 2 * 3 * kMaxM * kMaxM;
    const int k = c.k;
    T* in = buf;
    T* tmp1 = in + k * NR;
    T* tmp2 = tmp1 + k * NR;
    T* out = tmp2 + k * NR;
    __shared__ double zp[3 * kMaxM], zc[2 * 3 * kMaxM];
    const int p = parents[blockIdx.x];
    const int ch[2] = {t.child0[p], t.child1[p]};
    transfer_1d<T>(t, c, p, ch, E1, zp, zc);
    for (int q = 0; q < 2; ++q) {
        for (int e = threadIdx.x; e < k * NR; e += blockDim.x) in[e] = xh[(int64_t)ch[q] * k * NR + e];
        __syncthreads();
        kron_apply<T, NR, true>(E1 + q * 3 * c.m * c.m, c.m, in, tmp1, tmp2, out, q == 1);
    }
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) xh[(int64_t)p * k * NR + e] = out[e];
}

template <typename T, int NR>
__global__ void __launch_bounds__(256) k_downward(Tree t, Consts c, const int* __restrict__ parents,
                                                  T* __restrict__ yh) {
    extern __shared__ unsigned char smem_raw[];
    T* E1 = reinterpret_cast<T*>(smem_raw);
    T* buf = E1 + 2 * 3 * kMaxM * kMaxM;
    const int k = c.k;
    T* in = buf;
    T* tmp1 = in + k * NR;
    T* tmp2 = tmp1 + k * NR;
    T* out = tmp2 + k * NR;
    __shared__ double zp[3 * kMaxM], zc[2 * 3 * kMaxM];
    const int p = parents[blockIdx.x];
    const int ch[2] = {t.child0[p], t.child1[p]};
    transfer_1d<T>(t, c, p, ch, E1, zp, zc);
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) in[e] = yh[(int64_t)p * k * NR + e];
    __syncthreads();
    for (int q = 0; q < 2; ++q) {
        kron_apply<T, NR, false>(E1 + q * 3 * c.m * c.m, c.m, in, tmp1, tmp2, out, false);
        for (int e = threadIdx.x; e < k * NR; e += blockDim.x) yh[(int64_t)ch[q] * k * NR + e] += out[e];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Coupling, SIMT: one CTA per row cluster, S_ts generated on the fly from
// per-axis squared node differences.  Thread (nu, slice) sums over the mu of
// its slice; slices are reduced in shared memory at the end.
// ---------------------------------------------------------------------------
template <typename T, int NR>
__global__ void __launch_bounds__(256) k_coupling_simt(Tree t, Consts c, const int* __restrict__ rows,
                                                       const int* __restrict__ ptr, const int* __restrict__ col,
                                                       const T* __restrict__ xh, T* __restrict__ yh) {
    extern __shared__ unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);  // [k][NR], reused for the reduction [256][NR]
    __shared__ double zt[3 * kMaxM], zs[3 * kMaxM];
    __shared__ T D2[3 * kMaxM * kMaxM];
    const int row = rows[blockIdx.x];
    const int m = c.m, k = c.k;
    const int nslice = blockDim.x / k;
    const int nu = threadIdx.x % k, sl = threadIdx.x / k;
    const bool active = sl < nslice;
    const int ia = nu % m, ib = (nu / m) % m, ic = nu / (m * m);
    cluster_nodes(t, c, row, zt);
    T acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0;
    for (int b = ptr[blockIdx.x]; b < ptr[blockIdx.x + 1]; ++b) {
        const int s = col[b];
        __syncthreads();
        cluster_nodes(t, c, s, zs);
        for (int e = threadIdx.x; e < k * NR; e += blockDim.x) xs[e] = xh[(int64_t)s * k * NR + e];
        __syncthreads();
        for (int e = threadIdx.x; e < 3 * m * m; e += blockDim.x) {
            const int d = e / (m * m), a = (e / m) % m, a2 = e % m;
            const double df = zt[d * m + a] - zs[d * m + a2];
            D2[e] = (T)(df * df);
        }
        __syncthreads();
        if (active) {
            const T* Dx = D2 + ia * m;
            const T* Dy = D2 + m * m + ib * m;
            const T* Dz = D2 + 2 * m * m + ic * m;
            for (int mu = sl; mu < k; mu += nslice) {
                const int ja = mu % m, jb = (mu / m) % m, jc = mu / (m * m);
                const T sv = rsq<T>(Dx[ja] + Dy[jb] + Dz[jc]);
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[r] += sv * xs[mu * NR + r];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; ++r) xs[threadIdx.x * NR + r] = active ? acc[r] : (T)0;
    __syncthreads();
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) {
        const int v = e / NR, r = e % NR;
        T s = 0;
        for (int q = 0; q < nslice; ++q) s += xs[(q * k + v) * NR + r];
        yh[(int64_t)row * k * NR + e] = s * (T)kInv4Pi;
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

template <typename T, int NR>
static void leaf_fwd(bool dlpb, const Geom& g, const Tree& t, const Consts& c, const double* rule, int nl,
                     const int* leaves, const double* xp, void* xh, cudaStream_t s) {
    if (dlpb) k_leaf_forward<T, NR, true><<<nl, far_threads(c.k), 0, s>>>(g, t, c, rule, leaves, xp, (T*)xh);
    else k_leaf_forward<T, NR, false><<<nl, far_threads(c.k), 0, s>>>(g, t, c, rule, leaves, xp, (T*)xh);
}
template <typename T, int NR>
static void leaf_bwd(bool dlpb, const Geom& g, const Tree& t, const Consts& c, const double* rule, int nl,
                     const int* leaves, const void* yh, double* yp, cudaStream_t s) {
    if (dlpb) k_leaf_backward<T, NR, true><<<nl, far_threads(c.k), 0, s>>>(g, t, c, rule, leaves, (const T*)yh, yp);
    else k_leaf_backward<T, NR, false><<<nl, far_threads(c.k), 0, s>>>(g, t, c, rule, leaves, (const T*)yh, yp);
}

#define H2_NR_SWITCH(NR, CALL)          \
    switch (NR) {                       \
        case 1: { constexpr int R_ = 1; CALL; } break;  \
        case 4: { constexpr int R_ = 4; CALL; } break;  \
        case 8: { constexpr int R_ = 8; CALL; } break;  \
        default: { constexpr int R_ = 16; CALL; } break; \
    }

void launch_leaf_forward(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nleaves,
                         const int* leaves, bool dlp_basis, bool fp32, int NR, const double* xp, void* xh,
                         cudaStream_t s) {
    if (nleaves <= 0) return;
    if (fp32) { H2_NR_SWITCH(NR, (leaf_fwd<float, R_>(dlp_basis, g, t, c, rule, nleaves, leaves, xp, xh, s))) }
    else { H2_NR_SWITCH(NR, (leaf_fwd<double, R_>(dlp_basis, g, t, c, rule, nleaves, leaves, xp, xh, s))) }
}

void launch_leaf_backward(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nleaves,
                          const int* leaves, bool dlp_basis, bool fp32, int NR, const void* yh, double* yp,
                          cudaStream_t s) {
    if (nleaves <= 0) return;
    if (fp32) { H2_NR_SWITCH(NR, (leaf_bwd<float, R_>(dlp_basis, g, t, c, rule, nleaves, leaves, yh, yp, s))) }
    else { H2_NR_SWITCH(NR, (leaf_bwd<double, R_>(dlp_basis, g, t, c, rule, nleaves, leaves, yh, yp, s))) }
}

template <typename T, int NR, bool UP>
static void updown(const Tree& t, const Consts& c, int np, const int* parents, void* v, cudaStream_t s) {
    const size_t smem = sizeof(T) * (2 * 3 * kMaxM * kMaxM + 4 * (size_t)c.k * NR);
    if (UP) {
        cudaFuncSetAttribute(k_upward<T, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_upward<T, NR><<<np, 256, smem, s>>>(t, c, parents, (T*)v);
    } else {
        cudaFuncSetAttribute(k_downward<T, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_downward<T, NR><<<np, 256, smem, s>>>(t, c, parents, (T*)v);
    }
}

void launch_upward(const Tree& t, const Consts& c, int nparents, const int* parents, bool fp32, int NR, void* xh,
                   cudaStream_t s) {
    if (nparents <= 0) return;
    if (fp32) { H2_NR_SWITCH(NR, (updown<float, R_, true>(t, c, nparents, parents, xh, s))) }
    else { H2_NR_SWITCH(NR, (updown<double, R_, true>(t, c, nparents, parents, xh, s))) }
}

void launch_downward(const Tree& t, const Consts& c, int nparents, const int* parents, bool fp32, int NR, void* yh,
                     cudaStream_t s) {
    if (nparents <= 0) return;
    if (fp32) { H2_NR_SWITCH(NR, (updown<float, R_, false>(t, c, nparents, parents, yh, s))) }
    else { H2_NR_SWITCH(NR, (updown<double, R_, false>(t, c, nparents, parents, yh, s))) }
}

template <typename T, int NR>
static void coupling_simt(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                          const void* xh, void* yh, cudaStream_t s) {
    const size_t smem = sizeof(T) * (size_t)(256 > c.k ? 256 : c.k) * NR;
    cudaFuncSetAttribute(k_coupling_simt<T, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_coupling_simt<T, NR><<<nrows, 256, smem, s>>>(t, c, rows, ptr, col, (const T*)xh, (T*)yh);
}

void launch_coupling(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                     int precision, int NR, const void* xh, void* yh, cudaStream_t s) {
    if (nrows <= 0) return;
    if (precision == 0) { H2_NR_SWITCH(NR, (coupling_simt<double, R_>(t, c, nrows, rows, ptr, col, xh, yh, s))) }
    else { H2_NR_SWITCH(NR, (coupling_simt<float, R_>(t, c, nrows, rows, ptr, col, xh, yh, s))) }
}

}  // namespace h2
