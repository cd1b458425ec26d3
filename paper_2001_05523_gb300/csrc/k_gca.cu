// Farfield of the H^2 product with Green-cross-approximation cluster bases
// (section 4; the bases are built on the host in gca.cpp):
//   x-hat_s = V_s^T x|_s at the leaves (the stored-basis leaf kernels of
//   k_far.cu, bases zero-padded to K columns), x-hat_t = sum_t' E_t'^T
//   x-hat_t' upward, y-hat_t = sum_s S_ts x-hat_s with the stored coupling
//   matrices S_ts = G|_{t^ x s^} (Galerkin entries of the pivot triangles),
//   y-hat_t' += E_t' y-hat_t downward, y|_t += V_t y-hat_t at the leaves.
// Ranks differ per cluster: E_c (rank_c x rank_parent) and S_b (rank_t x
// rank_s) are stored compactly, row-major, at per-cluster / per-block
// offsets.  Cluster vectors keep K >= every rank entries per cluster; the
// entries beyond a cluster's rank are never read.
#include <algorithm>

#include "dmath.cuh"
#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;
}

// S_b[a][c] = int_{tau_i} int_{tau_j} g for the pivot triangles i = t^[a],
// j = s^[c] of every farfield block b = (t, s): the 7 x 7-point rule of the
// nearfield's regular pairs, in FP64 (pivot triangles of admissible clusters
// are apart, so no pair shares a vertex); stored as T, column by column
// (S_b[a][c] at c rank_t + a), so that the lanes of a warp owning rows a read
// a column in one coalesced access.
template <typename T>
__global__ void __launch_bounds__(256) k_gca_assemble(Geom g, Consts c, const int* __restrict__ rows,
                                                      const int* __restrict__ ptr, const int* __restrict__ col,
                                                      const int* __restrict__ rank, const int* __restrict__ piv_off,
                                                      const int* __restrict__ piv, const int64_t* __restrict__ soff,
                                                      T* __restrict__ S) {
    const int t = rows[blockIdx.x];
    const int rt = rank[t];
    const int n = g.n;
    for (int b = ptr[blockIdx.x]; b < ptr[blockIdx.x + 1]; ++b) {
        const int s = col[b], rs = rank[s];
        for (int e = threadIdx.x; e < rt * rs; e += blockDim.x) {  // column-major: e = c rt + a
            const int i = piv[piv_off[t] + e % rt], j = piv[piv_off[s] + e / rt];
            double yq[3][7];
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int q = 0; q < 7; ++q) yq[d][q] = g.qa[((int64_t)d * n + j) * 7 + q];
            double sum = 0.0;
#pragma unroll
            for (int p = 0; p < 7; ++p) {
                const double x0 = g.qa[((int64_t)0 * n + i) * 7 + p], x1 = g.qa[((int64_t)1 * n + i) * 7 + p],
                             x2 = g.qa[((int64_t)2 * n + i) * 7 + p];
                double sp = 0.0;
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    const double dx = x0 - yq[0][q], dy = x1 - yq[1][q], dz = x2 - yq[2][q];
                    sp = fma(c.rw[q], rsqrt_nr(fma(dz, dz, fma(dy, dy, dx * dx))), sp);
                }
                sum = fma(c.rw[p], sp, sum);
            }
            S[soff[b] + e] = (T)(sum * g.area[i] * g.area[j] * kInv4Pi);
        }
    }
}

// Upward (UP) or downward pass over the parents of one tree level, one CTA per
// parent p, thread nu for the entries of x-hat_p (upward) or of y-hat_c of a
// child (downward).
template <typename T, int NR, bool UP>
__global__ void __launch_bounds__(128) k_gca_updown(const int* __restrict__ parents, const int* __restrict__ child0,
                                                    const int* __restrict__ child1, const int* __restrict__ rank,
                                                    const int64_t* __restrict__ eoff, const T* __restrict__ E, int K,
                                                    T* __restrict__ v) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sv = reinterpret_cast<T*>(smem_raw);  // [K][NR]
    const int p = parents[blockIdx.x];
    const int kp = rank[p];
    const int ch[2] = {child0[p], child1[p]};
    const int tid = threadIdx.x;
    if constexpr (UP) {
        T acc[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = 0;
        for (int h = 0; h < 2; ++h) {
            const int cc = ch[h], kc = rank[cc];
            __syncthreads();
            for (int e = tid; e < kc * NR; e += blockDim.x) sv[e] = v[(int64_t)cc * K * NR + e];
            __syncthreads();
            if (tid < kp) {
                const T* Ec = E + eoff[cc];
                for (int a = 0; a < kc; ++a) {
                    const T w = Ec[(int64_t)a * kp + tid];
#pragma unroll
                    for (int r = 0; r < NR; ++r) acc[r] += w * sv[a * NR + r];
                }
            }
        }
        if (tid < kp)
#pragma unroll
            for (int r = 0; r < NR; ++r) v[((int64_t)p * K + tid) * NR + r] = acc[r];
    } else {
        for (int e = tid; e < kp * NR; e += blockDim.x) sv[e] = v[(int64_t)p * K * NR + e];
        __syncthreads();
        for (int h = 0; h < 2; ++h) {
            const int cc = ch[h], kc = rank[cc];
            if (tid < kc) {
                const T* Ec = E + eoff[cc] + (int64_t)tid * kp;
                T acc[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[r] = 0;
                for (int a = 0; a < kp; ++a) {
                    const T w = Ec[a];
#pragma unroll
                    for (int r = 0; r < NR; ++r) acc[r] += w * sv[a * NR + r];
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) v[((int64_t)cc * K + tid) * NR + r] += acc[r];
            }
        }
    }
}

// Coupling: y-hat_t = sum_b S_b x-hat_s over the farfield blocks b = (t, s) of
// row t, one CTA per row.  The blocks' S_b (stored column-major, each at a
// 16-byte aligned offset) and x-hat_s stream through a ring of NST shared-
// memory stages filled by 16-byte cp.async copies, NST - 1 blocks ahead of
// the one being multiplied, so that the HBM reads of later blocks overlap the
// products.  Output item (a, r) = e of the rank_t x NR entries per thread
// e, e + 256, ...
namespace {
// NR consecutive values of a cluster vector row, by 16-byte loads
template <typename T, int NR>
struct XRow {
    static __device__ __forceinline__ void load(const T* p, T* v) {
        constexpr int W = 16 / (int)sizeof(T);
        if constexpr (NR % W == 0) {
#pragma unroll
            for (int r = 0; r < NR; r += W) {
                if constexpr (W == 4) {
                    const float4 q = *reinterpret_cast<const float4*>(p + r);
                    v[r] = q.x, v[r + 1] = q.y, v[r + 2] = q.z, v[r + 3] = q.w;
                } else {
                    const double2 q = *reinterpret_cast<const double2*>(p + r);
                    v[r] = q.x, v[r + 1] = q.y;
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < NR; ++r) v[r] = p[r];
        }
    }
};
template <typename T>
struct GcaStages {
    static constexpr int NST = sizeof(T) == 4 ? 3 : 2;              // ring depth
    static constexpr int V = 16 / (int)sizeof(T);                   // elements per 16-byte copy
    static constexpr int SMAX = kGcaMaxRank * kGcaMaxRank;          // S_b
    template <int NR>
    static constexpr int xmax() { return (kGcaMaxRank * NR + V - 1) / V * V; }
    template <int NR>
    static constexpr size_t bytes() { return sizeof(T) * (size_t)NST * (SMAX + xmax<NR>()); }
};
__device__ __forceinline__ void cpa16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
}  // namespace

template <typename T, int NR>
__global__ void __launch_bounds__(256) k_gca_coupling(const int* __restrict__ rows, const int* __restrict__ ptr,
                                                      const int* __restrict__ col, const int* __restrict__ rank,
                                                      const int64_t* __restrict__ soff, const T* __restrict__ S,
                                                      int K, const T* __restrict__ xh, T* __restrict__ yh) {
    using G = GcaStages<T>;
    constexpr int NST = G::NST, V = G::V, SMAX = G::SMAX, XMAX = G::template xmax<NR>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ring = reinterpret_cast<T*>(smem_raw);  // NST x (S_b [SMAX], x-hat_s [XMAX])
    const int t = rows[blockIdx.x];
    const int rt = rank[t];
    const int tid = threadIdx.x;
    // thread (a, g): output row a of y-hat_t for every right-hand side, over
    // the columns mu = g, g + NG, ... of each block
    const int NG = 256 / max(rt, 1);
    const int a = tid % max(rt, 1), g = tid / max(rt, 1);
    const bool active = g < NG && rt > 0;
    const int b0 = ptr[blockIdx.x], nb = ptr[blockIdx.x + 1] - b0;
    auto issue = [&](int j) {
        const int b = b0 + j, s = col[b], rs = rank[s];
        T* st = ring + (size_t)(j % NST) * (SMAX + XMAX);
        const T* Sb = S + soff[b];
        const T* xs = xh + (int64_t)s * K * NR;
        const int nS = (rt * rs + V - 1) / V, nX = (rs * NR + V - 1) / V;
        for (int e = tid; e < nS; e += 256) cpa16(st + e * V, Sb + e * V);
        for (int e = tid; e < nX; e += 256) cpa16(st + SMAX + e * V, xs + e * V);
    };
#pragma unroll
    for (int j = 0; j < NST - 1; ++j) {
        if (j < nb) issue(j);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    T acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0;
    for (int j = 0; j < nb; ++j) {
        if (j + NST - 1 < nb) issue(j + NST - 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group %0;" ::"n"(NST - 1) : "memory");
        __syncthreads();
        const T* sS = ring + (size_t)(j % NST) * (SMAX + XMAX);
        const T* sx = sS + SMAX;
        const int rs = rank[col[b0 + j]];
        if (active)
            for (int mu = g; mu < rs; mu += NG) {
                const T sv = sS[mu * rt + a];
                T xv[NR];
                XRow<T, NR>::load(sx + mu * NR, xv);
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[r] += sv * xv[r];
            }
        __syncthreads();  // the stage is refilled NST - 1 blocks later
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // sum over the column slices g (the ring is free now)
    T* red = ring;  // [NG][rt][NR]
    if (active)
#pragma unroll
        for (int r = 0; r < NR; ++r) red[((size_t)g * rt + a) * NR + r] = acc[r];
    __syncthreads();
    for (int e = tid; e < rt * NR; e += 256) {
        T sum = 0;
        for (int q = 0; q < NG; ++q) sum += red[(size_t)q * rt * NR + e];
        yh[(int64_t)t * K * NR + e] = sum;
    }
}

#define GCA_NR_SWITCH(NR, CALL)                          \
    switch (NR) {                                        \
        case 1: { constexpr int R_ = 1; CALL; } break;   \
        case 4: { constexpr int R_ = 4; CALL; } break;   \
        case 8: { constexpr int R_ = 8; CALL; } break;   \
        default: { constexpr int R_ = 16; CALL; } break; \
    }

void launch_gca_assemble(const Geom& g, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                         const int* rank, const int* piv_off, const int* piv, const int64_t* soff, bool f32, void* S,
                         cudaStream_t s) {
    if (nrows <= 0) return;
    if (f32)
        k_gca_assemble<float><<<nrows, 256, 0, s>>>(g, c, rows, ptr, col, rank, piv_off, piv, soff, (float*)S);
    else
        k_gca_assemble<double><<<nrows, 256, 0, s>>>(g, c, rows, ptr, col, rank, piv_off, piv, soff, (double*)S);
}

template <typename T, int NR, bool UP>
static void updown_go(int np, const int* parents, const int* c0, const int* c1, const int* rank,
                      const int64_t* eoff, const void* E, int K, void* v, cudaStream_t s) {
    const size_t smem = sizeof(T) * (size_t)K * NR;
    k_gca_updown<T, NR, UP><<<np, 128, smem, s>>>(parents, c0, c1, rank, eoff, (const T*)E, K, (T*)v);
}

void launch_gca_updown(bool up, bool f32, int NR, int np, const int* parents, const int* child0, const int* child1,
                       const int* rank, const int64_t* eoff, const void* E, int K, void* v, cudaStream_t s) {
    if (np <= 0) return;
    if (f32) {
        if (up) { GCA_NR_SWITCH(NR, (updown_go<float, R_, true>(np, parents, child0, child1, rank, eoff, E, K, v, s))) }
        else { GCA_NR_SWITCH(NR, (updown_go<float, R_, false>(np, parents, child0, child1, rank, eoff, E, K, v, s))) }
    } else {
        if (up) { GCA_NR_SWITCH(NR, (updown_go<double, R_, true>(np, parents, child0, child1, rank, eoff, E, K, v, s))) }
        else { GCA_NR_SWITCH(NR, (updown_go<double, R_, false>(np, parents, child0, child1, rank, eoff, E, K, v, s))) }
    }
}

template <typename T, int NR>
static void coupling_go(int nrows, const int* rows, const int* ptr, const int* col, const int* rank,
                        const int64_t* soff, const void* S, int K, const void* xh, void* yh, cudaStream_t s) {
    constexpr size_t smem = GcaStages<T>::template bytes<NR>();
    cudaFuncSetAttribute(k_gca_coupling<T, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gca_coupling<T, NR><<<nrows, 256, smem, s>>>(rows, ptr, col, rank, soff, (const T*)S, K, (const T*)xh, (T*)yh);
}

void launch_gca_coupling(bool f32, int NR, int nrows, const int* rows, const int* ptr, const int* col,
                         const int* rank, const int64_t* soff, const void* S, int K, const void* xh, void* yh,
                         cudaStream_t s) {
    if (nrows <= 0) return;
    if (f32) { GCA_NR_SWITCH(NR, (coupling_go<float, R_>(nrows, rows, ptr, col, rank, soff, S, K, xh, yh, s))) }
    else { GCA_NR_SWITCH(NR, (coupling_go<double, R_>(nrows, rows, ptr, col, rank, soff, S, K, xh, yh, s))) }
}

}  // namespace h2
