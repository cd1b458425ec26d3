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
// are apart, so no pair shares a vertex); stored as T.
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
        for (int e = threadIdx.x; e < rt * rs; e += blockDim.x) {
            const int i = piv[piv_off[t] + e / rs], j = piv[piv_off[s] + e % rs];
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
// row t, one CTA per row; S_b and x-hat_s staged in shared memory, item
// (nu, r) = e of the rank_t x NR outputs per thread e, e + 256, ...
template <typename T, int NR>
__global__ void __launch_bounds__(256) k_gca_coupling(const int* __restrict__ rows, const int* __restrict__ ptr,
                                                      const int* __restrict__ col, const int* __restrict__ rank,
                                                      const int64_t* __restrict__ soff, const T* __restrict__ S,
                                                      int K, const T* __restrict__ xh, T* __restrict__ yh) {
    constexpr int J = (kGcaMaxRank * NR + 255) / 256;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sS = reinterpret_cast<T*>(smem_raw);                                  // [rank_t][rank_s]
    T* sx = reinterpret_cast<T*>(smem_raw + sizeof(T) * kGcaMaxRank * kGcaMaxRank);  // [rank_s][NR]
    const int t = rows[blockIdx.x];
    const int rt = rank[t];
    const int tid = threadIdx.x;
    T acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = 0;
    for (int b = ptr[blockIdx.x]; b < ptr[blockIdx.x + 1]; ++b) {
        const int s = col[b], rs = rank[s];
        __syncthreads();
        const T* Sb = S + soff[b];
        for (int e = tid; e < rt * rs; e += blockDim.x) sS[e] = Sb[e];
        for (int e = tid; e < rs * NR; e += blockDim.x) sx[e] = xh[(int64_t)s * K * NR + e];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int e = tid + 256 * j;
            if (e < rt * NR) {
                const int nu = e / NR, r = e % NR;
                const T* Srow = sS + nu * rs;
                T sum = 0;
                for (int mu = 0; mu < rs; ++mu) sum += Srow[mu] * sx[mu * NR + r];
                acc[j] += sum;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int e = tid + 256 * j;
        if (e < rt * NR) yh[(int64_t)t * K * NR + e] = acc[j];
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
    const size_t smem = sizeof(T) * ((size_t)kGcaMaxRank * kGcaMaxRank + (size_t)kGcaMaxRank * NR);
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
