// Stored nearfield (section 2: the nearfield blocks N_ts = A|_{t x s} of the
// leaves L^-, entries of section 1, eq. (slp) / eq. (dlp)).  The entries of
// every ordered nearfield block (t, s) are evaluated once at set-up (regular
// pairs by the nearfield kernel in its storing variant, Sauter-Schwab pairs
// scattered in afterwards) and every apply only streams them from HBM:
//   y|_t = sum_{s : (t, s) nearfield} N_ts x|_s          (A x)
//   y|_t = sum_{s : (s, t) nearfield} N_st^T x|_s        (A^T x, double layer)
// (the first stage of the apply; the farfield is added to y afterwards).
//
// Storage: block (t, s) holds |t| x |s| values (FP32 in the mixed tiers, FP64
// in the FP64 tier) column by column with the odd leading dimension
// ld = |t| | 1, and starts on a 16-byte boundary.  Lane i of a warp reads
// entry (i, j) at j ld + i (consecutive), and entry (j, i) of a transposed
// block at i ld' + j (stride ld' odd): neither access has bank conflicts.
//
// Apply: one CTA per row leaf t; warp w takes the blocks w, w + W, ... of the
// row.  Each block and its x|_s rows go to shared memory by cp.async (16-byte
// copies), two stages per warp so the next block is in flight while the
// current one is multiplied; a lane owns several rows and a chunk of the
// columns (LaneMap), sums in the working precision.  The column partials
// meet by shuffles and the warps' partials in shared memory, and row t of y
// is updated in FP64 without atomics (no other CTA writes it), so the result
// does not depend on scheduling.
#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace h2 {

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

constexpr int kMaxWarps = 4;

}  // namespace

// elements of T in one 16-byte unit
template <typename T>
__host__ __device__ constexpr int vec16() {
    return 16 / (int)sizeof(T);
}

// xs[pos][r] = x[pos][r] (r < NR), 0 for NR <= r < NX
template <typename T>
__global__ void k_store_x(int64_t total, int NR, int NX, const double* __restrict__ xp, T* __restrict__ xs) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t pos = e / NX;
    const int r = (int)(e % NX);
    xs[e] = r < NR ? (T)xp[pos * NR + r] : (T)0;
}

// multiply-add in the working precision (a plain fma(float, float, float)
// would resolve to the double overload and run on the FP64 pipe)
__device__ __forceinline__ float fma_w(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_w(double a, double b, double c) { return fma(a, b, c); }

// Lane layout of a warp on one block: IG lanes along the rows (lane ig owns
// rows ig, ig + IG, ...) times JG = 32 / IG lanes along the columns (lane jg
// owns the contiguous columns [jg c, jg c + c), c = ceil(|s| / JG)).  Each
// lane thus keeps (rows per lane) x NR sums in registers and reads one entry
// per row and one 16-byte vector of x per column step: the shared-memory
// instructions per multiply-add fall by the number of rows per lane, and the
// JG partial sums of a row are added once per CTA by shuffles.
template <int NR>
struct LaneMap {
    static constexpr int IG = NR == 1 ? 32 : NR >= 16 ? 16 : 8;
    static constexpr int JG = 32 / IG;
};

// Width of a staged x row: NR values, at least one 16-byte unit.
template <typename T, int NR>
struct XRow {
    static constexpr int NX = NR > vec16<T>() ? NR : vec16<T>();
    static constexpr int UPR = NX / vec16<T>();  // 16-byte units per row
};

// x rows of a block in shared memory: row j of column chunk g (j in
// [g c, g c + c)) at 16-byte unit j UPR + g (one unit of skew per chunk), so
// that the JG lanes of a column step, which read rows c apart, hit different
// banks.
template <int JG>
__device__ __forceinline__ int chunk_of(int j, int chunk) {
    int g = 0;
#pragma unroll
    for (int q = 1; q < JG; ++q) g += j >= q * chunk;
    return g;
}

// The blocks of row leaf t taken by this warp; acc[q][r] of lane (ig, jg)
// accumulates row ig + IG q over the lane's columns.  RPL: rows per lane
// (leaves of up to IG RPL triangles).  Returns with every copy this warp
// issued complete.
template <typename T, int NR, bool TRANS, int RPL>
__device__ __forceinline__ void stored_row(const NearBlock* __restrict__ blocks, const T* __restrict__ nst,
                                           const T* __restrict__ xs, int stageN, int stageX, T* sw, int W, int warp,
                                           int lane, int R, int b0, int b1, T (&acc)[RPL][NR]) {
    constexpr int IG = LaneMap<NR>::IG, JG = LaneMap<NR>::JG, V = vec16<T>();
    constexpr int UPR = XRow<T, NR>::UPR;
    const int ig = lane % IG, jg = lane / IG;
    const int ldt = R | 1;
    // stage block bk into buffer st of this warp
    auto issue = [&](const NearBlock& bk, int st) {
        const int cb = bk.cb, C = bk.C;
        const int chunk = (C + JG - 1) / JG;
        const int64_t ne = TRANS ? (int64_t)R * (C | 1) : (int64_t)C * ldt;
        const int nv = (int)((ne + V - 1) / V);  // whole 16-byte units (padding included)
        T* dN = sw + st * (stageN + stageX);
        T* dX = dN + stageN;
        const T* gN = nst + bk.off;
        for (int v = lane; v < nv; v += 32) cp16(dN + v * V, gN + v * V);
        const T* gX = xs + (int64_t)cb * XRow<T, NR>::NX;
        for (int v = lane; v < C * UPR; v += 32) {
            const int j = v / UPR, cc = v % UPR;
            cp16(dX + (j * UPR + chunk_of<JG>(j, chunk) + cc) * V, gX + v * V);
        }
    };
    int b = b0 + warp;
    NearBlock cur{}, nxt{};
    if (b < b1) {
        cur = blocks[b];
        issue(cur, 0);
    }
    cp_commit();
    for (int it = 0; b < b1; ++it, b += W) {
        const int st = it & 1;
        if (b + W < b1) {
            nxt = blocks[b + W];
            issue(nxt, st ^ 1);
        }
        cp_commit();
        cp_wait<1>();  // all but the group just issued: block b has landed
        __syncwarp();
        const int C = cur.C;
        const int chunk = (C + JG - 1) / JG;
        const T* N = sw + st * (stageN + stageX);
        const T* X = N + stageN;
        const int lds = C | 1;
        const int j0 = jg * chunk, j1 = min(C, j0 + chunk);
#pragma unroll 2
        for (int j = j0; j < j1; ++j) {
            T xv[NR];
            const T* xr = X + (j * UPR + jg) * V;
#pragma unroll
            for (int r = 0; r < NR; ++r) xv[r] = xr[r];
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int i = ig + IG * q;
                const T a = i < R ? (TRANS ? N[i * lds + j] : N[j * ldt + i]) : (T)0;
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[q][r] = fma_w(a, xv[r], acc[q][r]);
            }
        }
        __syncwarp();  // buffer st is refilled two blocks later
        cur = nxt;
    }
    cp_wait<0>();
}

template <typename T, int NR, bool TRANS, int RPL>
__device__ __forceinline__ void stored_cta(const NearBlock* __restrict__ blocks, const T* __restrict__ nst,
                                           const T* __restrict__ xs, int stageN, int stageX, int rb, int R, int b0,
                                           int b1, double* __restrict__ yp) {
    constexpr int IG = LaneMap<NR>::IG;
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* sw = reinterpret_cast<T*>(smem) + (size_t)warp * 2 * (stageN + stageX);
    T acc[RPL][NR];
#pragma unroll
    for (int q = 0; q < RPL; ++q)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[q][r] = (T)0;
    stored_row<T, NR, TRANS, RPL>(blocks, nst, xs, stageN, stageX, sw, W, warp, lane, R, b0, b1, acc);
    __syncthreads();  // every warp is done with its stages

    // the JG column partials of a row, then the warps' partials (at most 16
    // terms, in the working precision: FP64 arithmetic is ~1/46 of the FP32
    // rate here, and an FP64 epilogue per CTA would cost more than the
    // products) -> row t of y in FP64, written (not added: the farfield adds
    // to it afterwards, and every position belongs to exactly one row leaf)
    T* red = reinterpret_cast<T*>(smem);
    const int ig = lane % IG, jg = lane / IG;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        const int i = ig + IG * q;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            T v = acc[q][r];
#pragma unroll
            for (int o = IG; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (jg == 0 && i < R) red[((size_t)warp * kMaxLeaf + i) * NR + r] = v;
        }
    }
    __syncthreads();
    const int nw = min(W, b1 - b0);  // warps that received a block (the others hold zeros)
    for (int e = threadIdx.x; e < R * NR; e += blockDim.x) {
        T sum = (T)0;
        for (int w = 0; w < nw; ++w) sum += red[(size_t)w * kMaxLeaf * NR + e];
        yp[(int64_t)rb * NR + e] = (double)sum;
    }
}

// BIG: leaves of up to 64 triangles (else up to 32), chosen per operator so
// that operators with small leaves keep the smaller register footprint.
template <typename T, int NR, bool TRANS, bool BIG>
__global__ void __launch_bounds__(kMaxWarps * 32)
    k_near_stored(const NearRow* __restrict__ rows, const NearBlock* __restrict__ blocks, const T* __restrict__ nst,
                  const T* __restrict__ xs, int stageN, int stageX, double* __restrict__ yp) {
    constexpr int IG = LaneMap<NR>::IG;
    const NearRow rw = rows[blockIdx.x];
    stored_cta<T, NR, TRANS, (BIG ? 64 : 32) / IG>(blocks, nst, xs, stageN, stageX, rw.rb, rw.R, rw.b0, rw.b1, yp);
}

// N[pos0[p]] = v0[p], N[pos1[p]] = v1[p]: the Sauter-Schwab entries of the
// canonical pairs (lo, hi) into the stored blocks (entries (lo, hi), (hi, lo))
template <typename T>
__global__ void k_sing_scatter(int np, const int64_t* __restrict__ pos0, const int64_t* __restrict__ pos1,
                               const double* __restrict__ v0, const double* __restrict__ v1, T* __restrict__ nst) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    nst[pos0[p]] = (T)v0[p];
    nst[pos1[p]] = (T)v1[p];
}

int near_store_nx(bool f32, int NR) { return std::max(NR, f32 ? vec16<float>() : vec16<double>()); }

void launch_store_x(bool f32, int n, int NR, const double* xp, void* xs, cudaStream_t s) {
    const int NX = near_store_nx(f32, NR);
    const int64_t total = (int64_t)n * NX;
    const unsigned grid = (unsigned)((total + 255) / 256);
    if (f32) k_store_x<float><<<grid, 256, 0, s>>>(total, NR, NX, xp, (float*)xs);
    else k_store_x<double><<<grid, 256, 0, s>>>(total, NR, NX, xp, (double*)xs);
}

// shared memory of one warp, in elements: two stages of (block, x rows with
// one 16-byte unit of skew per column chunk, at most 4 chunks)
static void stage_elems(bool f32, int max_leaf, int NX, int& stageN, int& stageX) {
    const int v = f32 ? vec16<float>() : vec16<double>();
    const int64_t ne = (int64_t)max_leaf * (max_leaf | 1);
    stageN = (int)((ne + v - 1) / v * v);
    stageX = max_leaf * NX + 4 * v;
}

int near_stored_warps(bool f32, int max_leaf, int NR) {
    const int NX = near_store_nx(f32, NR);
    int sN, sX;
    stage_elems(f32, max_leaf, NX, sN, sX);
    const size_t per_warp = (size_t)2 * (sN + sX) * (f32 ? 4 : 8);
    int W = kMaxWarps;
    while (W > 1 && W * per_warp > 200 * 1024) --W;
    return W;
}

template <typename T, int NR>
static void stored_go(bool tr, int nrows, const NearRow* rows, const NearBlock* blocks, const T* nst, const T* xs,
                      int max_leaf, double* yp, cudaStream_t s) {
    constexpr bool F32 = std::is_same<T, float>::value;
    int sN, sX;
    stage_elems(F32, max_leaf, XRow<T, NR>::NX, sN, sX);
    const int W = near_stored_warps(F32, max_leaf, NR);
    const size_t stage_bytes = (size_t)W * 2 * (sN + sX) * sizeof(T);
    const size_t red_bytes = (size_t)W * kMaxLeaf * NR * sizeof(T);
    const size_t smem = std::max(stage_bytes, red_bytes);
    const bool big = max_leaf > 32;
    auto kern = tr ? (big ? k_near_stored<T, NR, true, true> : k_near_stored<T, NR, true, false>)
                   : (big ? k_near_stored<T, NR, false, true> : k_near_stored<T, NR, false, false>);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<nrows, W * 32, smem, s>>>(rows, blocks, nst, xs, sN, sX, yp);
}

template <typename T>
static void stored_nr(int NR, bool tr, int nrows, const NearRow* rows, const NearBlock* blocks, const T* nst,
                      const T* xs, int max_leaf, double* yp, cudaStream_t s) {
    switch (NR) {
        case 1: stored_go<T, 1>(tr, nrows, rows, blocks, nst, xs, max_leaf, yp, s); break;
        case 4: stored_go<T, 4>(tr, nrows, rows, blocks, nst, xs, max_leaf, yp, s); break;
        case 8: stored_go<T, 8>(tr, nrows, rows, blocks, nst, xs, max_leaf, yp, s); break;
        default: stored_go<T, 16>(tr, nrows, rows, blocks, nst, xs, max_leaf, yp, s); break;
    }
}

void launch_near_stored(bool f32, bool transpose, int NR, int nrows, const NearRow* rows, const NearBlock* blocks,
                        const void* nst, const void* xs, int max_leaf, double* yp, cudaStream_t s) {
    if (nrows <= 0) return;
    if (f32)
        stored_nr<float>(NR, transpose, nrows, rows, blocks, (const float*)nst, (const float*)xs, max_leaf, yp, s);
    else
        stored_nr<double>(NR, transpose, nrows, rows, blocks, (const double*)nst, (const double*)xs, max_leaf, yp, s);
}

void launch_sing_scatter(bool f32, int np, const int64_t* pos0, const int64_t* pos1, const double* v0,
                         const double* v1, void* nst, cudaStream_t s) {
    if (np <= 0) return;
    const unsigned grid = (unsigned)((np + 255) / 256);
    if (f32) k_sing_scatter<float><<<grid, 256, 0, s>>>(np, pos0, pos1, v0, v1, (float*)nst);
    else k_sing_scatter<double><<<grid, 256, 0, s>>>(np, pos0, pos1, v0, v1, (double*)nst);
}

}  // namespace h2
