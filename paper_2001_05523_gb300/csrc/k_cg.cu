// Vector kernels of the conjugate-gradient solver and of the mass term
// (section 1, eq. (matrix_dtn): G x = (M/2 + K) b).  Vectors are the
// caller's column-major n x nrhs blocks (leading dimension ld); every column
// is an independent system, so the scalars alpha, beta and the dot products
// are arrays of nrhs values in device memory.  FP64 throughout.
#include "internal.h"

namespace h2 {

namespace {
constexpr int kThreads = 256;
}

// out[r] += sum_i a[i + r lda] b[i + r ldb]; grid (blocks per column, nrhs)
__global__ void __launch_bounds__(kThreads) k_dots(int n, const double* __restrict__ a, int64_t lda,
                                                   const double* __restrict__ b, int64_t ldb, double* __restrict__ out) {
    const int r = blockIdx.y;
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s = fma(a[i + r * lda], b[i + r * ldb], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kThreads / 32 ? ws[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(&out[r], s);
    }
}

// x += alpha_r p, res -= alpha_r q
__global__ void k_cg_step(int n, int nrhs, const double* __restrict__ alpha, const double* __restrict__ p, int64_t ldp,
                          const double* __restrict__ q, int64_t ldq, double* __restrict__ x, int64_t ldx,
                          double* __restrict__ res, int64_t ldr) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nrhs) return;
    const int r = (int)(e / n), i = (int)(e % n);
    const double a = alpha[r];
    x[i + r * ldx] = fma(a, p[i + r * ldp], x[i + r * ldx]);
    res[i + r * ldr] = fma(-a, q[i + r * ldq], res[i + r * ldr]);
}

// p = res + beta_r p
__global__ void k_cg_dir(int n, int nrhs, const double* __restrict__ beta, const double* __restrict__ res, int64_t ldr,
                         double* __restrict__ p, int64_t ldp) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nrhs) return;
    const int r = (int)(e / n), i = (int)(e % n);
    p[i + r * ldp] = fma(beta[r], p[i + r * ldp], res[i + r * ldr]);
}

// q += m d_r (a rank-one term m m^T p with d_r = m . p_r computed before)
__global__ void k_rank1_add(int n, int nrhs, const double* __restrict__ m, const double* __restrict__ d,
                            double* __restrict__ q, int64_t ldq) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nrhs) return;
    const int r = (int)(e / n), i = (int)(e % n);
    q[i + r * ldq] = fma(m[i], d[r], q[i + r * ldq]);
}

void launch_rank1_add(int n, int nrhs, const double* m, const double* d, double* q, int64_t ldq, cudaStream_t s) {
    const int64_t tot = (int64_t)n * nrhs;
    if (tot <= 0) return;
    k_rank1_add<<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(n, nrhs, m, d, q, ldq);
}

// y += alpha |tau_i| x (P0 mass matrix); area in the caller's triangle order
__global__ void k_mass_add(int n, int nrhs, double alpha, const double* __restrict__ area_user,
                           const double* __restrict__ x, int64_t ldx, double* __restrict__ y, int64_t ldy) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nrhs) return;
    const int r = (int)(e / n), i = (int)(e % n);
    y[i + r * ldy] = fma(alpha * area_user[i], x[i + r * ldx], y[i + r * ldy]);
}

// tree-order areas to the caller's order: out[user i] = area[pos] with perm[pos] = i
__global__ void k_area_user(int n, const int* __restrict__ perm, const double* __restrict__ area,
                            double* __restrict__ out) {
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos < n) out[perm[pos]] = area[pos];
}

void launch_dots(int n, int nrhs, const double* a, int64_t lda, const double* b, int64_t ldb, double* out,
                 cudaStream_t s) {
    cudaMemsetAsync(out, 0, sizeof(double) * nrhs, s);
    int blocks = (n + kThreads - 1) / kThreads;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    k_dots<<<dim3(blocks, nrhs), kThreads, 0, s>>>(n, a, lda, b, ldb, out);
}

void launch_cg_step(int n, int nrhs, const double* alpha, const double* p, int64_t ldp, const double* q, int64_t ldq,
                    double* x, int64_t ldx, double* res, int64_t ldr, cudaStream_t s) {
    const int64_t tot = (int64_t)n * nrhs;
    k_cg_step<<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(n, nrhs, alpha, p, ldp, q, ldq, x, ldx,
                                                                            res, ldr);
}

void launch_cg_dir(int n, int nrhs, const double* beta, const double* res, int64_t ldr, double* p, int64_t ldp,
                   cudaStream_t s) {
    const int64_t tot = (int64_t)n * nrhs;
    k_cg_dir<<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(n, nrhs, beta, res, ldr, p, ldp);
}

void launch_mass_add(int n, int nrhs, double alpha, const double* area_user, const double* x, int64_t ldx, double* y,
                     int64_t ldy, cudaStream_t s) {
    const int64_t tot = (int64_t)n * nrhs;
    k_mass_add<<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(n, nrhs, alpha, area_user, x, ldx, y,
                                                                             ldy);
}

void launch_area_user(int n, const int* perm, const double* area, double* out, cudaStream_t s) {
    k_area_user<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(n, perm, area, out);
}

}  // namespace h2
