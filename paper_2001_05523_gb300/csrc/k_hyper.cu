// Hypersingular operator W on continuous piecewise-linear functions through
// its single-layer representation (section 1: W is set up from the single
// layer; for the Laplace kernel on a closed surface
//   w_ij = int int g(x, y) curl phi_i(x) . curl phi_j(y) dy dx,
// curl phi = n x grad phi).  The curl of a hat function is constant on each
// triangle tau = (a, b, c):
//   curl phi_a = (b - c) / (2 |tau|),  curl phi_b = (c - a) / (2 |tau|),  curl phi_c = (a - b) / (2 |tau|),
// so W = sum_d C_d^T G C_d with (C_d)_{tau j} = (curl phi_j |_tau)_d and G the
// piecewise-constant single layer (applied by the H^2 kernels).  These two
// kernels are C_d x (gather over the corners) and sum_d C_d^T w (gather over
// the triangles around each vertex, no atomics).  FP64; vertices and
// triangles in the caller's order.
#include "internal.h"

namespace h2 {

namespace {
constexpr int kThreads = 256;

// corner k of triangle tau: 2 |tau| curl phi_k = p_{k+1} - p_{k+2}; returns
// 1 / (2 |tau|) and the unscaled curl
__device__ __forceinline__ double corner_curl(const double* __restrict__ xyz, const int* __restrict__ tri, int tau,
                                              int k, double cv[3]) {
    const int ia = tri[3 * tau], ib = tri[3 * tau + 1], ic = tri[3 * tau + 2];
    double p[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        p[0][d] = xyz[3 * (int64_t)ia + d];
        p[1][d] = xyz[3 * (int64_t)ib + d];
        p[2][d] = xyz[3 * (int64_t)ic + d];
    }
    double e1[3], e2[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        e1[d] = p[1][d] - p[0][d];
        e2[d] = p[2][d] - p[0][d];
    }
    const double cx = e1[1] * e2[2] - e1[2] * e2[1];
    const double cy = e1[2] * e2[0] - e1[0] * e2[2];
    const double cz = e1[0] * e2[1] - e1[1] * e2[0];
    const int k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) cv[d] = p[k1][d] - p[k2][d];
    return 1.0 / sqrt(cx * cx + cy * cy + cz * cz);
}
}  // namespace

// z[tau + (d nrhs + r) n] = (C_d x)_tau for column r of x (nv x nrhs, leading dimension ldx)
__global__ void __launch_bounds__(kThreads) k_curl_fwd(int n, int nrhs, const double* __restrict__ xyz,
                                                       const int* __restrict__ tri, const double* __restrict__ x,
                                                       int64_t ldx, double* __restrict__ z) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nrhs) return;
    const int tau = (int)(e % n), r = (int)(e / n);
    double acc[3] = {0.0, 0.0, 0.0};
    double inv = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double cv[3];
        inv = corner_curl(xyz, tri, tau, k, cv);
        const double xv = x[tri[3 * tau + k] + r * ldx];
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[d] = fma(cv[d], xv, acc[d]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) z[tau + ((int64_t)d * nrhs + r) * n] = acc[d] * inv;
}

// y[j + r ldy] = sum_d sum_{tau at j} (curl phi_j |_tau)_d w[tau + (d nrhs + r) n];
// the triangles at vertex j are inc[vptr[j] .. vptr[j + 1]) as 3 tau + corner
__global__ void __launch_bounds__(kThreads) k_curl_bwd(int nv, int n, int nrhs, const int* __restrict__ vptr,
                                                       const int* __restrict__ inc, const double* __restrict__ xyz,
                                                       const int* __restrict__ tri, const double* __restrict__ w,
                                                       double* __restrict__ y, int64_t ldy) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)nv * nrhs) return;
    const int j = (int)(e % nv), r = (int)(e / nv);
    double acc = 0.0;
    for (int q = vptr[j]; q < vptr[j + 1]; ++q) {
        const int tau = inc[q] / 3, k = inc[q] % 3;
        double cv[3];
        const double inv = corner_curl(xyz, tri, tau, k, cv);
        double s = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) s = fma(cv[d], w[tau + ((int64_t)d * nrhs + r) * n], s);
        acc = fma(s, inv, acc);
    }
    y[j + r * ldy] = acc;
}

void launch_curl_fwd(int n, int nrhs, const double* xyz, const int* tri, const double* x, int64_t ldx, double* z,
                     cudaStream_t s) {
    const int64_t tot = (int64_t)n * nrhs;
    if (tot <= 0) return;
    k_curl_fwd<<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(n, nrhs, xyz, tri, x, ldx, z);
}

void launch_curl_bwd(int nv, int n, int nrhs, const int* vptr, const int* inc, const double* xyz, const int* tri,
                     const double* w, double* y, int64_t ldy, cudaStream_t s) {
    const int64_t tot = (int64_t)nv * nrhs;
    if (tot <= 0) return;
    k_curl_bwd<<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(nv, n, nrhs, vptr, inc, xyz, tri, w,
                                                                               y, ldy);
}

}  // namespace h2
