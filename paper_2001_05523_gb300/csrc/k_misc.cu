// Gather/scatter between the caller's column-major vectors (user triangle
// order, leading dimension ld) and the library's tree-ordered, RHS-interleaved
// work vectors xp[pos * NR + r] (NR >= nrhs, padded columns are zero).
#include <algorithm>

#include "internal.h"

namespace h2 {

__global__ void k_permute_in(const double* __restrict__ x, int64_t ldx, int nrhs, int NR,
                             const int* __restrict__ perm, int n, double* __restrict__ xp) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * NR) return;
    int pos = (int)(idx / NR), r = (int)(idx % NR);
    xp[idx] = r < nrhs ? x[perm[pos] + r * ldx] : 0.0;
}

// As k_permute_in, reading x in the caller's order (coalesced) and scattering
// into xp through iperm: for x in mapped host memory, read over the host link.
__global__ void k_permute_in_scatter(const double* __restrict__ x, int64_t ldx, int nrhs, int NR,
                                     const int* __restrict__ iperm, int n, double* __restrict__ xp) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * NR) return;
    int r = (int)(idx / n), i = (int)(idx % n);
    xp[(int64_t)iperm[i] * NR + r] = r < nrhs ? x[i + r * ldx] : 0.0;
}

// iperm: user index -> tree position; writes of y are coalesced.
__global__ void k_permute_out(const double* __restrict__ yp, int NR, int nrhs, const int* __restrict__ iperm,
                              int n, double* __restrict__ y, int64_t ldy) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * nrhs) return;
    int r = (int)(idx / n), i = (int)(idx % n);
    y[i + r * ldy] = yp[(int64_t)iperm[i] * NR + r];
}

// Geometry preparation: gathers the triangles into tree order and computes
// area |tau| = |(b-a) x (c-a)| / 2, the unit normal (b-a) x (c-a) / |...|, the
// centroid ((a+b)+c)/3 (section 1; the normal is outward for triangles oriented
// counter-clockwise seen from outside), the plane offset c . n, and the points
// y_q = a + u_q (b-a) + v_q (c-a) of the 7-point rule, in FP64 and as FP32
// offsets from the centroid, with a float split of the centroid; in FP32
// also the normal as hi + lo, the edge vectors b - a, c - a (with their low
// parts fl(e - hi)) and the area.
__global__ void k_geom(const double* __restrict__ xyz, const int* __restrict__ tri, const int* __restrict__ perm,
                       int n, Consts c, double* __restrict__ v, double* __restrict__ area, double* __restrict__ nrm,
                       double* __restrict__ ctr, int* __restrict__ vid, float* __restrict__ qo,
                       double* __restrict__ qa, float* __restrict__ chl, double* __restrict__ plane,
                       float* __restrict__ nef, float* __restrict__ areaf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int t = perm[i];
    double P[3][3];
    for (int k = 0; k < 3; ++k) {
        const int w = tri[3 * t + k];
        vid[k * n + i] = w;
        for (int d = 0; d < 3; ++d) {
            P[k][d] = xyz[3 * (int64_t)w + d];
            v[(3 * k + d) * n + i] = P[k][d];
        }
    }
    const double e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
    const double e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
    const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    area[i] = 0.5 * len;
    areaf[i] = (float)(0.5 * len);
    double pl = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double nd = cr[d] / len;
        const double cd = ((P[0][d] + P[1][d]) + P[2][d]) / 3.0;
        nrm[d * n + i] = nd;
        ctr[d * n + i] = cd;
        const float nh = (float)nd;
        nef[d * n + i] = nh;
        nef[(3 + d) * n + i] = (float)(nd - (double)nh);
        const float e1h = (float)e1[d], e2h = (float)e2[d];
        nef[(6 + d) * n + i] = e1h;
        nef[(9 + d) * n + i] = e2h;
        nef[(12 + d) * n + i] = (float)(e1[d] - (double)e1h);
        nef[(15 + d) * n + i] = (float)(e2[d] - (double)e2h);
        const float h = (float)cd;
        chl[d * n + i] = h;
        chl[(3 + d) * n + i] = (float)(cd - (double)h);
        pl += cd * nd;
        for (int q = 0; q < 7; ++q) {
            const double y = P[0][d] + c.ru[q] * e1[d] + c.rv[q] * e2[d];
            qa[((int64_t)d * n + i) * 7 + q] = y;
            qo[((int64_t)d * n + i) * 7 + q] = (float)(y - cd);
        }
    }
    plane[i] = pl;
}

void launch_geom(const double* xyz, const int* tri, const int* perm, int n, const Consts& c, double* v, double* area,
                 double* nrm, double* ctr, int* vid, float* qo, double* qa, float* chl, double* plane, float* nef,
                 float* areaf, cudaStream_t s) {
    k_geom<<<(n + 255) / 256, 256, 0, s>>>(xyz, tri, perm, n, c, v, area, nrm, ctr, vid, qo, qa, chl, plane, nef,
                                           areaf);
}

int resident_ctas(const void* func, int threads, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem);
    return std::max(1, per_sm) * std::max(1, sms);
}

void launch_permute_in(const double* x, int64_t ldx, int nrhs, int NR, const int* perm, int n, double* xp,
                       cudaStream_t s) {
    int64_t tot = (int64_t)n * NR;
    k_permute_in<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(x, ldx, nrhs, NR, perm, n, xp);
}

void launch_permute_in_scatter(const double* x, int64_t ldx, int nrhs, int NR, const int* iperm, int n, double* xp,
                               cudaStream_t s) {
    int64_t tot = (int64_t)n * NR;
    k_permute_in_scatter<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(x, ldx, nrhs, NR, iperm, n, xp);
}

void launch_permute_out(const double* yp, int NR, int nrhs, const int* iperm, int n, double* y, int64_t ldy,
                        cudaStream_t s) {
    int64_t tot = (int64_t)n * nrhs;
    k_permute_out<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(yp, NR, nrhs, iperm, n, y, ldy);
}

}  // namespace h2
