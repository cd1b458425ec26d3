// The double layer with continuous piecewise-linear trial functions, K1
// (section 1, eq. (dlp) with phi_j the hat functions of the vertices):
//   (K1)_{i v} = sum over the triangles j at vertex v of
//                int_{tau_i} int_{tau_j} dg/dn_y(x, y) lambda_{j,c(v)}(y) dy dx,
// lambda_{j,c} the barycentric coordinate of corner c of tau_j.  Per pair of
// triangles the trial function is lambda_c on the source panel, so a pair
// contributes three values k^c_ij.  Here: the corner gather of x (vertex
// values at the corners of every triangle, tree order), the vertex sum of
// the transpose, the regular nearfield (7 x 7-point rule, lambda_c at the
// source points; double-float arithmetic on the FP32 pipe in the FP64 tier,
// see k_p1_near; FP32 with cancellation-free heights in the mixed tiers, see
// k_p1_near32) and the Sauter-Schwab pairs (the full tensor rule with the
// source panel's barycentric coordinates as factors, FP64).  The farfield
// uses the per-corner leaf bases W1_c = int n . grad L lambda_c (k_far.cu's
// stored-basis kernels) and the passes of the double layer.
#include <algorithm>

#include "dmath.cuh"
#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;
constexpr int kThreadsP1 = 128;
}  // namespace

// x3[(c n + pos) NR + r] = x[vid_c(pos) + r ldx] (0 for r >= nrhs)
__global__ void k_p1_gather(int n, int NR, int nrhs, const int* __restrict__ vid, const double* __restrict__ x,
                            int64_t ldx, double* __restrict__ x3) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * (int64_t)n * NR) return;
    const int r = (int)(e % NR);
    const int64_t cp = e / NR;  // c n + pos
    x3[e] = r < nrhs ? x[vid[cp] + r * ldx] : 0.0;
}

// y[v + r ldy] = sum over the corners (tau, c) at v of y3[(c n + iperm[tau]) NR + r]
__global__ void k_p1_scatter(int nv, int n, int NR, int nrhs, const int* __restrict__ vptr,
                             const int* __restrict__ inc, const int* __restrict__ iperm, const double* __restrict__ y3,
                             double* __restrict__ y, int64_t ldy) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)nv * nrhs) return;
    const int v = (int)(e % nv), r = (int)(e / nv);
    double acc = 0.0;
    for (int q = vptr[v]; q < vptr[v + 1]; ++q) {
        const int tau = inc[q] / 3, c = inc[q] % 3;
        acc += y3[((int64_t)c * n + iperm[tau]) * NR + r];
    }
    y[v + r * ldy] = acc;
}

namespace {
// float-pair arithmetic (Knuth's TwoSum, Dekker's product through the FMA residual)
__device__ __forceinline__ void p1_tsum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void p1_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
    ph = __fmul_rn(ah, bh);
    pl = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fmaf_rn(ah, bh, -ph)));
}
__device__ __forceinline__ void p1_acc(float& sh, float& sl, float ph, float pl) {
    float e;
    p1_tsum(sh, ph, sh, e);
    sl = __fadd_rn(sl, __fadd_rn(e, pl));
}
}  // namespace

// point offsets from the centroid, y_q - c, as float pairs: off[(d n + i) 7 + q]
// (hi, d = 0..2) and off[((3 + d) n + i) 7 + q] (lo)
__global__ void k_p1_offsets(int n, const double* __restrict__ qa, const double* __restrict__ ctr,
                             float* __restrict__ off) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * (int64_t)n * 7) return;
    const int64_t di = e / 7;  // d n + i
    const double v = qa[e] - ctr[di];
    const float h = (float)v;
    off[e] = h;
    off[3 * (int64_t)n * 7 + e] = (float)(v - (double)h);
}

// Regular pairs of the nearfield blocks (t, s) of row t (CSR rows / ptr / col):
// forward (TR = false): y_i += sum_c k^c_ij x3_c[j], i in t, j in s;
// transposed: y3_c[j] += k^c_ij x_i, j in t, i in s.  Thread (a, part): output
// triangle a of t and the source triangles b = part, part + P, ... of each
// block; the parts meet in shared memory.  Pairs sharing a vertex are left to
// the Sauter-Schwab kernels.
//   k^c_ij = |tau_i||tau_j| / (4 pi) sum_q w_q lambda_c(y_q) sum_p w_p h_p / r_pq^3,
// h_p = (x_p - c_j) . n_j the height of the target point above the source's
// plane (y_q lies on it).  Double-float arithmetic on the FP32 pipe: the
// centroid difference formed in FP64 per pair and split, the point offsets as
// float pairs (set-up), the heights as float-pair dot products with the split
// normal, 1/r from the hardware reciprocal square root plus one Newton step,
// 1/r^3 and the sums as float pairs (about 1e-13 relative per entry).
template <int NR, bool TR>
__global__ void __launch_bounds__(kThreadsP1) k_p1_near(Geom g, Tree t, Consts c, const int* __restrict__ rows,
                                                        const int* __restrict__ ptr, const int* __restrict__ col,
                                                        const float* __restrict__ off,
                                                        const double* __restrict__ xin, double* __restrict__ yout) {
    constexpr int NO = TR ? 3 * NR : NR;  // outputs per output triangle
    extern __shared__ __align__(16) double red[];  // [P][R][NO]
    __shared__ float swh[7], swl[7], slh[21], sll[21];  // w_p; w_q lambda_c(q) at [3 q + c]
    const int tt = rows[blockIdx.x];
    const int tb = t.begin[tt], R = t.end[tt] - tb;
    const int n = g.n;
    const int tid = threadIdx.x;
    if (tid < 7) {
        const float h = (float)c.rw[tid];
        swh[tid] = h;
        swl[tid] = (float)(c.rw[tid] - (double)h);
    }
    if (tid < 21) {
        const int q = tid / 3, cc = tid % 3;
        const double lam = cc == 0 ? 1.0 - c.ru[q] - c.rv[q] : cc == 1 ? c.ru[q] : c.rv[q];
        const double v = c.rw[q] * lam;
        const float h = (float)v;
        slh[tid] = h;
        sll[tid] = (float)(v - (double)h);
    }
    __syncthreads();
    const int P = kThreadsP1 / R;
    const int a = tid % R, part = tid / R;
    const bool active = part < P;
    const int64_t n7 = (int64_t)n * 7, lo7 = 3 * n7;
    double acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = 0.0;
    if (active) {
        const int ia = tb + a;  // the output triangle (target forward, source transposed)
        for (int blk = ptr[blockIdx.x]; blk < ptr[blockIdx.x + 1]; ++blk) {
            const int s = col[blk];
            for (int jb = t.begin[s] + part; jb < t.end[s]; jb += P) {
                bool sing = false;
#pragma unroll
                for (int u = 0; u < 3; ++u)
#pragma unroll
                    for (int w = 0; w < 3; ++w) sing |= g.vid[u * n + ia] == g.vid[w * n + jb];
                if (sing) continue;
                const int it = TR ? jb : ia, js = TR ? ia : jb;  // target i, source j of k^c_ij
                float Dh[3], Dl[3], nh[3], nl[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const double Dd = g.ctr[d * n + it] - g.ctr[d * n + js];
                    Dh[d] = (float)Dd;
                    Dl[d] = (float)(Dd - (double)Dh[d]);
                    nh[d] = g.nef[d * n + js];
                    nl[d] = g.nef[(3 + d) * n + js];
                }
                // target offsets a_p and the weighted heights w_p h_p, h_p = (a_p + D) . n_j
                float aph[7][3], apl[7][3], whh[7], whl[7];
#pragma unroll
                for (int p = 0; p < 7; ++p) {
                    float vh[3], vl[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        aph[p][d] = off[(d * (int64_t)n + it) * 7 + p];
                        apl[p][d] = off[lo7 + (d * (int64_t)n + it) * 7 + p];
                        float e;
                        p1_tsum(aph[p][d], Dh[d], vh[d], e);
                        vl[d] = __fadd_rn(__fadd_rn(apl[p][d], Dl[d]), e);
                    }
                    float p0, q0, p1, q1, p2, q2, s1, e1, e2;
                    p1_mul(vh[0], vl[0], nh[0], nl[0], p0, q0);
                    p1_mul(vh[1], vl[1], nh[1], nl[1], p1, q1);
                    p1_mul(vh[2], vl[2], nh[2], nl[2], p2, q2);
                    p1_tsum(p0, p1, s1, e1);
                    float hh;
                    p1_tsum(s1, p2, hh, e2);
                    const float hl = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(q0, q1), q2));
                    p1_mul(swh[p], swl[p], hh, hl, whh[p], whl[p]);
                }
                float sch[3] = {0.0f, 0.0f, 0.0f}, scl[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll 1
                for (int q = 0; q < 7; ++q) {
                    // Y = D - (y_q - c_j)
                    float Yh[3], Yl[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        float e;
                        p1_tsum(Dh[d], -off[(d * (int64_t)n + js) * 7 + q], Yh[d], e);
                        Yl[d] = __fadd_rn(__fsub_rn(Dl[d], off[lo7 + (d * (int64_t)n + js) * 7 + q]), e);
                    }
                    float Ah = 0.0f, Al = 0.0f;
#pragma unroll
                    for (int p = 0; p < 7; ++p) {
                        float sq[3], sqe[3];
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            float dh, e;
                            p1_tsum(aph[p][d], Yh[d], dh, e);
                            const float dl = __fadd_rn(__fadd_rn(apl[p][d], Yl[d]), e);
                            sq[d] = __fmul_rn(dh, dh);
                            sqe[d] = __fmaf_rn(2.0f * dh, dl, __fmaf_rn(dh, dh, -sq[d]));
                        }
                        float s1, e1, Rh, e2;
                        p1_tsum(sq[0], sq[1], s1, e1);
                        p1_tsum(s1, sq[2], Rh, e2);
                        const float Rl = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(sqe[0], sqe[1]), sqe[2]));
                        float y0;
                        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(Rh));
                        const float y2 = __fmul_rn(y0, y0);
                        const float y2e = __fmaf_rn(y0, y0, -y2);
                        const float tq = __fmaf_rn(-Rh, y2, 1.0f);
                        const float ep = __fsub_rn(tq, __fmaf_rn(Rh, y2e, __fmul_rn(Rl, y2)));
                        const float yc = __fmul_rn(__fmul_rn(0.5f, y0), ep);  // 1/r = y0 + yc
                        const float yyl = __fmaf_rn(2.0f * y0, yc, y2e);       // (1/r)^2 = y2 + yyl
                        float y3h, y3l, th, tl;
                        p1_mul(y2, yyl, y0, yc, y3h, y3l);
                        p1_mul(whh[p], whl[p], y3h, y3l, th, tl);
                        p1_acc(Ah, Al, th, tl);
                    }
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) {
                        float th, tl;
                        p1_mul(slh[3 * q + cc], sll[3 * q + cc], Ah, Al, th, tl);
                        p1_acc(sch[cc], scl[cc], th, tl);
                    }
                }
                double sc[3];
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) sc[cc] = (double)sch[cc] + (double)scl[cc];
                const double f = g.area[it] * g.area[js] * kInv4Pi;
                if constexpr (!TR) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        double v = 0.0;
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) v = fma(sc[cc], xin[((int64_t)cc * n + js) * NR + r], v);
                        acc[r] = fma(f, v, acc[r]);
                    }
                } else {
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc)
#pragma unroll
                        for (int r = 0; r < NR; ++r) acc[cc * NR + r] = fma(f * sc[cc], xin[(int64_t)it * NR + r], acc[cc * NR + r]);
                }
            }
        }
    }
#pragma unroll
    for (int o = 0; o < NO; ++o)
        if (active) red[((size_t)part * R + a) * NO + o] = acc[o];
    __syncthreads();
    for (int e = tid; e < R * NO; e += kThreadsP1) {
        const int aa = e / NO, o = e % NO;
        double s = 0.0;
        for (int q = 0; q < P; ++q) s += red[((size_t)q * R + aa) * NO + o];
        if constexpr (!TR) {
            yout[(int64_t)(tb + aa) * NR + o] += s;
        } else {
            const int cc = o / NR, r = o % NR;
            yout[((int64_t)cc * n + tb + aa) * NR + r] += s;
        }
    }
}

// The same regular pairs in FP32 (mixed tiers).  The heights of the target
// points above the source's plane are O(h^2 kappa) against coordinates O(h),
// so they are formed without cancellation, as in the P0 double layer's FP32
// kernel: with delta = n_j - n_i from the split normals and the target point
// x_p = c_i + (u_p - 1/3) E1_i + (v_p - 1/3) E2_i (E1_i . n_i = E2_i . n_i = 0),
//   h_p = D . n_j + (u_p - 1/3) E1_i . delta + (v_p - 1/3) E2_i . delta,
// D = c_i - c_j from the centroids' float splits and D . n_j from Dekker's
// products and TwoSum (the cancelling part).  Distances from the points'
// FP32 offsets and D (hi difference exact for nearby centroids), 1/r the
// hardware reciprocal square root; the sums over p and q and the corner sums
// in FP32; the scale |tau_i||tau_j| / (4 pi) and the products with x in FP64.
template <int NR, bool TR>
__global__ void __launch_bounds__(kThreadsP1) k_p1_near32(Geom g, Tree t, Consts c, const int* __restrict__ rows,
                                                          const int* __restrict__ ptr, const int* __restrict__ col,
                                                          const double* __restrict__ xin, double* __restrict__ yout) {
    constexpr int NO = TR ? 3 * NR : NR;  // outputs per output triangle
    extern __shared__ __align__(16) double red[];  // [P][R][NO]
    __shared__ float slw[21];                      // w_q lambda_c(q) at [3 q + c]
    const int tt = rows[blockIdx.x];
    const int tb = t.begin[tt], R = t.end[tt] - tb;
    const int n = g.n;
    const int tid = threadIdx.x;
    if (tid < 21) {
        const int q = tid / 3, cc = tid % 3;
        const double lam = cc == 0 ? 1.0 - c.ru[q] - c.rv[q] : cc == 1 ? c.ru[q] : c.rv[q];
        slw[tid] = (float)(c.rw[q] * lam);
    }
    __syncthreads();
    const int P = kThreadsP1 / R;
    const int a = tid % R, part = tid / R;
    const bool active = part < P;
    double acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = 0.0;
    if (active) {
        const int ia = tb + a;  // the output triangle (target forward, source transposed)
        for (int blk = ptr[blockIdx.x]; blk < ptr[blockIdx.x + 1]; ++blk) {
            const int s = col[blk];
            for (int jb = t.begin[s] + part; jb < t.end[s]; jb += P) {
                bool sing = false;
#pragma unroll
                for (int u = 0; u < 3; ++u)
#pragma unroll
                    for (int w = 0; w < 3; ++w) sing |= g.vid[u * n + ia] == g.vid[w * n + jb];
                if (sing) continue;
                const int it = TR ? jb : ia, js = TR ? ia : jb;  // target i, source j of k^c_ij
                float Dh[3], Dl[3], nh[3], dl[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    Dh[d] = g.chl[d * n + it] - g.chl[d * n + js];
                    Dl[d] = g.chl[(3 + d) * n + it] - g.chl[(3 + d) * n + js];
                    nh[d] = g.nef[d * n + js];
                    dl[d] = (nh[d] - g.nef[d * n + it]) + (g.nef[(3 + d) * n + js] - g.nef[(3 + d) * n + it]);
                }
                // H0 = D . n_j: exact products and sums of the cancelling hi part
                const float p0 = __fmul_rn(Dh[0], nh[0]), p1 = __fmul_rn(Dh[1], nh[1]), p2 = __fmul_rn(Dh[2], nh[2]);
                const float r0 = __fmaf_rn(Dh[0], nh[0], -p0), r1 = __fmaf_rn(Dh[1], nh[1], -p1),
                            r2 = __fmaf_rn(Dh[2], nh[2], -p2);
                float s1, t1, s2, t2;
                p1_tsum(p0, p1, s1, t1);
                p1_tsum(s1, p2, s2, t2);
                float cr = (t1 + t2) + (r0 + r1 + r2);
#pragma unroll
                for (int d = 0; d < 3; ++d) cr = fmaf(Dh[d], g.nef[(3 + d) * n + js], fmaf(Dl[d], nh[d], cr));
                const float H0 = s2 + cr;
                const float e1 = g.nef[6 * n + it] * dl[0] + g.nef[7 * n + it] * dl[1] + g.nef[8 * n + it] * dl[2];
                const float e2 = g.nef[9 * n + it] * dl[0] + g.nef[10 * n + it] * dl[1] + g.nef[11 * n + it] * dl[2];
                float ax[7], ay[7], az[7], wh[7];
#pragma unroll
                for (int p = 0; p < 7; ++p) {
                    ax[p] = g.qo[((int64_t)0 * n + it) * 7 + p];
                    ay[p] = g.qo[((int64_t)1 * n + it) * 7 + p];
                    az[p] = g.qo[((int64_t)2 * n + it) * 7 + p];
                    wh[p] = c.rwf[p] * fmaf(c.ruf[p], e1, fmaf(c.rvf[p], e2, H0));
                }
                const float Dx = Dh[0] + Dl[0], Dy = Dh[1] + Dl[1], Dz = Dh[2] + Dl[2];
                float sc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    // Y = D - (y_q - c_j)
                    const float Yx = Dx - g.qo[((int64_t)0 * n + js) * 7 + q];
                    const float Yy = Dy - g.qo[((int64_t)1 * n + js) * 7 + q];
                    const float Yz = Dz - g.qo[((int64_t)2 * n + js) * 7 + q];
                    float A = 0.0f;
#pragma unroll
                    for (int p = 0; p < 7; ++p) {
                        const float dx = ax[p] + Yx, dy = ay[p] + Yy, dz = az[p] + Yz;
                        float y;
                        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(fmaf(dz, dz, fmaf(dy, dy, dx * dx))));
                        A = fmaf(wh[p], (y * y) * y, A);
                    }
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) sc[cc] = fmaf(slw[3 * q + cc], A, sc[cc]);
                }
                const double f = g.area[it] * g.area[js] * kInv4Pi;
                if constexpr (!TR) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        double v = 0.0;
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) v = fma((double)sc[cc], xin[((int64_t)cc * n + js) * NR + r], v);
                        acc[r] = fma(f, v, acc[r]);
                    }
                } else {
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc)
#pragma unroll
                        for (int r = 0; r < NR; ++r)
                            acc[cc * NR + r] = fma(f * (double)sc[cc], xin[(int64_t)it * NR + r], acc[cc * NR + r]);
                }
            }
        }
    }
#pragma unroll
    for (int o = 0; o < NO; ++o)
        if (active) red[((size_t)part * R + a) * NO + o] = acc[o];
    __syncthreads();
    for (int e = tid; e < R * NO; e += kThreadsP1) {
        const int aa = e / NO, o = e % NO;
        double sum = 0.0;
        for (int q = 0; q < P; ++q) sum += red[((size_t)q * R + aa) * NO + o];
        if constexpr (!TR) {
            yout[(int64_t)(tb + aa) * NR + o] += sum;
        } else {
            const int cc = o / NR, r = o % NR;
            yout[((int64_t)cc * n + tb + aa) * NR + r] += sum;
        }
    }
}

// Sauter-Schwab values of the canonical edge- and vertex-adjacent pairs
// (lo, hi) with code (rP | q0 << 2 | q1 << 4 | q2 << 6): P = corners rP, rP+1,
// rP+2 of lo, Q = corners q0, q1, q2 of hi, shared vertices first.  The full
// tensor rule `tab` (per point x1, x2, y1, y2, weight x Jacobian) on
// chi(z) = P0 + z1 (P1 - P0) + z2 (P2 - P1), lambda(z) = (1 - z1, z1 - z2, z2):
//   v[k]     = 4 |P||Q| sum w (x - y) . n_hi / (4 pi r^3) lambda_k(y)  (k^{q_k}_{lo,hi})
//   v[3 + k] = 4 |P||Q| sum w (y - x) . n_lo / (4 pi r^3) lambda_k(x)  (k^{(rP+k)%3}_{hi,lo})
__global__ void k_p1_sing_eval(Geom g, int np, const int* __restrict__ lo, const int* __restrict__ hi,
                               const int* __restrict__ code, const double* __restrict__ tab, int npts,
                               double* __restrict__ vals) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    const int n = g.n, il = lo[e], ih = hi[e], cd = code[e];
    const int rP = cd & 3, qc[3] = {(cd >> 2) & 3, (cd >> 4) & 3, (cd >> 6) & 3};
    double P[3][3], Q[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            P[k][d] = g.v[(3 * ((rP + k) % 3) + d) * n + il];
            Q[k][d] = g.v[(3 * qc[k] + d) * n + ih];
        }
    const double nl[3] = {g.nrm[il], g.nrm[n + il], g.nrm[2 * n + il]};
    const double nh[3] = {g.nrm[ih], g.nrm[n + ih], g.nrm[2 * n + ih]};
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int p = 0; p < npts; ++p) {
        const double x1 = tab[5 * p], x2 = tab[5 * p + 1], y1 = tab[5 * p + 2], y2 = tab[5 * p + 3],
                     w = tab[5 * p + 4];
        double d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double xp = P[0][k] + x1 * (P[1][k] - P[0][k]) + x2 * (P[2][k] - P[1][k]);
            const double yq = Q[0][k] + y1 * (Q[1][k] - Q[0][k]) + y2 * (Q[2][k] - Q[1][k]);
            d[k] = xp - yq;
        }
        const double r2 = fma(d[2], d[2], fma(d[1], d[1], d[0] * d[0]));
        const double ri = rsqrt_nr(r2);
        const double f = w * ri * ri * ri;
        const double kl = f * (d[0] * nh[0] + d[1] * nh[1] + d[2] * nh[2]);   // source hi
        const double kh = -f * (d[0] * nl[0] + d[1] * nl[1] + d[2] * nl[2]);  // source lo
        s[0] = fma(kl, 1.0 - y1, s[0]);
        s[1] = fma(kl, y1 - y2, s[1]);
        s[2] = fma(kl, y2, s[2]);
        s[3] = fma(kh, 1.0 - x1, s[3]);
        s[4] = fma(kh, x1 - x2, s[4]);
        s[5] = fma(kh, x2, s[5]);
    }
    const double sc = 4.0 * g.area[il] * g.area[ih] * kInv4Pi;
#pragma unroll
    for (int k = 0; k < 6; ++k) vals[6 * (int64_t)e + k] = sc * s[k];
}

// apply the stored values: forward y_lo += sum_k v[k] x3_{q_k}[hi],
// y_hi += sum_k v[3 + k] x3_{(rP+k)%3}[lo]; transposed y3_{q_k}[hi] += v[k] x_lo,
// y3_{(rP+k)%3}[lo] += v[3 + k] x_hi (FP64 atomics: a triangle is in several pairs)
template <bool TR>
__global__ void k_p1_sing_apply(int n, int np, int NR, const int* __restrict__ lo, const int* __restrict__ hi,
                                const int* __restrict__ code, const double* __restrict__ vals,
                                const double* __restrict__ xin, double* __restrict__ yout) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)np * NR) return;
    const int p = (int)(e / NR), r = (int)(e % NR);
    const int il = lo[p], ih = hi[p], cd = code[p];
    const int rP = cd & 3, qc[3] = {(cd >> 2) & 3, (cd >> 4) & 3, (cd >> 6) & 3};
    const double* v = vals + 6 * (int64_t)p;
    if constexpr (!TR) {
        double al = 0.0, ah = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            al = fma(v[k], xin[((int64_t)qc[k] * n + ih) * NR + r], al);
            ah = fma(v[3 + k], xin[((int64_t)((rP + k) % 3) * n + il) * NR + r], ah);
        }
        atomicAdd(&yout[(int64_t)il * NR + r], al);
        atomicAdd(&yout[(int64_t)ih * NR + r], ah);
    } else {
        const double xl = xin[(int64_t)il * NR + r], xh = xin[(int64_t)ih * NR + r];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicAdd(&yout[((int64_t)qc[k] * n + ih) * NR + r], v[k] * xl);
            atomicAdd(&yout[((int64_t)((rP + k) % 3) * n + il) * NR + r], v[3 + k] * xh);
        }
    }
}

// the P0 x P1 mass matrix, (M1)_{i v} = |tau_i| / 3 for the corners v of tau_i:
// forward y_pos += alpha |tau| / 3 sum_c x3_c[pos]; transposed y3_c[pos] +=
// alpha |tau| / 3 x_pos (the vertex sum follows)
template <bool TR>
__global__ void k_p1_mass(int n, int NR, double alpha, const double* __restrict__ area,
                          const double* __restrict__ xin, double* __restrict__ yout) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * NR) return;
    const int64_t pos = e / NR;
    const int r = (int)(e % NR);
    const double f = alpha * area[pos] * (1.0 / 3.0);
    if constexpr (!TR) {
        double sx = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) sx += xin[((int64_t)c * n + pos) * NR + r];
        yout[pos * NR + r] = fma(f, sx, yout[pos * NR + r]);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) yout[((int64_t)c * n + pos) * NR + r] = fma(f, xin[pos * NR + r], yout[((int64_t)c * n + pos) * NR + r]);
    }
}

void launch_p1_mass(bool transpose, int n, int NR, double alpha, const double* area, const double* xin, double* yout,
                    cudaStream_t s) {
    const int64_t tot = (int64_t)n * NR;
    if (tot <= 0 || alpha == 0.0) return;
    if (transpose) k_p1_mass<true><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, NR, alpha, area, xin, yout);
    else k_p1_mass<false><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, NR, alpha, area, xin, yout);
}

void launch_p1_gather(int n, int NR, int nrhs, const int* vid, const double* x, int64_t ldx, double* x3,
                      cudaStream_t s) {
    const int64_t tot = 3 * (int64_t)n * NR;
    if (tot <= 0) return;
    k_p1_gather<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, NR, nrhs, vid, x, ldx, x3);
}

void launch_p1_scatter(int nv, int n, int NR, int nrhs, const int* vptr, const int* inc, const int* iperm,
                       const double* y3, double* y, int64_t ldy, cudaStream_t s) {
    const int64_t tot = (int64_t)nv * nrhs;
    if (tot <= 0) return;
    k_p1_scatter<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(nv, n, NR, nrhs, vptr, inc, iperm, y3, y, ldy);
}

template <int NR>
static void p1_near_go(bool tr, bool fp32, const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows,
                       const int* ptr, const int* col, const float* off, const double* xin, double* yout,
                       cudaStream_t s) {
    const size_t smem = sizeof(double) * (size_t)kThreadsP1 * (tr ? 3 : 1) * NR;
    if (fp32) {
        auto kern = tr ? k_p1_near32<NR, true> : k_p1_near32<NR, false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<nrows, kThreadsP1, smem, s>>>(g, t, c, rows, ptr, col, xin, yout);
        return;
    }
    if (tr) {
        cudaFuncSetAttribute(k_p1_near<NR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_p1_near<NR, true><<<nrows, kThreadsP1, smem, s>>>(g, t, c, rows, ptr, col, off, xin, yout);
    } else {
        cudaFuncSetAttribute(k_p1_near<NR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_p1_near<NR, false><<<nrows, kThreadsP1, smem, s>>>(g, t, c, rows, ptr, col, off, xin, yout);
    }
}

void launch_p1_offsets(int n, const double* qa, const double* ctr, float* off, cudaStream_t s) {
    const int64_t tot = 3 * (int64_t)n * 7;
    if (tot <= 0) return;
    k_p1_offsets<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, qa, ctr, off);
}

void launch_p1_near(bool transpose, bool fp32, int NR, const Geom& g, const Tree& t, const Consts& c, int nrows,
                    const int* rows, const int* ptr, const int* col, const float* off, const double* xin,
                    double* yout, cudaStream_t s) {
    if (nrows <= 0) return;
    switch (NR) {
        case 1: p1_near_go<1>(transpose, fp32, g, t, c, nrows, rows, ptr, col, off, xin, yout, s); break;
        case 4: p1_near_go<4>(transpose, fp32, g, t, c, nrows, rows, ptr, col, off, xin, yout, s); break;
        case 8: p1_near_go<8>(transpose, fp32, g, t, c, nrows, rows, ptr, col, off, xin, yout, s); break;
        default: p1_near_go<16>(transpose, fp32, g, t, c, nrows, rows, ptr, col, off, xin, yout, s); break;
    }
}

void launch_p1_sing_eval(const Geom& g, int np, const int* lo, const int* hi, const int* code, const double* tab,
                         int npts, double* vals, cudaStream_t s) {
    if (np <= 0) return;
    k_p1_sing_eval<<<(np + 127) / 128, 128, 0, s>>>(g, np, lo, hi, code, tab, npts, vals);
}

void launch_p1_sing_apply(bool transpose, int n, int np, int NR, const int* lo, const int* hi, const int* code,
                          const double* vals, const double* xin, double* yout, cudaStream_t s) {
    const int64_t tot = (int64_t)np * NR;
    if (tot <= 0) return;
    if (transpose)
        k_p1_sing_apply<true><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, np, NR, lo, hi, code, vals, xin, yout);
    else
        k_p1_sing_apply<false><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, np, NR, lo, hi, code, vals, xin, yout);
}

}  // namespace h2
