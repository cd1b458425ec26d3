// Nearfield blocks, singular pairs (triangles sharing a vertex): Sauter-Schwab
// quadrature (cited in sections 1 and 5).  FP64-class points (FP64 tier, or
// on request in every tier): k_singular_df (k_sing_df.cu), double-float
// arithmetic on the FP32 pipe; k_singular_apply applies stored FP64 entries.
// k_singular32 (mixed tiers): every pair
// in FP32 - edge vectors as differences of the triangles' FP32 edge vectors
// (quantities of size h, no cancellation), Gram entries, quadrature points
// (hardware reciprocal square root, relative error below 2^-22) and sums; the
// area scale and the accumulation into y are FP64.  The double-layer
// projections use the difference of the split normals delta = n_hi - n_lo:
// an edge of one panel is orthogonal to its own normal (and the shared edge
// of an edge pair to both), so e . n_other = e . (+-delta), of size h^2 kappa
// and computed without cancellation.
//
// Each canonical pair {lo, hi} (outer panel P = triangle of lower user index,
// shared vertices first and in the same order in P and Q) is evaluated once.
// On every Sauter-Schwab region, x - y = lambda * w with lambda a monomial in
// the collapsed variables and w = alpha a + beta b (+ gamma c + delta d), a
// combination of the panels' edge vectors whose coefficients depend only on
// the remaining variables.  The Laplace kernels are homogeneous (degree -1 for
// g, -2 for dg/dn), so lambda cancels against the Jacobian up to a polynomial
// factor that the q-point Gauss rule integrates exactly; the host folds that
// factor into the point weights.  The tensor rule therefore reduces to
//   identical: 3 regions x q points   (mirror regions are equal for g)
//   edge:      5 regions x q^2 points
//   vertex:    2 regions x q^3 points
// with |w|^2 from the Gram matrix of the edge vectors.  The result equals the
// full 4-D tensor rule up to rounding.
//
// Vertex pairs (the bulk of the work): on both regions w = U(e1) - e2 V(e3)
// with U, V affine in one variable each, so
//   |w|^2 = A_i - 2 e2_k B_il + e2_k^2 C_l,   A_i = |U(e1_i)|^2, C_l = |V(e3_l)|^2,
//   B_il = U(e1_i) . V(e3_l),
// precomputed per pair from the Gram matrix of (a, b, c, d) (O(q^2) work);
// each of the q^3 points then costs two FMAs, a reciprocal square root and
// one accumulation.
//
// Single layer: a = 4 |P||Q| / (4 pi) sum_p W_p / |w_p|; g_ij = g_ji = a.
// Double layer: V = sum_p W_p w_p / |w_p|^3 (a vector), then
//   k_{lo,hi} = 4 |P||Q| / (4 pi)  V . n_hi,   k_{hi,lo} = -4 |P||Q| / (4 pi) V . n_lo.
#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;
constexpr int kThreads = 128;

}  // namespace

__device__ __forceinline__ float rsqrt_f32(float a) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}

// Stored FP64 entries of the canonical pairs (cache_singular) applied:
// y_lo += a_{lo,hi} x_hi, y_hi += a_{hi,lo} x_lo (swapped if transpose), by
// FP64 atomics; a pair with lo = hi adds once.  The FP64 evaluation itself is
// k_singular_df (k_sing_df.cu).
template <int NR>
__global__ void __launch_bounds__(kThreads) k_singular_apply(int npairs, const int* __restrict__ plo,
                                                             const int* __restrict__ phi, bool transpose,
                                                             const double* __restrict__ xp, double* __restrict__ yp,
                                                             const double* __restrict__ val0,
                                                             const double* __restrict__ val1) {
    const int pid = blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= npairs) return;
    const int lo = plo[pid], hi = phi[pid];
    const double a01 = transpose ? val1[pid] : val0[pid], a10 = transpose ? val0[pid] : val1[pid];
    if (lo == hi) {
#pragma unroll
        for (int r = 0; r < NR; ++r) atomicAdd(&yp[(int64_t)lo * NR + r], a01 * xp[(int64_t)lo * NR + r]);
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            atomicAdd(&yp[(int64_t)lo * NR + r], a01 * xp[(int64_t)hi * NR + r]);
            atomicAdd(&yp[(int64_t)hi * NR + r], a10 * xp[(int64_t)lo * NR + r]);
        }
    }
}

// FP32 evaluation (mixed tiers).  Table per point: identical (T0, T1, T2, T3)
// as the FP64 table; edge and vertex (x_k, w_k x_k, w_k, 0).  Q: the Gauss
// points per direction at compile time (edge and vertex pairs; 0: npts at run
// time), so that the nested point loops unroll.
template <int NR, int TYPE, int KER, int MODE, int Q = 0>
__global__ void __launch_bounds__(kThreads) k_singular32(Geom g, int npairs, const int* __restrict__ plo,
                                                         const int* __restrict__ phi, const int* __restrict__ pcode,
                                                         const double* __restrict__ tab, int npts, bool transpose,
                                                         const double* __restrict__ xp, double* __restrict__ yp,
                                                         double* __restrict__ val0, double* __restrict__ val1) {
    constexpr int W = TYPE == IDENTICAL ? 4 : TYPE == EDGE ? 4 : 3;  // doubles per point of the FP64 table
    extern __shared__ double stab[];
    float* stf = reinterpret_cast<float*>(stab);
    for (int p = threadIdx.x; p < npts; p += blockDim.x) {
        if (TYPE == IDENTICAL) {
            for (int j = 0; j < 4; ++j) stf[4 * p + j] = (float)tab[p * 4 + j];
        } else {
            stf[4 * p] = (float)tab[p * W];
            stf[4 * p + 1] = (float)(2.0 * tab[p * W + W - 1]);
            stf[4 * p + 2] = (float)tab[p * W + 1];
            stf[4 * p + 3] = 0.0f;
        }
    }
    __syncthreads();
    const int pid = blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= npairs) return;
    const int lo = plo[pid], hi = phi[pid], n = g.n;
    const int code = pcode[pid];
    const int rP = code & 3, q0 = (code >> 2) & 3, q1 = (code >> 4) & 3, q2 = (code >> 6) & 3;
    // corner k minus corner 0 of each panel, from the FP32 edge vectors (corner 0: zero)
    float EL[3][3], EH[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        EL[0][d] = 0.0f;
        EL[1][d] = g.nef[(6 + d) * n + lo];
        EL[2][d] = g.nef[(9 + d) * n + lo];
        EH[0][d] = 0.0f;
        EH[1][d] = g.nef[(6 + d) * n + hi];
        EH[2][d] = g.nef[(9 + d) * n + hi];
    }
    const int p0 = rP, p1 = (rP + 1) % 3, p2 = (rP + 2) % 3;
    float a[3], b[3], cc[3], dd[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        a[d] = EL[p1][d] - EL[p0][d];
        b[d] = EL[p2][d] - EL[p1][d];
        cc[d] = EH[q1][d] - EH[q0][d];
        dd[d] = EH[q2][d] - EH[q1][d];
    }
    auto dot3 = [](const float* u, const float* v) { return fmaf(u[2], v[2], fmaf(u[1], v[1], u[0] * v[0])); };
    // delta = n_hi - n_lo from the split normals (double layer)
    float del[3] = {0, 0, 0};
    if (KER != SLP) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
            del[d] = (g.nef[d * n + hi] - g.nef[d * n + lo]) + (g.nef[(3 + d) * n + hi] - g.nef[(3 + d) * n + lo]);
    }
    // MODE 3: the two entries as a float pair, scaled in FP32 (no FP64 arithmetic)
    const double sc = MODE == 3 ? 0.0 : 4.0 * g.area[lo] * g.area[hi] * kInv4Pi;
    const float scf = MODE == 3 ? (float)(4.0 * kInv4Pi) * (float)g.area[lo] * (float)g.area[hi] : 0.0f;
    double a01 = 0.0, a10 = 0.0;
    float v01 = 0.0f, v10 = 0.0f;
    if (TYPE == IDENTICAL) {
        const float aa = dot3(a, a), ab = dot3(a, b), bb = dot3(b, b);
        float sum = 0.0f;
        for (int p = 0; p < npts; ++p) {
            const float* T = stf + 4 * p;
            sum = fmaf(T[3], rsqrt_f32(fmaf(T[2], bb, fmaf(T[1], ab, T[0] * aa))), sum);
        }
        if (MODE == 3) v01 = v10 = scf * sum;
        else a01 = a10 = sc * (double)sum;
    } else if (TYPE == EDGE) {
        // vectors (a, b, d); regions and coefficient triples as in k_singular
        const float Gm[3][3] = {{dot3(a, a), dot3(a, b), dot3(a, dd)},
                                {dot3(a, b), dot3(b, b), dot3(b, dd)},
                                {dot3(a, dd), dot3(b, dd), dot3(dd, dd)}};
        const int q = Q > 0 ? Q : npts;
        float ssum = 0.0f, sb = 0.0f, sd = 0.0f;
        for (int reg = 0; reg < 5; ++reg) {
            float rs = 0.0f, rb = 0.0f, rd = 0.0f;
#pragma unroll
            for (int oi = 0; oi < q; ++oi) {
                const float o = stf[4 * oi], wo = stf[4 * oi + 2];
                float F[3], Gv[3];
                switch (reg) {
                    case 0: F[0] = o; F[1] = 0.0f; F[2] = o - 1.0f; Gv[0] = 0.0f; Gv[1] = 1.0f; Gv[2] = 0.0f; break;
                    case 1: F[0] = 0.0f; F[1] = 1.0f; F[2] = 0.0f; Gv[0] = o; Gv[1] = 0.0f; Gv[2] = o - 1.0f; break;
                    case 2: F[0] = 0.0f; F[1] = 1.0f; F[2] = 0.0f; Gv[0] = -1.0f; Gv[1] = -1.0f; Gv[2] = -o; break;
                    case 3: F[0] = 0.0f; F[1] = 0.0f; F[2] = -1.0f; Gv[0] = -o; Gv[1] = 1.0f - o; Gv[2] = 0.0f; break;
                    default: F[0] = 0.0f; F[1] = 1.0f; F[2] = 0.0f; Gv[0] = -o; Gv[1] = -o; Gv[2] = -1.0f; break;
                }
                float A = 0.0f, B2 = 0.0f, Cc = 0.0f;
#pragma unroll
                for (int u = 0; u < 3; ++u)
#pragma unroll
                    for (int v = 0; v < 3; ++v) {
                        A += F[u] * Gm[u][v] * F[v];
                        B2 += F[u] * Gm[u][v] * Gv[v];
                        Cc += Gv[u] * Gm[u][v] * Gv[v];
                    }
                B2 *= 2.0f;
                float f0 = 0.0f, f1 = 0.0f;
#pragma unroll
                for (int k = 0; k < q; ++k) {
                    const float tt = stf[4 * k];
                    const float wt = reg == 0 ? stf[4 * k + 2] : stf[4 * k + 1];  // w_t (R1) or w_t t
                    const float y = rsqrt_f32(fmaf(tt, fmaf(tt, Cc, B2), A));
                    if (KER == SLP) {
                        f0 = fmaf(wt, y, f0);
                    } else {
                        const float f = wt * (y * y * y);
                        f0 += f;
                        f1 = fmaf(f, tt, f1);
                    }
                }
                if (KER == SLP) {
                    rs = fmaf(wo, f0, rs);
                } else {
                    rb = fmaf(wo, f0 * F[1] + f1 * Gv[1], rb);
                    rd = fmaf(wo, f0 * F[2] + f1 * Gv[2], rd);
                }
            }
            ssum += rs;
            sb += rb;
            sd += rd;
        }
        if (KER == SLP) {
            if (MODE == 3) v01 = v10 = scf * ssum * (1.0f / 6.0f);
            else a01 = a10 = sc * (double)ssum * (1.0 / 6.0);
        } else if (MODE == 3) {
            v01 = 0.5f * scf * (sb * dot3(b, del));
            v10 = 0.5f * scf * (sd * dot3(dd, del));
        } else {
            // V = (sa a + sb b + sd d) / 2; a is in both planes, b in lo's, d in hi's
            a01 = 0.5 * sc * (double)(sb * dot3(b, del));
            a10 = 0.5 * sc * (double)(sd * dot3(dd, del));
        }
    } else {  // VERTEX: vectors (a, b, c, d)
        const float aa = dot3(a, a), bb = dot3(b, b), c2 = dot3(cc, cc), d2 = dot3(dd, dd);
        const float ab = dot3(a, b), ac = dot3(a, cc), ad = dot3(a, dd), bc = dot3(b, cc), bd = dot3(b, dd),
                    cd = dot3(cc, dd);
        const int q = Q > 0 ? Q : npts;
        float ssum = 0.0f, sa = 0.0f, sb = 0.0f, sc2 = 0.0f, sd = 0.0f;
        for (int reg = 0; reg < 2; ++reg) {
            const float uu = reg == 0 ? aa : c2, uv2 = reg == 0 ? ab : cd, vv2 = reg == 0 ? bb : d2;
            const float pp = reg == 0 ? c2 : aa, pq2 = reg == 0 ? cd : ab, qq2 = reg == 0 ? d2 : bb;
            const float b0 = ac, b1 = reg == 0 ? ad : bc, b2 = reg == 0 ? bc : ad;
#pragma unroll
            for (int i = 0; i < q; ++i) {
                const float e1 = stf[4 * i], w1 = stf[4 * i + 2];
                const float A = fmaf(e1, fmaf(e1, vv2, 2.0f * uv2), uu);
                const float Bi0 = fmaf(e1, b2, b0), Bi1 = fmaf(e1, bd, b1);
                float t0 = 0.0f, t1 = 0.0f, t2 = 0.0f;
#pragma unroll
                for (int l = 0; l < q; ++l) {
                    const float e3 = stf[4 * l], w3 = stf[4 * l + 2];
                    const float Cq = fmaf(e3, fmaf(e3, qq2, 2.0f * pq2), pp);
                    const float m2B = -2.0f * fmaf(e3, Bi1, Bi0);
                    float f0 = 0.0f, f1 = 0.0f;
#pragma unroll
                    for (int k = 0; k < q; ++k) {
                        const float2 T = *reinterpret_cast<const float2*>(stf + 4 * k);  // (e2, w e2)
                        const float y = rsqrt_f32(fmaf(T.x, fmaf(T.x, Cq, m2B), A));
                        if (KER == SLP) {
                            f0 = fmaf(T.y, y, f0);
                        } else {
                            const float f = T.y * (y * y * y);
                            f0 += f;
                            f1 = fmaf(f, T.x, f1);
                        }
                    }
                    t0 = fmaf(w3, f0, t0);
                    if (KER != SLP) {
                        t1 = fmaf(w3, f1, t1);
                        t2 = fmaf(w3 * e3, f1, t2);
                    }
                }
                const float T0 = w1 * t0;
                if (KER == SLP) {
                    ssum += T0;
                } else if (reg == 0) {  // w = a + e1 b - e2 c - e2 e3 d
                    sa += T0;
                    sb = fmaf(e1, T0, sb);
                    sc2 = fmaf(-w1, t1, sc2);
                    sd = fmaf(-w1, t2, sd);
                } else {                // w = e2 a + e2 e3 b - c - e1 d
                    sa = fmaf(w1, t1, sa);
                    sb = fmaf(w1, t2, sb);
                    sc2 -= T0;
                    sd = fmaf(-e1, T0, sd);
                }
            }
        }
        if (KER == SLP) {
            if (MODE == 3) v01 = v10 = scf * ssum * (1.0f / 3.0f);
            else a01 = a10 = sc * (double)ssum * (1.0 / 3.0);
        } else if (MODE == 3) {
            v01 = 0.5f * scf * fmaf(sa, dot3(a, del), sb * dot3(b, del));
            v10 = 0.5f * scf * fmaf(sc2, dot3(cc, del), sd * dot3(dd, del));
        } else {
            // V = (sa a + sb b + sc c + sd d) / 2; a, b in lo's plane, c, d in hi's
            a01 = 0.5 * sc * (double)fmaf(sa, dot3(a, del), sb * dot3(b, del));
            a10 = 0.5 * sc * (double)fmaf(sc2, dot3(cc, del), sd * dot3(dd, del));
        }
    }
    if (MODE == 3) {
        // each entry at its place in the row order of the gather: val1 holds
        // (position in row lo, position in row hi or -1) per pair
        const int2 ps = reinterpret_cast<const int2*>(val1)[pid];
        float* vo = reinterpret_cast<float*>(val0);
        vo[ps.x] = transpose ? v10 : v01;
        if (ps.y >= 0) vo[ps.y] = transpose ? v01 : v10;
        return;
    }
    if (MODE == 1) {
        val0[pid] = a01;
        val1[pid] = a10;
        return;
    }
    if (transpose) {
        const double tmp = a01;
        a01 = a10;
        a10 = tmp;
    }
    if (lo == hi) {
#pragma unroll
        for (int r = 0; r < NR; ++r) atomicAdd(&yp[(int64_t)lo * NR + r], a01 * xp[(int64_t)lo * NR + r]);
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            atomicAdd(&yp[(int64_t)lo * NR + r], a01 * xp[(int64_t)hi * NR + r]);
            atomicAdd(&yp[(int64_t)hi * NR + r], a10 * xp[(int64_t)lo * NR + r]);
        }
    }
}

template <int NR, int TYPE, int KER>
static void sing_mode32(int mode, int npairs, cudaStream_t s, const Geom& g, const int* lo, const int* hi,
                        const int* code, const double* tab, int npts, bool tr, const double* xp, double* yp,
                        double* v0, double* v1) {
    constexpr int W = TYPE == IDENTICAL ? 4 : TYPE == EDGE ? 4 : 3;
    const size_t smem = (size_t)npts * W * sizeof(double);
    dim3 grid((npairs + kThreads - 1) / kThreads);
    // the default 5 points per direction unrolled (edge and vertex pairs)
    const bool q5 = TYPE != IDENTICAL && npts == 5;
    auto k0 = q5 ? k_singular32<NR, TYPE, KER, 0, 5> : k_singular32<NR, TYPE, KER, 0>;
    auto k1 = q5 ? k_singular32<NR, TYPE, KER, 1, 5> : k_singular32<NR, TYPE, KER, 1>;
    auto k3 = q5 ? k_singular32<1, TYPE, KER, 3, 5> : k_singular32<1, TYPE, KER, 3>;
    auto kern = mode == 0 ? k0 : mode == 1 ? k1 : k3;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, kThreads, smem, s>>>(g, npairs, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
}

template <int NR, int TYPE>
static void sing_ker32(int ker, int mode, int npairs, cudaStream_t s, const Geom& g, const int* lo, const int* hi,
                       const int* code, const double* tab, int npts, bool tr, const double* xp, double* yp,
                       double* v0, double* v1) {
    if (ker == SLP) sing_mode32<NR, TYPE, SLP>(mode, npairs, s, g, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
    else sing_mode32<NR, TYPE, DLP>(mode, npairs, s, g, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
}

template <int NR>
static void sing_type32(int type, int ker, int mode, int npairs, cudaStream_t s, const Geom& g, const int* lo,
                        const int* hi, const int* code, const double* tab, int npts, bool tr, const double* xp,
                        double* yp, double* v0, double* v1) {
    if (type == IDENTICAL) sing_ker32<NR, IDENTICAL>(ker, mode, npairs, s, g, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
    else if (type == EDGE) sing_ker32<NR, EDGE>(ker, mode, npairs, s, g, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
    else sing_ker32<NR, VERTEX>(ker, mode, npairs, s, g, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
}

// Singular entries applied by rows: y_i += sum_e vals[e] x_{other[e]} over the
// entries e in [ptr[i], ptr[i+1]) of row i (tree position); the pair kernels
// write vals in this order.  FP32 products and row sums over the ~13 singular
// neighbours of a triangle, one FP64 addition per row and right-hand side; no
// atomics (one thread per row).
template <int NR>
__global__ void __launch_bounds__(kThreads) k_sing_gather(int n, const int* __restrict__ ptr,
                                                          const int* __restrict__ other,
                                                          const float* __restrict__ vals,
                                                          const float* __restrict__ xs, double* __restrict__ yp) {
    constexpr int NX = NR > 4 ? NR : 4;  // row width of the FP32 copy of x
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0f;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
        const float v = vals[e];
        const float* xo = xs + (int64_t)other[e] * NX;
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = fmaf(v, xo[r], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) yp[(int64_t)i * NR + r] += (double)acc[r];
}

void launch_sing_gather(int NR, int n, const int* ptr, const int* other, const float* vals, const float* xs,
                        double* yp, cudaStream_t s) {
    if (n <= 0) return;
    const unsigned grid = (unsigned)((n + kThreads - 1) / kThreads);
    switch (NR) {
        case 1: k_sing_gather<1><<<grid, kThreads, 0, s>>>(n, ptr, other, vals, xs, yp); break;
        case 4: k_sing_gather<4><<<grid, kThreads, 0, s>>>(n, ptr, other, vals, xs, yp); break;
        case 8: k_sing_gather<8><<<grid, kThreads, 0, s>>>(n, ptr, other, vals, xs, yp); break;
        default: k_sing_gather<16><<<grid, kThreads, 0, s>>>(n, ptr, other, vals, xs, yp); break;
    }
}

void launch_singular(const Geom& g, int type, int ker, int npairs, const int* lo, const int* hi, const int* code,
                     const double* tab, int npts, int mode, bool fp32, bool transpose, int NR, const double* xp,
                     double* yp, double* val0, double* val1, cudaStream_t s) {
    if (npairs <= 0) return;
    if (ker == DLP_T) ker = DLP;  // the transposed double layer swaps the two values
    if (mode == 2) {
        const unsigned grid = (unsigned)((npairs + kThreads - 1) / kThreads);
        switch (NR) {
            case 1: k_singular_apply<1><<<grid, kThreads, 0, s>>>(npairs, lo, hi, transpose, xp, yp, val0, val1); break;
            case 4: k_singular_apply<4><<<grid, kThreads, 0, s>>>(npairs, lo, hi, transpose, xp, yp, val0, val1); break;
            case 8: k_singular_apply<8><<<grid, kThreads, 0, s>>>(npairs, lo, hi, transpose, xp, yp, val0, val1); break;
            default: k_singular_apply<16><<<grid, kThreads, 0, s>>>(npairs, lo, hi, transpose, xp, yp, val0, val1); break;
        }
        return;
    }
    if (!fp32) {  // FP64-class points: double-float arithmetic (k_sing_df.cu)
        launch_singular_df(g, type, ker, npairs, lo, hi, code, tab, npts, mode, transpose, NR, xp, yp, val0, val1, s);
        return;
    }
    switch (NR) {
        case 1: sing_type32<1>(type, ker, mode, npairs, s, g, lo, hi, code, tab, npts, transpose, xp, yp, val0, val1); break;
        case 4: sing_type32<4>(type, ker, mode, npairs, s, g, lo, hi, code, tab, npts, transpose, xp, yp, val0, val1); break;
        case 8: sing_type32<8>(type, ker, mode, npairs, s, g, lo, hi, code, tab, npts, transpose, xp, yp, val0, val1); break;
        default: sing_type32<16>(type, ker, mode, npairs, s, g, lo, hi, code, tab, npts, transpose, xp, yp, val0, val1); break;
    }
}

}  // namespace h2
