// Nearfield blocks, singular pairs (triangles sharing a vertex): Sauter-Schwab
// quadrature (cited in sections 1 and 5), FP64 always.
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
#include "dmath.cuh"
#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;
constexpr int kThreads = 128;

__device__ __forceinline__ void load_corner(const Geom& g, int i, int corner, double* out) {
    out[0] = g.v[(3 * corner + 0) * g.n + i];
    out[1] = g.v[(3 * corner + 1) * g.n + i];
    out[2] = g.v[(3 * corner + 2) * g.n + i];
}
__device__ __forceinline__ double dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
}  // namespace

template <int NR, int TYPE, int KER, int MODE>
__global__ void __launch_bounds__(kThreads) k_singular(Geom g, int npairs, const int* __restrict__ plo,
                                                       const int* __restrict__ phi, const int* __restrict__ pcode,
                                                       const double* __restrict__ tab, int npts, bool transpose,
                                                       const double* __restrict__ xp, double* __restrict__ yp,
                                                       double* __restrict__ val0, double* __restrict__ val1) {
    constexpr int W = TYPE == IDENTICAL ? 4 : TYPE == EDGE ? 11 : 2;  // doubles per table point
    extern __shared__ double stab[];
    if (MODE != 2) {
        for (int e = threadIdx.x; e < npts * W; e += blockDim.x) stab[e] = tab[e];
        __syncthreads();
    }
    const int pid = blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= npairs) return;
    const int lo = plo[pid], hi = phi[pid];
    double a01, a10;  // a_{lo,hi}, a_{hi,lo}
    if (MODE == 2) {
        a01 = val0[pid];
        a10 = val1[pid];
    } else {
        const int code = pcode[pid];
        const int rP = code & 3, q0 = (code >> 2) & 3, q1 = (code >> 4) & 3, q2 = (code >> 6) & 3;
        double P0[3], P1[3], P2[3], Q0[3], Q1[3], Q2[3];
        load_corner(g, lo, rP, P0);
        load_corner(g, lo, (rP + 1) % 3, P1);
        load_corner(g, lo, (rP + 2) % 3, P2);
        load_corner(g, hi, q0, Q0);
        load_corner(g, hi, q1, Q1);
        load_corner(g, hi, q2, Q2);
        double ea[3], eb[3], ec[3], ed[3];
        for (int d = 0; d < 3; ++d) {
            ea[d] = P1[d] - P0[d];
            eb[d] = P2[d] - P1[d];
            ec[d] = Q1[d] - Q0[d];
            ed[d] = Q2[d] - Q1[d];
        }
        const double sc = 4.0 * g.area[lo] * g.area[hi] * kInv4Pi;
        if (TYPE == IDENTICAL) {
            const double aa = dot(ea, ea), ab = dot(ea, eb), bb = dot(eb, eb);
            double s = 0.0;
            for (int p = 0; p < npts; ++p) {
                const double* T = stab + p * W;
                const double r2 = T[0] * aa + T[1] * ab + T[2] * bb;
                s += T[3] * rsqrt_nr(r2);
            }
            a01 = a10 = sc * s;
        } else if (TYPE == EDGE) {
            // vectors (a, b, d) for coefficients (alpha, beta, gamma)
            const double G0 = dot(ea, ea), G1 = dot(eb, eb), G2 = dot(ed, ed);
            const double G3 = dot(ea, eb), G4 = dot(ea, ed), G5 = dot(eb, ed);
            if (KER == SLP) {
                double s = 0.0;
                for (int p = 0; p < npts; ++p) {
                    const double* T = stab + p * W;
                    const double r2 = T[0] * G0 + T[1] * G1 + T[2] * G2 + T[3] * G3 + T[4] * G4 + T[5] * G5;
                    s += T[9] * rsqrt_nr(r2);
                }
                a01 = a10 = sc * s;
            } else {
                double sa = 0.0, sb = 0.0, sd = 0.0;
                for (int p = 0; p < npts; ++p) {
                    const double* T = stab + p * W;
                    const double r2 = T[0] * G0 + T[1] * G1 + T[2] * G2 + T[3] * G3 + T[4] * G4 + T[5] * G5;
                    const double ri = rsqrt_nr(r2);
                    const double f = T[10] * ri * ri * ri;
                    sa += f * T[6];
                    sb += f * T[7];
                    sd += f * T[8];
                }
                double V[3];
                for (int d = 0; d < 3; ++d) V[d] = sa * ea[d] + sb * eb[d] + sd * ed[d];
                double nlo[3], nhi[3];
                for (int d = 0; d < 3; ++d) {
                    nlo[d] = g.nrm[d * g.n + lo];
                    nhi[d] = g.nrm[d * g.n + hi];
                }
                a01 = sc * dot(V, nhi);
                a10 = -sc * dot(V, nlo);
            }
        } else {  // VERTEX: vectors (a, b, c, d); stab holds the 1-D Gauss rule (x_k, w_k), npts = q
            const double aa = dot(ea, ea), bb = dot(eb, eb), cc = dot(ec, ec), dd = dot(ed, ed);
            const double ab = dot(ea, eb), ac = dot(ea, ec), ad = dot(ea, ed), bc = dot(eb, ec), bd = dot(eb, ed),
                         cd = dot(ec, ed);
            const int q = npts;
            double s = 0.0, sa = 0.0, sb = 0.0, sc2 = 0.0, sd = 0.0;
            for (int reg = 0; reg < 2; ++reg) {
                // R1: U = a + e1 b, V = c + e3 d;  R2: U = c + e1 d, V = a + e3 b
                const double uu = reg == 0 ? aa : cc, uv2 = reg == 0 ? ab : cd, vv2 = reg == 0 ? bb : dd;
                const double pp = reg == 0 ? cc : aa, pq2 = reg == 0 ? cd : ab, qq2 = reg == 0 ? dd : bb;
                const double b0 = ac, b1 = reg == 0 ? ad : bc, b2 = reg == 0 ? bc : ad;
                for (int i = 0; i < q; ++i) {
                    const double e1 = stab[2 * i], w1 = stab[2 * i + 1];
                    const double A = fma(e1, fma(e1, vv2, 2.0 * uv2), uu);
                    const double Bi0 = fma(e1, b2, b0), Bi1 = fma(e1, bd, b1);
                    for (int l = 0; l < q; ++l) {
                        const double e3 = stab[2 * l], w3 = stab[2 * l + 1];
                        const double Cc = fma(e3, fma(e3, qq2, 2.0 * pq2), pp);
                        const double m2B = -2.0 * fma(e3, Bi1, Bi0);
                        double f0 = 0.0, f1 = 0.0;
                        for (int k = 0; k < q; ++k) {
                            const double e2 = stab[2 * k], we2 = stab[2 * k + 1] * e2;
                            const double r2 = fma(e2, fma(e2, Cc, m2B), A);
                            const double ri = rsqrt_nr(r2);
                            if (KER == SLP) {
                                f0 = fma(we2, ri, f0);
                            } else {
                                const double f = we2 * (ri * ri * ri);
                                f0 += f;
                                f1 = fma(f, e2, f1);
                            }
                        }
                        const double ww = w1 * w3;
                        if (KER == SLP) {
                            s = fma(ww, f0, s);
                        } else {
                            f0 *= ww;
                            f1 *= ww;
                            if (reg == 0) {  // w = a + e1 b - e2 c - e2 e3 d
                                sa += f0;
                                sb = fma(e1, f0, sb);
                                sc2 -= f1;
                                sd = fma(-e3, f1, sd);
                            } else {         // w = e2 a + e2 e3 b - c - e1 d
                                sa += f1;
                                sb = fma(e3, f1, sb);
                                sc2 -= f0;
                                sd = fma(-e1, f0, sd);
                            }
                        }
                    }
                }
            }
            if (KER == SLP) {
                a01 = a10 = sc * s / 3.0;
            } else {
                double V[3];
                for (int d = 0; d < 3; ++d) V[d] = 0.5 * (sa * ea[d] + sb * eb[d] + sc2 * ec[d] + sd * ed[d]);
                double nlo[3], nhi[3];
                for (int d = 0; d < 3; ++d) {
                    nlo[d] = g.nrm[d * g.n + lo];
                    nhi[d] = g.nrm[d * g.n + hi];
                }
                a01 = sc * dot(V, nhi);
                a10 = -sc * dot(V, nlo);
            }
        }
        if (MODE == 1) {
            val0[pid] = a01;
            val1[pid] = a10;
            return;
        }
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
static void sing_mode(int mode, int npairs, cudaStream_t s, const Geom& g, const int* lo, const int* hi,
                      const int* code, const double* tab, int npts, bool tr, const double* xp, double* yp,
                      double* v0, double* v1) {
    constexpr int W = TYPE == IDENTICAL ? 4 : TYPE == EDGE ? 11 : 2;
    const size_t smem = mode == 2 ? 0 : (size_t)npts * W * sizeof(double);
    dim3 grid((npairs + kThreads - 1) / kThreads);
    if (mode == 0) {
        cudaFuncSetAttribute(k_singular<NR, TYPE, KER, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_singular<NR, TYPE, KER, 0><<<grid, kThreads, smem, s>>>(g, npairs, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
    } else if (mode == 1) {
        cudaFuncSetAttribute(k_singular<NR, TYPE, KER, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_singular<NR, TYPE, KER, 1><<<grid, kThreads, smem, s>>>(g, npairs, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
    } else {
        k_singular<NR, TYPE, KER, 2><<<grid, kThreads, 0, s>>>(g, npairs, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
    }
}

template <int NR, int TYPE>
static void sing_ker(int ker, int mode, int npairs, cudaStream_t s, const Geom& g, const int* lo, const int* hi,
                     const int* code, const double* tab, int npts, bool tr, const double* xp, double* yp, double* v0,
                     double* v1) {
    if (ker == SLP) sing_mode<NR, TYPE, SLP>(mode, npairs, s, g, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
    else sing_mode<NR, TYPE, DLP>(mode, npairs, s, g, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
}

template <int NR>
static void sing_type(int type, int ker, int mode, int npairs, cudaStream_t s, const Geom& g, const int* lo,
                      const int* hi, const int* code, const double* tab, int npts, bool tr, const double* xp,
                      double* yp, double* v0, double* v1) {
    if (type == IDENTICAL) sing_ker<NR, IDENTICAL>(ker, mode, npairs, s, g, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
    else if (type == EDGE) sing_ker<NR, EDGE>(ker, mode, npairs, s, g, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
    else sing_ker<NR, VERTEX>(ker, mode, npairs, s, g, lo, hi, code, tab, npts, tr, xp, yp, v0, v1);
}

void launch_singular(const Geom& g, int type, int ker, int npairs, const int* lo, const int* hi, const int* code,
                     const double* tab, int npts, int mode, bool transpose, int NR, const double* xp, double* yp,
                     double* val0, double* val1, cudaStream_t s) {
    if (npairs <= 0) return;
    if (ker == DLP_T) ker = DLP;  // the transposed double layer swaps the two values
    switch (NR) {
        case 1: sing_type<1>(type, ker, mode, npairs, s, g, lo, hi, code, tab, npts, transpose, xp, yp, val0, val1); break;
        case 4: sing_type<4>(type, ker, mode, npairs, s, g, lo, hi, code, tab, npts, transpose, xp, yp, val0, val1); break;
        case 8: sing_type<8>(type, ker, mode, npairs, s, g, lo, hi, code, tab, npts, transpose, xp, yp, val0, val1); break;
        default: sing_type<16>(type, ker, mode, npairs, s, g, lo, hi, code, tab, npts, transpose, xp, yp, val0, val1); break;
    }
}

}  // namespace h2
