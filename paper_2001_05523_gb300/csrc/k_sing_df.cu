// Singular pairs (triangles sharing a vertex) at FP64-class accuracy by
// double-float arithmetic on the FP32 pipe: the Sauter-Schwab quadrature
// (cited in sections 1 and 5) of the FP64 tier, and of the mixed tiers when
// the singular pairs are asked for in FP64.  The reduced rules are those of
// k_singular (k_sing.cu): per canonical pair {lo, hi}, x - y = lambda w on
// every region, lambda cancelled against the Jacobian, |w|^2 a quadratic in
// the innermost variable whose coefficients come from the Gram matrix of the
// panels' edge vectors:
//   identical: 3 regions x q points,  |w|^2 = T0 aa + T1 ab + T2 bb
//   edge:      5 regions x q^2,       |w|^2 = A(o) + t B2(o) + t^2 C(o)
//   vertex:    2 regions x q^3,       |w|^2 = A_i - 2 e2 B_il + e2^2 C_l
// GB300 issues FP64 at about 1/74 of its FP32 rate, and the FP64 points (six
// to seven FP64 operations each, 2.8e9 points per apply on the 2M sphere)
// bound that kernel.  Here every quantity is a float pair (dfloat.cuh):
//   - edge vectors from the triangles' FP64 edge vectors split into pairs
//     (geometry rows 6..17), Gram entries as float-pair dot products;
//   - the quadratic's coefficients and values as float pairs, r^2 renormalised
//     before the reciprocal square root (hardware seed plus the second-order
//     correction formed from the pairs, relative error about 1e-14);
//   - weights times 1/r (1/r^3 for the double layer) and every sum as pairs.
// Per pair, the area scale |P||Q|/(4 pi) and the products with x are FP64.
// Double layer: the entries need V . n_hi and -V . n_lo with V in the panels'
// planes; as in the FP32 kernel they are taken with delta = n_hi - n_lo, here
// formed in FP64 from the unit normals and split (a vector of size h kappa,
// so the pair keeps ~2^-48 of it, not of |n|).
#include <type_traits>

#include "dfloat.cuh"
#include "internal.h"

namespace h2 {

namespace {
using dfl::F2;
constexpr double kInv4PiS = 0.07957747154594766788;
constexpr int kThrS = 128;

// coefficient of edge vector u (0: a, 1: b, 2: d) in the region vectors of an
// edge pair, w = F(o) + t G(o), F = F0 + o F1, G = G0 + o G1 (which: 0 F0,
// 1 F1, 2 G0, 3 G1); the same regions as the FP64 kernel:
//   R1: F = (o, 0, o - 1), G = (0, 1, 0)      R2: F = (0, 1, 0), G = (o, 0, o - 1)
//   R3: F = (0, 1, 0), G = (-1, -1, -o)       R4: F = (0, 0, -1), G = (-o, 1 - o, 0)
//   R5: F = (0, 1, 0), G = (-o, -o, -1)
__host__ __device__ constexpr int ecoef(int r, int which, int u) {
    const int c[5][4][3] = {{{0, 0, -1}, {1, 0, 1}, {0, 1, 0}, {0, 0, 0}},
                            {{0, 1, 0}, {0, 0, 0}, {0, 0, -1}, {1, 0, 1}},
                            {{0, 1, 0}, {0, 0, 0}, {-1, -1, 0}, {0, 0, -1}},
                            {{0, 0, -1}, {0, 0, 0}, {0, 1, 0}, {-1, -1, 0}},
                            {{0, 1, 0}, {0, 0, 0}, {0, 0, -1}, {-1, -1, 0}}};
    return c[r][which][u];
}
// integer weight of the Gram entry (u, v) in the coefficient of o^p of
// A = F.F (Q = 0), B2 = 2 F.G (Q = 1) or C = G.G (Q = 2)
__host__ __device__ constexpr int qweight(int r, int Q, int p, int u, int v) {
    const int x0 = Q == 2 ? 2 : 0, y0 = Q == 0 ? 0 : 2;  // left and right vector: F (0) or G (2)
    const int w = p == 0 ? ecoef(r, x0, u) * ecoef(r, y0, v)
                : p == 1 ? ecoef(r, x0, u) * ecoef(r, y0 + 1, v) + ecoef(r, x0 + 1, u) * ecoef(r, y0, v)
                         : ecoef(r, x0 + 1, u) * ecoef(r, y0 + 1, v);
    return Q == 1 ? 2 * w : w;
}

__device__ __forceinline__ F2 ld(float4 v, int half) { return half ? F2{v.z, v.w} : F2{v.x, v.y}; }
__device__ __forceinline__ F2 horner2(F2 c0, F2 c1, F2 c2, F2 x) {
    return dfl::add(c0, dfl::mul(x, dfl::add(c1, dfl::mul(x, c2))));
}
}  // namespace

// Table in shared memory, two float4 per point (pairs split from the FP64
// table): identical (T0, T1), (T2, T3); edge and vertex (x_k, w_k), (w_k x_k, -).
// mode 0: y_lo += a_{lo,hi} x_hi, y_hi += a_{hi,lo} x_lo (swapped if transpose;
// FP64 atomics, nr right-hand sides); mode 1: val0 = a_{lo,hi}, val1 = a_{hi,lo}.
template <int TYPE, int KER, int Q>
__global__ void __launch_bounds__(kThrS) k_singular_df(Geom g, int npairs, const int* __restrict__ plo,
                                                       const int* __restrict__ phi, const int* __restrict__ pcode,
                                                       const double* __restrict__ tab, int npts, int mode,
                                                       bool transpose, int nr, const double* __restrict__ xp,
                                                       double* __restrict__ yp, double* __restrict__ val0,
                                                       double* __restrict__ val1) {
    extern __shared__ float4 st4[];
    float4* sA = st4;
    float4* sB = st4 + npts;
    for (int p = threadIdx.x; p < npts; p += blockDim.x) {
        if (TYPE == IDENTICAL) {
            const F2 t0 = dfl::split(tab[4 * p]), t1 = dfl::split(tab[4 * p + 1]), t2 = dfl::split(tab[4 * p + 2]),
                     t3 = dfl::split(tab[4 * p + 3]);
            sA[p] = make_float4(t0.h, t0.l, t1.h, t1.l);
            sB[p] = make_float4(t2.h, t2.l, t3.h, t3.l);
        } else {
            constexpr int W = TYPE == EDGE ? 4 : 3;  // FP64 table: (x, w, [w/2,] w x / 2)
            const F2 x = dfl::split(tab[W * p]), w = dfl::split(tab[W * p + 1]),
                     wx = dfl::split(2.0 * tab[W * p + W - 1]);
            sA[p] = make_float4(x.h, x.l, w.h, w.l);
            sB[p] = make_float4(wx.h, wx.l, 0.0f, 0.0f);
        }
    }
    __syncthreads();
    const int pid = blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= npairs) return;
    const int lo = plo[pid], hi = phi[pid], n = g.n;
    const int code = pcode[pid];
    const int rP = code & 3, q0 = (code >> 2) & 3, q1 = (code >> 4) & 3, q2 = (code >> 6) & 3;
    // corner k minus corner 0 of each panel as float pairs (corner 0: zero)
    F2 EL[3][3], EH[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        EL[0][d] = EH[0][d] = F2{0.0f, 0.0f};
        EL[1][d] = F2{g.nef[(6 + d) * n + lo], g.nef[(12 + d) * n + lo]};
        EL[2][d] = F2{g.nef[(9 + d) * n + lo], g.nef[(15 + d) * n + lo]};
        EH[1][d] = F2{g.nef[(6 + d) * n + hi], g.nef[(12 + d) * n + hi]};
        EH[2][d] = F2{g.nef[(9 + d) * n + hi], g.nef[(15 + d) * n + hi]};
    }
    const int p0 = rP, p1 = (rP + 1) % 3, p2 = (rP + 2) % 3;
    F2 a[3], b[3], c[3], d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a[k] = dfl::sub(EL[p1][k], EL[p0][k]);
        b[k] = dfl::sub(EL[p2][k], EL[p1][k]);
        c[k] = dfl::sub(EH[q1][k], EH[q0][k]);
        d[k] = dfl::sub(EH[q2][k], EH[q1][k]);
    }
    F2 del[3] = {};
    if (KER != SLP) {
#pragma unroll
        for (int k = 0; k < 3; ++k) del[k] = dfl::split(g.nrm[k * n + hi] - g.nrm[k * n + lo]);
    }
    const double sc = 4.0 * g.area[lo] * g.area[hi] * kInv4PiS;
    double a01 = 0.0, a10 = 0.0;
    if (TYPE == IDENTICAL) {
        if (KER == SLP) {  // the double layer's entry of a triangle with itself vanishes
            const F2 aa = dfl::dot3(a, a), ab = dfl::dot3(a, b), bb = dfl::dot3(b, b);
            F2 s{0.0f, 0.0f};
            for (int p = 0; p < npts; ++p) {
                const float4 A4 = sA[p], B4 = sB[p];
                const F2 r2 = dfl::renorm(
                    dfl::add(dfl::add(dfl::mul(ld(A4, 0), aa), dfl::mul(ld(A4, 1), ab)), dfl::mul(ld(B4, 0), bb)));
                s = dfl::add(s, dfl::mul(ld(B4, 1), dfl::rsqrt(r2)));
            }
            a01 = a10 = sc * dfl::to_double(s);
        }
    } else if (TYPE == EDGE) {
        // vectors (a, b, d) and their Gram matrix
        const F2* V[3] = {a, b, d};
        F2 G[3][3];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = u; v < 3; ++v) G[u][v] = G[v][u] = dfl::dot3(V[u], V[v]);
        const int q = Q > 0 ? Q : npts;
        F2 ssum{0.0f, 0.0f}, sb{0.0f, 0.0f}, sd{0.0f, 0.0f};
        auto region = [&](auto RC) {
            constexpr int R = decltype(RC)::value;
            // coefficients of A, B2, C in o: integer combinations of the Gram entries
            F2 co[3][3];
#pragma unroll
            for (int Qi = 0; Qi < 3; ++Qi)
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    F2 acc{0.0f, 0.0f};
#pragma unroll
                    for (int u = 0; u < 3; ++u)
#pragma unroll
                        for (int v = u; v < 3; ++v) {
                            const int k = u == v ? qweight(R, Qi, p, u, u) : qweight(R, Qi, p, u, v) + qweight(R, Qi, p, v, u);
                            if (k != 0) acc = dfl::add(acc, dfl::mul_k(G[u][v], (float)k));
                        }
                    co[Qi][p] = acc;
                }
#pragma unroll 1
            for (int oi = 0; oi < q; ++oi) {
                const float4 O = sA[oi];
                const F2 o = ld(O, 0), wo = ld(O, 1);
                const F2 A = horner2(co[0][0], co[0][1], co[0][2], o);
                const F2 B2 = horner2(co[1][0], co[1][1], co[1][2], o);
                const F2 C = horner2(co[2][0], co[2][1], co[2][2], o);
                F2 f0{0.0f, 0.0f}, f1{0.0f, 0.0f};
#pragma unroll
                for (int k = 0; k < q; ++k) {
                    const float4 T4 = sA[k];
                    const F2 tt = ld(T4, 0);
                    const F2 wt = R == 0 ? ld(T4, 1) : ld(sB[k], 0);  // w_t (R1) or w_t t
                    const F2 r2 = dfl::renorm(horner2(A, B2, C, tt));
                    const F2 y = dfl::rsqrt(r2);
                    if (KER == SLP) {
                        f0 = dfl::add(f0, dfl::mul(wt, y));
                    } else {
                        const F2 f = dfl::mul(wt, dfl::mul(dfl::mul(y, y), y));
                        f0 = dfl::add(f0, f);
                        f1 = dfl::add(f1, dfl::mul(f, tt));
                    }
                }
                if (KER == SLP) {
                    ssum = dfl::add(ssum, dfl::mul(wo, f0));
                } else {
                    // sum f w over the b and d components: f0 F(o) + f1 G(o)
                    const F2 of0 = dfl::mul(o, f0), of1 = dfl::mul(o, f1);
                    auto comp = [&](int u) {
                        F2 acc{0.0f, 0.0f};
                        const int k0 = ecoef(R, 0, u), k1 = ecoef(R, 1, u), k2 = ecoef(R, 2, u), k3 = ecoef(R, 3, u);
                        if (k0 != 0) acc = dfl::add(acc, dfl::mul_k(f0, (float)k0));
                        if (k1 != 0) acc = dfl::add(acc, dfl::mul_k(of0, (float)k1));
                        if (k2 != 0) acc = dfl::add(acc, dfl::mul_k(f1, (float)k2));
                        if (k3 != 0) acc = dfl::add(acc, dfl::mul_k(of1, (float)k3));
                        return acc;
                    };
                    sb = dfl::add(sb, dfl::mul(wo, comp(1)));
                    sd = dfl::add(sd, dfl::mul(wo, comp(2)));
                }
            }
        };
        region(std::integral_constant<int, 0>{});
        region(std::integral_constant<int, 1>{});
        region(std::integral_constant<int, 2>{});
        region(std::integral_constant<int, 3>{});
        region(std::integral_constant<int, 4>{});
        if (KER == SLP) {
            a01 = a10 = sc * dfl::to_double(ssum) * (1.0 / 6.0);
        } else {
            // V = (sa a + sb b + sd d) / 2; a lies in both planes, b in lo's, d in hi's
            a01 = 0.5 * sc * dfl::to_double(dfl::mul(sb, dfl::dot3(b, del)));
            a10 = 0.5 * sc * dfl::to_double(dfl::mul(sd, dfl::dot3(d, del)));
        }
    } else {  // VERTEX: vectors (a, b, c, d)
        const F2 aa = dfl::dot3(a, a), bb = dfl::dot3(b, b), cc = dfl::dot3(c, c), dd = dfl::dot3(d, d);
        const F2 ab = dfl::dot3(a, b), ac = dfl::dot3(a, c), ad = dfl::dot3(a, d), bc = dfl::dot3(b, c),
                 bd = dfl::dot3(b, d), cd = dfl::dot3(c, d);
        const int q = Q > 0 ? Q : npts;
        F2 ssum{0.0f, 0.0f}, sa{0.0f, 0.0f}, sb{0.0f, 0.0f}, sc2{0.0f, 0.0f}, sd{0.0f, 0.0f};
#pragma unroll 1
        for (int reg = 0; reg < 2; ++reg) {
            // R1: U = a + e1 b, V = c + e3 d;  R2: U = c + e1 d, V = a + e3 b
            const F2 uu = reg == 0 ? aa : cc, uv2 = dfl::mul_k(reg == 0 ? ab : cd, 2.0f), vv = reg == 0 ? bb : dd;
            const F2 pp = reg == 0 ? cc : aa, pq2 = dfl::mul_k(reg == 0 ? cd : ab, 2.0f), qq = reg == 0 ? dd : bb;
            const F2 b0 = ac, b1 = reg == 0 ? ad : bc, b2 = reg == 0 ? bc : ad;
            // C_l = |V(e3_l)|^2 (held for the default order)
            F2 Cl[Q > 0 ? Q : 1];
            if (Q > 0) {
#pragma unroll
                for (int l = 0; l < (Q > 0 ? Q : 1); ++l) Cl[l] = horner2(pp, pq2, qq, ld(sA[l], 0));
            }
#pragma unroll 1
            for (int i = 0; i < q; ++i) {
                const float4 I4 = sA[i];
                const F2 e1 = ld(I4, 0), w1 = ld(I4, 1);
                const F2 A = horner2(uu, uv2, vv, e1);
                const F2 Bi0 = dfl::add(b0, dfl::mul(e1, b2)), Bi1 = dfl::add(b1, dfl::mul(e1, bd));
                F2 t0{0.0f, 0.0f}, t1{0.0f, 0.0f}, t2{0.0f, 0.0f};
#pragma unroll
                for (int l = 0; l < q; ++l) {
                    const float4 L4 = sA[l];
                    const F2 e3 = ld(L4, 0), w3 = ld(L4, 1);
                    const F2 C = Q > 0 ? Cl[Q > 0 ? l : 0] : horner2(pp, pq2, qq, e3);
                    const F2 m2B = dfl::mul_k(dfl::add(Bi0, dfl::mul(e3, Bi1)), -2.0f);
                    F2 f0{0.0f, 0.0f}, f1{0.0f, 0.0f};
#pragma unroll
                    for (int k = 0; k < q; ++k) {
                        const F2 e2 = ld(sA[k], 0), W = ld(sB[k], 0);
                        const F2 r2 = dfl::renorm(horner2(A, m2B, C, e2));
                        const F2 y = dfl::rsqrt(r2);
                        if (KER == SLP) {
                            f0 = dfl::add(f0, dfl::mul(W, y));
                        } else {
                            const F2 f = dfl::mul(W, dfl::mul(dfl::mul(y, y), y));
                            f0 = dfl::add(f0, f);
                            f1 = dfl::add(f1, dfl::mul(f, e2));
                        }
                    }
                    t0 = dfl::add(t0, dfl::mul(w3, f0));
                    if (KER != SLP) {
                        t1 = dfl::add(t1, dfl::mul(w3, f1));
                        t2 = dfl::add(t2, dfl::mul(dfl::mul(w3, e3), f1));
                    }
                }
                const F2 T0 = dfl::mul(w1, t0);
                if (KER == SLP) {
                    ssum = dfl::add(ssum, T0);
                } else if (reg == 0) {  // w = a + e1 b - e2 c - e2 e3 d
                    sa = dfl::add(sa, T0);
                    sb = dfl::add(sb, dfl::mul(e1, T0));
                    sc2 = dfl::sub(sc2, dfl::mul(w1, t1));
                    sd = dfl::sub(sd, dfl::mul(w1, t2));
                } else {                // w = e2 a + e2 e3 b - c - e1 d
                    sa = dfl::add(sa, dfl::mul(w1, t1));
                    sb = dfl::add(sb, dfl::mul(w1, t2));
                    sc2 = dfl::sub(sc2, T0);
                    sd = dfl::sub(sd, dfl::mul(e1, T0));
                }
            }
        }
        if (KER == SLP) {
            a01 = a10 = sc * dfl::to_double(ssum) * (1.0 / 3.0);
        } else {
            // V = (sa a + sb b + sc c + sd d) / 2; a, b in lo's plane, c, d in hi's
            a01 = 0.5 * sc * dfl::to_double(dfl::add(dfl::mul(sa, dfl::dot3(a, del)), dfl::mul(sb, dfl::dot3(b, del))));
            a10 = 0.5 * sc * dfl::to_double(dfl::add(dfl::mul(sc2, dfl::dot3(c, del)), dfl::mul(sd, dfl::dot3(d, del))));
        }
    }
    if (mode == 1) {
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
        for (int r = 0; r < nr; ++r) atomicAdd(&yp[(int64_t)lo * nr + r], a01 * xp[(int64_t)lo * nr + r]);
    } else {
        for (int r = 0; r < nr; ++r) {
            atomicAdd(&yp[(int64_t)lo * nr + r], a01 * xp[(int64_t)hi * nr + r]);
            atomicAdd(&yp[(int64_t)hi * nr + r], a10 * xp[(int64_t)lo * nr + r]);
        }
    }
}

template <int TYPE, int KER>
static void sing_df_go(int mode, int npairs, cudaStream_t s, const Geom& g, const int* lo, const int* hi,
                       const int* code, const double* tab, int npts, bool tr, int nr, const double* xp, double* yp,
                       double* v0, double* v1) {
    const size_t smem = (size_t)npts * 2 * sizeof(float4);
    const dim3 grid((npairs + kThrS - 1) / kThrS);
    // the default 5 points per direction with the point loops unrolled (edge and vertex pairs)
    auto kern = TYPE != IDENTICAL && npts == 5 ? k_singular_df<TYPE, KER, 5> : k_singular_df<TYPE, KER, 0>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, kThrS, smem, s>>>(g, npairs, lo, hi, code, tab, npts, mode, tr, nr, xp, yp, v0, v1);
}

void launch_singular_df(const Geom& g, int type, int ker, int npairs, const int* lo, const int* hi, const int* code,
                        const double* tab, int npts, int mode, bool transpose, int NR, const double* xp, double* yp,
                        double* val0, double* val1, cudaStream_t s) {
    if (npairs <= 0) return;
    const bool slp = ker == SLP;
    if (type == IDENTICAL) {
        // the double layer's entry of a triangle with itself vanishes: zero values, nothing to add
        if (slp) sing_df_go<IDENTICAL, SLP>(mode, npairs, s, g, lo, hi, code, tab, npts, transpose, NR, xp, yp, val0, val1);
        else if (mode == 1) {
            cudaMemsetAsync(val0, 0, (size_t)npairs * sizeof(double), s);
            cudaMemsetAsync(val1, 0, (size_t)npairs * sizeof(double), s);
        }
    } else if (type == EDGE) {
        if (slp) sing_df_go<EDGE, SLP>(mode, npairs, s, g, lo, hi, code, tab, npts, transpose, NR, xp, yp, val0, val1);
        else sing_df_go<EDGE, DLP>(mode, npairs, s, g, lo, hi, code, tab, npts, transpose, NR, xp, yp, val0, val1);
    } else {
        if (slp) sing_df_go<VERTEX, SLP>(mode, npairs, s, g, lo, hi, code, tab, npts, transpose, NR, xp, yp, val0, val1);
        else sing_df_go<VERTEX, DLP>(mode, npairs, s, g, lo, hi, code, tab, npts, transpose, NR, xp, yp, val0, val1);
    }
}

}  // namespace h2
