// Nearfield blocks, regular pairs (section 2: nearfield leaves L^-; entries of
// section 1, eq. (slp) / eq. (dlp) by the 7-point rule on each triangle), each
// unordered pair of leaves {t, s} once.
//
// The single-layer matrix is symmetric, g_ij = g_ji, and the two double-layer
// entries of a pair share their 49 distances:
//   k_ij ~ sum_pq w_p w_q (x_p - y_q) . n_j / r^3,   k_ji ~ sum_pq w_p w_q (y_q - x_p) . n_i / r^3,
// where (x_p - y_q) . n_j is the height h_p of x_p above the plane of tau_j and
// (y_q - x_p) . n_i the height h_q of y_q above the plane of tau_i.  So the CTA
// of row leaf t walks the nearfield leaves s >= t, evaluates the |t| x |s|
// pairs once, adds the row-side products to y_t (registers) and the
// column-side products to y_s (an entry tile in shared memory, then a small
// product with x_t and FP64 atomics).  The diagonal block s = t is evaluated
// in full and applied on the row side only.
//
// Work layout: thread (il, kk), il < |t|, owns row triangle i = t.begin + il
// (its 7 points in registers) and every K-th column of a chunk of column
// leaves staged together (up to kCol triangles and kEnt entries), so that the
// threads of a CTA stay busy across leaf boundaries.  Pairs that share a
// vertex are left to the singular kernel (entry 0 here).
//
// FP32 (mixed tier): points are stored as offsets from their triangle's
// centroid and the centroid difference D = c_i - c_j is formed from float
// splits hi + lo (the hi difference is exact for nearby points, Sterbenz), so
// x_p - y_q keeps ~1e-7 relative accuracy even for touching neighbours.
// Double-layer heights are O(h^2 kappa) against coordinates O(h), so they are
// formed without cancellation in FP32:
//   h_p = D . n_j + (u_p - 1/3) E1_i . delta + (v_p - 1/3) E2_i . delta,
//   h_q = -D . n_j + D . delta - (u_q - 1/3) F1_j . delta - (v_q - 1/3) F2_j . delta,
// with delta = n_j - n_i from the split normals (E1, E2 edges of tau_i, F1, F2
// of tau_j; E . n_i = 0 on the plane of tau_i) and D . n_j as an exact
// double-float dot product: Dekker's product (the FMA residual of each
// product) and Knuth's TwoSum for the cancelling sum.
#include <algorithm>
#include <type_traits>

#include "dmath.cuh"
#include "f32x2.cuh"
#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;
constexpr int kThreads = 256;
constexpr int kEnt = 4096;  // entries of one chunk (rows of t x staged columns)
constexpr int kCol = 128;   // staged column triangles of one chunk

__device__ __forceinline__ float rsqrt_f32(float a) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}

// Knuth's TwoSum: s + e = a + b exactly (round to nearest, no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Byte offsets into the dynamic shared memory of one CTA.
template <typename T, int NR, bool DLPK, bool STORE = false>
struct Smem {
    static constexpr size_t al(size_t x) { return (x + 15) & ~size_t(15); }
    static constexpr bool F32 = std::is_same<T, float>::value;
    static constexpr size_t A = 0;                                   // T [kEnt] column-side entries [il][jc]
    static constexpr size_t Q = al(A + sizeof(T) * kEnt);            // T [3][kCol*7] column points
    static constexpr size_t CH = al(Q + sizeof(T) * 3 * kCol * 7);   // float [6][kCol] centroid hi, lo (F32)
    static constexpr size_t AR = al(CH + (F32 ? 4 * 6 * kCol : 0));  // T [kCol] areas
    static constexpr size_t VID = al(AR + sizeof(T) * kCol);         // int [3][kCol] vertex ids
    static constexpr size_t GID = al(VID + 4 * 3 * kCol);            // int [kCol] tree positions
    static constexpr size_t XC = al(GID + 4 * kCol);                 // T [kCol][NR] x of the columns
    static constexpr size_t XR = al(XC + sizeof(T) * kCol * NR);     // T [kMaxLeaf][NR] x of the row leaf
    // double layer: F32 float [12][kCol] (n hi, n lo, F1, F2); F64 double [4][kCol] (n, plane offset)
    static constexpr size_t NRM = al(XR + sizeof(T) * kMaxLeaf * NR);
    static constexpr size_t SB = al(NRM + (DLPK ? (F32 ? 4 * 12 * kCol : 8 * 4 * kCol) : 0));
    static constexpr size_t END = al(SB + (STORE ? 4 * kCol : 0));  // int [kCol] block of each column (storing)
    static constexpr size_t RED = sizeof(double) * kThreads * NR;  // final row reduction (reuses the front)
    static constexpr size_t BYTES = END > RED ? END : RED;
};
}  // namespace

// the work of one row leaf (index bi of the row list).  STORE: instead of
// applying the entries, write a_ij / (4 pi) of block (t, s) at
// ns.off_ts[b] + j' (|t| | 1) + i' and a_ji / (4 pi) of block (s, t) at
// ns.off_st[b] + i' (|s| | 1) + j' (i', j' positions within the leaves; the
// stored layout of the apply in k_nearstore.cu); pairs sharing a vertex get 0.
template <int NR, bool DLPK, bool F32, bool STORE = false>
__device__ __forceinline__ void near_sym_row(const Geom& g, const Tree& t, const Consts& c,
                                             const int* __restrict__ rows, const int* __restrict__ ptr,
                                             const int* __restrict__ col, bool transpose,
                                             const double* __restrict__ xp, double* __restrict__ yp, int bi,
                                             const NearStore& ns = NearStore{}) {
    using T = typename std::conditional<F32, float, double>::type;
    using L = Smem<T, NR, DLPK, STORE>;
    extern __shared__ __align__(16) unsigned char smem[];
    T* sA = reinterpret_cast<T*>(smem + L::A);
    T* sq = reinterpret_cast<T*>(smem + L::Q);
    float* sch = reinterpret_cast<float*>(smem + L::CH);
    T* sarea = reinterpret_cast<T*>(smem + L::AR);
    int* svid = reinterpret_cast<int*>(smem + L::VID);
    int* sgid = reinterpret_cast<int*>(smem + L::GID);
    T* sxc = reinterpret_cast<T*>(smem + L::XC);
    T* sxr = reinterpret_cast<T*>(smem + L::XR);
    float* snf = reinterpret_cast<float*>(smem + L::NRM);
    double* snd = reinterpret_cast<double*>(smem + L::NRM);
    int* sblk = reinterpret_cast<int*>(smem + L::SB);

    const int row = rows[bi];
    const int rb = t.begin[row], R = t.end[row] - rb;
    const int K = kThreads / R;
    const int tid = threadIdx.x;
    const int il = tid % R, kk = tid / R;
    const bool active = kk < K;
    const int n = g.n;
    const int cmax = min(kCol, kEnt / R);

    // rule constants in the working precision (kernel parameters)
    const T* w = F32 ? reinterpret_cast<const T*>(c.rwf) : reinterpret_cast<const T*>(c.rw);
    const float* ru = c.ruf;
    const float* rv = c.rvf;

    if (!STORE)
        for (int e = tid; e < R * NR; e += kThreads) sxr[e] = (T)xp[(int64_t)rb * NR + e];

    // row triangle i = rb + il
    T px[7], py[7], pz[7];
    float chi[3] = {0, 0, 0}, clo[3] = {0, 0, 0};
    float nhi[3] = {0, 0, 0}, nlo[3] = {0, 0, 0}, E1[3] = {0, 0, 0}, E2[3] = {0, 0, 0};
    double rn[3] = {0, 0, 0}, rplane = 0.0;
    T ai = 0;
    int vi[3] = {-1, -1, -1};
    if (active) {
        const int i = rb + il;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            vi[d] = g.vid[d * n + i];
            if (F32) {
                chi[d] = g.chl[d * n + i];
                clo[d] = g.chl[(3 + d) * n + i];
                if (DLPK) {
                    nhi[d] = g.nef[d * n + i];
                    nlo[d] = g.nef[(3 + d) * n + i];
                    E1[d] = g.nef[(6 + d) * n + i];
                    E2[d] = g.nef[(9 + d) * n + i];
                }
            } else if (DLPK) {
                rn[d] = g.nrm[d * n + i];
            }
        }
        if (!F32 && DLPK) rplane = g.plane[i];
        ai = (T)g.area[i];
#pragma unroll
        for (int p = 0; p < 7; ++p) {
            if (F32) {
                px[p] = (T)g.qo[((int64_t)0 * n + i) * 7 + p];
                py[p] = (T)g.qo[((int64_t)1 * n + i) * 7 + p];
                pz[p] = (T)g.qo[((int64_t)2 * n + i) * 7 + p];
            } else {
                px[p] = (T)g.qa[((int64_t)0 * n + i) * 7 + p];
                py[p] = (T)g.qa[((int64_t)1 * n + i) * 7 + p];
                pz[p] = (T)g.qa[((int64_t)2 * n + i) * 7 + p];
            }
        }
    }
    // FP32: the row points as packed pairs (0,1), (2,3), (4,5), and packed weights
    f2 PX[3], PY[3], PZ[3], W2[3];
    if constexpr (F32) {
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            PX[g] = pk(px[2 * g], px[2 * g + 1]);
            PY[g] = pk(py[2 * g], py[2 * g + 1]);
            PZ[g] = pk(pz[2 * g], pz[2 * g + 1]);
            W2[g] = pk(w[2 * g], w[2 * g + 1]);
        }
    }
    T acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0;

    const int bbeg = ptr[bi], bend = ptr[bi + 1];
    for (int b = bbeg; b < bend;) {
        // chunk: column leaves b .. b2-1 (the same decision in every thread)
        int ctot = 0, b2 = b;
        while (b2 < bend) {
            const int s = col[b2];
            const int C = t.end[s] - t.begin[s];
            if (ctot + C > cmax) break;
            ctot += C;
            ++b2;
        }
        if (b2 == b) break;  // a leaf larger than a chunk (excluded when the operator is created)
        const int cdiag = (b == bbeg && col[b] == row) ? R : 0;  // leading columns of the diagonal block
        __syncthreads();  // the previous chunk is done with the staging area
        for (int bl = b, off = 0; bl < b2; ++bl) {
            const int s = col[bl];
            const int cb = t.begin[s], C = t.end[s] - cb;
            for (int e = tid; e < C; e += kThreads) {
                sgid[off + e] = cb + e;
                if (STORE) sblk[off + e] = bl;
            }
            off += C;
        }
        __syncthreads();
        for (int e = tid; e < ctot * 7; e += kThreads) {
            const int j = sgid[e / 7], q = e % 7;
#pragma unroll
            for (int d = 0; d < 3; ++d)
                sq[d * (kCol * 7) + e] = F32 ? (T)g.qo[((int64_t)d * n + j) * 7 + q] : (T)g.qa[((int64_t)d * n + j) * 7 + q];
        }
        for (int e = tid; e < ctot; e += kThreads) {
            const int j = sgid[e];
            sarea[e] = (T)g.area[j];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                svid[d * kCol + e] = g.vid[d * n + j];
                if (F32) {
                    sch[d * kCol + e] = g.chl[d * n + j];
                    sch[(3 + d) * kCol + e] = g.chl[(3 + d) * n + j];
                }
            }
            if (DLPK) {
                if (F32) {
#pragma unroll
                    for (int d = 0; d < 12; ++d) snf[d * kCol + e] = g.nef[d * n + j];
                } else {
#pragma unroll
                    for (int d = 0; d < 3; ++d) snd[d * kCol + e] = g.nrm[d * n + j];
                    snd[3 * kCol + e] = g.plane[j];
                }
            }
        }
        if (!STORE)
            for (int e = tid; e < ctot * NR; e += kThreads) sxc[e] = (T)xp[(int64_t)sgid[e / NR] * NR + e % NR];
        __syncthreads();

        // phase 1: entries (row side into registers, column side into sA)
        if (active) {
            for (int jc = kk; jc < ctot; jc += K) {
                bool sing = false;
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb) sing |= (vi[a] == svid[bb * kCol + jc]);
                T arow = 0, acol = 0;
                if (!sing) {
                    T Dx = 0, Dy = 0, Dz = 0;
                    float Dh[3] = {0, 0, 0}, Dl[3] = {0, 0, 0};
                    if (F32) {
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            Dh[d] = chi[d] - sch[d * kCol + jc];
                            Dl[d] = clo[d] - sch[(3 + d) * kCol + jc];
                        }
                        Dx = Dh[0] + Dl[0];
                        Dy = Dh[1] + Dl[1];
                        Dz = Dh[2] + Dl[2];
                    }
                    // double layer: heights of the row points above plane j (hp)
                    // and of the column points above plane i (hq = H0q + ru_q f1 + rv_q f2)
                    T hp[7];
                    T H0q = 0, f1 = 0, f2v = 0;
                    double cn[3] = {0, 0, 0}, cplane = 0.0;
                    if (DLPK) {
                        if (F32) {
                            float nh[3], dl[3];
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                nh[d] = snf[d * kCol + jc];
                                dl[d] = (nh[d] - nhi[d]) + (snf[(3 + d) * kCol + jc] - nlo[d]);
                            }
                            // H0 = D . n_j, exact products and sums of the cancelling hi part
                            const float p0 = __fmul_rn(Dh[0], nh[0]), p1 = __fmul_rn(Dh[1], nh[1]),
                                        p2 = __fmul_rn(Dh[2], nh[2]);
                            const float r0 = fmaf(Dh[0], nh[0], -p0), r1 = fmaf(Dh[1], nh[1], -p1),
                                        r2 = fmaf(Dh[2], nh[2], -p2);
                            float s1, t1, s2, t2;
                            two_sum(p0, p1, s1, t1);
                            two_sum(s1, p2, s2, t2);
                            float cr = (t1 + t2) + (r0 + r1 + r2);
#pragma unroll
                            for (int d = 0; d < 3; ++d)
                                cr = fmaf(Dh[d], snf[(3 + d) * kCol + jc], fmaf(Dl[d], nh[d], cr));
                            const float H0 = s2 + cr;
                            const float e1 = E1[0] * dl[0] + E1[1] * dl[1] + E1[2] * dl[2];
                            const float e2 = E2[0] * dl[0] + E2[1] * dl[1] + E2[2] * dl[2];
#pragma unroll
                            for (int p = 0; p < 7; ++p) hp[p] = w[p] * fmaf(ru[p], e1, fmaf(rv[p], e2, H0));
                            H0q = (Dx * dl[0] + Dy * dl[1] + Dz * dl[2]) - H0;
                            f1 = -(snf[6 * kCol + jc] * dl[0] + snf[7 * kCol + jc] * dl[1] + snf[8 * kCol + jc] * dl[2]);
                            f2v = -(snf[9 * kCol + jc] * dl[0] + snf[10 * kCol + jc] * dl[1] + snf[11 * kCol + jc] * dl[2]);
                        } else {
                            cn[0] = snd[jc];
                            cn[1] = snd[kCol + jc];
                            cn[2] = snd[2 * kCol + jc];
                            cplane = snd[3 * kCol + jc];
#pragma unroll
                            for (int p = 0; p < 7; ++p)
                                hp[p] = w[p] * (T)(px[p] * cn[0] + py[p] * cn[1] + pz[p] * cn[2] - cplane);
                        }
                    }
                    T S1 = 0, S2 = 0;
                    if constexpr (F32) {
                        // row points in packed pairs (0,1), (2,3), (4,5) and point 6 alone
                        f2 HP[3];
                        if constexpr (DLPK) {
#pragma unroll
                            for (int g = 0; g < 3; ++g) HP[g] = pk(hp[2 * g], hp[2 * g + 1]);
                        }
#pragma unroll
                        for (int q = 0; q < 7; ++q) {
                            const float yx = Dx - sq[jc * 7 + q], yy = Dy - sq[kCol * 7 + jc * 7 + q],
                                        yz = Dz - sq[2 * kCol * 7 + jc * 7 + q];
                            const f2 YX = pk(yx, yx), YY = pk(yy, yy), YZ = pk(yz, yz);
                            f2 A1 = 0, A2 = 0;
#pragma unroll
                            for (int g = 0; g < 3; ++g) {
                                const f2 dx = add2(PX[g], YX), dy = add2(PY[g], YY), dz = add2(PZ[g], YZ);
                                const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                                float r0, r1;
                                upk(r2, r0, r1);
                                const f2 ri = pk(rsqrt_f32(r0), rsqrt_f32(r1));
                                if constexpr (!DLPK) {
                                    A1 = fma2(W2[g], ri, A1);
                                } else {
                                    const f2 ri3 = mul2(mul2(ri, ri), ri);
                                    A1 = fma2(HP[g], ri3, A1);
                                    A2 = fma2(W2[g], ri3, A2);
                                }
                            }
                            const float dx6 = px[6] + yx, dy6 = py[6] + yy, dz6 = pz[6] + yz;
                            const float ri6 = rsqrt_f32(dx6 * dx6 + dy6 * dy6 + dz6 * dz6);
                            float a0, a1;
                            upk(A1, a0, a1);
                            if constexpr (!DLPK) {
                                S1 = fmaf(w[q], fmaf(w[6], ri6, a0 + a1), S1);
                            } else {
                                const float r36 = ri6 * ri6 * ri6;
                                float b0, b1;
                                upk(A2, b0, b1);
                                const float hq = fmaf(ru[q], f1, fmaf(rv[q], f2v, H0q));
                                S1 = fmaf(w[q], fmaf(hp[6], r36, a0 + a1), S1);
                                S2 = fmaf(w[q] * hq, fmaf(w[6], r36, b0 + b1), S2);
                            }
                        }
                    } else {
#pragma unroll
                    for (int q = 0; q < 7; ++q) {
                        const T ex = sq[jc * 7 + q], ey = sq[kCol * 7 + jc * 7 + q], ez = sq[2 * kCol * 7 + jc * 7 + q];
                        const T yx = ex, yy = ey, yz = ez;
                        T sp1 = 0, sp2 = 0;
#pragma unroll
                        for (int p = 0; p < 7; ++p) {
                            const T dx = px[p] - yx;
                            const T dy = py[p] - yy;
                            const T dz = pz[p] - yz;
                            const T r2 = dx * dx + dy * dy + dz * dz;
                            if (!DLPK) {
                                // w/2 y (3 - r2 y^2): one Newton step for 1/sqrt(r2) folded in
                                double y;
                                asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"((double)r2));
                                const double tq = r2 * y;
                                sp1 = fma(w[p] * y, fma(-tq, y, 3.0), sp1);
                            } else {
                                const T ri = (T)rsqrt_nr((double)r2);
                                const T ri3 = ri * ri * ri;
                                sp1 += hp[p] * ri3;
                                sp2 += w[p] * ri3;
                            }
                        }
                        if (!DLPK) {
                            S1 += w[q] * sp1;
                        } else {
                            const T hq = (T)(ex * rn[0] + ey * rn[1] + ez * rn[2] - rplane);
                            S1 += w[q] * sp1;
                            S2 += (w[q] * hq) * sp2;
                        }
                    }
                    }
                    const T aa = ai * sarea[jc];
                    if (!DLPK) {
                        arow = acol = (F32 ? aa : (T)0.5 * aa) * S1;
                    } else {
                        // S1 -> k_ij (row i, column j), S2 -> k_ji
                        arow = aa * (transpose ? S2 : S1);
                        acol = aa * (transpose ? S1 : S2);
                    }
                }
                if constexpr (STORE) {
                    T* nout = reinterpret_cast<T*>(ns.N);
                    const int bl = sblk[jc];
                    const int s = col[bl];
                    const int jl = sgid[jc] - t.begin[s];
                    nout[ns.off_ts[bl] + (int64_t)jl * (R | 1) + il] = arow * (T)kInv4Pi;
                    if (jc >= cdiag)  // the diagonal block is written whole on the row side
                        nout[ns.off_st[bl] + (int64_t)il * ((t.end[s] - t.begin[s]) | 1) + jl] = acol * (T)kInv4Pi;
                } else {
#pragma unroll
                    for (int r = 0; r < NR; ++r) acc[r] += arow * sxc[jc * NR + r];
                    sA[il * cmax + jc] = acol;
                }
            }
        }
        __syncthreads();
        if (STORE) {
            b = b2;
            continue;
        }

        // phase 2: column side of the off-diagonal leaves, y_j += sum_i a_ji x_i
        for (int e = tid; e < (ctot - cdiag) * NR; e += kThreads) {
            const int jc = cdiag + e / NR, r = e % NR;
            T sum = 0;
            for (int i = 0; i < R; ++i) sum += sA[i * cmax + jc] * sxr[i * NR + r];
            atomicAdd(&yp[(int64_t)sgid[jc] * NR + r], (double)(sum * (T)kInv4Pi));
        }
        b = b2;
    }
    if (STORE) return;
    __syncthreads();
    // row side: reduce the K partial sums of each row (in the working precision)
    T* sred = reinterpret_cast<T*>(smem);
#pragma unroll
    for (int r = 0; r < NR; ++r) sred[tid * NR + r] = active ? acc[r] : (T)0;
    __syncthreads();
    for (int e = tid; e < R * NR; e += kThreads) {
        const int i = e / NR, r = e % NR;
        T s = 0;
        for (int q = 0; q < K; ++q) s += sred[(q * R + i) * NR + r];
        atomicAdd(&yp[(int64_t)(rb + i) * NR + r], (double)(s * (T)kInv4Pi));
    }
}

// One CTA per row leaf (work == nullptr), or persistent CTAs that take the
// next row from the counter *work (zero before the launch) until none is left.
// NB: CTAs per SM the register budget is sized for (0: 4 for the FP32 single
// layer, else 2); a launch shape the autotuner chooses.
template <int NR, bool DLPK, bool F32, bool PERSIST, int NB>
__global__ void __launch_bounds__(kThreads, NB > 0 ? NB : ((F32 && !DLPK) ? 4 : 2))
    k_near_sym(Geom g, Tree t, Consts c, int nrows, const int* __restrict__ rows, const int* __restrict__ ptr,
               const int* __restrict__ col, bool transpose, const double* __restrict__ xp, double* __restrict__ yp,
               int* __restrict__ work) {
    if constexpr (!PERSIST) {
        near_sym_row<NR, DLPK, F32>(g, t, c, rows, ptr, col, transpose, xp, yp, blockIdx.x);
        return;
    }
    __shared__ int s_bi;
    while (true) {
        __syncthreads();  // the previous row is done with shared memory and s_bi
        if (threadIdx.x == 0) s_bi = atomicAdd(work, 1);
        __syncthreads();
        const int bi = s_bi;
        if (bi >= nrows) break;
        near_sym_row<NR, DLPK, F32>(g, t, c, rows, ptr, col, transpose, xp, yp, bi);
    }
}

// Storing variant: one CTA per row of the unordered list, writes the entries.
template <bool DLPK, bool F32>
__global__ void __launch_bounds__(kThreads, 2)
    k_near_sym_store(Geom g, Tree t, Consts c, const int* __restrict__ rows, const int* __restrict__ ptr,
                     const int* __restrict__ col, NearStore ns) {
    near_sym_row<1, DLPK, F32, true>(g, t, c, rows, ptr, col, false, nullptr, nullptr, blockIdx.x, ns);
}

void launch_near_sym_store(const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                           const int* col, int ker, bool fp32, const NearStore& ns, cudaStream_t s) {
    if (nrows <= 0) return;
    auto go = [&](auto kern, size_t smem) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<nrows, kThreads, smem, s>>>(g, t, c, rows, ptr, col, ns);
    };
    const bool dlp = ker != SLP;
    if (fp32) {
        if (dlp) go(k_near_sym_store<true, true>, Smem<float, 1, true, true>::BYTES);
        else go(k_near_sym_store<false, true>, Smem<float, 1, false, true>::BYTES);
    } else {
        if (dlp) go(k_near_sym_store<true, false>, Smem<double, 1, true, true>::BYTES);
        else go(k_near_sym_store<false, false>, Smem<double, 1, false, true>::BYTES);
    }
}

template <int NR, bool DLPK, bool F32>
static void near_sym_go(int nrows, cudaStream_t s, const Geom& g, const Tree& t, const Consts& c, const int* rows,
                        const int* ptr, const int* col, bool tr, const double* xp, double* yp, int* work, int nb) {
    using T = typename std::conditional<F32, float, double>::type;
    constexpr size_t smem = Smem<T, NR, DLPK>::BYTES;
    auto go = [&](auto kplain, auto kpers) {
        if (!work) {
            cudaFuncSetAttribute(kplain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kplain<<<nrows, kThreads, smem, s>>>(g, t, c, nrows, rows, ptr, col, tr, xp, yp, nullptr);
            return;
        }
        cudaFuncSetAttribute(kpers, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int grid = std::min(nrows, resident_ctas((const void*)kpers, kThreads, smem));
        cudaMemsetAsync(work, 0, sizeof(int), s);
        kpers<<<grid, kThreads, smem, s>>>(g, t, c, nrows, rows, ptr, col, tr, xp, yp, work);
    };
    if constexpr (F32 && !DLPK) {
        if (nb == 3) go(k_near_sym<NR, DLPK, F32, false, 3>, k_near_sym<NR, DLPK, F32, true, 3>);
        else if (nb == 2) go(k_near_sym<NR, DLPK, F32, false, 2>, k_near_sym<NR, DLPK, F32, true, 2>);
        else go(k_near_sym<NR, DLPK, F32, false, 0>, k_near_sym<NR, DLPK, F32, true, 0>);
    } else {
        go(k_near_sym<NR, DLPK, F32, false, 0>, k_near_sym<NR, DLPK, F32, true, 0>);
    }
}

template <int NR>
static void near_sym_nr(int ker, bool fp32, int nrows, cudaStream_t s, const Geom& g, const Tree& t, const Consts& c,
                        const int* rows, const int* ptr, const int* col, bool tr, const double* xp, double* yp,
                        int* work, int nb) {
    const bool dlp = ker != SLP;
    if (fp32) {
        if (dlp) near_sym_go<NR, true, true>(nrows, s, g, t, c, rows, ptr, col, tr, xp, yp, work, nb);
        else near_sym_go<NR, false, true>(nrows, s, g, t, c, rows, ptr, col, tr, xp, yp, work, nb);
    } else {
        if (dlp) near_sym_go<NR, true, false>(nrows, s, g, t, c, rows, ptr, col, tr, xp, yp, work, nb);
        else near_sym_go<NR, false, false>(nrows, s, g, t, c, rows, ptr, col, tr, xp, yp, work, nb);
    }
}

void launch_near_sym(const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                     const int* col, int ker, bool transpose, bool fp32, int NR, const double* xp, double* yp,
                     const LaunchCfg& cfg, cudaStream_t s) {
    int* work = cfg.work;
    const int nb = cfg.nb;
    if (nrows <= 0) return;
    switch (NR) {
        case 1: near_sym_nr<1>(ker, fp32, nrows, s, g, t, c, rows, ptr, col, transpose, xp, yp, work, nb); break;
        case 4: near_sym_nr<4>(ker, fp32, nrows, s, g, t, c, rows, ptr, col, transpose, xp, yp, work, nb); break;
        case 8: near_sym_nr<8>(ker, fp32, nrows, s, g, t, c, rows, ptr, col, transpose, xp, yp, work, nb); break;
        default: near_sym_nr<16>(ker, fp32, nrows, s, g, t, c, rows, ptr, col, transpose, xp, yp, work, nb); break;
    }
}

}  // namespace h2
