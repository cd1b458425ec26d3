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

// ---------------------------------------------------------------------------
// FP32 single layer (the mixed tiers' hot case): packed over column pairs.
//
// Thread (il, kk) takes row triangle i = rb + il and the column pairs
// (2 pj, 2 pj + 1), pj = kk, kk + K, ...  Each f32x2 lane pair evaluates the
// same row point against the two columns' points, so all 7 x 7 point pairs of
// both entries are packed with no odd point left over, and the column data
// (centroid splits, point offsets, areas) arrive as natural pairs from one
// 64-bit shared-memory load: columns are stored [quantity][jc], adjacent.  The
// row's quantities are held duplicated (p, p) in registers.
// With P_p the row point's offset from the row centroid and Y_q = D - Q_q
// (D the centroid difference, Q_q the column point's offset), the squared
// distance is expanded as |P_p + Y_q|^2 = (|P_p|^2 + |Y_q|^2) + 2 P_p . Y_q:
// one add and three fma per evaluation instead of three add, one mul and two
// fma.  |P_p| is below the triangle's size and the rule's points of regular
// pairs stay apart, so the rounding of the expanded form is that of the
// direct one (float emulation over the nearest regular pairs of sphere, flat
// ellipsoid and jittered cube meshes: 2.3e-8 against 2.2e-8 relative in the
// product).  Per two kernel evaluations the loop issues 4 packed ops for the
// distance, 2 reciprocal square roots and 1 packed op for the sum, whose
// weights take the rule's three values (centre, two orbits).  A column sharing a
// vertex with the row is moved far away (its distance stays finite) and its
// entry masked to zero; the singular kernels supply those entries.  An odd
// column count is padded with one zero-area column far away.
//
// Staging: the column leaves of a row are taken in chunks of at most kColA
// triangles, copied into shared memory by cp.async in two stages, so that the
// next chunk's copies are in flight while the current one is evaluated.  All
// inputs are FP32 (x from the FP32 copy xs, areas from areaf): GB300's FP64
// pipe runs at 1/70 of FP32, and conversions from double would sit on the
// staging path.  The FP64 additions into y take their FP32 sums converted
// exactly by integer operations.
// ---------------------------------------------------------------------------
namespace {
constexpr int kColA = 104;   // staged column triangles of one chunk
constexpr int kEntA = 4160;  // column-side entries of one chunk, (R | 1) x columns: 65 x 64 for the largest leaves
constexpr int kSeg = 128;    // column leaves of a row described in shared memory at a time
static_assert(kColA >= kMaxLeaf && kEntA >= (kMaxLeaf | 1) * kMaxLeaf, "a chunk holds a column leaf of any row leaf");

template <int NR>
struct Smem32 {
    static constexpr size_t al(size_t x) { return (x + 15) & ~size_t(15); }
    // one stage of staged columns
    static constexpr size_t SQ = 0;                          // float [3][7][kColA] point offsets
    static constexpr size_t SCH = al(SQ + 4 * 21 * kColA);   // float [6][kColA] centroid hi, lo
    static constexpr size_t SVID = al(SCH + 4 * 6 * kColA);  // int [3][kColA] vertex ids
    static constexpr size_t SGID = al(SVID + 4 * 3 * kColA); // int [kColA] tree positions
    static constexpr size_t SAR = al(SGID + 4 * kColA);      // float [kColA] areas
    static constexpr size_t SX = al(SAR + 4 * kColA);        // float [kColA][NR] x
    static constexpr size_t STAGE = al(SX + 4 * kColA * NR);
    // CTA layout
    static constexpr size_t A = 0;                           // float [kEntA] column-side entries [jc][R | 1]
    static constexpr size_t ST = al(A + 4 * kEntA);          // two stages
    static constexpr size_t XR = al(ST + 2 * STAGE);         // float [kMaxLeaf][NR] x of the row leaf
    static constexpr size_t RC = al(XR + 4 * kMaxLeaf * NR); // f2 [kMaxLeaf][6] row centroid splits (duplicated)
    static constexpr size_t BL = al(RC + 8 * 6 * kMaxLeaf);  // int2 [kSeg] (first position, size) per block
    static constexpr size_t END = al(BL + 8 * kSeg);
    static constexpr size_t RED = 4 * kThreads * NR;         // final row reduction (reuses the front)
    static constexpr size_t BYTES = END > RED ? END : RED;
};

__device__ __forceinline__ f2 ld2(const float* p) { return *reinterpret_cast<const f2*>(p); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ void cp4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// float -> double, exact, by integer operations (zero and subnormal inputs give
// a signed zero; no infinities or NaNs reach it)
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned hi = (u & 0x80000000u) | (e ? (((e + 896u) << 20) | ((u >> 3) & 0xfffffu)) : 0u);
    const unsigned lo = e ? (u << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}

// one chunk of a row's column leaves: blocks [b, b2) of the staged list
struct Chunk {
    int b, b2, ctot;
};
}  // namespace

template <int NR>
__device__ __forceinline__ void near_slp32_row(const Geom& g, const Tree& t, const Consts& c,
                                               const int* __restrict__ rows, const int* __restrict__ ptr,
                                               const int* __restrict__ col, const float* __restrict__ xs,
                                               double* __restrict__ yp, int bi) {
    using L = Smem32<NR>;
    constexpr int NX = NR < 4 ? 4 : NR;  // row stride of xs
    extern __shared__ __align__(16) unsigned char smem[];
    float* sA = reinterpret_cast<float*>(smem + L::A);
    float* sxr = reinterpret_cast<float*>(smem + L::XR);
    f2* src = reinterpret_cast<f2*>(smem + L::RC);
    int2* sbl = reinterpret_cast<int2*>(smem + L::BL);

    const int row = rows[bi];
    const int rb = t.begin[row], R = t.end[row] - rb;
    const int K = kThreads / R;
    const int tid = threadIdx.x;
    const int il = tid % R, kk = tid / R;
    const bool active = kk < K;
    const int n = g.n;
    const int RS = R | 1;                         // odd stride of the entry tile: no bank conflicts
    const int cmax = min(kColA, kEntA / RS) & ~1;  // even: room for the padding column

    __syncthreads();  // a persistent CTA's previous row is done with shared memory
    for (int e = tid; e < R * NR; e += kThreads) sxr[e] = xs[(int64_t)(rb + e / NR) * NX + e % NR];
    for (int e = tid; e < R * 6; e += kThreads) {
        const float v = g.chl[(e % 6) * n + rb + e / 6];
        src[e] = pk(v, v);
    }

    // row triangle, duplicated into both lanes: 2 P_p, |P_p|^2 (centroid splits in shared memory)
    f2 PX[7], PY[7], PZ[7], CP[7];
    int vi[3];
    float ai;
    {
        const int i = rb + (active ? il : 0);
#pragma unroll
        for (int d = 0; d < 3; ++d) vi[d] = g.vid[d * n + i];
        ai = g.areaf[i];
#pragma unroll
        for (int p = 0; p < 7; ++p) {
            const float x = g.qo[((int64_t)0 * n + i) * 7 + p], y = g.qo[((int64_t)1 * n + i) * 7 + p],
                        z = g.qo[((int64_t)2 * n + i) * 7 + p];
            PX[p] = pk(2.0f * x, 2.0f * x);
            PY[p] = pk(2.0f * y, 2.0f * y);
            PZ[p] = pk(2.0f * z, 2.0f * z);
            const float cp = fmaf(z, z, fmaf(y, y, x * x));
            CP[p] = pk(cp, cp);
        }
    }
    // the rule's weights: centre (point 0), first orbit (1..3), second orbit (4..6)
    const f2 W0 = pk(c.rwf[0], c.rwf[0]), WA = pk(c.rwf[1], c.rwf[1]), WB = pk(c.rwf[4], c.rwf[4]);
    float acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0f;

    const int bbeg = ptr[bi], bend = ptr[bi + 1];
    const bool diag = bend > bbeg && col[bbeg] == row;  // the first column leaf is t itself
    for (int seg = bbeg; seg < bend; seg += kSeg) {
        const int nbl = min(kSeg, bend - seg);
        __syncthreads();
        if (tid < nbl) {
            const int s = col[seg + tid];
            sbl[tid] = make_int2(t.begin[s], t.end[s] - t.begin[s]);
        }
        __syncthreads();
        // the next chunk from block b of this segment; jc -> its tree position jpos
        auto next = [&](int b, int jc, int& jpos) {
            Chunk ch{b, b, 0};
            jpos = -1;
            while (ch.b2 < nbl) {
                const int2 bl = sbl[ch.b2];
                if (ch.ctot + bl.y > cmax) break;
                if (jc >= ch.ctot && jc < ch.ctot + bl.y) jpos = bl.x + (jc - ch.ctot);
                ch.ctot += bl.y;
                ++ch.b2;
            }
            return ch;
        };
        // copies of one chunk into a stage: thread jc (< 128) the point offsets,
        // thread 128 + jc the rest; the padding column by plain stores
        const int jc = tid & 127, half = tid >> 7;
        auto issue = [&](const Chunk& ch, int jpos, unsigned char* st) {
            float* q = reinterpret_cast<float*>(st + L::SQ);
            float* chs = reinterpret_cast<float*>(st + L::SCH);
            int* vid = reinterpret_cast<int*>(st + L::SVID);
            int* gid = reinterpret_cast<int*>(st + L::SGID);
            float* ar = reinterpret_cast<float*>(st + L::SAR);
            float* xc = reinterpret_cast<float*>(st + L::SX);
            if (jc < ch.ctot) {
                if (half == 0) {
#pragma unroll
                    for (int d = 0; d < 3; ++d)
#pragma unroll
                        for (int qq = 0; qq < 7; ++qq) cp4(q + (d * 7 + qq) * kColA + jc, g.qo + ((int64_t)d * n + jpos) * 7 + qq);
                } else {
#pragma unroll
                    for (int d = 0; d < 6; ++d) cp4(chs + d * kColA + jc, g.chl + (int64_t)d * n + jpos);
#pragma unroll
                    for (int d = 0; d < 3; ++d) cp4(vid + d * kColA + jc, g.vid + (int64_t)d * n + jpos);
                    cp4(ar + jc, g.areaf + jpos);
                    if constexpr (NR >= 4) {
#pragma unroll
                        for (int r = 0; r < NR; r += 4) cp16(xc + jc * NR + r, xs + (int64_t)jpos * NX + r);
                    } else {
                        cp4(xc + jc, xs + (int64_t)jpos * NX);
                    }
                    gid[jc] = jpos;
                }
            } else if (jc == ch.ctot && (ch.ctot & 1)) {  // padding column: zero area, far away, no vertex
                if (half == 0) {
#pragma unroll
                    for (int d = 0; d < 21; ++d) q[d * kColA + jc] = 0.0f;
                } else {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        chs[d * kColA + jc] = 1.0e4f;
                        chs[(3 + d) * kColA + jc] = 0.0f;
                        vid[d * kColA + jc] = -2;
                    }
                    ar[jc] = 0.0f;
#pragma unroll
                    for (int r = 0; r < NR; ++r) xc[jc * NR + r] = 0.0f;
                }
            }
        };

        int jpos;
        Chunk cur = next(0, jc, jpos);
        issue(cur, jpos, smem + L::ST);
        cp_commit();
        for (int it = 0; cur.b2 > cur.b; ++it) {
            unsigned char* st = smem + L::ST + (it & 1) * L::STAGE;
            int jn;
            const Chunk nxt = next(cur.b2, jc, jn);
            if (nxt.b2 > nxt.b) issue(nxt, jn, smem + L::ST + ((it + 1) & 1) * L::STAGE);
            cp_commit();
            cp_wait1();  // this thread's copies of the current chunk are done
            __syncthreads();
            const float* sq = reinterpret_cast<const float*>(st + L::SQ);
            const float* sch = reinterpret_cast<const float*>(st + L::SCH);
            const int* svid = reinterpret_cast<const int*>(st + L::SVID);
            const int* sgid = reinterpret_cast<const int*>(st + L::SGID);
            const float* sarea = reinterpret_cast<const float*>(st + L::SAR);
            const float* sxc = reinterpret_cast<const float*>(st + L::SX);
            const int ctot = cur.ctot, ctp = (ctot + 1) & ~1;
            const int cdiag = (diag && seg == bbeg && cur.b == 0) ? R : 0;  // leading columns of the diagonal block

            if (active) {
                for (int pj = kk; 2 * pj < ctp; pj += K) {
                    const int ja = 2 * pj;
                    bool sa = false, sb = false;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const int va = svid[d * kColA + ja], vb = svid[d * kColA + ja + 1];
                        sa |= (va == vi[0]) | (va == vi[1]) | (va == vi[2]);
                        sb |= (vb == vi[0]) | (vb == vi[1]) | (vb == vi[2]);
                    }
                    f2 D[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        D[d] = add2(sub2(src[il * 6 + d], ld2(sch + d * kColA + ja)),
                                    sub2(src[il * 6 + 3 + d], ld2(sch + (3 + d) * kColA + ja)));
                    // a column sharing a vertex: far away (finite distances), entry masked below
                    D[0] = add2(D[0], pk(sa ? 1.0e4f : 0.0f, sb ? 1.0e4f : 0.0f));
                    f2 S = 0;
#pragma unroll
                    for (int q = 0; q < 7; ++q) {
                        const f2 YX = sub2(D[0], ld2(sq + (0 * 7 + q) * kColA + ja));
                        const f2 YY = sub2(D[1], ld2(sq + (1 * 7 + q) * kColA + ja));
                        const f2 YZ = sub2(D[2], ld2(sq + (2 * 7 + q) * kColA + ja));
                        const f2 EQ = fma2(YZ, YZ, fma2(YY, YY, mul2(YX, YX)));
                        f2 ri[7];
#pragma unroll
                        for (int p = 0; p < 7; ++p) {
                            const f2 r2 = fma2(PZ[p], YZ, fma2(PY[p], YY, fma2(PX[p], YX, add2(CP[p], EQ))));
                            float r0, r1;
                            upk(r2, r0, r1);
                            ri[p] = pk(rsqrt_f32(r0), rsqrt_f32(r1));
                        }
                        f2 A = mul2(W0, ri[0]);
                        A = fma2(WA, add2(add2(ri[1], ri[2]), ri[3]), A);
                        A = fma2(WB, add2(add2(ri[4], ri[5]), ri[6]), A);
                        S = fma2(q == 0 ? W0 : q <= 3 ? WA : WB, A, S);
                    }
                    float a0, a1;
                    upk(mul2(S, ld2(sarea + ja)), a0, a1);
                    a0 = sa ? 0.0f : a0 * ai;
                    a1 = sb ? 0.0f : a1 * ai;
#pragma unroll
                    for (int r = 0; r < NR; ++r)
                        acc[r] = fmaf(a1, sxc[(ja + 1) * NR + r], fmaf(a0, sxc[ja * NR + r], acc[r]));
                    sA[ja * RS + il] = a0;
                    sA[(ja + 1) * RS + il] = a1;
                }
            }
            __syncthreads();

            // column side of the off-diagonal leaves, y_j += sum_i a_ji x_i
            constexpr int RV = NR >= 4 ? 4 : 1;
            for (int e = tid; e < (ctot - cdiag) * (NR / RV); e += kThreads) {
                const int j = cdiag + e / (NR / RV), r0 = (e % (NR / RV)) * RV;
                float sum[RV];
#pragma unroll
                for (int v = 0; v < RV; ++v) sum[v] = 0.0f;
                for (int i = 0; i < R; ++i) {
                    const float a = sA[j * RS + i];
                    if constexpr (RV == 4) {
                        const float4 xv = *reinterpret_cast<const float4*>(sxr + i * NR + r0);
                        sum[0] = fmaf(a, xv.x, sum[0]);
                        sum[1] = fmaf(a, xv.y, sum[1]);
                        sum[2] = fmaf(a, xv.z, sum[2]);
                        sum[3] = fmaf(a, xv.w, sum[3]);
                    } else {
                        sum[0] = fmaf(a, sxr[i * NR + r0], sum[0]);
                    }
                }
#pragma unroll
                for (int v = 0; v < RV; ++v)
                    atomicAdd(&yp[(int64_t)sgid[j] * NR + r0 + v], f2d_exact(sum[v] * (float)kInv4Pi));
            }
            __syncthreads();  // the stage and the entry tile are free for the chunk after next
            cur = nxt;
            jpos = jn;
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncthreads();
    float* sred = reinterpret_cast<float*>(smem);
#pragma unroll
    for (int r = 0; r < NR; ++r) sred[tid * NR + r] = active ? acc[r] : 0.0f;
    __syncthreads();
    for (int e = tid; e < R * NR; e += kThreads) {
        const int i = e / NR, r = e % NR;
        float s = 0.0f;
        for (int q = 0; q < K; ++q) s += sred[(q * R + i) * NR + r];
        atomicAdd(&yp[(int64_t)(rb + i) * NR + r], f2d_exact(s * (float)kInv4Pi));
    }
}

// One CTA per row leaf (work == nullptr), or persistent CTAs that take the
// next row from the counter *work (zero before the launch) until none is left.
// NB: CTAs per SM the register budget is sized for (0: 4 for the FP32 single
// layer, else 2); a launch shape the autotuner chooses.
template <int NR, bool DLPK, bool F32, bool PERSIST, int NB>
__global__ void __launch_bounds__(kThreads, NB > 0 ? NB : ((F32 && !DLPK) ? 4 : 2))
    k_near_sym(Geom g, Tree t, Consts c, int nrows, const int* __restrict__ rows, const int* __restrict__ ptr,
               const int* __restrict__ col, bool transpose, const double* __restrict__ xp,
               const float* __restrict__ xs, double* __restrict__ yp, int* __restrict__ work) {
    if constexpr (!PERSIST) {
        if constexpr (F32 && !DLPK) near_slp32_row<NR>(g, t, c, rows, ptr, col, xs, yp, blockIdx.x);
        else near_sym_row<NR, DLPK, F32>(g, t, c, rows, ptr, col, transpose, xp, yp, blockIdx.x);
        return;
    }
    __shared__ int s_bi;
    while (true) {
        __syncthreads();  // the previous row is done with shared memory and s_bi
        if (threadIdx.x == 0) s_bi = atomicAdd(work, 1);
        __syncthreads();
        const int bi = s_bi;
        if (bi >= nrows) break;
        if constexpr (F32 && !DLPK) near_slp32_row<NR>(g, t, c, rows, ptr, col, xs, yp, bi);
        else near_sym_row<NR, DLPK, F32>(g, t, c, rows, ptr, col, transpose, xp, yp, bi);
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
                        const int* ptr, const int* col, bool tr, const double* xp, const float* xs, double* yp,
                        int* work, int nb) {
    using T = typename std::conditional<F32, float, double>::type;
    constexpr size_t smem = (F32 && !DLPK) ? Smem32<NR>::BYTES : Smem<T, NR, DLPK>::BYTES;
    auto go = [&](auto kplain, auto kpers) {
        if (!work) {
            cudaFuncSetAttribute(kplain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kplain<<<nrows, kThreads, smem, s>>>(g, t, c, nrows, rows, ptr, col, tr, xp, xs, yp, nullptr);
            return;
        }
        cudaFuncSetAttribute(kpers, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int grid = std::min(nrows, resident_ctas((const void*)kpers, kThreads, smem));
        cudaMemsetAsync(work, 0, sizeof(int), s);
        kpers<<<grid, kThreads, smem, s>>>(g, t, c, nrows, rows, ptr, col, tr, xp, xs, yp, work);
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
                        const int* rows, const int* ptr, const int* col, bool tr, const double* xp, const float* xs,
                        double* yp, int* work, int nb) {
    const bool dlp = ker != SLP;
    if (fp32) {
        if (dlp) near_sym_go<NR, true, true>(nrows, s, g, t, c, rows, ptr, col, tr, xp, xs, yp, work, nb);
        else near_sym_go<NR, false, true>(nrows, s, g, t, c, rows, ptr, col, tr, xp, xs, yp, work, nb);
    } else {
        if (dlp) near_sym_go<NR, true, false>(nrows, s, g, t, c, rows, ptr, col, tr, xp, xs, yp, work, nb);
        else near_sym_go<NR, false, false>(nrows, s, g, t, c, rows, ptr, col, tr, xp, xs, yp, work, nb);
    }
}

void launch_near_sym(const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                     const int* col, int ker, bool transpose, bool fp32, int NR, const double* xp, const float* xs,
                     double* yp, const LaunchCfg& cfg, cudaStream_t s) {
    int* work = cfg.work;
    const int nb = cfg.nb;
    if (nrows <= 0) return;
    if (!fp32) {  // FP64 tier: double-float evaluation (k_near_df.cu)
        launch_near_df(g, t, c, nrows, rows, ptr, col, ker != SLP, transpose, NR, xp, yp, s);
        return;
    }
    switch (NR) {
        case 1: near_sym_nr<1>(ker, fp32, nrows, s, g, t, c, rows, ptr, col, transpose, xp, xs, yp, work, nb); break;
        case 4: near_sym_nr<4>(ker, fp32, nrows, s, g, t, c, rows, ptr, col, transpose, xp, xs, yp, work, nb); break;
        case 8: near_sym_nr<8>(ker, fp32, nrows, s, g, t, c, rows, ptr, col, transpose, xp, xs, yp, work, nb); break;
        default: near_sym_nr<16>(ker, fp32, nrows, s, g, t, c, rows, ptr, col, transpose, xp, xs, yp, work, nb); break;
    }
}

}  // namespace h2
