// Regular nearfield of the single layer in the FP64 tier (section 1,
// eq. (slp): the 7 x 7-point rule on the pairs of nearfield leaves that share
// no vertex) by double-float arithmetic on the FP32 pipe.
//
// GB300 issues FP64 at about 1/74 of its FP32 rate, and the FP64 evaluation
// (about ten FP64 operations per point pair) made this stage take most of the
// FP64 tier's time.  Here every quantity of a point pair is carried as an
// unevaluated float pair hi + lo (about 48 significant bits), formed with
// Knuth's TwoSum and Dekker's product (the FMA residual of a rounded product):
//   - the centroid difference D = c_i - c_j, formed in FP64 once per pair and
//     split (so it keeps ~2^-48 of |D|, not of |c|: the double layer's plane
//     heights are O(h^2) and need that), and the point offsets from each
//     centroid as float pairs, so d = (x_p - c_i) + D - (y_q - c_j) keeps
//     ~1e-14 of |d|;
//   - r^2 = |d|^2 as a float pair;
//   - 1/r from the hardware reciprocal square root y0 (rel. error < 2^-22)
//     and one Newton step y = y0 (1 + e / 2), e = 1 - r^2 y0^2 formed from
//     the float pairs (relative error of y about (3/8) e^2 < 3e-14);
//   - the rule sums sum_q w_q sum_p w_p / r_pq as float pairs.
// The entry |tau_i| |tau_j| S / (4 pi) and the products with x are FP64, once
// per pair.  Work layout as for the other nearfield kernels: one CTA per row
// leaf t over the nearfield leaves s >= t (each unordered pair once, the
// single layer being symmetric), thread (il, kk) owns row triangle
// t.begin + il and every K-th column of a chunk of staged column leaves; the
// row side accumulates in registers, the column side through an entry tile
// in shared memory and FP64 atomics.  The diagonal block is applied on the row
// side only.
//
// Double layer (FP64 tier): the two entries of a pair share their distances,
//   k_ij ~ sum_pq w_p w_q h_p / r^3,  h_p = (x_p - c_j) . n_j (height of x_p above the plane of tau_j),
//   k_ji ~ sum_pq w_p w_q h_q / r^3,  h_q = (y_q - c_i) . n_i,
// the heights as float-pair dot products with the split normals, once per pair
// and point; per point pair then 1/r^3 as a float pair and two float-pair sums.
#include <algorithm>

#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4PiD = 0.07957747154594766788;
constexpr int kThrD = 256;
constexpr int kColD = 128;   // staged column triangles of one chunk
constexpr int kEntD = 4096;  // column-side entries of one chunk (rows x columns)
static_assert(kColD >= kMaxLeaf && kEntD >= kMaxLeaf * kMaxLeaf, "a chunk holds a column leaf of any row leaf");

// Knuth's TwoSum: s + e = a + b exactly
__device__ __forceinline__ void tsum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (ah + al)(bh + bl) as a float pair (Dekker's product for the hi parts)
__device__ __forceinline__ void dmul(float ah, float al, float bh, float bl, float& ph, float& pl) {
    ph = __fmul_rn(ah, bh);
    pl = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fmaf_rn(ah, bh, -ph)));
}
// (sh, sl) += (ph, pl)
__device__ __forceinline__ void dacc(float& sh, float& sl, float ph, float pl) {
    float e;
    tsum(sh, ph, sh, e);
    sl = __fadd_rn(sl, __fadd_rn(e, pl));
}
// the dot product of the float-pair vectors a and b as a float pair
__device__ __forceinline__ void ddot3(const float* ah, const float* al, const float* bh, const float* bl, float& rh,
                                      float& rl) {
    float p0, q0, p1, q1, p2, q2;
    dmul(ah[0], al[0], bh[0], bl[0], p0, q0);
    dmul(ah[1], al[1], bh[1], bl[1], p1, q1);
    dmul(ah[2], al[2], bh[2], bl[2], p2, q2);
    float s1, e1, e2;
    tsum(p0, p1, s1, e1);
    tsum(s1, p2, rh, e2);
    rl = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(q0, q1), q2));
}

template <int NR>
struct SmemD {
    static constexpr size_t al(size_t x) { return (x + 15) & ~size_t(15); }
    static constexpr size_t A = 0;                           // double [kEntD] column-side entries [il][jc]
    static constexpr size_t BH = al(A + 8 * kEntD);          // float [3][kColD][7] point offsets, hi
    static constexpr size_t BL = al(BH + 4 * 3 * kColD * 7);  // float [3][kColD][7] point offsets, lo
    static constexpr size_t CT = al(BL + 4 * 3 * kColD * 7);  // double [3][kColD] centroids
    static constexpr size_t AR = al(CT + 8 * 3 * kColD);      // double [kColD] areas
    static constexpr size_t VID = al(AR + 8 * kColD);         // int [3][kColD] vertex ids
    static constexpr size_t GID = al(VID + 4 * 3 * kColD);    // int [kColD] tree positions
    static constexpr size_t XC = al(GID + 4 * kColD);         // double [kColD][NR] x of the columns
    static constexpr size_t XR = al(XC + 8 * kColD * NR);     // double [kMaxLeaf][NR] x of the row leaf
    static constexpr size_t NM = al(XR + 8 * kMaxLeaf * NR);  // float [6][kColD] normal hi, lo (double layer)
    static constexpr size_t END = al(NM + 4 * 6 * kColD);
    static constexpr size_t RED = 8 * kThrD * NR;  // final row reduction (reuses the front)
    static constexpr size_t BYTES = END > RED ? END : RED;
};
}  // namespace

template <int NR, bool DLPK>
__global__ void __launch_bounds__(kThrD) k_near_df(Geom g, Tree t, Consts c, const int* __restrict__ rows,
                                                   const int* __restrict__ ptr, const int* __restrict__ col,
                                                   bool transpose, const double* __restrict__ xp,
                                                   double* __restrict__ yp) {
    using L = SmemD<NR>;
    extern __shared__ __align__(16) unsigned char smem[];
    double* sA = reinterpret_cast<double*>(smem + L::A);
    float* sbh = reinterpret_cast<float*>(smem + L::BH);
    float* sbl = reinterpret_cast<float*>(smem + L::BL);
    double* sct = reinterpret_cast<double*>(smem + L::CT);
    double* sarea = reinterpret_cast<double*>(smem + L::AR);
    int* svid = reinterpret_cast<int*>(smem + L::VID);
    int* sgid = reinterpret_cast<int*>(smem + L::GID);
    double* sxc = reinterpret_cast<double*>(smem + L::XC);
    double* sxr = reinterpret_cast<double*>(smem + L::XR);
    float* snm = reinterpret_cast<float*>(smem + L::NM);

    const int row = rows[blockIdx.x];
    const int rb = t.begin[row], R = t.end[row] - rb;
    const int K = kThrD / R;
    const int tid = threadIdx.x;
    const int il = tid % R, kk = tid / R;
    const bool active = kk < K;
    const int n = g.n;
    const int cmax = min(kColD, kEntD / R);

    for (int e = tid; e < R * NR; e += kThrD) sxr[e] = xp[(int64_t)rb * NR + e];
    // the rule's weights as float pairs
    float wh[7], wl[7];
#pragma unroll
    for (int p = 0; p < 7; ++p) {
        wh[p] = (float)c.rw[p];
        wl[p] = (float)(c.rw[p] - (double)wh[p]);
    }
    // row triangle: its points as offsets from its centroid (float pairs), the
    // centroid split, and (double layer) the split normal
    float ah[7][3], alo[7][3], nih[3] = {0, 0, 0}, nil[3] = {0, 0, 0};
    double ci[3] = {0.0, 0.0, 0.0};
    double ai = 0.0;
    int vi[3] = {-1, -1, -1};
#pragma unroll
    for (int p = 0; p < 7; ++p)
#pragma unroll
        for (int d = 0; d < 3; ++d) ah[p][d] = alo[p][d] = 0.0f;
    if (active) {
        const int i = rb + il;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            vi[d] = g.vid[d * n + i];
            ci[d] = g.ctr[d * n + i];
            if (DLPK) {
                nih[d] = g.nef[d * n + i];
                nil[d] = g.nef[(3 + d) * n + i];
            }
            const double cd = g.ctr[d * n + i];
#pragma unroll
            for (int p = 0; p < 7; ++p) {
                const double off = g.qa[((int64_t)d * n + i) * 7 + p] - cd;
                ah[p][d] = (float)off;
                alo[p][d] = (float)(off - (double)ah[p][d]);
            }
        }
        ai = g.area[i];
    }
    double acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0;

    const int bbeg = ptr[blockIdx.x], bend = ptr[blockIdx.x + 1];
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
            for (int e = tid; e < C; e += kThrD) sgid[off + e] = cb + e;
            off += C;
        }
        __syncthreads();
        for (int e = tid; e < ctot * 7; e += kThrD) {
            const int j = sgid[e / 7], q = e % 7;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double off = g.qa[((int64_t)d * n + j) * 7 + q] - g.ctr[d * n + j];
                const float h = (float)off;
                sbh[d * (kColD * 7) + e] = h;
                sbl[d * (kColD * 7) + e] = (float)(off - (double)h);
            }
        }
        for (int e = tid; e < ctot; e += kThrD) {
            const int j = sgid[e];
            sarea[e] = g.area[j];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                svid[d * kColD + e] = g.vid[d * n + j];
                sct[d * kColD + e] = g.ctr[d * n + j];
                if (DLPK) {
                    snm[d * kColD + e] = g.nef[d * n + j];
                    snm[(3 + d) * kColD + e] = g.nef[(3 + d) * n + j];
                }
            }
        }
        for (int e = tid; e < ctot * NR; e += kThrD) sxc[e] = xp[(int64_t)sgid[e / NR] * NR + e % NR];
        __syncthreads();

        // phase 1: entries (row side into registers, column side into sA)
        if (active) {
            for (int jc = kk; jc < ctot; jc += K) {
                bool sing = false;
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb) sing |= (vi[a] == svid[bb * kColD + jc]);
                double arow = 0.0, acol = 0.0;
                if (!sing) {
                    // D = c_i - c_j in FP64, split into a float pair
                    float Dh[3], Dl[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const double Dd = ci[d] - sct[d * kColD + jc];
                        Dh[d] = (float)Dd;
                        Dl[d] = (float)(Dd - (double)Dh[d]);
                    }
                    // double layer: w_p h_p, h_p = (x_p - c_j) . n_j = ((x_p - c_i) + D) . n_j
                    float hph[7], hpl[7];
                    float njh[3], njl[3];
                    if (DLPK) {
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            njh[d] = snm[d * kColD + jc];
                            njl[d] = snm[(3 + d) * kColD + jc];
                        }
#pragma unroll
                        for (int p = 0; p < 7; ++p) {
                            float vh[3], vl[3];
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                float e;
                                tsum(ah[p][d], Dh[d], vh[d], e);
                                vl[d] = __fadd_rn(__fadd_rn(alo[p][d], Dl[d]), e);
                            }
                            float hh, hl;
                            ddot3(vh, vl, njh, njl, hh, hl);
                            dmul(wh[p], wl[p], hh, hl, hph[p], hpl[p]);
                        }
                    }
                    float Sh = 0.0f, Sl = 0.0f, S2h = 0.0f, S2l = 0.0f;
#pragma unroll 1
                    for (int q = 0; q < 7; ++q) {
                        // Y = D - (y_q - c_j)
                        float Yh[3], Yl[3];
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            float e;
                            tsum(Dh[d], -sbh[d * (kColD * 7) + jc * 7 + q], Yh[d], e);
                            Yl[d] = __fadd_rn(__fsub_rn(Dl[d], sbl[d * (kColD * 7) + jc * 7 + q]), e);
                        }
                        float Ph = 0.0f, Pl = 0.0f, P2h = 0.0f, P2l = 0.0f;
#pragma unroll
                        for (int p = 0; p < 7; ++p) {
                            // d = (x_p - c_i) + Y and r^2 = |d|^2, float pairs
                            float sq[3], sqe[3];
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                float dh, e;
                                tsum(ah[p][d], Yh[d], dh, e);
                                const float dl = __fadd_rn(__fadd_rn(alo[p][d], Yl[d]), e);
                                sq[d] = __fmul_rn(dh, dh);
                                sqe[d] = __fmaf_rn(2.0f * dh, dl, __fmaf_rn(dh, dh, -sq[d]));
                            }
                            float s1, e1, Rh, e2;
                            tsum(sq[0], sq[1], s1, e1);
                            tsum(s1, sq[2], Rh, e2);
                            const float Rl = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(sqe[0], sqe[1]), sqe[2]));
                            // 1/r: y0 (hardware) and one Newton step from e = 1 - r^2 y0^2
                            float y0;
                            asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(Rh));
                            const float y2 = __fmul_rn(y0, y0);
                            const float y2e = __fmaf_rn(y0, y0, -y2);
                            const float tq = __fmaf_rn(-Rh, y2, 1.0f);
                            const float ep = __fsub_rn(tq, __fmaf_rn(Rh, y2e, __fmul_rn(Rl, y2)));
                            const float yc = __fmul_rn(__fmul_rn(0.5f, y0), ep);  // y = y0 + yc
                            if constexpr (!DLPK) {
                                // P += w_p y
                                const float th = __fmul_rn(wh[p], y0);
                                const float tl = __fmaf_rn(wh[p], yc, __fmaf_rn(wl[p], y0, __fmaf_rn(wh[p], y0, -th)));
                                dacc(Ph, Pl, th, tl);
                            } else {
                                // y^3 as a float pair, then P += w_p h_p y^3 and P2 += w_p y^3
                                const float yy = __fmul_rn(y0, y0);
                                const float yyl = __fmaf_rn(2.0f * y0, yc, __fmaf_rn(y0, y0, -yy));
                                float y3h, y3l;
                                dmul(yy, yyl, y0, yc, y3h, y3l);
                                float th, tl;
                                dmul(hph[p], hpl[p], y3h, y3l, th, tl);
                                dacc(Ph, Pl, th, tl);
                                dmul(wh[p], wl[p], y3h, y3l, th, tl);
                                dacc(P2h, P2l, th, tl);
                            }
                        }
                        // S += w_q P;  double layer: S2 += w_q h_q P2, h_q = (y_q - c_i) . n_i = -Y . n_i
                        float qh, ql;
                        dmul(wh[q], wl[q], Ph, Pl, qh, ql);
                        dacc(Sh, Sl, qh, ql);
                        if (DLPK) {
                            float hqh, hql;
                            ddot3(Yh, Yl, nih, nil, hqh, hql);
                            float wqh, wql;
                            dmul(wh[q], wl[q], -hqh, -hql, wqh, wql);
                            dmul(wqh, wql, P2h, P2l, qh, ql);
                            dacc(S2h, S2l, qh, ql);
                        }
                    }
                    const double aa = ai * sarea[jc];
                    const double S1 = (double)Sh + (double)Sl;
                    if (!DLPK) {
                        arow = acol = aa * S1;
                    } else {
                        // S1 -> k_ij (row i, column j), S2 -> k_ji
                        const double S2 = (double)S2h + (double)S2l;
                        arow = aa * (transpose ? S2 : S1);
                        acol = aa * (transpose ? S1 : S2);
                    }
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[r] = fma(arow, sxc[jc * NR + r], acc[r]);
                sA[il * cmax + jc] = acol;
            }
        }
        __syncthreads();
        // phase 2: column side of the off-diagonal leaves, y_j += sum_i a_ji x_i
        for (int e = tid; e < (ctot - cdiag) * NR; e += kThrD) {
            const int jc = cdiag + e / NR, r = e % NR;
            double sum = 0.0;
            for (int i = 0; i < R; ++i) sum = fma(sA[i * cmax + jc], sxr[i * NR + r], sum);
            atomicAdd(&yp[(int64_t)sgid[jc] * NR + r], sum * kInv4PiD);
        }
        b = b2;
    }
    __syncthreads();
    // row side: reduce the K partial sums of each row
    double* sred = reinterpret_cast<double*>(smem);
#pragma unroll
    for (int r = 0; r < NR; ++r) sred[tid * NR + r] = active ? acc[r] : 0.0;
    __syncthreads();
    for (int e = tid; e < R * NR; e += kThrD) {
        const int i = e / NR, r = e % NR;
        double s = 0.0;
        for (int q = 0; q < K; ++q) s += sred[(q * R + i) * NR + r];
        atomicAdd(&yp[(int64_t)(rb + i) * NR + r], s * kInv4PiD);
    }
}

void launch_near_df(const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                    const int* col, bool dlp, bool transpose, int NR, const double* xp, double* yp, cudaStream_t s) {
    if (nrows <= 0) return;
    auto go = [&](auto kern, size_t smem) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<nrows, kThrD, smem, s>>>(g, t, c, rows, ptr, col, transpose, xp, yp);
    };
    if (dlp) {
        switch (NR) {
            case 1: go(k_near_df<1, true>, SmemD<1>::BYTES); break;
            case 4: go(k_near_df<4, true>, SmemD<4>::BYTES); break;
            case 8: go(k_near_df<8, true>, SmemD<8>::BYTES); break;
            default: go(k_near_df<16, true>, SmemD<16>::BYTES); break;
        }
    } else {
        switch (NR) {
            case 1: go(k_near_df<1, false>, SmemD<1>::BYTES); break;
            case 4: go(k_near_df<4, false>, SmemD<4>::BYTES); break;
            case 8: go(k_near_df<8, false>, SmemD<8>::BYTES); break;
            default: go(k_near_df<16, false>, SmemD<16>::BYTES); break;
        }
    }
}

}  // namespace h2
