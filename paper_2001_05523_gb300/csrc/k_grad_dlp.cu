// Shape gradient of L = sum_r <w_r, K(X) x_r> for the double layer (FP64),
// cluster tree and block lists frozen (section 1, eq. (dlp); section 2,
// eq. (vsw); section 3).  With N_j = |tau_j| n_j = (e1 x e2) / 2 the
// area-normal of the source triangle, every entry is
//   k_ij = |tau_i| sum_pq w_pq F(x_p, y_q, N_j),
//   F(x, y, N) = (x - y).N / (4 pi |x - y|^3),
// (Sauter-Schwab pairs: 4 |tau_i| sum w J F with the canonical points), so it
// depends on the points of both triangles, on |tau_i| and on N_j; d(g.N)/dY_k
// = (Y_{k+1} - Y_{k+2}) x g / 2 in the triangle's own vertex order.
//   nearfield    thread i gathers everything that moves the vertices of
//                tau_i: from k_ij (target side: |tau_i|, the points x_p) and
//                from k_ji (source side: the points y_p and N_i); one
//                reciprocal square root serves both, since d_ji = -d_ij
//   singular     thread per canonical pair, both orientations, full tensor rule
//   farfield     as for the single layer with x-hat = W^T x; the row side's
//                leaf term (V) runs k_grad_leaf with beta = w y-hat only, the
//                column side's W = sum_p w_p N . grad L(y_p) here, through N,
//                the points (Hessian of L) and the box centre and half-widths
#include "dmath.cuh"
#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;

// reference-interval Lagrange value, first and second derivative of node a at t
__device__ __forceinline__ void lag012(const Consts& c, int a, double t, double* l0, double* l1, double* l2) {
    double p = 1.0, s1 = 0.0, s2 = 0.0;
    for (int b = 0; b < c.m; ++b) {
        if (b == a) continue;
        p *= t - c.cheb[b];
        double q = 1.0;
        for (int e = 0; e < c.m; ++e)
            if (e != a && e != b) q *= t - c.cheb[e];
        s1 += q;
        for (int d = 0; d < c.m; ++d) {
            if (d == a || d == b) continue;
            double r = 1.0;
            for (int e = 0; e < c.m; ++e)
                if (e != a && e != b && e != d) r *= t - c.cheb[e];
            s2 += r;
        }
    }
    *l0 = c.bary[a] * p;
    *l1 = c.bary[a] * s1;
    *l2 = c.bary[a] * s2;
}

template <int NV>
__device__ void cta_sum(double* v, double* red /* [32][NV] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    __syncthreads();
    if (lane == 0)
        for (int q = 0; q < NV; ++q) red[warp * NV + q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[w * NV + q];
            v[q] = s;
        }
}

// (Y_{k+1} - Y_{k+2}) x g / 2 for the corners k of the triangle at tree
// position i (its own vertex order), added with factor f to the vertices
__device__ __forceinline__ void add_area_normal(const Geom& g, int i, const double* gv, double f, double* dX) {
    const int n = g.n;
    for (int k = 0; k < 3; ++k) {
        const int a = (k + 1) % 3, b = (k + 2) % 3;
        const double e[3] = {g.v[(3 * a) * n + i] - g.v[(3 * b) * n + i], g.v[(3 * a + 1) * n + i] - g.v[(3 * b + 1) * n + i],
                             g.v[(3 * a + 2) * n + i] - g.v[(3 * b + 2) * n + i]};
        const double cr[3] = {e[1] * gv[2] - e[2] * gv[1], e[2] * gv[0] - e[0] * gv[2], e[0] * gv[1] - e[1] * gv[0]};
        const int vid = g.vid[k * n + i];
        for (int d = 0; d < 3; ++d) atomicAdd(&dX[3 * (int64_t)vid + d], 0.5 * f * cr[d]);
    }
}

// d|tau|/dX_k = n x (X_{k+2} - X_{k+1}) / 2 for the listed corners X
__device__ __forceinline__ void area_grad3(const double (*X)[3], double (*dA)[3]) {
    const double e1[3] = {X[1][0] - X[0][0], X[1][1] - X[0][1], X[1][2] - X[0][2]};
    const double e2[3] = {X[2][0] - X[0][0], X[2][1] - X[0][1], X[2][2] - X[0][2]};
    double nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double len = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    for (int d = 0; d < 3; ++d) nn[d] /= len;
    for (int k = 0; k < 3; ++k) {
        const double* a = X[(k + 1) % 3];
        const double* b = X[(k + 2) % 3];
        const double e[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        dA[k][0] = 0.5 * (nn[1] * e[2] - nn[2] * e[1]);
        dA[k][1] = 0.5 * (nn[2] * e[0] - nn[0] * e[2]);
        dA[k][2] = 0.5 * (nn[0] * e[1] - nn[1] * e[0]);
    }
}
}  // namespace

// ---------------------------------------------------------------------------
// column-side leaf basis W_c[i,nu] = sum_p w_p N_i . grad L_nu(y_p): CTA per
// leaf, triangle by triangle; beta_nu = sum_r x_i zh_c[nu]; thread p the
// gradient Pw = sum beta grad L and HN = (sum beta Hess L) N at point p
// ---------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(128) k_grad_leaf_w(Geom g, Tree t, Consts c, const double* __restrict__ rule,
                                                     const int* __restrict__ leaves, const double* __restrict__ xp,
                                                     const double* __restrict__ zh, double* __restrict__ dbox,
                                                     double* __restrict__ dX) {
    __shared__ double beta[kMaxK], red[32 * 18], boxacc[6];
    const int cl = leaves[blockIdx.x];
    const int b0 = t.begin[cl], R = t.end[cl] - b0;
    const int m = c.m, k = c.k, nb = c.nb, n = g.n;
    double ctr[3], ih[3];
    for (int d = 0; d < 3; ++d) {
        ctr[d] = t.box[d * t.nc + cl];
        ih[d] = t.box[(6 + d) * t.nc + cl];
    }
    if (threadIdx.x < 6) boxacc[threadIdx.x] = 0.0;
    for (int il = 0; il < R; ++il) {
        const int i = b0 + il;
        __syncthreads();
        for (int nu = threadIdx.x; nu < k; nu += blockDim.x) {
            double s = 0.0;
#pragma unroll
            for (int r = 0; r < NR; ++r) s += xp[(int64_t)i * NR + r] * zh[((int64_t)cl * k + nu) * NR + r];
            beta[nu] = s;
        }
        __syncthreads();
        const double area = g.area[i];
        const double N[3] = {area * g.nrm[i], area * g.nrm[n + i], area * g.nrm[2 * n + i]};
        // v[0..2] sum_p w Pw; v[3 + 3k + d] sum_p w lambda_k HN; v[12..14] box centre; v[15..17] half-width
        double v[18];
        for (int q = 0; q < 18; ++q) v[q] = 0.0;
        for (int p = threadIdx.x; p < nb; p += blockDim.x) {
            double y[3], tt[3], l0[3][kMaxM], l1[3][kMaxM], l2[3][kMaxM];
            for (int d = 0; d < 3; ++d) {
                const double v0 = g.v[d * n + i];
                y[d] = v0 + rule[3 * p] * (g.v[(3 + d) * n + i] - v0) + rule[3 * p + 1] * (g.v[(6 + d) * n + i] - v0);
                tt[d] = (y[d] - ctr[d]) * ih[d];
                for (int a = 0; a < m; ++a) {
                    lag012(c, a, tt[d], &l0[d][a], &l1[d][a], &l2[d][a]);
                    l1[d][a] *= ih[d];
                    l2[d][a] *= ih[d] * ih[d];
                }
            }
            double Pw[3] = {0, 0, 0}, Hs[3][3] = {{0}};
            for (int nu = 0; nu < k; ++nu) {
                const int ia[3] = {nu % m, (nu / m) % m, nu / (m * m)};
                const double bv = beta[nu];
                const double a0 = l0[0][ia[0]], a1 = l1[0][ia[0]], a2 = l2[0][ia[0]];
                const double b0v = l0[1][ia[1]], b1 = l1[1][ia[1]], b2 = l2[1][ia[1]];
                const double c0 = l0[2][ia[2]], c1 = l1[2][ia[2]], c2 = l2[2][ia[2]];
                Pw[0] += bv * a1 * b0v * c0;
                Pw[1] += bv * a0 * b1 * c0;
                Pw[2] += bv * a0 * b0v * c1;
                Hs[0][0] += bv * a2 * b0v * c0;
                Hs[1][1] += bv * a0 * b2 * c0;
                Hs[2][2] += bv * a0 * b0v * c2;
                Hs[0][1] += bv * a1 * b1 * c0;
                Hs[0][2] += bv * a1 * b0v * c1;
                Hs[1][2] += bv * a0 * b1 * c1;
            }
            Hs[1][0] = Hs[0][1];
            Hs[2][0] = Hs[0][2];
            Hs[2][1] = Hs[1][2];
            double HN[3];
            for (int d = 0; d < 3; ++d) HN[d] = Hs[d][0] * N[0] + Hs[d][1] * N[1] + Hs[d][2] * N[2];
            const double w = rule[3 * p + 2];
            const double lam[3] = {1.0 - rule[3 * p] - rule[3 * p + 1], rule[3 * p], rule[3 * p + 1]};
            for (int d = 0; d < 3; ++d) {
                v[d] += w * Pw[d];
                for (int kk = 0; kk < 3; ++kk) v[3 + 3 * kk + d] += w * lam[kk] * HN[d];
                v[12 + d] -= w * HN[d];
                v[15 + d] -= w * (N[d] * Pw[d] * ih[d] + tt[d] * HN[d]);
            }
        }
        cta_sum<18>(v, red);
        if (threadIdx.x == 0) {
            add_area_normal(g, i, v, 1.0, dX);
            for (int kk = 0; kk < 3; ++kk) {
                const int vid = g.vid[kk * n + i];
                for (int d = 0; d < 3; ++d) atomicAdd(&dX[3 * (int64_t)vid + d], v[3 + 3 * kk + d]);
            }
            for (int q = 0; q < 6; ++q) boxacc[q] += v[12 + q];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; ++d) {
            atomicAdd(&dbox[d * t.nc + cl], boxacc[d]);
            atomicAdd(&dbox[(3 + d) * t.nc + cl], boxacc[3 + d]);
        }
}

// ---------------------------------------------------------------------------
// regular nearfield pairs (FP64): CTA per row leaf over its ordered nearfield
// blocks, thread (i, part).  For a pair (i, j) sharing no vertex, with
// d = x_p - y_q (x_p on tau_i, y_q on tau_j), i3 = 1 / |d|^3,
// A = c_ij |tau_i|, B = c_ji |tau_j|:
//   point p of tau_i:  w_pq i3 [(A N_j - B N_i) + 3 (B d.N_i - A d.N_j) d / |d|^2]
//   |tau_i|:           c_ij w_pq i3 d.N_j
//   N_i:               -B w_pq i3 d
// (times 1 / (4 pi)), the first two from k_ij, the rest from k_ji.
// ---------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(256) k_grad_near_dlp(Geom g, Tree t, Consts c, const int* __restrict__ rows,
                                                       const int* __restrict__ ptr, const int* __restrict__ col,
                                                       const double* __restrict__ xp, const double* __restrict__ wp,
                                                       double* __restrict__ dX) {
    __shared__ double sq[3 * kMaxLeaf * 7], sarea[kMaxLeaf], snrm[3 * kMaxLeaf], sx[kMaxLeaf * NR],
        sw[kMaxLeaf * NR];
    __shared__ int svid[3 * kMaxLeaf];
    __shared__ double sbuf[256];
    const int row = rows[blockIdx.x];
    const int rb = t.begin[row], R = t.end[row] - rb;
    const int K = 256 / R;
    const int tid = threadIdx.x, il = tid % R, kk = tid / R;
    const bool active = kk < K;
    const int n = g.n;
    double px[7], py[7], pz[7], xr[NR], wr[NR], Ni[3] = {0, 0, 0};
    int vi[3] = {-1, -1, -1};
    double ai = 0.0;
    if (active) {
        const int i = rb + il;
        for (int p = 0; p < 7; ++p) {
            px[p] = g.qa[((int64_t)0 * n + i) * 7 + p];
            py[p] = g.qa[((int64_t)1 * n + i) * 7 + p];
            pz[p] = g.qa[((int64_t)2 * n + i) * 7 + p];
        }
        for (int d = 0; d < 3; ++d) vi[d] = g.vid[d * n + i];
        for (int r = 0; r < NR; ++r) {
            xr[r] = xp[(int64_t)i * NR + r];
            wr[r] = wp[(int64_t)i * NR + r];
        }
        ai = g.area[i];
        for (int d = 0; d < 3; ++d) Ni[d] = ai * g.nrm[d * n + i];
    }
    double sA = 0.0, GN[3] = {0, 0, 0}, Gp[7][3];
    for (int p = 0; p < 7; ++p) Gp[p][0] = Gp[p][1] = Gp[p][2] = 0.0;
    for (int b = ptr[blockIdx.x]; b < ptr[blockIdx.x + 1]; ++b) {
        const int s = col[b];
        const int cb = t.begin[s], C = t.end[s] - cb;
        __syncthreads();
        for (int e = tid; e < C * 7; e += 256)
            for (int d = 0; d < 3; ++d) sq[d * kMaxLeaf * 7 + e] = g.qa[((int64_t)d * n + cb) * 7 + e];
        for (int e = tid; e < C; e += 256) {
            sarea[e] = g.area[cb + e];
            for (int d = 0; d < 3; ++d) {
                svid[d * kMaxLeaf + e] = g.vid[d * n + cb + e];
                snrm[d * kMaxLeaf + e] = g.nrm[d * n + cb + e];
            }
        }
        for (int e = tid; e < C * NR; e += 256) {
            sx[e] = xp[(int64_t)cb * NR + e];
            sw[e] = wp[(int64_t)cb * NR + e];
        }
        __syncthreads();
        if (!active) continue;
        for (int jl = kk; jl < C; jl += K) {
            bool sing = false;
            for (int a = 0; a < 3; ++a)
                for (int bb = 0; bb < 3; ++bb) sing |= (vi[a] == svid[bb * kMaxLeaf + jl]);
            if (sing) continue;
            double cij = 0.0, cji = 0.0;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                cij += wr[r] * sx[jl * NR + r];
                cji += sw[jl * NR + r] * xr[r];
            }
            const double aj = sarea[jl];
            const double Nj[3] = {aj * snrm[jl], aj * snrm[kMaxLeaf + jl], aj * snrm[2 * kMaxLeaf + jl]};
            const double A = cij * ai, B = cji * aj;
            const double VN[3] = {A * Nj[0] - B * Ni[0], A * Nj[1] - B * Ni[1], A * Nj[2] - B * Ni[2]};
            for (int q = 0; q < 7; ++q) {
                const double yx = sq[jl * 7 + q], yy = sq[kMaxLeaf * 7 + jl * 7 + q], yz = sq[2 * kMaxLeaf * 7 + jl * 7 + q];
                const double wq = c.rw[q];
#pragma unroll
                for (int p = 0; p < 7; ++p) {
                    const double dx = px[p] - yx, dy = py[p] - yy, dz = pz[p] - yz;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    const double ri = rsqrt_nr(r2);
                    const double i3 = wq * ri * ri * ri;
                    const double dNj = dx * Nj[0] + dy * Nj[1] + dz * Nj[2];
                    const double dNi = dx * Ni[0] + dy * Ni[1] + dz * Ni[2];
                    const double f = 3.0 * i3 * (B * dNi - A * dNj) * ri * ri;
                    Gp[p][0] += i3 * VN[0] + f * dx;
                    Gp[p][1] += i3 * VN[1] + f * dy;
                    Gp[p][2] += i3 * VN[2] + f * dz;
                    const double cw = c.rw[p] * i3;
                    sA += cij * cw * dNj;
                    GN[0] -= B * cw * dx;
                    GN[1] -= B * cw * dy;
                    GN[2] -= B * cw * dz;
                }
            }
        }
    }
    // per row triangle: v[0] |tau| factor, v[1 + 3k + d] the points, v[10..12] N
    double v[13];
    v[0] = active ? sA : 0.0;
    for (int q = 1; q < 13; ++q) v[q] = 0.0;
    if (active) {
        for (int p = 0; p < 7; ++p) {
            const double lam[3] = {1.0 - c.ru[p] - c.rv[p], c.ru[p], c.rv[p]};
            for (int k3 = 0; k3 < 3; ++k3)
                for (int d = 0; d < 3; ++d) v[1 + 3 * k3 + d] += c.rw[p] * lam[k3] * Gp[p][d];
        }
        for (int d = 0; d < 3; ++d) v[10 + d] = GN[d];
    }
    for (int q = 0; q < 13; ++q) {
        __syncthreads();
        sbuf[tid] = v[q];
        __syncthreads();
        if (tid < R) {
            double s = 0.0;
            for (int e = 0; e < K; ++e) s += sbuf[e * R + tid];
            v[q] = s;
        }
    }
    if (tid < R) {
        const int i = rb + tid;
        double X[3][3], dA[3][3];
        for (int k3 = 0; k3 < 3; ++k3)
            for (int d = 0; d < 3; ++d) X[k3][d] = g.v[(3 * k3 + d) * n + i];
        area_grad3(X, dA);
        for (int k3 = 0; k3 < 3; ++k3) {
            const int vid = g.vid[k3 * n + i];
            for (int d = 0; d < 3; ++d)
                atomicAdd(&dX[3 * (int64_t)vid + d], kInv4Pi * (dA[k3][d] * v[0] + v[1 + 3 * k3 + d]));
        }
        add_area_normal(g, i, v + 10, kInv4Pi, dX);
    }
}

// ---------------------------------------------------------------------------
// singular (edge / vertex) pairs: thread per canonical pair (lo, hi), code
// (rP | q0 << 2 | q1 << 4 | q2 << 6): P = corners rP, rP+1, rP+2 of lo, Q =
// corners q0, q1, q2 of hi; the full tensor rule tab (per point x1, x2, y1,
// y2, weight x Jacobian) on chi(z) = P0 + z1 (P1 - P0) + z2 (P2 - P1), both
// orientations: k_lo,hi = 4 |P| sum F(x, y, N_hi) and k_hi,lo = 4 |Q| sum
// F(y, x, N_lo), x on P, y on Q.
// ---------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(128) k_grad_singular_dlp(Geom g, int npairs, const int* __restrict__ plo,
                                                           const int* __restrict__ phi, const int* __restrict__ pcode,
                                                           const double* __restrict__ tab, int npts,
                                                           const double* __restrict__ xp, const double* __restrict__ wp,
                                                           double* __restrict__ dX) {
    const int pid = blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= npairs) return;
    const int lo = plo[pid], hi = phi[pid], code = pcode[pid], n = g.n;
    const int rP = code & 3;
    const int cq[3] = {(code >> 2) & 3, (code >> 4) & 3, (code >> 6) & 3};
    double P[3][3], Q[3][3];
    int pv[3], qv[3];
    for (int k3 = 0; k3 < 3; ++k3) {
        const int cp = (rP + k3) % 3;
        pv[k3] = g.vid[cp * n + lo];
        qv[k3] = g.vid[cq[k3] * n + hi];
        for (int d = 0; d < 3; ++d) {
            P[k3][d] = g.v[(3 * cp + d) * n + lo];
            Q[k3][d] = g.v[(3 * cq[k3] + d) * n + hi];
        }
    }
    const double ap = g.area[lo], aq = g.area[hi];
    const double Nlo[3] = {ap * g.nrm[lo], ap * g.nrm[n + lo], ap * g.nrm[2 * n + lo]};
    const double Nhi[3] = {aq * g.nrm[hi], aq * g.nrm[n + hi], aq * g.nrm[2 * n + hi]};
    double c1 = 0.0, c2 = 0.0;  // c_lo,hi and c_hi,lo
    for (int r = 0; r < NR; ++r) {
        c1 += wp[(int64_t)lo * NR + r] * xp[(int64_t)hi * NR + r];
        c2 += wp[(int64_t)hi * NR + r] * xp[(int64_t)lo * NR + r];
    }
    const double A = c1 * ap, B = c2 * aq;  // k_lo,hi = 4 |P| S1, k_hi,lo = 4 |Q| S2
    double S1 = 0.0, S2 = 0.0, gP[3][3] = {{0}}, gQ[3][3] = {{0}}, GNhi[3] = {0, 0, 0}, GNlo[3] = {0, 0, 0};
    for (int e = 0; e < npts; ++e) {
        const double* T = tab + 5 * e;
        const double x1 = T[0], x2 = T[1], y1 = T[2], y2 = T[3], wj = T[4];
        double d[3];
        for (int k = 0; k < 3; ++k) {
            const double x = P[0][k] + x1 * (P[1][k] - P[0][k]) + x2 * (P[2][k] - P[1][k]);
            const double y = Q[0][k] + y1 * (Q[1][k] - Q[0][k]) + y2 * (Q[2][k] - Q[1][k]);
            d[k] = x - y;
        }
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double ri = rsqrt_nr(r2);
        const double i3 = wj * ri * ri * ri;
        const double dNh = d[0] * Nhi[0] + d[1] * Nhi[1] + d[2] * Nhi[2];
        const double dNl = d[0] * Nlo[0] + d[1] * Nlo[1] + d[2] * Nlo[2];
        S1 += i3 * dNh;   // F(x, y, N_hi)
        S2 -= i3 * dNl;   // F(y, x, N_lo), y - x = -d
        // gradient in x (on P) of A F1 + B F2 and in y (on Q) is its negative
        const double f = 3.0 * i3 * (B * dNl - A * dNh) * ri * ri;
        double gx[3];
        for (int k = 0; k < 3; ++k) gx[k] = i3 * (A * Nhi[k] - B * Nlo[k]) + f * d[k];
        const double lx[3] = {1.0 - x1, x1 - x2, x2}, ly[3] = {1.0 - y1, y1 - y2, y2};
        for (int k3 = 0; k3 < 3; ++k3)
            for (int k = 0; k < 3; ++k) {
                gP[k3][k] += lx[k3] * gx[k];
                gQ[k3][k] -= ly[k3] * gx[k];
            }
        for (int k = 0; k < 3; ++k) {
            GNhi[k] += A * i3 * d[k];  // d F1 / d N_hi
            GNlo[k] -= B * i3 * d[k];  // d F2 / d N_lo
        }
    }
    double dAP[3][3], dAQ[3][3];
    area_grad3(P, dAP);
    area_grad3(Q, dAQ);
    const double f4 = 4.0 * kInv4Pi;
    for (int k3 = 0; k3 < 3; ++k3)
        for (int k = 0; k < 3; ++k) {
            atomicAdd(&dX[3 * (int64_t)pv[k3] + k], f4 * (c1 * dAP[k3][k] * S1 + gP[k3][k]));
            atomicAdd(&dX[3 * (int64_t)qv[k3] + k], f4 * (c2 * dAQ[k3][k] * S2 + gQ[k3][k]));
        }
    add_area_normal(g, hi, GNhi, f4, dX);
    add_area_normal(g, lo, GNlo, f4, dX);
}

// ---------------------------------------------------------------------------
void launch_grad_leaf_w(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nl, const int* leaves,
                        int NR, const double* xp, const double* zh, double* dbox, double* dX, cudaStream_t s) {
    if (nl <= 0) return;
    const int th = c.nb > 64 ? 128 : 64;
    switch (NR) {
        case 1: k_grad_leaf_w<1><<<nl, th, 0, s>>>(g, t, c, rule, leaves, xp, zh, dbox, dX); break;
        case 4: k_grad_leaf_w<4><<<nl, th, 0, s>>>(g, t, c, rule, leaves, xp, zh, dbox, dX); break;
        case 8: k_grad_leaf_w<8><<<nl, th, 0, s>>>(g, t, c, rule, leaves, xp, zh, dbox, dX); break;
        default: k_grad_leaf_w<16><<<nl, th, 0, s>>>(g, t, c, rule, leaves, xp, zh, dbox, dX); break;
    }
}

void launch_grad_near_dlp(const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                          const int* col, int NR, const double* xp, const double* wp, double* dX, cudaStream_t s) {
    if (nrows <= 0) return;
    switch (NR) {
        case 1: k_grad_near_dlp<1><<<nrows, 256, 0, s>>>(g, t, c, rows, ptr, col, xp, wp, dX); break;
        case 4: k_grad_near_dlp<4><<<nrows, 256, 0, s>>>(g, t, c, rows, ptr, col, xp, wp, dX); break;
        case 8: k_grad_near_dlp<8><<<nrows, 256, 0, s>>>(g, t, c, rows, ptr, col, xp, wp, dX); break;
        default: k_grad_near_dlp<16><<<nrows, 256, 0, s>>>(g, t, c, rows, ptr, col, xp, wp, dX); break;
    }
}

void launch_grad_singular_dlp(const Geom& g, int npairs, const int* lo, const int* hi, const int* code,
                              const double* tab, int npts, int NR, const double* xp, const double* wp, double* dX,
                              cudaStream_t s) {
    if (npairs <= 0) return;
    const int nb = (npairs + 127) / 128;
    switch (NR) {
        case 1: k_grad_singular_dlp<1><<<nb, 128, 0, s>>>(g, npairs, lo, hi, code, tab, npts, xp, wp, dX); break;
        case 4: k_grad_singular_dlp<4><<<nb, 128, 0, s>>>(g, npairs, lo, hi, code, tab, npts, xp, wp, dX); break;
        case 8: k_grad_singular_dlp<8><<<nb, 128, 0, s>>>(g, npairs, lo, hi, code, tab, npts, xp, wp, dX); break;
        default: k_grad_singular_dlp<16><<<nb, 128, 0, s>>>(g, npairs, lo, hi, code, tab, npts, xp, wp, dX); break;
    }
}

}  // namespace h2
