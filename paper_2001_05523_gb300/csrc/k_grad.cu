// Shape gradient of L = sum_r <w_r, G(X) x_r> for the single layer (FP64),
// with the cluster tree and block lists frozen (section 2, eq. (vsw) and
// eq. (transfer); section 3, tensor Chebyshev interpolation; section 1,
// eq. (slp) quadrature for the nearfield).
//
// The farfield part L = sum_{(t,s)} wh_t^T S_ts xh_s is differentiated through
// the interpolation nodes xi = c + h cos-node of every cluster box (centre c,
// floored half-width h), with the forward vectors xh = V^T x, wh = V^T w
// (upward passes) and the downward-accumulated coupling outputs yh = S xh,
// zh = S^T wh:
//   coupling   dL/dxi_t = sum_s sum_mu (wh_t . xh_s) grad_x g(xi_t, xi_s),  dL/dxi_s = -(...)
//   transfers  dL/dE_c'[nu',nu] = xh_c'[nu'] zh_p[nu] + wh_c'[nu'] yh_p[nu] through
//              E_c'[nu',nu] = L_{p,nu}(xi_{c',nu'})
//   leaves     dL/dV_c[i,nu] = x_i zh_c[nu] + w_i yh_c[nu] through
//              V_c[i,nu] = |tau_i| sum_p w_p L_{c,nu}(x_p)
// The box derivatives dL/dc, dL/dh are collected per cluster (dbox) and then
// passed to the vertices that realise the bounding-box extremes.
// Nearfield: regular pairs are differentiated on the row side only, with the
// coefficient c_kj + c_jk (c_ij = sum_r w_ir x_jr); the single-layer entry is a
// symmetric function of the two triangles, so this covers the column side.
// Singular pairs are differentiated through the Gram entries of the edge
// vectors and the two areas.
#include "dmath.cuh"
#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;

__device__ __forceinline__ void cluster_nodes(const Tree& t, const Consts& c, int cl, double* z) {
    for (int e = threadIdx.x; e < 3 * c.m; e += blockDim.x) {
        const int d = e / c.m, a = e % c.m;
        z[e] = t.box[d * t.nc + cl] + t.box[(3 + d) * t.nc + cl] * c.cheb[a];
    }
}

// reference-interval Lagrange value and derivative of node a at t
__device__ __forceinline__ void lag1(const Consts& c, int a, double t, double* l, double* dl) {
    double p = c.bary[a], s = 0.0;
    for (int b = 0; b < c.m; ++b) {
        if (b == a) continue;
        double q = 1.0;
        for (int e = 0; e < c.m; ++e)
            if (e != a && e != b) q *= t - c.cheb[e];
        s += q;
        p *= t - c.cheb[b];
    }
    *l = p;
    *dl = s * c.bary[a];
}

// sum of NV values over the CTA; result valid in thread 0
template <int NV>
__device__ void block_sum(double* v, double* red /* [32][NV] */) {
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

__device__ __forceinline__ void atomic_box(double* dbox, int nc, int cl, const double* gc, const double* gh,
                                           double sign) {
    for (int d = 0; d < 3; ++d) {
        atomicAdd(&dbox[d * nc + cl], sign * gc[d]);
        atomicAdd(&dbox[(3 + d) * nc + cl], sign * gh[d]);
    }
}
}  // namespace

// ---------------------------------------------------------------------------
// coupling: one CTA per row cluster t; thread (nu, slice of mu)
// ---------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(256) k_grad_coupling(Tree t, Consts c, const int* __restrict__ rows,
                                                       const int* __restrict__ ptr, const int* __restrict__ col,
                                                       const double* __restrict__ wh, const double* __restrict__ xh,
                                                       double* __restrict__ dbox) {
    extern __shared__ double xs[];  // [k][NR]
    __shared__ double zt[3 * kMaxM], zs[3 * kMaxM], D[3 * kMaxM * kMaxM], red[32 * 6];
    const int row = rows[blockIdx.x];
    const int m = c.m, k = c.k;
    const int nslice = blockDim.x / k;
    const int nu = threadIdx.x % k, sl = threadIdx.x / k;
    const bool active = sl < nslice;
    const int ia = nu % m, ib = (nu / m) % m, ic = nu / (m * m);
    cluster_nodes(t, c, row, zt);
    double wv[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) wv[r] = active ? wh[((int64_t)row * k + nu) * NR + r] : 0.0;
    double At[3] = {0, 0, 0};
    for (int b = ptr[blockIdx.x]; b < ptr[blockIdx.x + 1]; ++b) {
        const int s = col[b];
        __syncthreads();
        cluster_nodes(t, c, s, zs);
        for (int e = threadIdx.x; e < k * NR; e += blockDim.x) xs[e] = xh[(int64_t)s * k * NR + e];
        __syncthreads();
        for (int e = threadIdx.x; e < 3 * m * m; e += blockDim.x) {
            const int d = e / (m * m), a = (e / m) % m, a2 = e % m;
            D[e] = zt[d * m + a] - zs[d * m + a2];
        }
        __syncthreads();
        double As[6] = {0, 0, 0, 0, 0, 0};
        if (active) {
            for (int mu = sl; mu < k; mu += nslice) {
                const int ja = mu % m, jb = (mu / m) % m, jc = mu / (m * m);
                const double dx = D[ia * m + ja], dy = D[m * m + ib * m + jb], dz = D[2 * m * m + ic * m + jc];
                const double ri = rsqrt_nr(dx * dx + dy * dy + dz * dz);
                double coef = 0.0;
#pragma unroll
                for (int r = 0; r < NR; ++r) coef += wv[r] * xs[mu * NR + r];
                const double f = -coef * kInv4Pi * ri * ri * ri;
                const double g[3] = {f * dx, f * dy, f * dz};
                At[0] += g[0];
                At[1] += g[1];
                At[2] += g[2];
                As[0] -= g[0];
                As[1] -= g[1];
                As[2] -= g[2];
                As[3] -= c.cheb[ja] * g[0];
                As[4] -= c.cheb[jb] * g[1];
                As[5] -= c.cheb[jc] * g[2];
            }
        }
        block_sum<6>(As, red);
        if (threadIdx.x == 0) atomic_box(dbox, t.nc, s, As, As + 3, 1.0);
    }
    double Ar[6] = {At[0], At[1], At[2], c.cheb[ia] * At[0], c.cheb[ib] * At[1], c.cheb[ic] * At[2]};
    if (!active)
        for (int q = 0; q < 6; ++q) Ar[q] = 0.0;
    block_sum<6>(Ar, red);
    if (threadIdx.x == 0) atomic_box(dbox, t.nc, row, Ar, Ar + 3, 1.0);
}

// ---------------------------------------------------------------------------
// transfers: one CTA per non-root cluster c' (parent p); thread (nu', slice of nu)
// ---------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(256) k_grad_transfer(Tree t, Consts c, const int* __restrict__ children,
                                                       const int* __restrict__ parent, const double* __restrict__ xh,
                                                       const double* __restrict__ wh, const double* __restrict__ yh,
                                                       const double* __restrict__ zh, double* __restrict__ dbox) {
    extern __shared__ double sm[];  // xc, wc, zp, yp: 4 x [k][NR]
    __shared__ double L1[3 * kMaxM * kMaxM], dL1[3 * kMaxM * kMaxM], T1[3 * kMaxM], red[32 * 12];
    const int cc = children[blockIdx.x], p = parent[cc];
    const int m = c.m, k = c.k;
    double* xc = sm;
    double* wc = xc + k * NR;
    double* zp = wc + k * NR;
    double* yp = zp + k * NR;
    for (int e = threadIdx.x; e < k * NR; e += blockDim.x) {
        xc[e] = xh[(int64_t)cc * k * NR + e];
        wc[e] = wh[(int64_t)cc * k * NR + e];
        zp[e] = zh[(int64_t)p * k * NR + e];
        yp[e] = yh[(int64_t)p * k * NR + e];
    }
    // 1-D tables: child node a' along d in the parent's reference interval
    for (int e = threadIdx.x; e < 3 * m * m; e += blockDim.x) {
        const int d = e / (m * m), ap = (e / m) % m, a = e % m;
        const double xi = t.box[d * t.nc + cc] + t.box[(3 + d) * t.nc + cc] * c.cheb[ap];
        const double tr = (xi - t.box[d * t.nc + p]) * t.box[(6 + d) * t.nc + p];
        double l, dl;
        lag1(c, a, tr, &l, &dl);
        L1[e] = l;
        dL1[e] = dl * t.box[(6 + d) * t.nc + p];
        if (a == 0) T1[d * m + ap] = tr;
    }
    __syncthreads();
    const int nslice = blockDim.x / k;
    const int nup = threadIdx.x % k, sl = threadIdx.x / k;
    const bool active = sl < nslice;
    const int pa = nup % m, pb = (nup / m) % m, pc = nup / (m * m);
    double A[3] = {0, 0, 0};
    if (active) {
        for (int nu = sl; nu < k; nu += nslice) {
            const int a = nu % m, b = (nu / m) % m, cz = nu / (m * m);
            double M = 0.0;
#pragma unroll
            for (int r = 0; r < NR; ++r) M += xc[nup * NR + r] * zp[nu * NR + r] + wc[nup * NR + r] * yp[nu * NR + r];
            const double lx = L1[pa * m + a], ly = L1[m * m + pb * m + b], lz = L1[2 * m * m + pc * m + cz];
            A[0] += M * dL1[pa * m + a] * ly * lz;
            A[1] += M * lx * dL1[m * m + pb * m + b] * lz;
            A[2] += M * lx * ly * dL1[2 * m * m + pc * m + cz];
        }
    }
    double v[12];
    const double cn[3] = {c.cheb[pa], c.cheb[pb], c.cheb[pc]};
    const double tp[3] = {T1[pa], T1[m + pb], T1[2 * m + pc]};
    for (int d = 0; d < 3; ++d) {
        v[d] = active ? A[d] : 0.0;               // child centre
        v[3 + d] = active ? cn[d] * A[d] : 0.0;   // child half-width
        v[6 + d] = active ? -A[d] : 0.0;          // parent centre
        v[9 + d] = active ? -tp[d] * A[d] : 0.0;  // parent half-width
    }
    block_sum<12>(v, red);
    if (threadIdx.x == 0) {
        atomic_box(dbox, t.nc, cc, v, v + 3, 1.0);
        atomic_box(dbox, t.nc, p, v + 6, v + 9, 1.0);
    }
}

// ---------------------------------------------------------------------------
// leaf bases: one CTA per leaf; per triangle, thread nu forms
// beta_nu = sum_r (x_i zh_c[nu] + w_i yh_c[nu]) (zh = NULL: the row side
// w_i yh_c[nu] only, for the double layer), thread p the interpolant
// P = sum beta_nu L_nu and its gradient at quadrature point p.
// ---------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(256) k_grad_leaf(Geom g, Tree t, Consts c, const double* __restrict__ rule,
                                                   const int* __restrict__ leaves, const double* __restrict__ xp,
                                                   const double* __restrict__ wp, const double* __restrict__ yh,
                                                   const double* __restrict__ zh, double* __restrict__ dbox,
                                                   double* __restrict__ dX) {
    __shared__ double beta[kMaxK], red[32 * 16], boxacc[6];
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
            for (int r = 0; r < NR; ++r) {
                s += wp[(int64_t)i * NR + r] * yh[((int64_t)cl * k + nu) * NR + r];
                if (zh) s += xp[(int64_t)i * NR + r] * zh[((int64_t)cl * k + nu) * NR + r];
            }
            beta[nu] = s;
        }
        __syncthreads();
        const double area = g.area[i];
        double v[16];
        for (int q = 0; q < 16; ++q) v[q] = 0.0;
        for (int p = threadIdx.x; p < nb; p += blockDim.x) {
            double y[3], tt[3], l[3][kMaxM], dl[3][kMaxM];
            for (int d = 0; d < 3; ++d) {
                const double v0 = g.v[d * n + i];
                y[d] = v0 + rule[3 * p] * (g.v[(3 + d) * n + i] - v0) + rule[3 * p + 1] * (g.v[(6 + d) * n + i] - v0);
                tt[d] = (y[d] - ctr[d]) * ih[d];
                for (int a = 0; a < m; ++a) {
                    lag1(c, a, tt[d], &l[d][a], &dl[d][a]);
                    dl[d][a] *= ih[d];
                }
            }
            double P = 0.0, G[3] = {0, 0, 0};
            for (int nu = 0; nu < k; ++nu) {
                const int a = nu % m, bq = (nu / m) % m, cz = nu / (m * m);
                const double bv = beta[nu];
                P += bv * l[0][a] * l[1][bq] * l[2][cz];
                G[0] += bv * dl[0][a] * l[1][bq] * l[2][cz];
                G[1] += bv * l[0][a] * dl[1][bq] * l[2][cz];
                G[2] += bv * l[0][a] * l[1][bq] * dl[2][cz];
            }
            const double w = rule[3 * p + 2];
            const double lam[3] = {1.0 - rule[3 * p] - rule[3 * p + 1], rule[3 * p], rule[3 * p + 1]};
            v[0] += w * P;
            for (int kk = 0; kk < 3; ++kk)
                for (int d = 0; d < 3; ++d) v[1 + 3 * kk + d] += w * lam[kk] * G[d];
            for (int d = 0; d < 3; ++d) {
                v[10 + d] -= area * w * G[d];
                v[13 + d] -= area * w * G[d] * tt[d];
            }
        }
        block_sum<16>(v, red);
        if (threadIdx.x == 0) {
            double X[9];
            for (int q = 0; q < 9; ++q) X[q] = g.v[q * n + i];
            const double nx = g.nrm[i], ny = g.nrm[n + i], nz = g.nrm[2 * n + i];
            for (int kk = 0; kk < 3; ++kk) {
                const double* a = X + 3 * ((kk + 1) % 3);
                const double* bb = X + 3 * ((kk + 2) % 3);
                const double e[3] = {bb[0] - a[0], bb[1] - a[1], bb[2] - a[2]};
                const double dA[3] = {0.5 * (ny * e[2] - nz * e[1]), 0.5 * (nz * e[0] - nx * e[2]),
                                      0.5 * (nx * e[1] - ny * e[0])};
                const int vid = g.vid[kk * n + i];
                for (int d = 0; d < 3; ++d) atomicAdd(&dX[3 * (int64_t)vid + d], dA[d] * v[0] + area * v[1 + 3 * kk + d]);
            }
            for (int q = 0; q < 6; ++q) boxacc[q] += v[10 + q];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) atomic_box(dbox, t.nc, cl, boxacc, boxacc + 3, 1.0);
}

// ---------------------------------------------------------------------------
// regular nearfield pairs, row side (FP64): CTA per row leaf, thread (i, kk)
// ---------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(256) k_grad_near(Geom g, Tree t, Consts c, const int* __restrict__ rows,
                                                   const int* __restrict__ ptr, const int* __restrict__ col,
                                                   const double* __restrict__ xp, const double* __restrict__ wp,
                                                   double* __restrict__ dX) {
    __shared__ double sq[3 * kMaxLeaf * 7], sarea[kMaxLeaf], sx[kMaxLeaf * NR], sw[kMaxLeaf * NR];
    __shared__ int svid[3 * kMaxLeaf];
    __shared__ double sbuf[256];
    const int row = rows[blockIdx.x];
    const int rb = t.begin[row], R = t.end[row] - rb;
    const int K = 256 / R;
    const int tid = threadIdx.x, il = tid % R, kk = tid / R;
    const bool active = kk < K;
    const int n = g.n;
    double px[7], py[7], pz[7], xr[NR], wr[NR];
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
    }
    double sA = 0.0, Gp[7][3];
    for (int p = 0; p < 7; ++p) Gp[p][0] = Gp[p][1] = Gp[p][2] = 0.0;
    for (int b = ptr[blockIdx.x]; b < ptr[blockIdx.x + 1]; ++b) {
        const int s = col[b];
        const int cb = t.begin[s], C = t.end[s] - cb;
        __syncthreads();
        for (int e = tid; e < C * 7; e += 256)
            for (int d = 0; d < 3; ++d) sq[d * kMaxLeaf * 7 + e] = g.qa[((int64_t)d * n + cb) * 7 + e];
        for (int e = tid; e < C; e += 256) {
            sarea[e] = g.area[cb + e];
            for (int d = 0; d < 3; ++d) svid[d * kMaxLeaf + e] = g.vid[d * n + cb + e];
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
            double gam = 0.0;
#pragma unroll
            for (int r = 0; r < NR; ++r) gam += wr[r] * sx[jl * NR + r] + sw[jl * NR + r] * xr[r];
            const double ga = gam * sarea[jl];
            double S = 0.0;
            for (int q = 0; q < 7; ++q) {
                const double yx = sq[jl * 7 + q], yy = sq[kMaxLeaf * 7 + jl * 7 + q], yz = sq[2 * kMaxLeaf * 7 + jl * 7 + q];
                const double wq = c.rw[q];
                for (int p = 0; p < 7; ++p) {
                    const double dx = px[p] - yx, dy = py[p] - yy, dz = pz[p] - yz;
                    const double ri = rsqrt_nr(dx * dx + dy * dy + dz * dz);
                    S += c.rw[p] * wq * ri;
                    const double f = -ga * wq * ri * ri * ri;
                    Gp[p][0] += f * dx;
                    Gp[p][1] += f * dy;
                    Gp[p][2] += f * dz;
                }
            }
            sA += ga * S;
        }
    }
    // per row triangle: v[0] = sum gamma |tau_j| S, v[1 + 3k + d] = sum_p w_p lambda_pk G_p,d
    double v[10];
    v[0] = active ? sA : 0.0;
    for (int q = 1; q < 10; ++q) v[q] = 0.0;
    if (active)
        for (int p = 0; p < 7; ++p) {
            const double lam[3] = {1.0 - c.ru[p] - c.rv[p], c.ru[p], c.rv[p]};
            for (int k3 = 0; k3 < 3; ++k3)
                for (int d = 0; d < 3; ++d) v[1 + 3 * k3 + d] += c.rw[p] * lam[k3] * Gp[p][d];
        }
    for (int q = 0; q < 10; ++q) {
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
        double X[9];
        for (int q = 0; q < 9; ++q) X[q] = g.v[q * n + i];
        const double area = g.area[i];
        const double nx = g.nrm[i], ny = g.nrm[n + i], nz = g.nrm[2 * n + i];
        for (int k3 = 0; k3 < 3; ++k3) {
            const double* a = X + 3 * ((k3 + 1) % 3);
            const double* bb = X + 3 * ((k3 + 2) % 3);
            const double e[3] = {bb[0] - a[0], bb[1] - a[1], bb[2] - a[2]};
            const double dA[3] = {0.5 * (ny * e[2] - nz * e[1]), 0.5 * (nz * e[0] - nx * e[2]), 0.5 * (nx * e[1] - ny * e[0])};
            const int vid = g.vid[k3 * n + i];
            for (int d = 0; d < 3; ++d)
                atomicAdd(&dX[3 * (int64_t)vid + d], kInv4Pi * (dA[d] * v[0] + area * v[1 + 3 * k3 + d]));
        }
    }
}

// ---------------------------------------------------------------------------
// singular pairs: thread per canonical pair, Gram-form tables
// (identical [aa, 2ab, bb, W]; edge [aa, bb, dd, 2ab, 2ad, 2bd, ..., W at 9];
//  vertex [aa, bb, cc, dd, 2ab, 2ac, 2ad, 2bc, 2bd, 2cd, W])
// ---------------------------------------------------------------------------
template <int NR, int TYPE>
__global__ void __launch_bounds__(128) k_grad_singular(Geom g, int npairs, const int* __restrict__ plo,
                                                       const int* __restrict__ phi, const int* __restrict__ pcode,
                                                       const double* __restrict__ tab, int npts,
                                                       const double* __restrict__ xp, const double* __restrict__ wp,
                                                       double* __restrict__ dX) {
    constexpr int W = TYPE == IDENTICAL ? 4 : TYPE == EDGE ? 11 : 11;
    constexpr int NG = TYPE == IDENTICAL ? 3 : TYPE == EDGE ? 6 : 10;
    constexpr int WI = TYPE == IDENTICAL ? 3 : TYPE == EDGE ? 9 : 10;  // index of the weight
    constexpr int NVEC = TYPE == IDENTICAL ? 2 : TYPE == EDGE ? 3 : 4;
    extern __shared__ double stab[];
    for (int e = threadIdx.x; e < npts * W; e += blockDim.x) stab[e] = tab[e];
    __syncthreads();
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
    // edge vectors: identical (a, b); edge (a, b, d); vertex (a, b, c, d)
    double ev[4][3];
    for (int d = 0; d < 3; ++d) {
        ev[0][d] = P[1][d] - P[0][d];
        ev[1][d] = P[2][d] - P[1][d];
        if (TYPE == EDGE) ev[2][d] = Q[2][d] - Q[1][d];
        if (TYPE == VERTEX) {
            ev[2][d] = Q[1][d] - Q[0][d];
            ev[3][d] = Q[2][d] - Q[1][d];
        }
    }
    // Gram entry q couples vectors (ga[q], gb[q])
    int ga[NG], gb[NG];
    if (TYPE == IDENTICAL) {
        ga[0] = 0; gb[0] = 0; ga[1] = 0; gb[1] = 1; ga[2] = 1; gb[2] = 1;
    } else if (TYPE == EDGE) {
        const int A[6] = {0, 1, 2, 0, 0, 1}, B[6] = {0, 1, 2, 1, 2, 2};
        for (int q = 0; q < 6; ++q) { ga[q] = A[q]; gb[q] = B[q]; }
    } else {
        const int A[10] = {0, 1, 2, 3, 0, 0, 0, 1, 1, 2}, B[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
        for (int q = 0; q < 10; ++q) { ga[q] = A[q]; gb[q] = B[q]; }
    }
    double G[NG], Hk[NG];
    for (int q = 0; q < NG; ++q) {
        G[q] = ev[ga[q]][0] * ev[gb[q]][0] + ev[ga[q]][1] * ev[gb[q]][1] + ev[ga[q]][2] * ev[gb[q]][2];
        Hk[q] = 0.0;
    }
    double S = 0.0;
    for (int p = 0; p < npts; ++p) {
        const double* T = stab + p * W;
        double r2 = 0.0;
#pragma unroll
        for (int q = 0; q < NG; ++q) r2 += T[q] * G[q];
        const double ri = rsqrt_nr(r2);
        S += T[WI] * ri;
        const double f = -0.5 * T[WI] * ri * ri * ri;
#pragma unroll
        for (int q = 0; q < NG; ++q) Hk[q] += f * T[q];
    }
    const double ap = g.area[lo], aq = g.area[hi];
    const double sc = 4.0 * ap * aq * kInv4Pi;
    double gam = 0.0;
    for (int r = 0; r < NR; ++r)
        gam += lo == hi ? wp[(int64_t)lo * NR + r] * xp[(int64_t)lo * NR + r]
                        : wp[(int64_t)lo * NR + r] * xp[(int64_t)hi * NR + r] + wp[(int64_t)hi * NR + r] * xp[(int64_t)lo * NR + r];
    // d value / d edge vector
    double dv[4][3] = {{0}};
    for (int q = 0; q < NG; ++q) {
        const double dG = sc * Hk[q];
        for (int d = 0; d < 3; ++d) {
            dv[ga[q]][d] += dG * ev[gb[q]][d];
            dv[gb[q]][d] += dG * ev[ga[q]][d];
        }
    }
    // corners: a = P1-P0, b = P2-P1; edge d = Q2-Q1; vertex c = Q1-Q0, d = Q2-Q1
    double dP[3][3], dQ[3][3];
    for (int d = 0; d < 3; ++d) {
        dP[0][d] = -dv[0][d];
        dP[1][d] = dv[0][d] - dv[1][d];
        dP[2][d] = dv[1][d];
        dQ[0][d] = dQ[1][d] = dQ[2][d] = 0.0;
        if (TYPE == EDGE) {
            dQ[1][d] = -dv[2][d];
            dQ[2][d] = dv[2][d];
        }
        if (TYPE == VERTEX) {
            dQ[0][d] = -dv[2][d];
            dQ[1][d] = dv[2][d] - dv[3][d];
            dQ[2][d] = dv[3][d];
        }
    }
    // area factors |P| |Q|
    const double sp = 4.0 * kInv4Pi * aq * S, sq2 = 4.0 * kInv4Pi * ap * S;
    for (int side = 0; side < 2; ++side) {
        const double(*X)[3] = side == 0 ? P : Q;
        double nn[3];
        {
            const double e1[3] = {X[1][0] - X[0][0], X[1][1] - X[0][1], X[1][2] - X[0][2]};
            const double e2[3] = {X[2][0] - X[0][0], X[2][1] - X[0][1], X[2][2] - X[0][2]};
            nn[0] = e1[1] * e2[2] - e1[2] * e2[1];
            nn[1] = e1[2] * e2[0] - e1[0] * e2[2];
            nn[2] = e1[0] * e2[1] - e1[1] * e2[0];
            const double len = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
            nn[0] /= len;
            nn[1] /= len;
            nn[2] /= len;
        }
        const double f = side == 0 ? sp : sq2;
        double(*dXs)[3] = side == 0 ? dP : dQ;
        for (int k3 = 0; k3 < 3; ++k3) {
            const double* a = X[(k3 + 1) % 3];
            const double* bb = X[(k3 + 2) % 3];
            const double e[3] = {bb[0] - a[0], bb[1] - a[1], bb[2] - a[2]};
            dXs[k3][0] += f * 0.5 * (nn[1] * e[2] - nn[2] * e[1]);
            dXs[k3][1] += f * 0.5 * (nn[2] * e[0] - nn[0] * e[2]);
            dXs[k3][2] += f * 0.5 * (nn[0] * e[1] - nn[1] * e[0]);
        }
    }
    for (int k3 = 0; k3 < 3; ++k3)
        for (int d = 0; d < 3; ++d) {
            atomicAdd(&dX[3 * (int64_t)pv[k3] + d], gam * dP[k3][d]);
            atomicAdd(&dX[3 * (int64_t)qv[k3] + d], gam * dQ[k3][d]);
        }
    (void)NVEC;
}

// ---------------------------------------------------------------------------
// boxes -> extreme vertices: centre c = (lo+hi)/2, half-width h = (hi-lo)/2
// raised to 1e-2 of the largest half-width where smaller (then it follows the
// largest axis' extremes)
// ---------------------------------------------------------------------------
__global__ void k_grad_box(int nc, const int* __restrict__ cext, const int* __restrict__ cflag,
                           const double* __restrict__ dbox, double* __restrict__ dX) {
    const int cl = blockIdx.x * blockDim.x + threadIdx.x;
    if (cl >= nc) return;
    const int fl = cflag[cl], am = (fl >> 3) & 3;
    double glo[3] = {0, 0, 0}, ghi[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
        const double gc = dbox[d * nc + cl], gh = dbox[(3 + d) * nc + cl];
        glo[d] += 0.5 * gc;
        ghi[d] += 0.5 * gc;
        const bool floored = (fl >> d) & 1;
        const int e = floored ? am : d;
        const double f = floored ? 1e-2 : 1.0;
        glo[e] -= 0.5 * f * gh;
        ghi[e] += 0.5 * f * gh;
    }
    for (int d = 0; d < 3; ++d) {
        atomicAdd(&dX[3 * (int64_t)cext[d * nc + cl] + d], glo[d]);
        atomicAdd(&dX[3 * (int64_t)cext[(3 + d) * nc + cl] + d], ghi[d]);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define H2G_NR(NR, CALL)                                \
    switch (NR) {                                       \
        case 1: { constexpr int R_ = 1; CALL; } break;   \
        case 4: { constexpr int R_ = 4; CALL; } break;   \
        case 8: { constexpr int R_ = 8; CALL; } break;   \
        default: { constexpr int R_ = 16; CALL; } break;  \
    }

void launch_grad_coupling(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                          int NR, const double* wh, const double* xh, double* dbox, cudaStream_t s) {
    if (nrows <= 0) return;
    const size_t smem = sizeof(double) * (size_t)c.k * NR;
    H2G_NR(NR, (cudaFuncSetAttribute(k_grad_coupling<R_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                k_grad_coupling<R_><<<nrows, 256, smem, s>>>(t, c, rows, ptr, col, wh, xh, dbox)))
}

void launch_grad_transfer(const Tree& t, const Consts& c, int nch, const int* children, const int* parent, int NR,
                          const double* xh, const double* wh, const double* yh, const double* zh, double* dbox,
                          cudaStream_t s) {
    if (nch <= 0) return;
    const size_t smem = sizeof(double) * 4 * (size_t)c.k * NR;
    H2G_NR(NR, (cudaFuncSetAttribute(k_grad_transfer<R_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                k_grad_transfer<R_><<<nch, 256, smem, s>>>(t, c, children, parent, xh, wh, yh, zh, dbox)))
}

void launch_grad_leaf(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nl, const int* leaves,
                      int NR, const double* xp, const double* wp, const double* yh, const double* zh, double* dbox,
                      double* dX, cudaStream_t s) {
    if (nl <= 0) return;
    const int th = c.nb > 64 ? 128 : 64;
    H2G_NR(NR, (k_grad_leaf<R_><<<nl, th, 0, s>>>(g, t, c, rule, leaves, xp, wp, yh, zh, dbox, dX)))
}

void launch_grad_near(const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                      const int* col, int NR, const double* xp, const double* wp, double* dX, cudaStream_t s) {
    if (nrows <= 0) return;
    H2G_NR(NR, (k_grad_near<R_><<<nrows, 256, 0, s>>>(g, t, c, rows, ptr, col, xp, wp, dX)))
}

void launch_grad_singular(const Geom& g, int type, int npairs, const int* lo, const int* hi, const int* code,
                          const double* tab, int npts, int NR, const double* xp, const double* wp, double* dX,
                          cudaStream_t s) {
    if (npairs <= 0) return;
    const int W = type == IDENTICAL ? 4 : 11;
    const size_t smem = sizeof(double) * (size_t)npts * W;
    const dim3 grid((npairs + 127) / 128);
    if (type == IDENTICAL) {
        H2G_NR(NR, (cudaFuncSetAttribute(k_grad_singular<R_, IDENTICAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    k_grad_singular<R_, IDENTICAL><<<grid, 128, smem, s>>>(g, npairs, lo, hi, code, tab, npts, xp, wp, dX)))
    } else if (type == EDGE) {
        H2G_NR(NR, (cudaFuncSetAttribute(k_grad_singular<R_, EDGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    k_grad_singular<R_, EDGE><<<grid, 128, smem, s>>>(g, npairs, lo, hi, code, tab, npts, xp, wp, dX)))
    } else {
        H2G_NR(NR, (cudaFuncSetAttribute(k_grad_singular<R_, VERTEX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    k_grad_singular<R_, VERTEX><<<grid, 128, smem, s>>>(g, npairs, lo, hi, code, tab, npts, xp, wp, dX)))
    }
}

void launch_grad_box(int nc, const int* cext, const int* cflag, const double* dbox, double* dX, cudaStream_t s) {
    if (nc <= 0) return;
    k_grad_box<<<(nc + 127) / 128, 128, 0, s>>>(nc, cext, cflag, dbox, dX);
}

}  // namespace h2
