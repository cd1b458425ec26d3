// Green cross approximation (section 4) of the single layer: construction of
// the cluster bases on the host, level by level from the leaves up.
//
// For a cluster t with box B_t = [a, b]:
//  - omega_t = [a - delta, b + delta] on every axis, delta = the largest side
//    of B_t (the choice of the paper's experiments, section 5);
//  - Green's representation formula on omega_t (section 4),
//      g(x,y) = int g(x,z) dg/dn_z(z,y) dz - int dg/dn_z(x,z) g(z,y) dz,
//    discretised on the six faces of d omega_t, face f = 2d + side (side 0:
//    x_d = lo_d with normal -e_d, side 1: x_d = hi_d with normal +e_d), by
//    q x q Gauss-Legendre points over the face's other axes d1 < d2, point
//    index (f q + a) q + b, weight gw_a gw_b |side d1| |side d2|;
//  - L = (A C) over the row set (the triangles of a leaf; the children's
//    pivot triangles, first child first, for other clusters), with
//    A_i,nu = w_nu^(1/2) int_tau_i g(x, z_nu), C_i,nu = w_nu^(1/2) int_tau_i
//    dg/dn_z(x, z_nu), both by the 7-point rule on tau_i;
//  - adaptive cross approximation of L with full pivoting: the pivot is the
//    first entry in row-major order within a relative 2^-40 of the largest
//    residual entry, so that rounding far below that cannot change the choice;
//    stop at rank kmax, at a zero residual or when the pivot falls to eps
//    times the first one;
//  - V^_t = L|_{rows x sigma} (L|_{tau x sigma})^{-1} (eq. gca_onesided):
//    the leaf basis V_t of a leaf, else the transfer matrices of the children
//    (E_t1; E_t2) = V^_t split by rows (eq. (transfer)); the pivot triangles
//    t^ = rows[tau].
// The coupling matrices are Galerkin entries between pivot triangles,
// S_ts = G|_{t^ x s^}; they are evaluated on the GPU (k_gca.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;

struct Boundary {
    int k = 0;
    std::vector<double> z, sw, nz;  // points [k][3], w^(1/2), normals [k][3]
};

void boundary_rule(const double* lo, const double* hi, int q, const std::vector<double>& g,
                   const std::vector<double>& gw, Boundary& B) {
    B.k = 6 * q * q;
    B.z.assign(3 * B.k, 0.0);
    B.sw.assign(B.k, 0.0);
    B.nz.assign(3 * B.k, 0.0);
    for (int f = 0; f < 6; ++f) {
        const int d = f >> 1, side = f & 1;
        const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
        const double l1 = hi[d1] - lo[d1], l2 = hi[d2] - lo[d2];
        for (int a = 0; a < q; ++a)
            for (int b = 0; b < q; ++b) {
                const int nu = (f * q + a) * q + b;
                B.z[3 * nu + d] = side ? hi[d] : lo[d];
                B.z[3 * nu + d1] = lo[d1] + l1 * g[a];
                B.z[3 * nu + d2] = lo[d2] + l2 * g[b];
                B.sw[nu] = std::sqrt(gw[a] * gw[b] * l1 * l2);
                B.nz[3 * nu + d] = side ? 1.0 : -1.0;
            }
    }
}

// row of L for the triangle at tree position pos
void L_row(const GcaSetup& S, int64_t pos, const Boundary& B, double* L) {
    const int32_t* t = S.tri + 3 * S.perm[pos];
    double P[3][3];
    for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) P[c][d] = S.xyz[3 * (int64_t)t[c] + d];
    double e1[3], e2[3];
    for (int d = 0; d < 3; ++d) {
        e1[d] = P[1][d] - P[0][d];
        e2[d] = P[2][d] - P[0][d];
    }
    const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                 cz = e1[0] * e2[1] - e1[1] * e2[0];
    const double area = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    double X[7][3];
    for (int p = 0; p < 7; ++p)
        for (int d = 0; d < 3; ++d) X[p][d] = P[0][d] + S.ru[p] * e1[d] + S.rv[p] * e2[d];
    for (int nu = 0; nu < B.k; ++nu) {
        const double* z = &B.z[3 * nu];
        const double* nz = &B.nz[3 * nu];
        double sa = 0.0, sc = 0.0;
        for (int p = 0; p < 7; ++p) {
            const double dx = X[p][0] - z[0], dy = X[p][1] - z[1], dz = X[p][2] - z[2];
            const double r2 = dx * dx + dy * dy + dz * dz, r = std::sqrt(r2);
            sa += S.rw[p] * (kInv4Pi / r);
            sc += S.rw[p] * (kInv4Pi * (dx * nz[0] + dy * nz[1] + dz * nz[2]) / (r2 * r));
        }
        L[nu] = B.sw[nu] * area * sa;
        L[B.k + nu] = B.sw[nu] * area * sc;
    }
}

}  // namespace

// full-pivot cross approximation of the rows x cols matrix A (destroyed)
int cross_approx(std::vector<double>& A, int rows, int cols, double eps, int kmax, std::vector<int>& tau,
                 std::vector<int>& sigma) {
    tau.clear();
    sigma.clear();
    std::vector<double> cv(rows), rv(cols);
    double first = 0.0;
    const size_t total = (size_t)rows * cols;
    while ((int)tau.size() < std::min({kmax, rows, cols})) {
        double M = 0.0;
        for (size_t e = 0; e < total; ++e) M = std::max(M, std::fabs(A[e]));
        if (M == 0.0) break;
        const double thr = M * (1.0 - std::ldexp(1.0, -40));
        size_t e = 0;
        while (std::fabs(A[e]) < thr) ++e;
        const int pi = (int)(e / cols), pj = (int)(e % cols);
        const double p = A[e];
        if (tau.empty()) first = std::fabs(p);
        else if (std::fabs(p) <= eps * first) break;
        tau.push_back(pi);
        sigma.push_back(pj);
        for (int i = 0; i < rows; ++i) cv[i] = A[(size_t)i * cols + pj];
        for (int j = 0; j < cols; ++j) rv[j] = A[(size_t)pi * cols + j] / p;
        for (int i = 0; i < rows; ++i) {
            double* Ai = &A[(size_t)i * cols];
            const double c = cv[i];
            for (int j = 0; j < cols; ++j) Ai[j] -= c * rv[j];
        }
    }
    return (int)tau.size();
}

namespace {
// V = L|_{: x sigma} (L|_{tau x sigma})^{-1}: LU with partial pivoting of
// M = L|_{tau x sigma}, then V M = B row by row (B = L|_{: x sigma}).
void interp(const std::vector<double>& L, int rows, int cols, const std::vector<int>& tau,
            const std::vector<int>& sigma, std::vector<double>& V) {
    const int k = (int)tau.size();
    V.assign((size_t)rows * k, 0.0);
    if (!k) return;
    // solve V M = B  <=>  M^T V^T = B^T; factor Mt = M^T = P^T L U
    std::vector<double> Mt((size_t)k * k);
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) Mt[(size_t)a * k + b] = L[(size_t)tau[b] * cols + sigma[a]];
    std::vector<int> pv(k);
    for (int c = 0; c < k; ++c) {
        int pr = c;
        for (int a = c + 1; a < k; ++a)
            if (std::fabs(Mt[(size_t)a * k + c]) > std::fabs(Mt[(size_t)pr * k + c])) pr = a;
        pv[c] = pr;
        if (pr != c)
            for (int b = 0; b < k; ++b) std::swap(Mt[(size_t)c * k + b], Mt[(size_t)pr * k + b]);
        for (int a = c + 1; a < k; ++a) {
            const double f = Mt[(size_t)a * k + c] / Mt[(size_t)c * k + c];
            Mt[(size_t)a * k + c] = f;
            for (int b = c + 1; b < k; ++b) Mt[(size_t)a * k + b] -= f * Mt[(size_t)c * k + b];
        }
    }
    std::vector<double> y(k);
    for (int r = 0; r < rows; ++r) {
        for (int a = 0; a < k; ++a) y[a] = L[(size_t)r * cols + sigma[a]];
        for (int c = 0; c < k; ++c) std::swap(y[c], y[pv[c]]);
        for (int a = 1; a < k; ++a)
            for (int c = 0; c < a; ++c) y[a] -= Mt[(size_t)a * k + c] * y[c];
        for (int a = k - 1; a >= 0; --a) {
            double s = y[a];
            for (int b = a + 1; b < k; ++b) s -= Mt[(size_t)a * k + b] * y[b];
            y[a] = s / Mt[(size_t)a * k + a];
        }
        for (int a = 0; a < k; ++a) V[(size_t)r * k + a] = y[a];
    }
}
}  // namespace

int gca_build(const GcaSetup& S, GcaResult& R) {
    const int64_t nc = S.nc;
    const std::vector<double> g(S.gl_x, S.gl_x + S.q), gw(S.gl_w, S.gl_w + S.q);
    R.rank.assign(nc, 0);
    std::vector<std::vector<int64_t>> piv(nc);   // pivot tree positions
    std::vector<std::vector<double>> V(nc), E(nc);
    int64_t maxlev = 0;
    for (int64_t c = 0; c < nc; ++c) maxlev = std::max(maxlev, S.level[c]);
    std::vector<std::vector<int64_t>> bylev(maxlev + 1);
    for (int64_t c = 0; c < nc; ++c) bylev[S.level[c]].push_back(c);
    for (int64_t lev = maxlev; lev >= 0; --lev) {
        const auto& cl = bylev[lev];
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t ii = 0; ii < (int64_t)cl.size(); ++ii) {
            const int64_t c = cl[ii];
            double lo[3], hi[3], delta = 0.0;
            for (int d = 0; d < 3; ++d) delta = std::max(delta, S.bmax[3 * c + d] - S.bmin[3 * c + d]);
            for (int d = 0; d < 3; ++d) {
                lo[d] = S.bmin[3 * c + d] - delta;
                hi[d] = S.bmax[3 * c + d] + delta;
            }
            Boundary B;
            boundary_rule(lo, hi, S.q, g, gw, B);
            std::vector<int64_t> rows;
            const bool leaf = S.child0[c] < 0;
            if (leaf) {
                for (int64_t a = S.begin[c]; a < S.end[c]; ++a) rows.push_back(a);
            } else {
                for (int64_t ch : {S.child0[c], S.child1[c]}) rows.insert(rows.end(), piv[ch].begin(), piv[ch].end());
            }
            const int nr = (int)rows.size(), cols = 2 * B.k;
            std::vector<double> L((size_t)nr * cols);
            for (int r = 0; r < nr; ++r) L_row(S, rows[r], B, &L[(size_t)r * cols]);
            std::vector<double> A = L;
            std::vector<int> tau, sigma;
            const int rk = cross_approx(A, nr, cols, S.eps, S.kmax, tau, sigma);
            std::vector<double> Vh;
            interp(L, nr, cols, tau, sigma, Vh);
            R.rank[c] = rk;
            for (int a = 0; a < rk; ++a) piv[c].push_back(rows[tau[a]]);
            if (leaf) {
                V[c] = std::move(Vh);
            } else {
                int off = 0;
                for (int64_t ch : {S.child0[c], S.child1[c]}) {
                    const int kc = (int)piv[ch].size();
                    E[ch].assign(Vh.begin() + (size_t)off * rk, Vh.begin() + (size_t)(off + kc) * rk);
                    off += kc;
                }
            }
        }
    }
    // flatten
    R.piv_off.assign(nc + 1, 0);
    R.voff.assign(nc, -1);
    R.eoff.assign(nc, -1);
    R.piv.clear();
    R.V.clear();
    R.E.clear();
    for (int64_t c = 0; c < nc; ++c) {
        R.piv_off[c + 1] = R.piv_off[c] + (int)piv[c].size();
        for (int64_t p : piv[c]) R.piv.push_back((int)p);
        if (!V[c].empty()) {
            R.voff[c] = (int64_t)R.V.size();
            R.V.insert(R.V.end(), V[c].begin(), V[c].end());
        }
        if (!E[c].empty()) {
            R.eoff[c] = (int64_t)R.E.size();
            R.E.insert(R.E.end(), E[c].begin(), E[c].end());
        }
    }
    return 0;
}

}  // namespace h2
