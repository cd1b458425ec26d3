// Hybrid cross approximation (section 3) of the single layer and its
// hierarchical compression into an H^2-matrix: construction on the host
// (OpenMP), stored for the GPU apply of the stored-basis passes (k_gca.cu).
//
// Per farfield block b = (t, s), with the tensor Chebyshev nodes xi of both
// clusters (m per axis, k = m^3; the node rule of the interpolation bases):
//  - S = g(xi_t, xi_s) (k x k) and its cross approximation with full pivoting
//    (cross_approx, the rule of the GCA construction) to eps_aca, at most kaca
//    steps: row pivots tau, column pivots sigma, rank r;
//  - C = (S|_{tau x sigma})^{-1} by LU with partial pivoting, indexed
//    [sigma position][tau position];
//  - the take-back factors of eq. (hca_discrete), A[i,kappa] = int_{tau_i}
//    g(x, xi_{s,sigma_kappa}) for i in t and B[j,lambda] = int_{tau_j}
//    g(xi_{t,tau_lambda}, y) for j in s (7-point rule): G|_{t x s} ~ A C B^T.
// Compression into orthonormal nested cluster bases, from the leaves up (the
// paper cites hierarchical compression without fixing its steps; this follows
// the construction of total cluster bases):
//  - the block row of cluster c is every block (a, s) with a = c or an
//    ancestor of c, restricted to the rows of c; with B = Q R (Householder),
//    A C B^T = (A C R^T) Q^T and Q^T has orthonormal rows, so the columns
//    A|_c W, W = C R^T, carry the block row's left singular vectors and values;
//  - leaves: Q_c = the left singular vectors of Z_c = [A_b|_c W_b]_b with
//    singular values above eps_c times the largest (at most kmax);
//    other clusters: the same for [Q_c1^T Z_c|_c1 ; Q_c2^T Z_c|_c2], whose
//    vectors split by rows into the transfer matrices E_c1, E_c2;
//  - the singular vectors: the triangular factor of Z^T (Householder), then
//    one-sided Jacobi on its transpose, vectors = normalised rotated columns;
//  - coupling matrices S_b = (Q_t^T A_b) C_b (Q_s^T B_b)^T.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"

namespace h2 {

namespace {
constexpr double kInv4Pi = 0.07957747154594766788;
constexpr double kPi = 3.14159265358979323846;

inline double green(const double* x, const double* y) {
    const double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
    const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
    return kInv4Pi / r;
}

// the 7 rule points and the area of the triangle at tree position pos
struct Panel {
    double X[7][3];
    double area;
};
void make_panel(const HcaSetup& S, int64_t pos, Panel& P) {
    const int32_t* t = S.tri + 3 * S.perm[pos];
    double V[3][3];
    for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) V[c][d] = S.xyz[3 * (int64_t)t[c] + d];
    double e1[3], e2[3];
    for (int d = 0; d < 3; ++d) {
        e1[d] = V[1][d] - V[0][d];
        e2[d] = V[2][d] - V[0][d];
    }
    const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                 cz = e1[0] * e2[1] - e1[1] * e2[0];
    P.area = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    for (int q = 0; q < 7; ++q)
        for (int d = 0; d < 3; ++d) P.X[q][d] = V[0][d] + S.ru[q] * e1[d] + S.rv[q] * e2[d];
}
inline double potential(const HcaSetup& S, const Panel& P, const double* p) {
    double s = 0.0;
    for (int q = 0; q < 7; ++q) s += S.rw[q] * green(P.X[q], p);
    return P.area * s;
}

// Upper-triangular (trapezoidal) factor R (p x cols, row-major, p =
// min(rows, cols)) of the Householder QR of the rows x cols matrix X
// (row-major, overwritten).
void householder_r(std::vector<double>& X, int rows, int cols, std::vector<double>& R) {
    const int p = std::min(rows, cols);
    std::vector<double> v(rows);
    for (int j = 0; j < p; ++j) {
        double nn = 0.0;
        for (int i = j; i < rows; ++i) nn += X[(size_t)i * cols + j] * X[(size_t)i * cols + j];
        if (nn == 0.0) continue;
        const double nrm = std::sqrt(nn);
        const double x0 = X[(size_t)j * cols + j];
        const double beta = x0 > 0 ? -nrm : nrm;  // new diagonal entry
        // v = x - beta e_j, |v|^2 = 2 nrm (nrm + |x0|)
        for (int i = j; i < rows; ++i) v[i] = X[(size_t)i * cols + j];
        v[j] = x0 - beta;
        const double vv = 2.0 * nrm * (nrm + std::fabs(x0));
        X[(size_t)j * cols + j] = beta;
        for (int i = j + 1; i < rows; ++i) X[(size_t)i * cols + j] = 0.0;
        for (int c = j + 1; c < cols; ++c) {
            double d = 0.0;
            for (int i = j; i < rows; ++i) d += v[i] * X[(size_t)i * cols + c];
            const double f = 2.0 * d / vv;
            for (int i = j; i < rows; ++i) X[(size_t)i * cols + c] -= f * v[i];
        }
    }
    R.assign((size_t)p * cols, 0.0);
    for (int i = 0; i < p; ++i)
        for (int c = i; c < cols; ++c) R[(size_t)i * cols + c] = X[(size_t)i * cols + c];
}

// Left singular vectors and values of Z (rows x cols) from the factor R of
// Z^T = Q R (R: p x rows, row-major): Z = R^T Q^T, one-sided Jacobi on the
// columns of Y = R^T (rows x p) until they are orthogonal; the singular values
// are the column norms, the vectors the normalised columns.  U: rows x p
// (column j = j-th vector), sorted by decreasing value.
void left_singular(const std::vector<double>& R, int p, int rows, std::vector<double>& U, std::vector<double>& sv) {
    std::vector<double> Y((size_t)p * rows);  // column-major: column j = Y[j*rows ...]
    for (int j = 0; j < p; ++j)
        for (int i = 0; i < rows; ++i) Y[(size_t)j * rows + i] = R[(size_t)j * rows + i];
    for (int sweep = 0; sweep < 60; ++sweep) {
        bool any = false;
        for (int a = 0; a < p - 1; ++a)
            for (int b = a + 1; b < p; ++b) {
                double* ya = &Y[(size_t)a * rows];
                double* yb = &Y[(size_t)b * rows];
                double aa = 0.0, bb = 0.0, ab = 0.0;
                for (int i = 0; i < rows; ++i) {
                    aa += ya[i] * ya[i];
                    bb += yb[i] * yb[i];
                    ab += ya[i] * yb[i];
                }
                if (ab == 0.0 || std::fabs(ab) <= 1e-15 * std::sqrt(aa * bb)) continue;
                any = true;
                const double tau = (bb - aa) / (2.0 * ab);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < rows; ++i) {
                    const double u = ya[i], w = yb[i];
                    ya[i] = c * u - s * w;
                    yb[i] = s * u + c * w;
                }
            }
        if (!any) break;
    }
    std::vector<double> nrm(p);
    for (int j = 0; j < p; ++j) {
        double s = 0.0;
        for (int i = 0; i < rows; ++i) s += Y[(size_t)j * rows + i] * Y[(size_t)j * rows + i];
        nrm[j] = std::sqrt(s);
    }
    std::vector<int> ord(p);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return nrm[a] > nrm[b]; });
    U.assign((size_t)rows * p, 0.0);
    sv.assign(p, 0.0);
    for (int j = 0; j < p; ++j) {
        const int o = ord[j];
        sv[j] = nrm[o];
        if (nrm[o] > 0.0)
            for (int i = 0; i < rows; ++i) U[(size_t)i * p + j] = Y[(size_t)o * rows + i] / nrm[o];
    }
}

// inverse of the r x r matrix M (row-major) by LU with partial pivoting;
// false if a pivot vanishes
bool invert(const std::vector<double>& M, int r, std::vector<double>& Inv) {
    std::vector<double> F(M);
    std::vector<int> pv(r);
    for (int c = 0; c < r; ++c) {
        int p = c;
        for (int i = c + 1; i < r; ++i)
            if (std::fabs(F[(size_t)i * r + c]) > std::fabs(F[(size_t)p * r + c])) p = i;
        if (F[(size_t)p * r + c] == 0.0) return false;
        pv[c] = p;
        if (p != c)
            for (int j = 0; j < r; ++j) std::swap(F[(size_t)c * r + j], F[(size_t)p * r + j]);
        for (int i = c + 1; i < r; ++i) {
            const double f = F[(size_t)i * r + c] / F[(size_t)c * r + c];
            F[(size_t)i * r + c] = f;
            for (int j = c + 1; j < r; ++j) F[(size_t)i * r + j] -= f * F[(size_t)c * r + j];
        }
    }
    Inv.assign((size_t)r * r, 0.0);
    std::vector<double> y(r);
    for (int col = 0; col < r; ++col) {
        for (int i = 0; i < r; ++i) y[i] = i == col ? 1.0 : 0.0;
        for (int c = 0; c < r; ++c) std::swap(y[c], y[pv[c]]);
        for (int i = 1; i < r; ++i)
            for (int c = 0; c < i; ++c) y[i] -= F[(size_t)i * r + c] * y[c];
        for (int i = r - 1; i >= 0; --i) {
            double s = y[i];
            for (int j = i + 1; j < r; ++j) s -= F[(size_t)i * r + j] * y[j];
            y[i] = s / F[(size_t)i * r + i];
        }
        for (int i = 0; i < r; ++i) Inv[(size_t)i * r + col] = y[i];
    }
    return true;
}
}  // namespace

int hca_build(const HcaSetup& S, HcaResult& R) {
    const int64_t nc = S.nc, nf = S.nfar;
    const int m = S.m, k = m * m * m;
    // Chebyshev nodes per cluster and axis (half-widths raised to 1e-2 of the largest)
    std::vector<double> nodes((size_t)nc * 3 * m);
    for (int64_t c = 0; c < nc; ++c) {
        double ctr[3], h[3], hmax = 0.0;
        for (int d = 0; d < 3; ++d) {
            ctr[d] = 0.5 * (S.bmin[3 * c + d] + S.bmax[3 * c + d]);
            h[d] = 0.5 * (S.bmax[3 * c + d] - S.bmin[3 * c + d]);
            hmax = std::max(hmax, h[d]);
        }
        for (int d = 0; d < 3; ++d) {
            const double hd = h[d] < 1e-2 * hmax ? 1e-2 * hmax : h[d];
            for (int a = 0; a < m; ++a) nodes[(c * 3 + d) * m + a] = ctr[d] + hd * std::cos((2.0 * a + 1.0) * kPi / (2.0 * m));
        }
    }
    auto node = [&](int64_t c, int nu, double* x) {
        x[0] = nodes[(c * 3 + 0) * m + nu % m];
        x[1] = nodes[(c * 3 + 1) * m + (nu / m) % m];
        x[2] = nodes[(c * 3 + 2) * m + nu / (m * m)];
    };
    std::vector<int64_t> parent(nc, -1);
    for (int64_t c = 0; c < nc; ++c)
        if (S.child0[c] >= 0) parent[S.child0[c]] = parent[S.child1[c]] = c;
    // blocks by row cluster
    std::vector<int64_t> bptr(nc + 1, 0), bidx(nf);
    for (int64_t b = 0; b < nf; ++b) bptr[S.far_t[b] + 1]++;
    for (int64_t c = 0; c < nc; ++c) bptr[c + 1] += bptr[c];
    {
        std::vector<int64_t> fill(bptr.begin(), bptr.end() - 1);
        for (int64_t b = 0; b < nf; ++b) bidx[fill[S.far_t[b]]++] = b;
    }

    // ---- per block: cross approximation, C, W = C R^T --------------------
    R.brank.assign(nf, 0);
    std::vector<std::vector<int>> btau(nf), bsig(nf);
    std::vector<std::vector<double>> bC(nf), bW(nf);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < nf; ++b) {
        const int64_t t = S.far_t[b], s = S.far_s[b];
        std::vector<double> Sm((size_t)k * k);
        double xt[3], xs[3];
        for (int nu = 0; nu < k; ++nu) {
            node(t, nu, xt);
            for (int mu = 0; mu < k; ++mu) {
                node(s, mu, xs);
                Sm[(size_t)nu * k + mu] = green(xt, xs);
            }
        }
        std::vector<double> Sc(Sm);
        std::vector<int> tau, sig;
        int r = cross_approx(Sc, k, k, S.eps_aca, std::min(S.kaca, k), tau, sig);
        std::vector<double> M((size_t)r * r), C;
        for (int a = 0; a < r; ++a)
            for (int c = 0; c < r; ++c) M[(size_t)a * r + c] = Sm[(size_t)tau[a] * k + sig[c]];
        if (!invert(M, r, C)) r = 0;
        tau.resize(r);
        sig.resize(r);
        std::vector<double> W((size_t)r * r, 0.0);
        if (r > 0) {
            const int64_t ns = S.end[s] - S.begin[s];
            std::vector<double> Bm((size_t)ns * r);
            Panel P;
            for (int64_t j = 0; j < ns; ++j) {
                make_panel(S, S.begin[s] + j, P);
                for (int l = 0; l < r; ++l) {
                    node(t, tau[l], xt);
                    Bm[(size_t)j * r + l] = potential(S, P, xt);
                }
            }
            std::vector<double> Rf;
            householder_r(Bm, (int)ns, r, Rf);
            const int p = std::min<int>((int)ns, r);
            for (int a = 0; a < r; ++a)
                for (int c = 0; c < p; ++c) {
                    double acc = 0.0;
                    for (int l = 0; l < r; ++l) acc += C[(size_t)a * r + l] * Rf[(size_t)c * r + l];
                    W[(size_t)a * r + c] = acc;
                }
        }
        R.brank[b] = r;
        btau[b] = std::move(tau);
        bsig[b] = std::move(sig);
        bC[b] = std::move(C);
        bW[b] = std::move(W);
    }

    // ---- compression, level by level from the leaves -----------------------
    R.rank.assign(nc, 0);
    std::vector<std::vector<double>> Q(nc), E(nc);  // Q_c: |c| x rank row-major (tree order)
    // Q_c^T A_b|_c (rank_c x r) for a cluster c inside the row cluster of b
    auto projected_A = [&](int64_t b, int64_t c, double* out) {
        const int r = R.brank[b], kc = R.rank[c];
        const int64_t s = S.far_s[b];
        std::fill(out, out + (size_t)kc * r, 0.0);
        std::vector<double> a(r);
        Panel P;
        double p[3];
        for (int64_t i = 0; i < S.end[c] - S.begin[c]; ++i) {
            make_panel(S, S.begin[c] + i, P);
            for (int l = 0; l < r; ++l) {
                node(s, bsig[b][l], p);
                a[l] = potential(S, P, p);
            }
            const double* q = &Q[c][(size_t)i * kc];
            for (int nu = 0; nu < kc; ++nu)
                for (int l = 0; l < r; ++l) out[(size_t)nu * r + l] += q[nu] * a[l];
        }
    };
    int64_t maxlev = 0;
    for (int64_t c = 0; c < nc; ++c) maxlev = std::max(maxlev, S.level[c]);
    std::vector<std::vector<int64_t>> bylev(maxlev + 1);
    for (int64_t c = 0; c < nc; ++c) bylev[S.level[c]].push_back(c);
    for (int64_t lev = maxlev; lev >= 0; --lev) {
        const auto& cl = bylev[lev];
        const int64_t ncl = (int64_t)cl.size();
        // the columns of Z_c, transposed: Zt[c] is cols x rows (row-major), one
        // row per column of Z; the (cluster, block) pieces run in parallel
        std::vector<int> rows(ncl);
        std::vector<int64_t> cols(ncl, 0);
        std::vector<std::vector<double>> Zt(ncl);
        struct Piece {
            int64_t ci, b, off;
        };
        std::vector<Piece> pieces;
        for (int64_t ii = 0; ii < ncl; ++ii) {
            const int64_t c = cl[ii];
            const bool leaf = S.child0[c] < 0;
            rows[ii] = leaf ? (int)(S.end[c] - S.begin[c]) : R.rank[S.child0[c]] + R.rank[S.child1[c]];
            for (int64_t a = c; a >= 0; a = parent[a])
                for (int64_t q = bptr[a]; q < bptr[a + 1]; ++q) {
                    const int64_t b = bidx[q];
                    if (R.brank[b] == 0) continue;
                    pieces.push_back({ii, b, cols[ii]});
                    cols[ii] += R.brank[b];
                }
            Zt[ii].assign((size_t)cols[ii] * rows[ii], 0.0);
        }
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t pi = 0; pi < (int64_t)pieces.size(); ++pi) {
            const Piece& pc = pieces[pi];
            const int64_t c = cl[pc.ci];
            const int64_t b = pc.b;
            const int r = R.brank[b], nr = rows[pc.ci];
            std::vector<double> Ah((size_t)nr * r);
            if (S.child0[c] < 0) {
                Panel P;
                double p[3];
                for (int i = 0; i < nr; ++i) {
                    make_panel(S, S.begin[c] + i, P);
                    for (int l = 0; l < r; ++l) {
                        node(S.far_s[b], bsig[b][l], p);
                        Ah[(size_t)i * r + l] = potential(S, P, p);
                    }
                }
            } else {
                const int k1 = R.rank[S.child0[c]];
                projected_A(b, S.child0[c], Ah.data());
                projected_A(b, S.child1[c], Ah.data() + (size_t)k1 * r);
            }
            // columns off .. off + r of Z: Ah W
            for (int j = 0; j < r; ++j)
                for (int i = 0; i < nr; ++i) {
                    double acc = 0.0;
                    for (int l = 0; l < r; ++l) acc += Ah[(size_t)i * r + l] * bW[b][(size_t)l * r + j];
                    Zt[pc.ci][(size_t)(pc.off + j) * nr + i] = acc;
                }
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t ii = 0; ii < ncl; ++ii) {
            const int64_t c = cl[ii];
            const bool leaf = S.child0[c] < 0;
            const int nr = rows[ii];
            const int64_t nct = S.end[c] - S.begin[c];
            int kt = 0;
            std::vector<double> U, sv;
            int p = 0;
            if (nr > 0 && cols[ii] > 0) {
                std::vector<double> Rf;
                householder_r(Zt[ii], (int)cols[ii], nr, Rf);
                p = (int)std::min<int64_t>(cols[ii], nr);
                left_singular(Rf, p, nr, U, sv);
                if (sv[0] > 0.0)
                    while (kt < p && kt < S.kmax && sv[kt] > S.eps_c * sv[0]) ++kt;
            }
            std::vector<double>().swap(Zt[ii]);
            R.rank[c] = kt;
            Q[c].assign((size_t)nct * kt, 0.0);
            if (leaf) {
                for (int64_t i = 0; i < nct; ++i)
                    for (int j = 0; j < kt; ++j) Q[c][(size_t)i * kt + j] = U[(size_t)i * p + j];
            } else {
                int roff = 0;
                for (int64_t ch : {S.child0[c], S.child1[c]}) {
                    const int kc = R.rank[ch];
                    E[ch].assign((size_t)kc * kt, 0.0);
                    for (int a = 0; a < kc; ++a)
                        for (int j = 0; j < kt; ++j) E[ch][(size_t)a * kt + j] = U[(size_t)(roff + a) * p + j];
                    const int64_t b0 = S.begin[ch] - S.begin[c], nch = S.end[ch] - S.begin[ch];
                    for (int64_t i = 0; i < nch; ++i)
                        for (int j = 0; j < kt; ++j) {
                            double acc = 0.0;
                            for (int a = 0; a < kc; ++a) acc += Q[ch][(size_t)i * kc + a] * E[ch][(size_t)a * kt + j];
                            Q[c][(size_t)(b0 + i) * kt + j] = acc;
                        }
                    roff += kc;
                }
            }
        }
    }

    // ---- coupling matrices -------------------------------------------------
    std::vector<std::vector<double>> Sb(nf);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < nf; ++b) {
        const int64_t t = S.far_t[b], s = S.far_s[b];
        const int r = R.brank[b], kt = R.rank[t], ks = R.rank[s];
        Sb[b].assign((size_t)kt * ks, 0.0);
        if (!r || !kt || !ks) continue;
        std::vector<double> QA((size_t)kt * r), QB((size_t)ks * r, 0.0), CQ((size_t)r * ks, 0.0);
        projected_A(b, t, QA.data());
        Panel P;
        double p[3];
        std::vector<double> bv(r);
        for (int64_t j = 0; j < S.end[s] - S.begin[s]; ++j) {
            make_panel(S, S.begin[s] + j, P);
            for (int l = 0; l < r; ++l) {
                node(t, btau[b][l], p);
                bv[l] = potential(S, P, p);
            }
            for (int mu = 0; mu < ks; ++mu)
                for (int l = 0; l < r; ++l) QB[(size_t)mu * r + l] += Q[s][(size_t)j * ks + mu] * bv[l];
        }
        for (int a = 0; a < r; ++a)
            for (int mu = 0; mu < ks; ++mu) {
                double acc = 0.0;
                for (int l = 0; l < r; ++l) acc += bC[b][(size_t)a * r + l] * QB[(size_t)mu * r + l];
                CQ[(size_t)a * ks + mu] = acc;
            }
        for (int nu = 0; nu < kt; ++nu)
            for (int mu = 0; mu < ks; ++mu) {
                double acc = 0.0;
                for (int a = 0; a < r; ++a) acc += QA[(size_t)nu * r + a] * CQ[(size_t)a * ks + mu];
                Sb[b][(size_t)nu * ks + mu] = acc;
            }
    }

    // ---- flatten -----------------------------------------------------------
    R.voff.assign(nc, -1);
    R.eoff.assign(nc, -1);
    R.V.clear();
    R.E.clear();
    for (int64_t c = 0; c < nc; ++c) {
        if (S.child0[c] < 0) {
            R.voff[c] = (int64_t)R.V.size();
            R.V.insert(R.V.end(), Q[c].begin(), Q[c].end());
        }
        if (!E[c].empty()) {
            R.eoff[c] = (int64_t)R.E.size();
            R.E.insert(R.E.end(), E[c].begin(), E[c].end());
        }
    }
    R.soff.assign(nf + 1, 0);
    for (int64_t b = 0; b < nf; ++b) R.soff[b + 1] = R.soff[b] + (int64_t)Sb[b].size();
    R.S.resize(R.soff[nf]);
    for (int64_t b = 0; b < nf; ++b) std::copy(Sb[b].begin(), Sb[b].end(), R.S.begin() + R.soff[b]);
    return 0;
}

}  // namespace h2
