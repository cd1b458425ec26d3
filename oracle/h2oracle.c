/*
 * FP64 CPU oracle for the Galerkin BEM single-layer (G) and double-layer (K)
 * Laplace operators with piecewise-constant basis functions, and for their
 * H^2-matrix approximation by tensor Chebyshev interpolation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares no source, no
 * header, no table and no constant generator with the CUDA library; the two
 * implement the same written specification independently.
 *
 * Plain, slow and direct: every function follows the definition it names, in
 * the paper's order and notation, in double precision.  OpenMP only spreads
 * independent rows (or row clusters) over threads.
 *
 * Paper: S. Boerm, "Fast large-scale boundary element algorithms".
 *   - Green's function g and its normal derivative: section 1.
 *   - Matrix entries g_ij, k_ij: section 1, eq. (slp) and eq. (dlp).
 *   - Cluster tree, block tree, farfield/nearfield leaves: section 2,
 *     Definitions "cluster tree" and "block tree".
 *   - Cluster basis, transfer matrices: section 2, eq. (transfer).
 *   - H^2-matrix blocks G|_{t x s} = V_t S_ts W_s^*: section 2, eq. (vsw).
 *   - Bounding boxes, admissibility: section 3, eq. (admissibility).
 *   - Tensor Chebyshev interpolation g_int, k = m^3: section 3.
 *   - Singular (Sauter-Schwab-Erichsen) quadrature is cited, not printed, in
 *     sections 1 and 5; the region maps used here are the standard relative-
 *     coordinate Duffy decompositions for identical, edge- and vertex-adjacent
 *     triangles (6, 5 and 2 regions), written out in h2oracle.h.
 *
 * Parity status per function is listed in h2oracle.h.
 */
#include "h2oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288
#define OR_INV4PI (1.0 / (4.0 * OR_PI))

/* ------------------------------------------------------------------------- */
/* 1-D Gauss-Legendre rule on [0,1] (Newton iteration on the three-term      */
/* recurrence of the Legendre polynomials).                                  */
/* ------------------------------------------------------------------------- */
int or_gauss_legendre01(int q, double* x, double* w) {
    if (q < 1 || q > 64) return -1;
    for (int i = 0; i < q; ++i) {
        /* node i of P_q on [-1,1], counted from the right end */
        double z = cos(OR_PI * (i + 0.75) / (q + 0.5));
        double pk = 1.0, pkm1 = 0.0, dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            /* P_q(z) and P_{q-1}(z) by the three-term recurrence */
            pkm1 = 1.0;
            pk = z;
            for (int k = 2; k <= q; ++k) {
                double pkp1 = ((2.0 * k - 1.0) * z * pk - (k - 1.0) * pkm1) / k;
                pkm1 = pk;
                pk = pkp1;
            }
            if (q == 1) pkm1 = 1.0;
            dp = q * (z * pk - pkm1) / (z * z - 1.0); /* P_q'(z) */
            double dz = pk / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        pkm1 = 1.0;
        pk = z;
        for (int k = 2; k <= q; ++k) {
            double pkp1 = ((2.0 * k - 1.0) * z * pk - (k - 1.0) * pkm1) / k;
            pkm1 = pk;
            pk = pkp1;
        }
        dp = q * (z * pk - pkm1) / (z * z - 1.0);
        /* map [-1,1] -> [0,1]; ascending order */
        x[q - 1 - i] = 0.5 * (1.0 + z);
        w[q - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* 7-point rule of degree 5 on the unit simplex {u,v >= 0, u+v <= 1} (Radon's
 * rule).  Points as (u,v), weights normalised to sum 1, so that
 * int_tau f ~= |tau| sum_p w_p f(x_p) with x_p = V0 + u(V1-V0) + v(V2-V0). */
void or_radon7(double* uv, double* w) {
    const double r = sqrt(15.0);
    const double a = (6.0 - r) / 21.0, b = (6.0 + r) / 21.0;
    const double wa = (155.0 - r) / 1200.0, wb = (155.0 + r) / 1200.0;
    const double pts[7][2] = {{1.0 / 3.0, 1.0 / 3.0}, {a, a}, {1.0 - 2.0 * a, a}, {a, 1.0 - 2.0 * a},
                              {b, b}, {1.0 - 2.0 * b, b}, {b, 1.0 - 2.0 * b}};
    const double ws[7] = {9.0 / 40.0, wa, wa, wa, wb, wb, wb};
    for (int p = 0; p < 7; ++p) {
        uv[2 * p] = pts[p][0];
        uv[2 * p + 1] = pts[p][1];
        w[p] = ws[p];
    }
}

/* Collapsed (Duffy) tensor Gauss rule on the unit simplex: u = s,
 * v = (1-s) t with s,t Gauss-Legendre on [0,1]; exact for total degree
 * <= 2q-2.  Weights normalised to sum 1.  Returns the point count q*q. */
int or_collapsed_rule(int q, double* uv, double* w) {
    double x[64], wx[64];
    if (or_gauss_legendre01(q, x, wx)) return -1;
    int k = 0;
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
            uv[2 * k] = x[i];
            uv[2 * k + 1] = (1.0 - x[i]) * x[j];
            w[k] = 2.0 * wx[i] * wx[j] * (1.0 - x[i]);
            ++k;
        }
    return k;
}

/* ------------------------------------------------------------------------- */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------- */
static void sub3(const double* a, const double* b, double* c) {
    c[0] = a[0] - b[0];
    c[1] = a[1] - b[1];
    c[2] = a[2] - b[2];
}
static void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* area |tau| and outward unit normal of the triangle (a, b, c). */
void or_tri_geom(const double* a, const double* b, const double* c, double* area, double* normal) {
    double e1[3], e2[3], cr[3];
    sub3(b, a, e1);
    sub3(c, a, e2);
    cross3(e1, e2, cr);
    double len = sqrt(dot3(cr, cr));
    *area = 0.5 * len;
    normal[0] = cr[0] / len;
    normal[1] = cr[1] / len;
    normal[2] = cr[2] / len;
}

static void tri_vertices(const or_mesh* M, int64_t i, double* V /* 9 */) {
    for (int k = 0; k < 3; ++k) {
        int64_t v = M->tri[3 * i + k];
        V[3 * k + 0] = M->xyz[3 * v + 0];
        V[3 * k + 1] = M->xyz[3 * v + 1];
        V[3 * k + 2] = M->xyz[3 * v + 2];
    }
}

/* ------------------------------------------------------------------------- */
/* Kernel functions (section 1): g(x,y) = 1/(4 pi |x-y|), g(x,x) = 0;        */
/* d g / d n_y (x,y) = (x-y).n_y / (4 pi |x-y|^3).                           */
/* ------------------------------------------------------------------------- */
static double kernel_slp(const double* x, const double* y) {
    double d[3];
    sub3(x, y, d);
    double r = sqrt(dot3(d, d));
    return r > 0.0 ? OR_INV4PI / r : 0.0;
}
static double kernel_dlp(const double* x, const double* y, const double* ny) {
    double d[3];
    sub3(x, y, d);
    double r2 = dot3(d, d);
    if (r2 == 0.0) return 0.0;
    double r = sqrt(r2);
    return OR_INV4PI * dot3(d, ny) / (r2 * r);
}

/* ------------------------------------------------------------------------- */
/* Regular pairs: 7 x 7 point tensor rule on tau x sigma.                    */
/* ------------------------------------------------------------------------- */
double or_pair_regular(int kernel, const double* X, const double* Y) {
    double uv[14], w[7];
    or_radon7(uv, w);
    double ax, nx[3], ay, ny[3];
    or_tri_geom(X, X + 3, X + 6, &ax, nx);
    or_tri_geom(Y, Y + 3, Y + 6, &ay, ny);
    double xp[7][3], yq[7][3];
    for (int p = 0; p < 7; ++p)
        for (int d = 0; d < 3; ++d) {
            xp[p][d] = X[d] + uv[2 * p] * (X[3 + d] - X[d]) + uv[2 * p + 1] * (X[6 + d] - X[d]);
            yq[p][d] = Y[d] + uv[2 * p] * (Y[3 + d] - Y[d]) + uv[2 * p + 1] * (Y[6 + d] - Y[d]);
        }
    double s = 0.0;
    for (int p = 0; p < 7; ++p) {
        double sq = 0.0;
        for (int q = 0; q < 7; ++q) {
            double k = kernel == OR_SLP ? kernel_slp(xp[p], yq[q]) : kernel_dlp(xp[p], yq[q], ny);
            sq += w[q] * k;
        }
        s += w[p] * sq;
    }
    return ax * ay * s;
}

/* ------------------------------------------------------------------------- */
/* Sauter-Schwab quadrature (full 4-D tensor Gauss, q points per direction). */
/*                                                                           */
/* Reference triangle T = {(x1,x2): 0 <= x2 <= x1 <= 1}, parametrisation     */
/* chi(x) = P0 + x1 (P1 - P0) + x2 (P2 - P1), |det| = 2 |tau|.               */
/* int_tau int_sigma k = 4 |tau||sigma| int_T int_T k(chi_t(x), chi_s(y)).   */
/* The regions and Jacobians are listed in h2oracle.h.                       */
/*                                                                           */
/* kernel: OR_SLP -> g;  OR_DLP -> (x-y).nrm/(4 pi |x-y|^3) with a caller-   */
/* given normal and sign (sgn=+1: (x-y).n, sgn=-1: (y-x).n).                 */
/* ------------------------------------------------------------------------- */
static void chi(const double* P, double x1, double x2, double* out) {
    for (int d = 0; d < 3; ++d) out[d] = P[d] + x1 * (P[3 + d] - P[d]) + x2 * (P[6 + d] - P[3 + d]);
}

static double ss_kernel(int kernel, const double* x, const double* y, const double* nrm, double sgn) {
    if (kernel == OR_SLP) return kernel_slp(x, y);
    return sgn * kernel_dlp(x, y, nrm);
}

/* regions: fill up to 6 (x1,x2,y1,y2,jac) tuples for one (xi, e1, e2, e3). */
static int ss_regions(int type, double xi, double a, double b, double c, double out[6][5]) {
    if (type == OR_IDENTICAL) {
        double j = xi * xi * xi * a * a * b;
        double r[3][4] = {{xi, xi * (1.0 - a + a * b), xi * (1.0 - a * b * c), xi * (1.0 - a)},
                          {xi, xi * a * (1.0 - b + b * c), xi * (1.0 - a * b), xi * a * (1.0 - b)},
                          {xi * (1.0 - a * b * c), xi * a * (1.0 - b * c), xi, xi * a * (1.0 - b)}};
        for (int k = 0; k < 3; ++k) {
            out[2 * k][0] = r[k][0]; out[2 * k][1] = r[k][1];
            out[2 * k][2] = r[k][2]; out[2 * k][3] = r[k][3]; out[2 * k][4] = j;
            out[2 * k + 1][0] = r[k][2]; out[2 * k + 1][1] = r[k][3];
            out[2 * k + 1][2] = r[k][0]; out[2 * k + 1][3] = r[k][1]; out[2 * k + 1][4] = j;
        }
        return 6;
    }
    if (type == OR_EDGE) {
        double j1 = xi * xi * xi * a * a, j2 = j1 * b;
        double r[5][5] = {
            {xi, xi * a * c, xi * (1.0 - a * b), xi * a * (1.0 - b), j1},
            {xi, xi * a, xi * (1.0 - a * b * c), xi * a * b * (1.0 - c), j2},
            {xi * (1.0 - a * b), xi * a * (1.0 - b), xi, xi * a * b * c, j2},
            {xi * (1.0 - a * b * c), xi * a * b * (1.0 - c), xi, xi * a, j2},
            {xi * (1.0 - a * b * c), xi * a * (1.0 - b * c), xi, xi * a * b, j2}};
        memcpy(out, r, sizeof(r));
        return 5;
    }
    /* OR_VERTEX */
    double j = xi * xi * xi * b;
    out[0][0] = xi; out[0][1] = xi * a; out[0][2] = xi * b; out[0][3] = xi * b * c; out[0][4] = j;
    out[1][0] = xi * b; out[1][1] = xi * b * c; out[1][2] = xi; out[1][3] = xi * a; out[1][4] = j;
    return 2;
}

double or_ss_pair(int kernel, int type, const double* P, const double* Q, const double* nrm, double sgn,
                  int q) {
    double g[64], gw[64];
    if (or_gauss_legendre01(q, g, gw)) return NAN;
    double ap, np_[3], aq, nq[3];
    or_tri_geom(P, P + 3, P + 6, &ap, np_);
    or_tri_geom(Q, Q + 3, Q + 6, &aq, nq);
    /* the parametrisation chi uses (P1-P0, P2-P1); |det| = 2|tau| either way */
    double s = 0.0;
    for (int i0 = 0; i0 < q; ++i0)
        for (int i1 = 0; i1 < q; ++i1)
            for (int i2 = 0; i2 < q; ++i2)
                for (int i3 = 0; i3 < q; ++i3) {
                    double wt = gw[i0] * gw[i1] * gw[i2] * gw[i3];
                    double reg[6][5];
                    int nr = ss_regions(type, g[i0], g[i1], g[i2], g[i3], reg);
                    for (int r = 0; r < nr; ++r) {
                        double x[3], y[3];
                        chi(P, reg[r][0], reg[r][1], x);
                        chi(Q, reg[r][2], reg[r][3], y);
                        s += wt * reg[r][4] * ss_kernel(kernel, x, y, nrm, sgn);
                    }
                }
    return 4.0 * ap * aq * s;
}

/* Moment of x1^a x2^b y1^c y2^d over T x T computed through the same regions
 * and Jacobians as or_ss_pair (used to pin the region maps). */
double or_ss_moment(int type, int q, int a, int b, int c, int d) {
    double g[64], gw[64];
    if (or_gauss_legendre01(q, g, gw)) return NAN;
    double s = 0.0;
    for (int i0 = 0; i0 < q; ++i0)
        for (int i1 = 0; i1 < q; ++i1)
            for (int i2 = 0; i2 < q; ++i2)
                for (int i3 = 0; i3 < q; ++i3) {
                    double wt = gw[i0] * gw[i1] * gw[i2] * gw[i3];
                    double reg[6][5];
                    int nr = ss_regions(type, g[i0], g[i1], g[i2], g[i3], reg);
                    for (int r = 0; r < nr; ++r)
                        s += wt * reg[r][4] * pow(reg[r][0], a) * pow(reg[r][1], b) * pow(reg[r][2], c) *
                             pow(reg[r][3], d);
                }
    return s;
}

/* ------------------------------------------------------------------------- */
/* Pair classification from shared vertex indices and canonical orientation  */
/* ------------------------------------------------------------------------- */
int or_shared_vertices(const or_mesh* M, int64_t i, int64_t j) {
    int c = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (M->tri[3 * i + a] == M->tri[3 * j + b]) ++c;
    return c;
}

/* Orient a singular pair (lo, hi) (lo < hi, user numbering): the vertices of
 * the outer panel P = tau_lo and of the inner panel Q = tau_hi are listed so
 * that the shared vertices come first and in the same order.  Edge: P is the
 * cyclic rotation of tau_lo with its unshared vertex last, Q = (P0, P1, the
 * unshared vertex of tau_hi).  Vertex: both are the cyclic rotations that
 * start at the shared vertex. */
/* canonical vertex order of the pair (lo, hi): pv (outer panel), qv (inner) */
static void orient_ids(const or_mesh* M, int64_t lo, int64_t hi, int* type_out, int32_t* pv, int32_t* qv) {
    const int32_t* tl = M->tri + 3 * lo;
    const int32_t* th = M->tri + 3 * hi;
    int ns = or_shared_vertices(M, lo, hi);
    if (ns == 3) {
        *type_out = OR_IDENTICAL;
        for (int k = 0; k < 3; ++k) pv[k] = qv[k] = tl[k];
    } else if (ns == 2) {
        *type_out = OR_EDGE;
        int un = -1; /* unshared local vertex of tau_lo */
        for (int a = 0; a < 3; ++a) {
            int found = 0;
            for (int b = 0; b < 3; ++b) found |= (tl[a] == th[b]);
            if (!found) un = a;
        }
        pv[0] = tl[(un + 1) % 3];
        pv[1] = tl[(un + 2) % 3];
        pv[2] = tl[un];
        int32_t other = -1;
        for (int b = 0; b < 3; ++b)
            if (th[b] != pv[0] && th[b] != pv[1]) other = th[b];
        qv[0] = pv[0];
        qv[1] = pv[1];
        qv[2] = other;
    } else {
        *type_out = OR_VERTEX;
        int a0 = -1, b0 = -1;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (tl[a] == th[b]) { a0 = a; b0 = b; }
        for (int k = 0; k < 3; ++k) {
            pv[k] = tl[(a0 + k) % 3];
            qv[k] = th[(b0 + k) % 3];
        }
    }
}

void or_orient_pair(const or_mesh* M, int64_t lo, int64_t hi, int* type_out, double* P, double* Q) {
    int32_t pv[3], qv[3];
    orient_ids(M, lo, hi, type_out, pv, qv);
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) {
            P[3 * k + d] = M->xyz[3 * (int64_t)pv[k] + d];
            Q[3 * k + d] = M->xyz[3 * (int64_t)qv[k] + d];
        }
}

/* One Galerkin matrix entry a_ij (section 1, eq. (slp) / eq. (dlp)) with
 * psi_i = 1 on tau_i.  Pairs that share no vertex use the 7 x 7 rule; pairs
 * that share vertices use the Sauter-Schwab rule in the canonical orientation
 * (outer panel = lower user index), so that G is exactly symmetric and k_ij,
 * k_ji come from one point set.  The double-layer entry of a triangle with
 * itself vanishes (x - y lies in the plane of tau) and is set to 0. */
double or_entry(int kernel, const or_mesh* M, int64_t i, int64_t j, int q_ss) {
    int ns = or_shared_vertices(M, i, j);
    if (ns == 0) {
        double X[9], Y[9];
        tri_vertices(M, i, X);
        tri_vertices(M, j, Y);
        return or_pair_regular(kernel, X, Y);
    }
    if (i == j && kernel == OR_DLP) return 0.0;
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    double P[9], Q[9];
    int type;
    or_orient_pair(M, lo, hi, &type, P, Q);
    if (kernel == OR_SLP) return or_ss_pair(OR_SLP, type, P, Q, NULL, 1.0, q_ss);
    /* k_ij uses the normal of tau_j; x in tau_i, y in tau_j. */
    double aj, nj[3], Yj[9];
    tri_vertices(M, j, Yj);
    or_tri_geom(Yj, Yj + 3, Yj + 6, &aj, nj);
    /* outer panel points p in tau_lo, inner q in tau_hi.
     * i == lo: x = p, y = q -> (p - q).n_j  (sgn +1)
     * i == hi: x = q, y = p -> (q - p).n_j  (sgn -1) */
    return or_ss_pair(OR_DLP, type, P, Q, nj, i == lo ? 1.0 : -1.0, q_ss);
}

/* ------------------------------------------------------------------------- */
/* Double layer with continuous piecewise-linear trial functions (section 1,  */
/* eq. (dlp) with phi_j the hat functions of the vertices): on each pair of   */
/* triangles the trial function is the barycentric coordinate of one corner   */
/* of the source panel, so the pair contributes three values                  */
/*   int_tau int_sigma dg/dn_y(x, y) lambda_c(y) dy dx,  c = corners of sigma, */
/* with the quadrature of or_pair_regular / or_ss_pair and the factor          */
/* lambda_c(y) at the source points.                                           */
/* ------------------------------------------------------------------------- */

/* As or_ss_pair, with the barycentric coordinates of the point on panel
 * `side` (0: P, 1: Q) as factors: out[k], k = corner k of that panel in its
 * given order.  chi(x) = P0 + x1 (P1 - P0) + x2 (P2 - P1) gives
 * lambda = (1 - x1, x1 - x2, x2). */
void or_ss_pair3(int kernel, int type, const double* P, const double* Q, const double* nrm, double sgn, int q,
                 int side, double* out) {
    double g[64], gw[64];
    out[0] = out[1] = out[2] = 0.0;
    if (or_gauss_legendre01(q, g, gw)) {
        out[0] = out[1] = out[2] = NAN;
        return;
    }
    double ap, np_[3], aq, nq[3];
    or_tri_geom(P, P + 3, P + 6, &ap, np_);
    or_tri_geom(Q, Q + 3, Q + 6, &aq, nq);
    double s[3] = {0.0, 0.0, 0.0};
    for (int i0 = 0; i0 < q; ++i0)
        for (int i1 = 0; i1 < q; ++i1)
            for (int i2 = 0; i2 < q; ++i2)
                for (int i3 = 0; i3 < q; ++i3) {
                    double wt = gw[i0] * gw[i1] * gw[i2] * gw[i3];
                    double reg[6][5];
                    int nr = ss_regions(type, g[i0], g[i1], g[i2], g[i3], reg);
                    for (int r = 0; r < nr; ++r) {
                        double x[3], y[3];
                        chi(P, reg[r][0], reg[r][1], x);
                        chi(Q, reg[r][2], reg[r][3], y);
                        const double f = wt * reg[r][4] * ss_kernel(kernel, x, y, nrm, sgn);
                        const double z1 = reg[r][side ? 2 : 0], z2 = reg[r][side ? 3 : 1];
                        s[0] += f * (1.0 - z1);
                        s[1] += f * (z1 - z2);
                        s[2] += f * z2;
                    }
                }
    for (int k = 0; k < 3; ++k) out[k] = 4.0 * ap * aq * s[k];
}

/* out[c] = int_{tau_i} int_{tau_j} dg/dn_y(x, y) lambda_{j,c}(y) dy dx, c = 0, 1, 2
 * the corners of tau_j in the caller's order (n_y the normal of tau_j).  Pairs
 * sharing no vertex: the 7 x 7 rule (lambda = (1 - u - v, u, v) at the rule's
 * points); pairs sharing vertices: Sauter-Schwab in the canonical orientation
 * of or_entry; a triangle with itself: 0 (x - y lies in its plane). */
void or_entry_dlp_p1(const or_mesh* M, int64_t i, int64_t j, int q_ss, double* out) {
    out[0] = out[1] = out[2] = 0.0;
    int ns = or_shared_vertices(M, i, j);
    double Yj[9], aj, nj[3];
    tri_vertices(M, j, Yj);
    or_tri_geom(Yj, Yj + 3, Yj + 6, &aj, nj);
    if (ns == 0) {
        double X[9], ax, nx[3], uv[14], w[7];
        tri_vertices(M, i, X);
        or_tri_geom(X, X + 3, X + 6, &ax, nx);
        or_radon7(uv, w);
        double xp[7][3], yq[7][3];
        for (int p = 0; p < 7; ++p)
            for (int d = 0; d < 3; ++d) {
                xp[p][d] = X[d] + uv[2 * p] * (X[3 + d] - X[d]) + uv[2 * p + 1] * (X[6 + d] - X[d]);
                yq[p][d] = Yj[d] + uv[2 * p] * (Yj[3 + d] - Yj[d]) + uv[2 * p + 1] * (Yj[6 + d] - Yj[d]);
            }
        for (int p = 0; p < 7; ++p)
            for (int qq = 0; qq < 7; ++qq) {
                const double f = w[p] * w[qq] * kernel_dlp(xp[p], yq[qq], nj);
                const double u = uv[2 * qq], v = uv[2 * qq + 1];
                out[0] += f * (1.0 - u - v);
                out[1] += f * u;
                out[2] += f * v;
            }
        for (int c = 0; c < 3; ++c) out[c] *= ax * aj;
        return;
    }
    if (i == j) return;
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    int type;
    int32_t pv[3], qv[3];
    orient_ids(M, lo, hi, &type, pv, qv);
    double P[9], Q[9];
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) {
            P[3 * k + d] = M->xyz[3 * (int64_t)pv[k] + d];
            Q[3 * k + d] = M->xyz[3 * (int64_t)qv[k] + d];
        }
    /* the source panel is tau_j: Q (side 1) if i == lo, else P (side 0) */
    const int side = i == lo ? 1 : 0;
    double can[3];
    or_ss_pair3(OR_DLP, type, P, Q, nj, i == lo ? 1.0 : -1.0, q_ss, side, can);
    const int32_t* sv = side ? qv : pv;
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c)
            if (M->tri[3 * j + c] == sv[k]) out[c] += can[k];
}

/* The matrix K1 (nt x nv, row-major): K1[i, v] = sum over the triangles j at
 * vertex v of or_entry_dlp_p1(i, j)[corner of v in j]. */
void or_dense_dlp_p1(const or_mesh* M, int q_ss, double* A) {
    const int64_t n = M->nt, nv = M->nv;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        double* row = A + i * nv;
        for (int64_t v = 0; v < nv; ++v) row[v] = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double e[3];
            or_entry_dlp_p1(M, i, j, q_ss, e);
            for (int c = 0; c < 3; ++c) row[M->tri[3 * j + c]] += e[c];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Dense matrix-vector products (the plain definition)                       */
/* x, y column-major n x nrhs with leading dimension n.                      */
/* ------------------------------------------------------------------------- */
void or_dense_matvec(int kernel, const or_mesh* M, int q_ss, const double* x, int nrhs, double* y,
                     int transpose) {
    int64_t n = M->nt;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        double acc[64];
        for (int r = 0; r < nrhs; ++r) acc[r] = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double a = transpose ? or_entry(kernel, M, j, i, q_ss) : or_entry(kernel, M, i, j, q_ss);
            for (int r = 0; r < nrhs; ++r) acc[r] += a * x[j + r * n];
        }
        for (int r = 0; r < nrhs; ++r) y[i + r * n] = acc[r];
    }
}

void or_dense_rows(int kernel, const or_mesh* M, int q_ss, const int64_t* rows, int64_t nrows,
                   const double* x, int nrhs, double* y /* nrows x nrhs, col-major ld nrows */) {
    int64_t n = M->nt;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nrows; ++k) {
        int64_t i = rows[k];
        double acc[64];
        for (int r = 0; r < nrhs; ++r) acc[r] = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double a = or_entry(kernel, M, i, j, q_ss);
            for (int r = 0; r < nrhs; ++r) acc[r] += a * x[j + r * n];
        }
        for (int r = 0; r < nrhs; ++r) y[k + r * nrows] = acc[r];
    }
}

void or_dense_matrix(int kernel, const or_mesh* M, int q_ss, double* A /* n x n row-major */) {
    int64_t n = M->nt;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) A[i * n + j] = or_entry(kernel, M, i, j, q_ss);
}

/* ------------------------------------------------------------------------- */
/* Cluster tree (section 2, Definition "cluster tree"; boxes: section 3)     */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t n, cap, count;
    int64_t* perm;
    int64_t *begin, *end, *child0, *child1, *parent;
    int32_t* level;
    double *bmin, *bmax;
} tree_t;

static void tree_box(const or_mesh* M, const int64_t* idx, int64_t cnt, double* lo, double* hi) {
    for (int d = 0; d < 3; ++d) { lo[d] = INFINITY; hi[d] = -INFINITY; }
    for (int64_t a = 0; a < cnt; ++a)
        for (int k = 0; k < 3; ++k) {
            const double* v = M->xyz + 3 * (int64_t)M->tri[3 * idx[a] + k];
            for (int d = 0; d < 3; ++d) {
                if (v[d] < lo[d]) lo[d] = v[d];
                if (v[d] > hi[d]) hi[d] = v[d];
            }
        }
}

static double centroid_coord(const or_mesh* M, int64_t t, int d) {
    const int32_t* tv = M->tri + 3 * t;
    return ((M->xyz[3 * (int64_t)tv[0] + d] + M->xyz[3 * (int64_t)tv[1] + d]) + M->xyz[3 * (int64_t)tv[2] + d]) /
           3.0;
}

typedef struct { double key; int64_t pos; int64_t id; } sort_item;
static int cmp_item(const void* a, const void* b) {
    const sort_item* x = a;
    const sort_item* y = b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->pos > y->pos) - (x->pos < y->pos);
}

static int64_t tree_new(tree_t* T) {
    if (T->count == T->cap) {
        T->cap = T->cap ? 2 * T->cap : 1024;
        T->begin = realloc(T->begin, T->cap * sizeof(int64_t));
        T->end = realloc(T->end, T->cap * sizeof(int64_t));
        T->child0 = realloc(T->child0, T->cap * sizeof(int64_t));
        T->child1 = realloc(T->child1, T->cap * sizeof(int64_t));
        T->parent = realloc(T->parent, T->cap * sizeof(int64_t));
        T->level = realloc(T->level, T->cap * sizeof(int32_t));
        T->bmin = realloc(T->bmin, 3 * T->cap * sizeof(double));
        T->bmax = realloc(T->bmax, 3 * T->cap * sizeof(double));
    }
    return T->count++;
}

static int64_t tree_split(const or_mesh* M, tree_t* T, int64_t b, int64_t e, int64_t parent, int level,
                          int leaf, int64_t* tmp) {
    int64_t c = tree_new(T);
    T->begin[c] = b;
    T->end[c] = e;
    T->parent[c] = parent;
    T->level[c] = level;
    T->child0[c] = T->child1[c] = -1;
    tree_box(M, T->perm + b, e - b, T->bmin + 3 * c, T->bmax + 3 * c);
    if (e - b <= leaf) return c;
    const double* lo = T->bmin + 3 * c;
    const double* hi = T->bmax + 3 * c;
    int axis = 0;
    for (int d = 1; d < 3; ++d)
        if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
    double mid = 0.5 * (lo[axis] + hi[axis]);
    int64_t n0 = 0;
    for (int64_t a = b; a < e; ++a)
        if (centroid_coord(M, T->perm[a], axis) < mid) ++n0;
    int64_t split;
    if (n0 == 0 || n0 == e - b) {
        /* stable median split */
        sort_item* it = malloc((e - b) * sizeof(sort_item));
        for (int64_t a = b; a < e; ++a) {
            it[a - b].key = centroid_coord(M, T->perm[a], axis);
            it[a - b].pos = a;
            it[a - b].id = T->perm[a];
        }
        qsort(it, e - b, sizeof(sort_item), cmp_item);
        for (int64_t a = b; a < e; ++a) T->perm[a] = it[a - b].id;
        free(it);
        split = b + (e - b) / 2;
    } else {
        int64_t k0 = 0, k1 = 0;
        for (int64_t a = b; a < e; ++a) {
            int64_t t = T->perm[a];
            if (centroid_coord(M, t, axis) < mid) T->perm[b + k0++] = t;
            else tmp[k1++] = t;
        }
        for (int64_t a = 0; a < k1; ++a) T->perm[b + n0 + a] = tmp[a];
        split = b + n0;
    }
    int64_t c0 = tree_split(M, T, b, split, c, level + 1, leaf, tmp);
    int64_t c1 = tree_split(M, T, split, e, c, level + 1, leaf, tmp);
    T->child0[c] = c0;
    T->child1[c] = c1;
    return c;
}

/* ------------------------------------------------------------------------- */
/* Block tree (section 2, Definition "block tree"; eq. (admissibility) with  */
/* max(diam B_t, diam B_s) <= eta dist(B_t, B_s), dist > 0).                 */
/* ------------------------------------------------------------------------- */
typedef struct { int64_t* t; int64_t* s; int64_t n, cap; } blist;
static void blist_push(blist* L, int64_t t, int64_t s) {
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 1024;
        L->t = realloc(L->t, L->cap * sizeof(int64_t));
        L->s = realloc(L->s, L->cap * sizeof(int64_t));
    }
    L->t[L->n] = t;
    L->s[L->n] = s;
    L->n++;
}

static double box_diam(const double* lo, const double* hi) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) s += (hi[d] - lo[d]) * (hi[d] - lo[d]);
    return sqrt(s);
}
static double box_dist(const double* lo1, const double* hi1, const double* lo2, const double* hi2) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
        double g = 0.0;
        if (lo2[d] > hi1[d]) g = lo2[d] - hi1[d];
        else if (lo1[d] > hi2[d]) g = lo1[d] - hi2[d];
        s += g * g;
    }
    return sqrt(s);
}

static void block_build(const tree_t* T, double eta, int64_t t, int64_t s, blist* far, blist* near) {
    const double *lt = T->bmin + 3 * t, *ht = T->bmax + 3 * t, *ls = T->bmin + 3 * s, *hs = T->bmax + 3 * s;
    double dt = box_diam(lt, ht), ds = box_diam(ls, hs), dist = box_dist(lt, ht, ls, hs);
    double dm = dt > ds ? dt : ds;
    if (dist > 0.0 && dm <= eta * dist) {
        blist_push(far, t, s);
        return;
    }
    int tl = T->child0[t] < 0, sl = T->child0[s] < 0;
    if (tl && sl) {
        blist_push(near, t, s);
        return;
    }
    if (tl) {
        block_build(T, eta, t, T->child0[s], far, near);
        block_build(T, eta, t, T->child1[s], far, near);
    } else if (sl) {
        block_build(T, eta, T->child0[t], s, far, near);
        block_build(T, eta, T->child1[t], s, far, near);
    } else {
        block_build(T, eta, T->child0[t], T->child0[s], far, near);
        block_build(T, eta, T->child0[t], T->child1[s], far, near);
        block_build(T, eta, T->child1[t], T->child0[s], far, near);
        block_build(T, eta, T->child1[t], T->child1[s], far, near);
    }
}

/* ------------------------------------------------------------------------- */
/* Tensor Chebyshev interpolation (section 3)                                */
/* ------------------------------------------------------------------------- */
/* 1-D Lagrange polynomial L_nu on the nodes z[0..m-1], and its derivative. */
static double lagrange(const double* z, int m, int nu, double x) {
    double p = 1.0;
    for (int k = 0; k < m; ++k)
        if (k != nu) p *= (x - z[k]) / (z[nu] - z[k]);
    return p;
}
static double lagrange_deriv(const double* z, int m, int nu, double x) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) {
        if (k == nu) continue;
        double p = 1.0 / (z[nu] - z[k]);
        for (int l = 0; l < m; ++l)
            if (l != nu && l != k) p *= (x - z[l]) / (z[nu] - z[l]);
        s += p;
    }
    return s;
}

struct or_h2 {
    or_mesh mesh;
    double* xyz;
    int32_t* tri;
    int kernel, m, k, q_ss, qb;
    double eta;
    tree_t T;
    blist far, near;
    /* per cluster: Chebyshev nodes per axis, m per axis: nodes[c*3*m + d*m + a] */
    double* nodes;
    /* per leaf cluster c: V (|c| x k row-major), W (|c| x k) */
    double** V;
    double** W;
    /* per non-root cluster c: E_c (k x k row-major, E[nu' * k + nu]) */
    double** E;
    /* CSR of farfield/nearfield blocks by row cluster */
    int64_t *far_ptr, *far_col, *near_ptr, *near_col;
    int64_t *far_ptr_t, *far_row_t; /* by column cluster (transpose) */
    int64_t *near_ptr_t, *near_row_t;
};

static void cluster_nodes(const double* lo, const double* hi, int m, double* z /* 3*m */) {
    double c[3], h[3], hmax = 0.0;
    for (int d = 0; d < 3; ++d) {
        c[d] = 0.5 * (lo[d] + hi[d]);
        h[d] = 0.5 * (hi[d] - lo[d]);
        if (h[d] > hmax) hmax = h[d];
    }
    for (int d = 0; d < 3; ++d) {
        double hd = h[d] < 1e-2 * hmax ? 1e-2 * hmax : h[d];
        for (int a = 0; a < m; ++a) z[d * m + a] = c[d] + hd * cos((2.0 * a + 1.0) * OR_PI / (2.0 * m));
    }
}

/* L_{t,nu}(x) for the tensor index nu = a + m (b + m c). */
static double tensor_lagrange(const double* z, int m, int nu, const double* x) {
    int a = nu % m, b = (nu / m) % m, c = nu / (m * m);
    return lagrange(z, m, a, x[0]) * lagrange(z + m, m, b, x[1]) * lagrange(z + 2 * m, m, c, x[2]);
}
static void tensor_lagrange_grad(const double* z, int m, int nu, const double* x, double* g) {
    int a = nu % m, b = (nu / m) % m, c = nu / (m * m);
    double la = lagrange(z, m, a, x[0]), lb = lagrange(z + m, m, b, x[1]), lc = lagrange(z + 2 * m, m, c, x[2]);
    g[0] = lagrange_deriv(z, m, a, x[0]) * lb * lc;
    g[1] = la * lagrange_deriv(z + m, m, b, x[1]) * lc;
    g[2] = la * lb * lagrange_deriv(z + 2 * m, m, c, x[2]);
}

/* second derivative of the 1-D Lagrange polynomial: the sum over ordered
 * pairs k != l (both != nu) of the product with factors (x - z_o) / (z_nu -
 * z_o) for the other nodes o and 1 / (z_nu - z_k), 1 / (z_nu - z_l) */
static double lagrange_deriv2(const double* z, int m, int nu, double x) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) {
        if (k == nu) continue;
        for (int l = 0; l < m; ++l) {
            if (l == nu || l == k) continue;
            double p = 1.0 / ((z[nu] - z[k]) * (z[nu] - z[l]));
            for (int o = 0; o < m; ++o)
                if (o != nu && o != k && o != l) p *= (x - z[o]) / (z[nu] - z[o]);
            s += p;
        }
    }
    return s;
}
/* Hessian of L_{t,nu} at x: h[3 d + e] = d^2 L / dx_d dx_e */
static void tensor_lagrange_hess(const double* z, int m, int nu, const double* x, double* h) {
    const int a[3] = {nu % m, (nu / m) % m, nu / (m * m)};
    double l0[3], l1[3], l2[3];
    for (int d = 0; d < 3; ++d) {
        l0[d] = lagrange(z + d * m, m, a[d], x[d]);
        l1[d] = lagrange_deriv(z + d * m, m, a[d], x[d]);
        l2[d] = lagrange_deriv2(z + d * m, m, a[d], x[d]);
    }
    for (int d = 0; d < 3; ++d)
        for (int e = 0; e < 3; ++e) {
            double v = 1.0;
            for (int f = 0; f < 3; ++f) {
                if (d == e) v *= f == d ? l2[f] : l0[f];
                else v *= (f == d || f == e) ? l1[f] : l0[f];
            }
            h[3 * d + e] = v;
        }
}

static int64_t* csr_from(int64_t nrows, const int64_t* key, const int64_t* val, int64_t n, int64_t** col_out) {
    int64_t* ptr = calloc(nrows + 1, sizeof(int64_t));
    for (int64_t b = 0; b < n; ++b) ptr[key[b] + 1]++;
    for (int64_t r = 0; r < nrows; ++r) ptr[r + 1] += ptr[r];
    int64_t* fill = malloc(nrows * sizeof(int64_t));
    memcpy(fill, ptr, nrows * sizeof(int64_t));
    int64_t* col = malloc((n ? n : 1) * sizeof(int64_t));
    for (int64_t b = 0; b < n; ++b) col[fill[key[b]]++] = val[b];
    free(fill);
    *col_out = col;
    return ptr;
}

/* Geometry-dependent parts of the H^2 approximation for the current vertex
 * positions, with the cluster tree and the block lists unchanged: cluster
 * boxes, interpolation nodes, leaf bases and transfer matrices. */
static void h2_geometry(or_h2* H) {
    tree_t* T = &H->T;
    int64_t nc = T->count;
    int m = H->m;
    int kernel = H->kernel;
    for (int64_t c = 0; c < nc; ++c)
        tree_box(&H->mesh, T->perm + T->begin[c], T->end[c] - T->begin[c], T->bmin + 3 * c, T->bmax + 3 * c);
    free(H->nodes);
    if (H->V)
        for (int64_t c = 0; c < nc; ++c) {
            if (H->W[c] && H->W[c] != H->V[c]) free(H->W[c]);
            free(H->V[c]);
        }
    if (H->E)
        for (int64_t c = 0; c < nc; ++c) free(H->E[c]);
    free(H->V);
    free(H->W);
    free(H->E);
    /* interpolation nodes */
    H->nodes = malloc(nc * 3 * m * sizeof(double));
    for (int64_t c = 0; c < nc; ++c) cluster_nodes(T->bmin + 3 * c, T->bmax + 3 * c, m, H->nodes + c * 3 * m);
    /* leaf bases V_t[i,nu] = int_{tau_i} L_{t,nu};  W_s = V_s (SLP) or
     * W_s[j,mu] = int_{tau_j} n_j . grad L_{s,mu} (DLP) */
    H->V = calloc(nc, sizeof(double*));
    H->W = calloc(nc, sizeof(double*));
    double ruv[2 * 64 * 64], rw[64 * 64];
    int np = or_collapsed_rule(H->qb, ruv, rw);
    int k = H->k;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] >= 0) continue;
        int64_t sz = T->end[c] - T->begin[c];
        double* V = calloc(sz * k, sizeof(double));
        double* W = kernel == OR_DLP ? calloc(sz * k, sizeof(double)) : V; /* W_s = V_s */
        const double* z = H->nodes + c * 3 * m;
        for (int64_t a = 0; a < sz; ++a) {
            double X[9], area, nrm[3];
            tri_vertices(&H->mesh, T->perm[T->begin[c] + a], X);
            or_tri_geom(X, X + 3, X + 6, &area, nrm);
            for (int p = 0; p < np; ++p) {
                double x[3];
                for (int d = 0; d < 3; ++d)
                    x[d] = X[d] + ruv[2 * p] * (X[3 + d] - X[d]) + ruv[2 * p + 1] * (X[6 + d] - X[d]);
                for (int nu = 0; nu < k; ++nu) {
                    V[a * k + nu] += area * rw[p] * tensor_lagrange(z, m, nu, x);
                    if (kernel == OR_DLP) {
                        double g[3];
                        tensor_lagrange_grad(z, m, nu, x, g);
                        W[a * k + nu] += area * rw[p] * dot3(nrm, g);
                    }
                }
            }
        }
        H->V[c] = V;
        H->W[c] = W;
    }
    /* transfer matrices E_{t'}[nu', nu] = L_{t,nu}(xi_{t',nu'}), t = parent */
    H->E = calloc(nc, sizeof(double*));
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t c = 1; c < nc; ++c) {
        int64_t p = T->parent[c];
        double* E = malloc((size_t)k * k * sizeof(double));
        const double* zc = H->nodes + c * 3 * m;
        const double* zp = H->nodes + p * 3 * m;
        for (int nup = 0; nup < k; ++nup) {
            double xi[3] = {zc[nup % m], zc[m + (nup / m) % m], zc[2 * m + nup / (m * m)]};
            for (int nu = 0; nu < k; ++nu) E[nup * k + nu] = tensor_lagrange(zp, m, nu, xi);
        }
        H->E[c] = E;
    }
}

or_h2* or_h2_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, int kernel, int m, double eta,
                    int leaf, int q_ss) {
    if (m < 1 || m > 10 || leaf < 1 || nt < 1) return NULL;
    or_h2* H = calloc(1, sizeof(or_h2));
    H->xyz = malloc(3 * nv * sizeof(double));
    H->tri = malloc(3 * nt * sizeof(int32_t));
    memcpy(H->xyz, xyz, 3 * nv * sizeof(double));
    memcpy(H->tri, tri, 3 * nt * sizeof(int32_t));
    H->mesh.xyz = H->xyz;
    H->mesh.tri = H->tri;
    H->mesh.nv = nv;
    H->mesh.nt = nt;
    H->kernel = kernel;
    H->m = m;
    H->k = m * m * m;
    H->eta = eta;
    H->q_ss = q_ss;
    /* basis rule exact for total degree 3(m-1): collapsed Gauss, qb points */
    H->qb = (3 * (m - 1) + 2 + 1) / 2;
    if (H->qb < 1) H->qb = 1;
    /* cluster tree */
    tree_t* T = &H->T;
    T->n = nt;
    T->perm = malloc(nt * sizeof(int64_t));
    for (int64_t i = 0; i < nt; ++i) T->perm[i] = i;
    int64_t* tmp = malloc(nt * sizeof(int64_t));
    tree_split(&H->mesh, T, 0, nt, -1, 0, leaf, tmp);
    free(tmp);
    /* block tree */
    block_build(T, eta, 0, 0, &H->far, &H->near);
    int64_t nc = T->count;
    H->far_ptr = csr_from(nc, H->far.t, H->far.s, H->far.n, &H->far_col);
    H->near_ptr = csr_from(nc, H->near.t, H->near.s, H->near.n, &H->near_col);
    H->far_ptr_t = csr_from(nc, H->far.s, H->far.t, H->far.n, &H->far_row_t);
    H->near_ptr_t = csr_from(nc, H->near.s, H->near.t, H->near.n, &H->near_row_t);
    h2_geometry(H);
    return H;
}

void or_h2_destroy(or_h2* H) {
    if (!H) return;
    tree_t* T = &H->T;
    for (int64_t c = 0; c < T->count; ++c) {
        if (H->W && H->W[c] && H->W[c] != H->V[c]) free(H->W[c]);
        if (H->V) free(H->V[c]);
        if (H->E) free(H->E[c]);
    }
    free(H->V); free(H->W); free(H->E); free(H->nodes);
    free(H->far_ptr); free(H->far_col); free(H->near_ptr); free(H->near_col);
    free(H->far_ptr_t); free(H->far_row_t); free(H->near_ptr_t); free(H->near_row_t);
    free(H->far.t); free(H->far.s); free(H->near.t); free(H->near.s);
    free(T->perm); free(T->begin); free(T->end); free(T->child0); free(T->child1); free(T->parent);
    free(T->level); free(T->bmin); free(T->bmax);
    free(H->xyz); free(H->tri);
    free(H);
}

/* ------------------------------------------------------------------------- */
/* Introspection                                                             */
/* ------------------------------------------------------------------------- */
void or_h2_sizes(const or_h2* H, int64_t* out /* 6 */) {
    out[0] = H->T.count;
    out[1] = H->far.n;
    out[2] = H->near.n;
    out[3] = H->k;
    int64_t leaves = 0;
    for (int64_t c = 0; c < H->T.count; ++c) leaves += H->T.child0[c] < 0;
    out[4] = leaves;
    out[5] = H->qb;
}
void or_h2_tree(const or_h2* H, int64_t* perm, int64_t* begin, int64_t* end, int64_t* child0, int64_t* child1,
                double* bmin, double* bmax) {
    const tree_t* T = &H->T;
    memcpy(perm, T->perm, T->n * sizeof(int64_t));
    memcpy(begin, T->begin, T->count * sizeof(int64_t));
    memcpy(end, T->end, T->count * sizeof(int64_t));
    memcpy(child0, T->child0, T->count * sizeof(int64_t));
    memcpy(child1, T->child1, T->count * sizeof(int64_t));
    memcpy(bmin, T->bmin, 3 * T->count * sizeof(double));
    memcpy(bmax, T->bmax, 3 * T->count * sizeof(double));
}
void or_h2_blocks(const or_h2* H, int64_t* far_t, int64_t* far_s, int64_t* near_t, int64_t* near_s) {
    memcpy(far_t, H->far.t, H->far.n * sizeof(int64_t));
    memcpy(far_s, H->far.s, H->far.n * sizeof(int64_t));
    memcpy(near_t, H->near.t, H->near.n * sizeof(int64_t));
    memcpy(near_s, H->near.s, H->near.n * sizeof(int64_t));
}
/* V_t, W_t of a leaf (|t| x k) and E_c (k x k) */
int or_h2_leaf_basis(const or_h2* H, int64_t c, double* V, double* W) {
    if (c < 0 || c >= H->T.count || H->T.child0[c] >= 0) return -1;
    int64_t sz = (H->T.end[c] - H->T.begin[c]) * H->k;
    memcpy(V, H->V[c], sz * sizeof(double));
    memcpy(W, H->W[c], sz * sizeof(double));
    return 0;
}
int or_h2_transfer(const or_h2* H, int64_t c, double* E) {
    if (c <= 0 || c >= H->T.count) return -1;
    memcpy(E, H->E[c], (size_t)H->k * H->k * sizeof(double));
    return 0;
}
void or_h2_nodes(const or_h2* H, double* nodes) { memcpy(nodes, H->nodes, H->T.count * 3 * H->m * sizeof(double)); }

/* ------------------------------------------------------------------------- */
/* H^2 matrix-vector product (section 2, eq. (vsw), eq. (transfer))          */
/*   forward:   xh_s = W_s^T x|_s (leaves),  xh_t = sum_{t'} E_{t'}^T xh_{t'} */
/*   coupling:  yh_t = sum_{(t,s) farfield} S_ts xh_s,                        */
/*              S_ts[nu,mu] = g(xi_{t,nu}, xi_{s,mu})                         */
/*   backward:  yh_{t'} += E_{t'} yh_t,  y|_t += V_t yh_t (leaves)            */
/*   nearfield: y|_t += A|_{t x s} x|_s                                       */
/* transpose != 0 computes y = A^T x with the roles of V and W, rows and      */
/* columns exchanged.                                                         */
/* x, y column-major n x nrhs (ld n), user triangle order.                   */
/* ------------------------------------------------------------------------- */
/* Test kernel P(x) Q(y), degree 3 in each coordinate of x and of y; with
 * m >= 4 tensor interpolation reproduces it exactly, so the H^2 farfield of
 * this kernel is exact and pins the tree, blocks, bases and passes. */
double or_test_poly_P(const double* x) {
    return (1.0 + x[0] - 2.0 * x[0] * x[0] * x[0]) * (2.0 - x[1] + x[1] * x[1]) * (0.5 + x[2] * x[2] * x[2] - 3.0 * x[2]);
}
double or_test_poly_Q(const double* y) {
    return (y[0] * y[0] * y[0] - y[0] + 0.25) * (1.0 + y[1] * y[1]) * (2.0 + y[2] - y[2] * y[2]);
}
static double test_poly_kernel(const double* x, const double* y) { return or_test_poly_P(x) * or_test_poly_Q(y); }

static void coupling_matrix(const or_h2* H, int64_t t, int64_t s, double* S) {
    int m = H->m, k = H->k;
    const double* zt = H->nodes + t * 3 * m;
    const double* zs = H->nodes + s * 3 * m;
    for (int nu = 0; nu < k; ++nu) {
        double xt[3] = {zt[nu % m], zt[m + (nu / m) % m], zt[2 * m + nu / (m * m)]};
        for (int mu = 0; mu < k; ++mu) {
            double xs[3] = {zs[mu % m], zs[m + (mu / m) % m], zs[2 * m + mu / (m * m)]};
            S[nu * k + mu] = H->kernel == OR_TEST_POLY ? test_poly_kernel(xt, xs) : kernel_slp(xt, xs);
        }
    }
}

/* The passes between the leaf transformations (section 2, eq. (vsw) and
 * eq. (transfer)): upward x-hat_t += E_t'^T x-hat_t', coupling y-hat_t +=
 * S_ts x-hat_s over the farfield blocks (S_st^T for the transpose), downward
 * y-hat_t' += E_t' y-hat_t.  xh, yh: [nc][k][nrhs], yh zero on entry. */
static void h2_far_passes(const or_h2* H, double* xh, double* yh, int nrhs, int transpose) {
    const tree_t* T = &H->T;
    int64_t nc = T->count;
    int k = H->k;
    /* upward pass: children carry larger DFS numbers than their parents */
    for (int64_t c = nc - 1; c >= 0; --c) {
        if (T->child0[c] < 0) continue;
        int64_t ch[2] = {T->child0[c], T->child1[c]};
        for (int q = 0; q < 2; ++q) {
            const double* E = H->E[ch[q]];
            for (int nu = 0; nu < k; ++nu)
                for (int r = 0; r < nrhs; ++r) {
                    double s = 0.0;
                    for (int nup = 0; nup < k; ++nup) s += E[nup * k + nu] * xh[(ch[q] * k + nup) * nrhs + r];
                    xh[(c * k + nu) * nrhs + r] += s;
                }
        }
    }
    /* coupling */
    const int64_t* ptr = transpose ? H->far_ptr_t : H->far_ptr;
    const int64_t* col = transpose ? H->far_row_t : H->far_col;
#pragma omp parallel
    {
        double* S = malloc((size_t)k * k * sizeof(double));
#pragma omp for schedule(dynamic, 4)
        for (int64_t t = 0; t < nc; ++t) {
            for (int64_t b = ptr[t]; b < ptr[t + 1]; ++b) {
                int64_t s = col[b];
                if (!transpose) coupling_matrix(H, t, s, S);  /* S_ts */
                else coupling_matrix(H, s, t, S);             /* S_st, used transposed */
                for (int nu = 0; nu < k; ++nu)
                    for (int r = 0; r < nrhs; ++r) {
                        double acc = 0.0;
                        for (int mu = 0; mu < k; ++mu) {
                            double smu = transpose ? S[mu * k + nu] : S[nu * k + mu];
                            acc += smu * xh[(s * k + mu) * nrhs + r];
                        }
                        yh[(t * k + nu) * nrhs + r] += acc;
                    }
            }
        }
        free(S);
    }
    /* downward pass */
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] < 0) continue;
        int64_t ch[2] = {T->child0[c], T->child1[c]};
        for (int q = 0; q < 2; ++q) {
            const double* E = H->E[ch[q]];
            for (int nup = 0; nup < k; ++nup)
                for (int r = 0; r < nrhs; ++r) {
                    double s = 0.0;
                    for (int nu = 0; nu < k; ++nu) s += E[nup * k + nu] * yh[(c * k + nu) * nrhs + r];
                    yh[(ch[q] * k + nup) * nrhs + r] += s;
                }
        }
    }
}

void or_h2_matvec(const or_h2* H, const double* x, int nrhs, double* y, int transpose, int parts) {
    const tree_t* T = &H->T;
    int64_t n = T->n, nc = T->count;
    int k = H->k;
    double* xh = calloc((size_t)nc * k * nrhs, sizeof(double)); /* xh[c][nu][r] */
    double* yh = calloc((size_t)nc * k * nrhs, sizeof(double));
    double** Bin = transpose ? H->V : H->W;   /* basis applied to the input  */
    double** Bout = transpose ? H->W : H->V;  /* basis applied to the output */
    /* forward transformation at the leaves */
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] >= 0) continue;
        int64_t b = T->begin[c], sz = T->end[c] - b;
        for (int nu = 0; nu < k; ++nu)
            for (int r = 0; r < nrhs; ++r) {
                double s = 0.0;
                for (int64_t a = 0; a < sz; ++a) s += Bin[c][a * k + nu] * x[T->perm[b + a] + r * n];
                xh[(c * k + nu) * nrhs + r] = s;
            }
    }
    h2_far_passes(H, xh, yh, nrhs, transpose);
    for (int64_t i = 0; i < n * nrhs; ++i) y[i] = 0.0;
    /* backward transformation at the leaves, then the nearfield */
    const int64_t* nptr = transpose ? H->near_ptr_t : H->near_ptr;
    const int64_t* ncol = transpose ? H->near_row_t : H->near_col;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] >= 0) continue;
        int64_t b = T->begin[c], sz = T->end[c] - b;
        for (int64_t a = 0; a < sz && (parts & OR_PART_FAR); ++a) {
            int64_t i = T->perm[b + a];
            for (int r = 0; r < nrhs; ++r) {
                double s = 0.0;
                for (int nu = 0; nu < k; ++nu) s += Bout[c][a * k + nu] * yh[(c * k + nu) * nrhs + r];
                y[i + r * n] += s;
            }
        }
        for (int64_t q = nptr[c]; q < nptr[c + 1] && (parts & OR_PART_NEAR); ++q) {
            int64_t s = ncol[q];
            for (int64_t a = 0; a < sz; ++a) {
                int64_t i = T->perm[b + a];
                for (int64_t bb = T->begin[s]; bb < T->end[s]; ++bb) {
                    int64_t j = T->perm[bb];
                    double e = transpose ? or_entry(H->kernel, &H->mesh, j, i, H->q_ss)
                                         : or_entry(H->kernel, &H->mesh, i, j, H->q_ss);
                    for (int r = 0; r < nrhs; ++r) y[i + r * n] += e * x[j + r * n];
                }
            }
        }
    }
    free(xh);
    free(yh);
}

/* K1 x and K1^T x: the double layer with piecewise-linear trial functions
 * (section 1, eq. (dlp), phi_j the hat functions) in the same H^2 form.  The
 * vertex side takes the per-corner basis
 *   W1_s[a, c, mu] = int_{tau_a} n_a . grad L_{s,mu}(y) lambda_c(y) dy
 * (the collapsed rule of the leaf bases, lambda = (1 - u - v, u, v) at its
 * points; the integrand's degree 3(m-1) is within the rule's exactness); the
 * triangle side takes V; the passes are those of or_h2_matvec (transposed for
 * K1^T); the nearfield uses or_entry_dlp_p1.
 *   forward:   x nv x nrhs, y nt x nrhs;   transpose: x nt x nrhs, y nv x nrhs
 * (column-major). */
static void leaf_w1(const or_h2* H, int64_t j, const double* z, double* W1 /* 3 x k */) {
    int k = H->k, m = H->m;
    double ruv[2 * 64 * 64], rw[64 * 64];
    int np = or_collapsed_rule(H->qb, ruv, rw);
    double X[9], area, nrm[3];
    tri_vertices(&H->mesh, j, X);
    or_tri_geom(X, X + 3, X + 6, &area, nrm);
    for (int e = 0; e < 3 * k; ++e) W1[e] = 0.0;
    for (int p = 0; p < np; ++p) {
        const double u = ruv[2 * p], v = ruv[2 * p + 1];
        const double lam[3] = {1.0 - u - v, u, v};
        double xq[3], g[3];
        for (int d = 0; d < 3; ++d) xq[d] = X[d] + u * (X[3 + d] - X[d]) + v * (X[6 + d] - X[d]);
        for (int mu = 0; mu < k; ++mu) {
            tensor_lagrange_grad(z, m, mu, xq, g);
            const double f = area * rw[p] * dot3(nrm, g);
            for (int cc = 0; cc < 3; ++cc) W1[cc * k + mu] += f * lam[cc];
        }
    }
}

void or_h2_matvec_dlp_p1(const or_h2* H, const double* x, int nrhs, double* y, int transpose, int parts) {
    const tree_t* T = &H->T;
    int64_t n = T->n, nc = T->count, nv = H->mesh.nv;
    int k = H->k, m = H->m;
    const int64_t nin = transpose ? n : nv, nout = transpose ? nv : n;
    double* xh = calloc((size_t)nc * k * nrhs, sizeof(double));
    double* yh = calloc((size_t)nc * k * nrhs, sizeof(double));
    /* input side at the leaves */
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] >= 0) continue;
        const double* z = H->nodes + c * 3 * m;
        int64_t b = T->begin[c], sz = T->end[c] - b;
        double* W1 = malloc((size_t)3 * k * sizeof(double));
        for (int64_t a = 0; a < sz; ++a) {
            const int64_t j = T->perm[b + a];
            if (transpose) {
                for (int mu = 0; mu < k; ++mu)
                    for (int r = 0; r < nrhs; ++r) xh[(c * k + mu) * nrhs + r] += H->V[c][a * k + mu] * x[j + r * nin];
                continue;
            }
            leaf_w1(H, j, z, W1);
            for (int cc = 0; cc < 3; ++cc) {
                const int64_t vtx = H->mesh.tri[3 * j + cc];
                for (int mu = 0; mu < k; ++mu)
                    for (int r = 0; r < nrhs; ++r) xh[(c * k + mu) * nrhs + r] += W1[cc * k + mu] * x[vtx + r * nin];
            }
        }
        free(W1);
    }
    h2_far_passes(H, xh, yh, nrhs, transpose);
    for (int64_t i = 0; i < nout * nrhs; ++i) y[i] = 0.0;
    /* output side and nearfield, one leaf at a time (vertex rows of different
     * leaves may coincide, so the transpose runs serially) */
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] >= 0) continue;
        const double* z = H->nodes + c * 3 * m;
        int64_t b = T->begin[c], sz = T->end[c] - b;
        double W1[3 * 216];
        for (int64_t a = 0; a < sz && (parts & OR_PART_FAR); ++a) {
            int64_t i = T->perm[b + a];
            if (!transpose) {
                for (int r = 0; r < nrhs; ++r) {
                    double s = 0.0;
                    for (int nu = 0; nu < k; ++nu) s += H->V[c][a * k + nu] * yh[(c * k + nu) * nrhs + r];
                    y[i + r * nout] += s;
                }
            } else {
                leaf_w1(H, i, z, W1);
                for (int cc = 0; cc < 3; ++cc) {
                    const int64_t vtx = H->mesh.tri[3 * i + cc];
                    for (int r = 0; r < nrhs; ++r) {
                        double s = 0.0;
                        for (int nu = 0; nu < k; ++nu) s += W1[cc * k + nu] * yh[(c * k + nu) * nrhs + r];
                        y[vtx + r * nout] += s;
                    }
                }
            }
        }
        for (int64_t q = H->near_ptr[c]; q < H->near_ptr[c + 1] && (parts & OR_PART_NEAR); ++q) {
            int64_t s = H->near_col[q];
            for (int64_t a = 0; a < sz; ++a) {
                int64_t i = T->perm[b + a];
                for (int64_t bb = T->begin[s]; bb < T->end[s]; ++bb) {
                    int64_t j = T->perm[bb];
                    double e[3];
                    or_entry_dlp_p1(&H->mesh, i, j, H->q_ss, e);
                    for (int cc = 0; cc < 3; ++cc) {
                        const int64_t vtx = H->mesh.tri[3 * j + cc];
                        for (int r = 0; r < nrhs; ++r) {
                            if (!transpose) y[i + r * nout] += e[cc] * x[vtx + r * nin];
                            else y[vtx + r * nout] += e[cc] * x[i + r * nin];
                        }
                    }
                }
            }
        }
    }
    free(xh);
    free(yh);
}

/* Selected rows of the H^2 product, one by one (forward only).  The forward
 * transformation and the upward pass run in full; then row i in leaf t sums
 * v S_as xh_s over the farfield blocks (a, s) of t and its ancestors a, with
 * the row vector v = V_t[i,:] E_t E_parent(t) ... (eq. (transfer)), plus the
 * nearfield row.  y: nrows x nrhs col-major (ld nrows). */
void or_h2_rows(const or_h2* H, const int64_t* rows, int64_t nrows, const double* x, int nrhs, double* y) {
    const tree_t* T = &H->T;
    int64_t n = T->n, nc = T->count;
    int k = H->k;
    double* xh = calloc((size_t)nc * k * nrhs, sizeof(double));
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] >= 0) continue;
        int64_t b = T->begin[c], sz = T->end[c] - b;
        for (int nu = 0; nu < k; ++nu)
            for (int r = 0; r < nrhs; ++r) {
                double s = 0.0;
                for (int64_t a = 0; a < sz; ++a) s += H->W[c][a * k + nu] * x[T->perm[b + a] + r * n];
                xh[(c * k + nu) * nrhs + r] = s;
            }
    }
    for (int64_t c = nc - 1; c >= 0; --c) {
        if (T->child0[c] < 0) continue;
        int64_t ch[2] = {T->child0[c], T->child1[c]};
        for (int q = 0; q < 2; ++q) {
            const double* E = H->E[ch[q]];
            for (int nu = 0; nu < k; ++nu)
                for (int r = 0; r < nrhs; ++r) {
                    double s = 0.0;
                    for (int nup = 0; nup < k; ++nup) s += E[nup * k + nu] * xh[(ch[q] * k + nup) * nrhs + r];
                    xh[(c * k + nu) * nrhs + r] += s;
                }
        }
    }
    /* inverse permutation and leaf of each position */
    int64_t* pos = malloc(n * sizeof(int64_t));
    for (int64_t a = 0; a < n; ++a) pos[T->perm[a]] = a;
    int64_t* leaf_of = malloc(n * sizeof(int64_t));
    for (int64_t c = 0; c < nc; ++c)
        if (T->child0[c] < 0)
            for (int64_t a = T->begin[c]; a < T->end[c]; ++a) leaf_of[a] = c;
#pragma omp parallel
    {
        double* S = malloc((size_t)k * k * sizeof(double));
        double* v = malloc(k * sizeof(double));
        double* v2 = malloc(k * sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < nrows; ++q) {
            int64_t i = rows[q], a = pos[i], t = leaf_of[a];
            double acc[64];
            for (int r = 0; r < nrhs; ++r) acc[r] = 0.0;
            for (int nu = 0; nu < k; ++nu) v[nu] = H->V[t][(a - T->begin[t]) * k + nu];
            int64_t c = t;
            while (c >= 0) {
                for (int64_t b = H->far_ptr[c]; b < H->far_ptr[c + 1]; ++b) {
                    int64_t s = H->far_col[b];
                    coupling_matrix(H, c, s, S);
                    for (int nu = 0; nu < k; ++nu)
                        for (int r = 0; r < nrhs; ++r) {
                            double sm = 0.0;
                            for (int mu = 0; mu < k; ++mu) sm += S[nu * k + mu] * xh[(s * k + mu) * nrhs + r];
                            acc[r] += v[nu] * sm;
                        }
                }
                if (T->parent[c] < 0) break;
                /* V_parent|_c = V_c E_c */
                for (int nu = 0; nu < k; ++nu) {
                    double s = 0.0;
                    for (int nup = 0; nup < k; ++nup) s += v[nup] * H->E[c][nup * k + nu];
                    v2[nu] = s;
                }
                memcpy(v, v2, k * sizeof(double));
                c = T->parent[c];
            }
            for (int64_t b = H->near_ptr[t]; b < H->near_ptr[t + 1]; ++b) {
                int64_t s = H->near_col[b];
                for (int64_t bb = T->begin[s]; bb < T->end[s]; ++bb) {
                    int64_t j = T->perm[bb];
                    double e = or_entry(H->kernel, &H->mesh, i, j, H->q_ss);
                    for (int r = 0; r < nrhs; ++r) acc[r] += e * x[j + r * n];
                }
            }
            for (int r = 0; r < nrhs; ++r) y[q + r * nrows] = acc[r];
        }
        free(S);
        free(v);
        free(v2);
    }
    free(pos);
    free(leaf_of);
    free(xh);
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* Shape gradient of L = sum_r <w_r, A x_r> for the single layer, with the    */
/* cluster tree and the block lists frozen: derivative with respect to every  */
/* vertex coordinate, through the nearfield entries (7 x 7 rule and the full  */
/* Sauter-Schwab rule, areas included), the leaf bases, the transfer and      */
/* coupling matrices and, through their interpolation nodes, the cluster      */
/* boxes (centre and floored half-width) and the extreme vertices that define */
/* them.                                                                      */
/* ------------------------------------------------------------------------- */
void or_h2_update_geometry(or_h2* H, const double* xyz) {
    memcpy(H->xyz, xyz, 3 * H->mesh.nv * sizeof(double));
    h2_geometry(H);
}

/* grad_x g(x, y) = -(x - y) / (4 pi |x - y|^3) */
static void grad_g(const double* x, const double* y, double* out) {
    double d[3];
    sub3(x, y, d);
    double r2 = dot3(d, d);
    double c = -OR_INV4PI / (r2 * sqrt(r2));
    out[0] = c * d[0];
    out[1] = c * d[1];
    out[2] = c * d[2];
}

/* d|tau|/dX_k = 1/2 n x (X_{k+2} - X_{k+1}) (indices mod 3) */
static void area_grad(const double* X, double* dA) {
    double area, n[3];
    or_tri_geom(X, X + 3, X + 6, &area, n);
    for (int k = 0; k < 3; ++k) {
        double e[3];
        sub3(X + 3 * ((k + 2) % 3), X + 3 * ((k + 1) % 3), e);
        double c[3];
        cross3(n, e, c);
        for (int d = 0; d < 3; ++d) dA[3 * k + d] = 0.5 * c[d];
    }
}

static void add_vertex(double* gX, int32_t v, const double* g, double s) {
    for (int d = 0; d < 3; ++d) gX[3 * (int64_t)v + d] += s * g[d];
}

/* coef * d a_ij / d(vertices), single layer, accumulated into gX */
static void entry_grad_slp(const or_mesh* M, int64_t i, int64_t j, int q_ss, double coef, double* gX) {
    int ns = or_shared_vertices(M, i, j);
    if (ns == 0) {
        double X[9], Y[9], ax, ay, nx[3], ny[3], uv[14], w[7];
        tri_vertices(M, i, X);
        tri_vertices(M, j, Y);
        or_tri_geom(X, X + 3, X + 6, &ax, nx);
        or_tri_geom(Y, Y + 3, Y + 6, &ay, ny);
        or_radon7(uv, w);
        double xp[7][3], yq[7][3];
        for (int p = 0; p < 7; ++p)
            for (int d = 0; d < 3; ++d) {
                xp[p][d] = X[d] + uv[2 * p] * (X[3 + d] - X[d]) + uv[2 * p + 1] * (X[6 + d] - X[d]);
                yq[p][d] = Y[d] + uv[2 * p] * (Y[3 + d] - Y[d]) + uv[2 * p + 1] * (Y[6 + d] - Y[d]);
            }
        double S = 0.0, gx[3][3] = {{0}}, gy[3][3] = {{0}};
        for (int p = 0; p < 7; ++p)
            for (int q = 0; q < 7; ++q) {
                double wpq = w[p] * w[q], g[3];
                S += wpq * kernel_slp(xp[p], yq[q]);
                grad_g(xp[p], yq[q], g);
                double lx[3] = {1.0 - uv[2 * p] - uv[2 * p + 1], uv[2 * p], uv[2 * p + 1]};
                double ly[3] = {1.0 - uv[2 * q] - uv[2 * q + 1], uv[2 * q], uv[2 * q + 1]};
                for (int k = 0; k < 3; ++k)
                    for (int d = 0; d < 3; ++d) {
                        gx[k][d] += wpq * lx[k] * g[d];
                        gy[k][d] -= wpq * ly[k] * g[d];
                    }
            }
        double dAx[9], dAy[9];
        area_grad(X, dAx);
        area_grad(Y, dAy);
        for (int k = 0; k < 3; ++k) {
            double vx[3], vy[3];
            for (int d = 0; d < 3; ++d) {
                vx[d] = dAx[3 * k + d] * ay * S + ax * ay * gx[k][d];
                vy[d] = dAy[3 * k + d] * ax * S + ax * ay * gy[k][d];
            }
            add_vertex(gX, M->tri[3 * i + k], vx, coef);
            add_vertex(gX, M->tri[3 * j + k], vy, coef);
        }
        return;
    }
    /* singular: canonical orientation, full tensor rule */
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    double P[9], Q[9];
    int type;
    or_orient_pair(M, lo, hi, &type, P, Q);
    /* vertex ids of P and Q in their listed order */
    int32_t pv[3], qv[3];
    for (int k = 0; k < 3; ++k) {
        pv[k] = qv[k] = -1;
        for (int a = 0; a < 3; ++a) {
            const double* va = M->xyz + 3 * (int64_t)M->tri[3 * lo + a];
            const double* vb = M->xyz + 3 * (int64_t)M->tri[3 * hi + a];
            if (va[0] == P[3 * k] && va[1] == P[3 * k + 1] && va[2] == P[3 * k + 2]) pv[k] = M->tri[3 * lo + a];
            if (vb[0] == Q[3 * k] && vb[1] == Q[3 * k + 1] && vb[2] == Q[3 * k + 2]) qv[k] = M->tri[3 * hi + a];
        }
    }
    double g[64], gw[64];
    or_gauss_legendre01(q_ss, g, gw);
    double ap, np_[3], aq, nq[3];
    or_tri_geom(P, P + 3, P + 6, &ap, np_);
    or_tri_geom(Q, Q + 3, Q + 6, &aq, nq);
    double S = 0.0, gp[3][3] = {{0}}, gq[3][3] = {{0}};
    for (int i0 = 0; i0 < q_ss; ++i0)
        for (int i1 = 0; i1 < q_ss; ++i1)
            for (int i2 = 0; i2 < q_ss; ++i2)
                for (int i3 = 0; i3 < q_ss; ++i3) {
                    double wt = gw[i0] * gw[i1] * gw[i2] * gw[i3];
                    double reg[6][5];
                    int nr = ss_regions(type, g[i0], g[i1], g[i2], g[i3], reg);
                    for (int r = 0; r < nr; ++r) {
                        double x[3], y[3], gg[3];
                        chi(P, reg[r][0], reg[r][1], x);
                        chi(Q, reg[r][2], reg[r][3], y);
                        double c = wt * reg[r][4];
                        S += c * kernel_slp(x, y);
                        grad_g(x, y, gg);
                        /* d chi / d corner: (1 - x1, x1 - x2, x2) */
                        double lx[3] = {1.0 - reg[r][0], reg[r][0] - reg[r][1], reg[r][1]};
                        double ly[3] = {1.0 - reg[r][2], reg[r][2] - reg[r][3], reg[r][3]};
                        for (int k = 0; k < 3; ++k)
                            for (int d = 0; d < 3; ++d) {
                                gp[k][d] += c * lx[k] * gg[d];
                                gq[k][d] -= c * ly[k] * gg[d];
                            }
                    }
                }
    double dAp[9], dAq[9];
    area_grad(P, dAp);
    area_grad(Q, dAq);
    for (int k = 0; k < 3; ++k) {
        double vp[3], vq[3];
        for (int d = 0; d < 3; ++d) {
            vp[d] = 4.0 * (dAp[3 * k + d] * aq * S + ap * aq * gp[k][d]);
            vq[d] = 4.0 * (dAq[3 * k + d] * ap * S + ap * aq * gq[k][d]);
        }
        add_vertex(gX, pv[k], vp, coef);
        add_vertex(gX, qv[k], vq, coef);
    }
}

/* F(x, y, N) = (x - y).N / (4 pi |x - y|^3): its value, its gradient in x
 * (the gradient in y is the negative) and in N */
static double dlp_F(const double* x, const double* y, const double* N, double* gx, double* gN) {
    double d[3];
    sub3(x, y, d);
    const double r2 = dot3(d, d), r = sqrt(r2);
    const double i3 = OR_INV4PI / (r2 * r), dn = dot3(d, N);
    for (int e = 0; e < 3; ++e) {
        gx[e] = i3 * N[e] - 3.0 * i3 * dn * d[e] / r2;
        gN[e] = i3 * d[e];
    }
    return i3 * dn;
}

/* d(g . N)/dY_k for the area-normal N = (Y1 - Y0) x (Y2 - Y0) / 2 of the
 * triangle Y in its own vertex order: (Y_{k+1} - Y_{k+2}) x g / 2 */
static void area_normal_grad(const double* Y, const double* g, double* out /* 9 */) {
    for (int k = 0; k < 3; ++k) {
        double e[3], c[3];
        sub3(Y + 3 * ((k + 1) % 3), Y + 3 * ((k + 2) % 3), e);
        cross3(e, g, c);
        for (int d = 0; d < 3; ++d) out[3 * k + d] = 0.5 * c[d];
    }
}

/* coef * d k_ij / d(vertices), double layer (eq. (dlp), piecewise constant):
 * k_ij = |tau_i| sum w F(x, y, N_j) with N_j = |tau_j| n_j, so the entry
 * depends on the points of both triangles, on |tau_i| and on N_j. */
static void entry_grad_dlp(const or_mesh* M, int64_t i, int64_t j, int q_ss, double coef, double* gX) {
    if (i == j) return; /* identical pair: 0 for every flat triangle */
    double Yj[9], aj, nj[3], Nj[3];
    tri_vertices(M, j, Yj);
    or_tri_geom(Yj, Yj + 3, Yj + 6, &aj, nj);
    for (int d = 0; d < 3; ++d) Nj[d] = aj * nj[d];
    double Ssum = 0.0, gN[3] = {0, 0, 0};
    double gxi[3][3] = {{0}}, gyj[3][3] = {{0}};  /* per listed corner of tau_i / tau_j */
    int32_t iv[3], jv[3];
    double ai, scale;
    double Xi[9];
    int ns = or_shared_vertices(M, i, j);
    if (ns == 0) {
        double ni[3], uv[14], w[7];
        tri_vertices(M, i, Xi);
        or_tri_geom(Xi, Xi + 3, Xi + 6, &ai, ni);
        or_radon7(uv, w);
        for (int k = 0; k < 3; ++k) {
            iv[k] = M->tri[3 * i + k];
            jv[k] = M->tri[3 * j + k];
        }
        for (int p = 0; p < 7; ++p)
            for (int q = 0; q < 7; ++q) {
                double x[3], y[3], gx[3], gn[3];
                for (int d = 0; d < 3; ++d) {
                    x[d] = Xi[d] + uv[2 * p] * (Xi[3 + d] - Xi[d]) + uv[2 * p + 1] * (Xi[6 + d] - Xi[d]);
                    y[d] = Yj[d] + uv[2 * q] * (Yj[3 + d] - Yj[d]) + uv[2 * q + 1] * (Yj[6 + d] - Yj[d]);
                }
                const double wpq = w[p] * w[q];
                Ssum += wpq * dlp_F(x, y, Nj, gx, gn);
                const double lx[3] = {1.0 - uv[2 * p] - uv[2 * p + 1], uv[2 * p], uv[2 * p + 1]};
                const double ly[3] = {1.0 - uv[2 * q] - uv[2 * q + 1], uv[2 * q], uv[2 * q + 1]};
                for (int k = 0; k < 3; ++k)
                    for (int d = 0; d < 3; ++d) {
                        gxi[k][d] += wpq * lx[k] * gx[d];
                        gyj[k][d] -= wpq * ly[k] * gx[d];
                    }
                for (int d = 0; d < 3; ++d) gN[d] += wpq * gn[d];
            }
        scale = 1.0;
    } else {
        /* canonical orientation: the outer panel P is tau_lo, Q is tau_hi */
        const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
        double P[9], Q[9];
        int type;
        or_orient_pair(M, lo, hi, &type, P, Q);
        int32_t pv[3], qv[3];
        for (int k = 0; k < 3; ++k) {
            pv[k] = qv[k] = -1;
            for (int a = 0; a < 3; ++a) {
                const double* va = M->xyz + 3 * (int64_t)M->tri[3 * lo + a];
                const double* vb = M->xyz + 3 * (int64_t)M->tri[3 * hi + a];
                if (va[0] == P[3 * k] && va[1] == P[3 * k + 1] && va[2] == P[3 * k + 2]) pv[k] = M->tri[3 * lo + a];
                if (vb[0] == Q[3 * k] && vb[1] == Q[3 * k + 1] && vb[2] == Q[3 * k + 2]) qv[k] = M->tri[3 * hi + a];
            }
        }
        const int ilo = i == lo;
        const double* Xl = ilo ? P : Q; /* tau_i in its listed order */
        for (int k = 0; k < 3; ++k) {
            iv[k] = ilo ? pv[k] : qv[k];
            jv[k] = ilo ? qv[k] : pv[k];
        }
        memcpy(Xi, Xl, sizeof Xi);
        double ni[3];
        or_tri_geom(Xi, Xi + 3, Xi + 6, &ai, ni);
        double g[64], gw[64];
        or_gauss_legendre01(q_ss, g, gw);
        for (int i0 = 0; i0 < q_ss; ++i0)
            for (int i1 = 0; i1 < q_ss; ++i1)
                for (int i2 = 0; i2 < q_ss; ++i2)
                    for (int i3 = 0; i3 < q_ss; ++i3) {
                        const double wt = gw[i0] * gw[i1] * gw[i2] * gw[i3];
                        double reg[6][5];
                        const int nr = ss_regions(type, g[i0], g[i1], g[i2], g[i3], reg);
                        for (int r = 0; r < nr; ++r) {
                            double pp[3], qq[3], gx[3], gn[3];
                            chi(P, reg[r][0], reg[r][1], pp);
                            chi(Q, reg[r][2], reg[r][3], qq);
                            const double c = wt * reg[r][4];
                            const double lp[3] = {1.0 - reg[r][0], reg[r][0] - reg[r][1], reg[r][1]};
                            const double lq[3] = {1.0 - reg[r][2], reg[r][2] - reg[r][3], reg[r][3]};
                            const double* x = ilo ? pp : qq;
                            const double* y = ilo ? qq : pp;
                            const double* lx = ilo ? lp : lq;
                            const double* ly = ilo ? lq : lp;
                            Ssum += c * dlp_F(x, y, Nj, gx, gn);
                            for (int k = 0; k < 3; ++k)
                                for (int d = 0; d < 3; ++d) {
                                    gxi[k][d] += c * lx[k] * gx[d];
                                    gyj[k][d] -= c * ly[k] * gx[d];
                                }
                            for (int d = 0; d < 3; ++d) gN[d] += c * gn[d];
                        }
                    }
        scale = 4.0; /* int_tau int_sigma = 4 |tau||sigma| int_T int_T, |sigma| inside N_j */
    }
    /* k_ij = scale |tau_i| Ssum */
    double dAi[9], dN[9];
    area_grad(Xi, dAi);
    area_normal_grad(Yj, gN, dN);
    for (int k = 0; k < 3; ++k) {
        double vi[3], vj[3], vn[3];
        for (int d = 0; d < 3; ++d) {
            vi[d] = scale * (dAi[3 * k + d] * Ssum + ai * gxi[k][d]);
            vj[d] = scale * ai * gyj[k][d];
            vn[d] = scale * ai * dN[3 * k + d];
        }
        add_vertex(gX, iv[k], vi, coef);
        add_vertex(gX, jv[k], vj, coef);
        add_vertex(gX, M->tri[3 * j + k], vn, coef); /* N_j in tau_j's own vertex order */
    }
}

/* nodes of cluster c along axis e, centre, floored half-width */
static void box_ch(const tree_t* T, int64_t c, double* ctr, double* half, int* floored, int* amax) {
    double h[3], hmax = 0.0;
    int am = 0;
    for (int d = 0; d < 3; ++d) {
        ctr[d] = 0.5 * (T->bmin[3 * c + d] + T->bmax[3 * c + d]);
        h[d] = 0.5 * (T->bmax[3 * c + d] - T->bmin[3 * c + d]);
        if (h[d] > hmax) {
            hmax = h[d];
            am = d;
        }
    }
    for (int d = 0; d < 3; ++d) {
        floored[d] = h[d] < 1e-2 * hmax;
        half[d] = floored[d] ? 1e-2 * hmax : h[d];
    }
    *amax = am;
}

int or_h2_grad(const or_h2* H, const double* w, const double* x, int nrhs, double* gX, int parts) {
    if (H->kernel != OR_SLP && H->kernel != OR_DLP) return -1;
    const int dlp = H->kernel == OR_DLP;
    const tree_t* T = &H->T;
    int64_t n = T->n, nc = T->count, nv = H->mesh.nv;
    int k = H->k, m = H->m;
    for (int64_t a = 0; a < 3 * nv; ++a) gX[a] = 0.0;
    if (parts & OR_PART_NEAR) {
        /* nearfield entries, coefficient c_ij = sum_r w_ir x_jr */
        for (int64_t t = 0; t < nc; ++t)
            for (int64_t b = H->near_ptr[t]; b < H->near_ptr[t + 1]; ++b) {
                int64_t s = H->near_col[b];
                for (int64_t a = T->begin[t]; a < T->end[t]; ++a)
                    for (int64_t bb = T->begin[s]; bb < T->end[s]; ++bb) {
                        int64_t i = T->perm[a], j = T->perm[bb];
                        double c = 0.0;
                        for (int r = 0; r < nrhs; ++r) c += w[i + r * n] * x[j + r * n];
                        if (dlp) entry_grad_dlp(&H->mesh, i, j, H->q_ss, c, gX);
                        else entry_grad_slp(&H->mesh, i, j, H->q_ss, c, gX);
                    }
            }
    }
    if (!(parts & OR_PART_FAR) || H->far.n == 0) return 0;
    /* forward quantities: xh = W^T x, wh = V^T w (upward), yh = S xh, zh = S^T wh, then downward
     * (W = V for the single layer) */
    size_t vs = (size_t)nc * k * nrhs;
    double* xh = calloc(vs, sizeof(double));
    double* wh = calloc(vs, sizeof(double));
    double* yh = calloc(vs, sizeof(double));
    double* zh = calloc(vs, sizeof(double));
    double* S = malloc((size_t)k * k * sizeof(double));
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] >= 0) continue;
        int64_t b = T->begin[c], sz = T->end[c] - b;
        for (int nu = 0; nu < k; ++nu)
            for (int r = 0; r < nrhs; ++r) {
                double sx = 0.0, sw = 0.0;
                for (int64_t a = 0; a < sz; ++a) {
                    sx += H->W[c][a * k + nu] * x[T->perm[b + a] + r * n];
                    sw += H->V[c][a * k + nu] * w[T->perm[b + a] + r * n];
                }
                xh[(c * k + nu) * nrhs + r] = sx;
                wh[(c * k + nu) * nrhs + r] = sw;
            }
    }
    for (int64_t c = nc - 1; c >= 0; --c) {
        if (T->child0[c] < 0) continue;
        int64_t ch[2] = {T->child0[c], T->child1[c]};
        for (int q = 0; q < 2; ++q)
            for (int nu = 0; nu < k; ++nu)
                for (int r = 0; r < nrhs; ++r) {
                    double sx = 0.0, sw = 0.0;
                    for (int nup = 0; nup < k; ++nup) {
                        sx += H->E[ch[q]][nup * k + nu] * xh[(ch[q] * k + nup) * nrhs + r];
                        sw += H->E[ch[q]][nup * k + nu] * wh[(ch[q] * k + nup) * nrhs + r];
                    }
                    xh[(c * k + nu) * nrhs + r] += sx;
                    wh[(c * k + nu) * nrhs + r] += sw;
                }
    }
    for (int b = 0; b < H->far.n; ++b) {
        int64_t t = H->far.t[b], s = H->far.s[b];
        coupling_matrix(H, t, s, S);
        for (int nu = 0; nu < k; ++nu)
            for (int mu = 0; mu < k; ++mu)
                for (int r = 0; r < nrhs; ++r) {
                    yh[(t * k + nu) * nrhs + r] += S[nu * k + mu] * xh[(s * k + mu) * nrhs + r];
                    zh[(s * k + mu) * nrhs + r] += S[nu * k + mu] * wh[(t * k + nu) * nrhs + r];
                }
    }
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] < 0) continue;
        int64_t ch[2] = {T->child0[c], T->child1[c]};
        for (int q = 0; q < 2; ++q)
            for (int nup = 0; nup < k; ++nup)
                for (int r = 0; r < nrhs; ++r) {
                    double sy = 0.0, sz = 0.0;
                    for (int nu = 0; nu < k; ++nu) {
                        sy += H->E[ch[q]][nup * k + nu] * yh[(c * k + nu) * nrhs + r];
                        sz += H->E[ch[q]][nup * k + nu] * zh[(c * k + nu) * nrhs + r];
                    }
                    yh[(ch[q] * k + nup) * nrhs + r] += sy;
                    zh[(ch[q] * k + nup) * nrhs + r] += sz;
                }
    }
    /* dL/d(centre), dL/d(half-width) of every cluster's interpolation box */
    double* gc = calloc(3 * nc, sizeof(double));
    double* gh = calloc(3 * nc, sizeof(double));
    /* coupling: L contains wh_t^T S_ts xh_s */
    for (int b = 0; b < H->far.n; ++b) {
        int64_t t = H->far.t[b], s = H->far.s[b];
        const double* zt = H->nodes + t * 3 * m;
        const double* zs = H->nodes + s * 3 * m;
        double ct[3], htt[3], cs[3], hs[3];
        int fl[3], am;
        box_ch(T, t, ct, htt, fl, &am);
        box_ch(T, s, cs, hs, fl, &am);
        for (int nu = 0; nu < k; ++nu) {
            int ia[3] = {nu % m, (nu / m) % m, nu / (m * m)};
            double xt[3] = {zt[ia[0]], zt[m + ia[1]], zt[2 * m + ia[2]]};
            for (int mu = 0; mu < k; ++mu) {
                int ja[3] = {mu % m, (mu / m) % m, mu / (m * m)};
                double xs[3] = {zs[ja[0]], zs[m + ja[1]], zs[2 * m + ja[2]]};
                double c = 0.0;
                for (int r = 0; r < nrhs; ++r) c += wh[(t * k + nu) * nrhs + r] * xh[(s * k + mu) * nrhs + r];
                double gg[3];
                grad_g(xt, xs, gg);
                for (int d = 0; d < 3; ++d) {
                    /* xi = centre + half * cos-node: d xi / d centre = 1, d xi / d half = (xi - centre) / half */
                    gc[3 * t + d] += c * gg[d];
                    gh[3 * t + d] += c * gg[d] * (xt[d] - ct[d]) / htt[d];
                    gc[3 * s + d] -= c * gg[d];
                    gh[3 * s + d] -= c * gg[d] * (xs[d] - cs[d]) / hs[d];
                }
            }
        }
    }
    /* transfers: L contains sum E_c'[nu',nu] (xh_c'[nu'] zh_p[nu] + wh_c'[nu'] yh_p[nu]) */
    for (int64_t c = 1; c < nc; ++c) {
        int64_t p = T->parent[c];
        const double* zc = H->nodes + c * 3 * m;
        const double* zp = H->nodes + p * 3 * m;
        double cc[3], hc[3], cp[3], hp[3];
        int fl[3], am;
        box_ch(T, c, cc, hc, fl, &am);
        box_ch(T, p, cp, hp, fl, &am);
        for (int nup = 0; nup < k; ++nup) {
            double xi[3] = {zc[nup % m], zc[m + (nup / m) % m], zc[2 * m + nup / (m * m)]};
            for (int nu = 0; nu < k; ++nu) {
                double M = 0.0;
                for (int r = 0; r < nrhs; ++r)
                    M += xh[(c * k + nup) * nrhs + r] * zh[(p * k + nu) * nrhs + r] +
                         wh[(c * k + nup) * nrhs + r] * yh[(p * k + nu) * nrhs + r];
                double gl[3];
                tensor_lagrange_grad(zp, m, nu, xi, gl);
                for (int d = 0; d < 3; ++d) {
                    gc[3 * c + d] += M * gl[d];
                    gh[3 * c + d] += M * gl[d] * (xi[d] - cc[d]) / hc[d];
                    gc[3 * p + d] -= M * gl[d];
                    gh[3 * p + d] -= M * gl[d] * (xi[d] - cp[d]) / hp[d];
                }
            }
        }
    }
    /* leaf bases: L contains sum_i sum_nu V_c[i,nu] w_i yh_c[nu] + W_c[i,nu] x_i zh_c[nu]
     * (W = V for the single layer) */
    double ruv[2 * 64 * 64], rw[64 * 64];
    int np = or_collapsed_rule(H->qb, ruv, rw);
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] >= 0) continue;
        const double* z = H->nodes + c * 3 * m;
        double cc[3], hc[3];
        int fl[3], am;
        box_ch(T, c, cc, hc, fl, &am);
        for (int64_t a = T->begin[c]; a < T->end[c]; ++a) {
            int64_t i = T->perm[a];
            double beta[512], betaW[512];
            for (int nu = 0; nu < k; ++nu) {
                double bv = 0.0, bw = 0.0;
                for (int r = 0; r < nrhs; ++r) {
                    bv += w[i + r * n] * yh[(c * k + nu) * nrhs + r];
                    bw += x[i + r * n] * zh[(c * k + nu) * nrhs + r];
                }
                beta[nu] = dlp ? bv : bv + bw;
                betaW[nu] = dlp ? bw : 0.0;
            }
            double X[9], area, nrm[3], dA[9];
            tri_vertices(&H->mesh, i, X);
            or_tri_geom(X, X + 3, X + 6, &area, nrm);
            area_grad(X, dA);
            double Psum = 0.0, gv[3][3] = {{0}};
            for (int pp = 0; pp < np; ++pp) {
                double y[3];
                for (int d = 0; d < 3; ++d)
                    y[d] = X[d] + ruv[2 * pp] * (X[3 + d] - X[d]) + ruv[2 * pp + 1] * (X[6 + d] - X[d]);
                double P = 0.0, gP[3] = {0, 0, 0};
                for (int nu = 0; nu < k; ++nu) {
                    double gl[3];
                    P += beta[nu] * tensor_lagrange(z, m, nu, y);
                    tensor_lagrange_grad(z, m, nu, y, gl);
                    for (int d = 0; d < 3; ++d) gP[d] += beta[nu] * gl[d];
                }
                Psum += rw[pp] * P;
                double lam[3] = {1.0 - ruv[2 * pp] - ruv[2 * pp + 1], ruv[2 * pp], ruv[2 * pp + 1]};
                for (int kk = 0; kk < 3; ++kk)
                    for (int d = 0; d < 3; ++d) gv[kk][d] += rw[pp] * lam[kk] * gP[d];
                for (int d = 0; d < 3; ++d) {
                    gc[3 * c + d] -= area * rw[pp] * gP[d];
                    gh[3 * c + d] -= area * rw[pp] * gP[d] * (y[d] - cc[d]) / hc[d];
                }
            }
            for (int kk = 0; kk < 3; ++kk) {
                double v[3];
                for (int d = 0; d < 3; ++d) v[d] = dA[3 * kk + d] * Psum + area * gv[kk][d];
                add_vertex(gX, H->tri[3 * i + kk], v, 1.0);
            }
            if (!dlp) continue;
            /* double layer: sum_nu betaW[nu] W_c[i,nu] = sum_p rw_p N . grad Pw(y_p), with
             * Pw = sum_nu betaW[nu] L_nu and N = area n (the rule's weights sum to 1) */
            double N[3], G[3] = {0, 0, 0}, gw2[3][3] = {{0}};
            for (int d = 0; d < 3; ++d) N[d] = area * nrm[d];
            for (int pp = 0; pp < np; ++pp) {
                double y[3];
                for (int d = 0; d < 3; ++d)
                    y[d] = X[d] + ruv[2 * pp] * (X[3 + d] - X[d]) + ruv[2 * pp + 1] * (X[6 + d] - X[d]);
                double gP[3] = {0, 0, 0}, HN[3] = {0, 0, 0};
                for (int nu = 0; nu < k; ++nu) {
                    double gl[3], hl[9];
                    tensor_lagrange_grad(z, m, nu, y, gl);
                    tensor_lagrange_hess(z, m, nu, y, hl);
                    for (int d = 0; d < 3; ++d) {
                        gP[d] += betaW[nu] * gl[d];
                        HN[d] += betaW[nu] * (hl[3 * d] * N[0] + hl[3 * d + 1] * N[1] + hl[3 * d + 2] * N[2]);
                    }
                }
                const double lam[3] = {1.0 - ruv[2 * pp] - ruv[2 * pp + 1], ruv[2 * pp], ruv[2 * pp + 1]};
                for (int d = 0; d < 3; ++d) {
                    G[d] += rw[pp] * gP[d];
                    for (int kk = 0; kk < 3; ++kk) gw2[kk][d] += rw[pp] * lam[kk] * HN[d];
                    /* the nodes: d(grad L)/d centre = -Hess L; d(d_e L)/d h_d = -delta_de d_d L / h_d
                     * - (y_d - c_d) / h_d d_d d_e L */
                    gc[3 * c + d] -= rw[pp] * HN[d];
                    gh[3 * c + d] -= rw[pp] * (N[d] * gP[d] + (y[d] - cc[d]) * HN[d]) / hc[d];
                }
            }
            double dN[9];
            area_normal_grad(X, G, dN);
            for (int kk = 0; kk < 3; ++kk) {
                double v[3];
                for (int d = 0; d < 3; ++d) v[d] = dN[3 * kk + d] + gw2[kk][d];
                add_vertex(gX, H->tri[3 * i + kk], v, 1.0);
            }
        }
    }
    /* boxes -> bounding-box extremes -> vertices */
    for (int64_t c = 0; c < nc; ++c) {
        double cc[3], hc[3];
        int fl[3], am;
        box_ch(T, c, cc, hc, fl, &am);
        double glo[3] = {0, 0, 0}, ghi[3] = {0, 0, 0};
        for (int d = 0; d < 3; ++d) {
            glo[d] += 0.5 * gc[3 * c + d];
            ghi[d] += 0.5 * gc[3 * c + d];
            int e = fl[d] ? am : d;
            double f = fl[d] ? 1e-2 : 1.0;
            glo[e] -= 0.5 * f * gh[3 * c + d];
            ghi[e] += 0.5 * f * gh[3 * c + d];
        }
        /* the vertex realising each extreme: first in traversal order (as tree_box) */
        for (int d = 0; d < 3; ++d) {
            double lo = INFINITY, hi = -INFINITY;
            int32_t vlo = -1, vhi = -1;
            for (int64_t a = T->begin[c]; a < T->end[c]; ++a)
                for (int q = 0; q < 3; ++q) {
                    int32_t v = H->tri[3 * T->perm[a] + q];
                    double val = H->xyz[3 * (int64_t)v + d];
                    if (val < lo) { lo = val; vlo = v; }
                    if (val > hi) { hi = val; vhi = v; }
                }
            gX[3 * (int64_t)vlo + d] += glo[d];
            gX[3 * (int64_t)vhi + d] += ghi[d];
        }
    }
    free(gc); free(gh); free(S); free(xh); free(wh); free(yh); free(zh);
    return 0;
}

/* ========================================================================= */
/* Green cross approximation, GCA (section 4), single layer G               */
/* ========================================================================= */
/* For a cluster t with box B_t = [a, b]:                                     */
/*  1. The auxiliary box omega_t = [a - delta_t, b + delta_t] on every axis,  */
/*     delta_t = max_d (b_d - a_d) (the choice of the experiments, section 5, */
/*     dist(d omega_t, B_t) = delta_t).                                       */
/*  2. Green's representation formula on omega_t (section 4):                 */
/*       g(x,y) = int g(x,z) dg/dn_z(z,y) dz - int dg/dn_z(x,z) g(z,y) dz,    */
/*     discretised by a composite Gauss rule on the six faces of d omega_t:   */
/*     face f = 2 d + side (side 0: x_d = lo_d, normal -e_d; side 1: x_d =   */
/*     hi_d, normal +e_d), q x q Gauss-Legendre points over its two other     */
/*     axes d1 < d2, point nu = (f q + a) q + b, weight w_nu = gw_a gw_b      */
/*     len_d1 len_d2; k = 6 q^2 points.                                       */
/*  3. L = (A C), rows = the row set of t, A_i,nu = w_nu^(1/2) int_tau_i      */
/*     g(x, z_nu) dx, C_i,nu = w_nu^(1/2) int_tau_i dg/dn_z(x, z_nu) dx (the  */
/*     7-point rule on tau_i; z_nu is at distance >= delta_t from B_t).       */
/*     The row set is the triangles of t (a leaf, in tree order) or          */
/*     t^_{t1} followed by t^_{t2} (the children's pivots, nested form).     */
/*  4. Adaptive cross approximation of L with full pivoting (the pivoted LU  */
/*     of section 3): residual R = L; while rank < kmax and rank < min(rows, */
/*     cols): with M = max |R|, the pivot (i*, j*) is the first entry in     */
/*     row-major order with |R_ij| >= (1 - 2^-40) M (the paper leaves ties   */
/*     open; this makes the choice insensitive to rounding far below 2^-40,  */
/*     so exact ties of symmetric meshes resolve alike everywhere); stop if  */
/*     M = 0 or (rank > 0 and |R_i*j*| <= eps |first pivot|);                */
/*     R_ij -= R_ij* (R_i*j / R_i*j*) for all i, j (the row of the pivot      */
/*     divided first); tau += i*, sigma += j*.                                */
/*  5. V^_t = L|_{rows x sigma} (L|_{tau x sigma})^{-1} (eq. gca_onesided);  */
/*     t^ = rows[tau] in pivot order.  Leaf: V_t = V^_t.  Otherwise          */
/*     (E_t1; E_t2) = V^_t split by rows (eq. (transfer)).                   */
/*  6. Coupling S_ts = G|_{t^ x s^} (Galerkin entries of the pivot           */
/*     triangles, eq. (slp)); the single layer is symmetric, so W_s = V_s.   */
/* The H^2 product then runs the passes of section 2 with these V, E, S.     */

struct or_gca {
    or_mesh mesh;
    double* xyz;
    int32_t* tri;
    int q, q_ss, kmax;
    double eta, eps;
    tree_t T;
    blist far, near;
    int64_t *far_ptr, *far_col, *near_ptr, *near_col;
    int* rank;      /* k~_t */
    int64_t** piv;  /* pivot triangles (user indices) of t, pivot order */
    double** V;     /* leaves: |t| x rank_t, rows in tree order */
    double** E;     /* non-root clusters: rank_c x rank_parent */
};

/* The composite Gauss rule on the boundary of the box [lo, hi] (step 2):
 * z[3 k], w[k], nz[3 k] with k = 6 q^2. */
int or_gca_boundary_rule(const double* lo, const double* hi, int q, double* z, double* w, double* nz) {
    double g[64], gw[64];
    if (or_gauss_legendre01(q, g, gw)) return -1;
    for (int f = 0; f < 6; ++f) {
        const int d = f / 2, side = f % 2;
        const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
        const double l1 = hi[d1] - lo[d1], l2 = hi[d2] - lo[d2];
        for (int a = 0; a < q; ++a)
            for (int b = 0; b < q; ++b) {
                const int nu = (f * q + a) * q + b;
                z[3 * nu + d] = side ? hi[d] : lo[d];
                z[3 * nu + d1] = lo[d1] + l1 * g[a];
                z[3 * nu + d2] = lo[d2] + l2 * g[b];
                w[nu] = gw[a] * gw[b] * l1 * l2;
                nz[3 * nu + 0] = nz[3 * nu + 1] = nz[3 * nu + 2] = 0.0;
                nz[3 * nu + d] = side ? 1.0 : -1.0;
            }
    }
    return 6 * q * q;
}

/* g~_grn(x, y) of step 2 with the boundary rule of [lo, hi]. */
double or_gca_green(const double* lo, const double* hi, int q, const double* x, const double* y) {
    const int k = 6 * q * q;
    double* z = malloc(3 * k * sizeof(double));
    double* w = malloc(k * sizeof(double));
    double* nz = malloc(3 * k * sizeof(double));
    or_gca_boundary_rule(lo, hi, q, z, w, nz);
    double s = 0.0;
    for (int nu = 0; nu < k; ++nu)
        s += w[nu] * (kernel_slp(x, z + 3 * nu) * kernel_dlp(y, z + 3 * nu, nz + 3 * nu) -
                      kernel_dlp(x, z + 3 * nu, nz + 3 * nu) * kernel_slp(z + 3 * nu, y));
    free(z);
    free(w);
    free(nz);
    return s;
}

/* Row of L for triangle i (step 3): 2k values. */
static void gca_L_row(const or_mesh* M, int64_t i, int k, const double* z, const double* w, const double* nz,
                      double* L) {
    double X[9], area, nrm[3], uv[14], rw[7], xp[7][3];
    tri_vertices(M, i, X);
    or_tri_geom(X, X + 3, X + 6, &area, nrm);
    or_radon7(uv, rw);
    for (int p = 0; p < 7; ++p)
        for (int d = 0; d < 3; ++d) xp[p][d] = X[d] + uv[2 * p] * (X[3 + d] - X[d]) + uv[2 * p + 1] * (X[6 + d] - X[d]);
    for (int nu = 0; nu < k; ++nu) {
        double a = 0.0, c = 0.0;
        for (int p = 0; p < 7; ++p) {
            a += rw[p] * kernel_slp(xp[p], z + 3 * nu);
            c += rw[p] * kernel_dlp(xp[p], z + 3 * nu, nz + 3 * nu);
        }
        const double sw = sqrt(w[nu]);
        L[nu] = sw * area * a;
        L[k + nu] = sw * area * c;
    }
}

/* omega_t of step 1 */
static void gca_omega(const tree_t* T, int64_t c, double* lo, double* hi) {
    const double* a = T->bmin + 3 * c;
    const double* b = T->bmax + 3 * c;
    double delta = 0.0;
    for (int d = 0; d < 3; ++d)
        if (b[d] - a[d] > delta) delta = b[d] - a[d];
    for (int d = 0; d < 3; ++d) {
        lo[d] = a[d] - delta;
        hi[d] = b[d] + delta;
    }
}

/* Row set of cluster c (step 3): user triangle indices; returns the count. */
static int64_t gca_rows(const or_gca* G, int64_t c, int64_t* rows) {
    const tree_t* T = &G->T;
    if (T->child0[c] < 0) {
        for (int64_t a = T->begin[c]; a < T->end[c]; ++a) rows[a - T->begin[c]] = T->perm[a];
        return T->end[c] - T->begin[c];
    }
    int64_t n = 0;
    const int64_t ch[2] = {T->child0[c], T->child1[c]};
    for (int h = 0; h < 2; ++h)
        for (int r = 0; r < G->rank[ch[h]]; ++r) rows[n++] = G->piv[ch[h]][r];
    return n;
}

/* L of cluster c (rows x 2k, row-major) for its row set; returns rows. */
static int64_t gca_L(const or_gca* G, int64_t c, int64_t* rows, double* L) {
    const int k = 6 * G->q * G->q;
    double lo[3], hi[3];
    gca_omega(&G->T, c, lo, hi);
    double* z = malloc(3 * k * sizeof(double));
    double* w = malloc(k * sizeof(double));
    double* nz = malloc(3 * k * sizeof(double));
    or_gca_boundary_rule(lo, hi, G->q, z, w, nz);
    const int64_t nr = gca_rows(G, c, rows);
    for (int64_t r = 0; r < nr; ++r) gca_L_row(&G->mesh, rows[r], k, z, w, nz, L + r * 2 * k);
    free(z);
    free(w);
    free(nz);
    return nr;
}

/* Step 4: full-pivot cross approximation; returns the rank. */
int or_gca_aca(const double* L, int rows, int cols, double eps, int kmax, int* tau, int* sigma) {
    double* R = malloc((size_t)rows * cols * sizeof(double));
    double* col = malloc(rows * sizeof(double));
    double* row = malloc(cols * sizeof(double));
    memcpy(R, L, (size_t)rows * cols * sizeof(double));
    int k = 0;
    double first = 0.0;
    while (k < kmax && k < rows && k < cols) {
        double M = 0.0;
        for (size_t e = 0; e < (size_t)rows * cols; ++e)
            if (fabs(R[e]) > M) M = fabs(R[e]);
        if (M == 0.0) break;
        const double thr = M * (1.0 - ldexp(1.0, -40));
        size_t e = 0;
        while (fabs(R[e]) < thr) ++e;
        const int bi = (int)(e / cols), bj = (int)(e % cols);
        const double p = R[(size_t)bi * cols + bj];
        if (k == 0) first = fabs(p);
        else if (fabs(p) <= eps * first) break;
        tau[k] = bi;
        sigma[k] = bj;
        ++k;
        for (int i = 0; i < rows; ++i) col[i] = R[(size_t)i * cols + bj];
        for (int j = 0; j < cols; ++j) row[j] = R[(size_t)bi * cols + j] / p;
        for (int i = 0; i < rows; ++i)
            for (int j = 0; j < cols; ++j) R[(size_t)i * cols + j] -= col[i] * row[j];
    }
    free(R);
    free(col);
    free(row);
    return k;
}

/* Step 5: V = L|_{: x sigma} (L|_{tau x sigma})^{-1} (rows x k), by Gaussian
 * elimination with partial pivoting on M^T V^T = L|_{: x sigma}^T. */
static void gca_interp(const double* L, int rows, int cols, int k, const int* tau, const int* sigma, double* V) {
    double* Mt = malloc((size_t)k * k * sizeof(double));  /* Mt[a][b] = L[tau[b]][sigma[a]] */
    double* B = malloc((size_t)k * rows * sizeof(double)); /* B[a][r] = L[r][sigma[a]] */
    for (int a = 0; a < k; ++a) {
        for (int b = 0; b < k; ++b) Mt[a * k + b] = L[(size_t)tau[b] * cols + sigma[a]];
        for (int r = 0; r < rows; ++r) B[(size_t)a * rows + r] = L[(size_t)r * cols + sigma[a]];
    }
    for (int c = 0; c < k; ++c) {
        int pr = c;
        for (int a = c + 1; a < k; ++a)
            if (fabs(Mt[a * k + c]) > fabs(Mt[pr * k + c])) pr = a;
        if (pr != c) {
            for (int b = 0; b < k; ++b) {
                double t = Mt[c * k + b];
                Mt[c * k + b] = Mt[pr * k + b];
                Mt[pr * k + b] = t;
            }
            for (int r = 0; r < rows; ++r) {
                double t = B[(size_t)c * rows + r];
                B[(size_t)c * rows + r] = B[(size_t)pr * rows + r];
                B[(size_t)pr * rows + r] = t;
            }
        }
        for (int a = c + 1; a < k; ++a) {
            const double f = Mt[a * k + c] / Mt[c * k + c];
            for (int b = c; b < k; ++b) Mt[a * k + b] -= f * Mt[c * k + b];
            for (int r = 0; r < rows; ++r) B[(size_t)a * rows + r] -= f * B[(size_t)c * rows + r];
        }
    }
    for (int c = k - 1; c >= 0; --c)
        for (int r = 0; r < rows; ++r) {
            double s = B[(size_t)c * rows + r];
            for (int b = c + 1; b < k; ++b) s -= Mt[c * k + b] * V[(size_t)r * k + b];
            V[(size_t)r * k + c] = s / Mt[c * k + c];
        }
    free(Mt);
    free(B);
}

or_gca* or_gca_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, int q, double eta, int leaf,
                      double eps, int kmax, int q_ss) {
    if (q < 1 || q > 16 || leaf < 1 || nt < 1 || kmax < 1) return NULL;
    or_gca* G = calloc(1, sizeof(or_gca));
    G->xyz = malloc(3 * nv * sizeof(double));
    G->tri = malloc(3 * nt * sizeof(int32_t));
    memcpy(G->xyz, xyz, 3 * nv * sizeof(double));
    memcpy(G->tri, tri, 3 * nt * sizeof(int32_t));
    G->mesh.xyz = G->xyz;
    G->mesh.tri = G->tri;
    G->mesh.nv = nv;
    G->mesh.nt = nt;
    G->q = q;
    G->eta = eta;
    G->eps = eps;
    G->kmax = kmax;
    G->q_ss = q_ss;
    tree_t* T = &G->T;
    T->n = nt;
    T->perm = malloc(nt * sizeof(int64_t));
    for (int64_t i = 0; i < nt; ++i) T->perm[i] = i;
    int64_t* tmp = malloc(nt * sizeof(int64_t));
    tree_split(&G->mesh, T, 0, nt, -1, 0, leaf, tmp);
    free(tmp);
    block_build(T, eta, 0, 0, &G->far, &G->near);
    const int64_t nc = T->count;
    G->far_ptr = csr_from(nc, G->far.t, G->far.s, G->far.n, &G->far_col);
    G->near_ptr = csr_from(nc, G->near.t, G->near.s, G->near.n, &G->near_col);
    G->rank = calloc(nc, sizeof(int));
    G->piv = calloc(nc, sizeof(int64_t*));
    G->V = calloc(nc, sizeof(double*));
    G->E = calloc(nc, sizeof(double*));
    const int k = 6 * q * q;
    /* children before parents: clusters are numbered in pre-order; a level of
     * the tree at a time, its clusters in parallel */
    int maxlev = 0;
    for (int64_t c = 0; c < nc; ++c)
        if (T->level[c] > maxlev) maxlev = T->level[c];
    for (int lev = maxlev; lev >= 0; --lev) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t c = 0; c < nc; ++c) {
            if (T->level[c] != lev) continue;
            const int64_t cap = (T->end[c] - T->begin[c]) > 2 * kmax ? (T->end[c] - T->begin[c]) : 2 * kmax;
            int64_t* rows = malloc(cap * sizeof(int64_t));
            double* L = malloc((size_t)cap * 2 * k * sizeof(double));
            const int64_t nr = gca_L(G, c, rows, L);
            int* tau = malloc((kmax + 1) * sizeof(int));
            int* sigma = malloc((kmax + 1) * sizeof(int));
            const int rk = or_gca_aca(L, (int)nr, 2 * k, eps, kmax, tau, sigma);
            double* Vh = malloc(((size_t)nr * rk + 1) * sizeof(double));
            gca_interp(L, (int)nr, 2 * k, rk, tau, sigma, Vh);
            G->rank[c] = rk;
            G->piv[c] = malloc((rk + 1) * sizeof(int64_t));
            for (int r = 0; r < rk; ++r) G->piv[c][r] = rows[tau[r]];
            if (T->child0[c] < 0) {
                G->V[c] = Vh;
            } else {
                const int64_t ch[2] = {T->child0[c], T->child1[c]};
                int off = 0;
                for (int h = 0; h < 2; ++h) {
                    const int kc = G->rank[ch[h]];
                    G->E[ch[h]] = malloc(((size_t)kc * rk + 1) * sizeof(double));
                    memcpy(G->E[ch[h]], Vh + (size_t)off * rk, (size_t)kc * rk * sizeof(double));
                    off += kc;
                }
                free(Vh);
            }
            free(rows);
            free(L);
            free(tau);
            free(sigma);
        }
    }
    return G;
}

void or_gca_destroy(or_gca* G) {
    if (!G) return;
    tree_t* T = &G->T;
    for (int64_t c = 0; c < T->count; ++c) {
        free(G->piv[c]);
        free(G->V[c]);
        free(G->E[c]);
    }
    free(G->piv); free(G->V); free(G->E); free(G->rank);
    free(G->far_ptr); free(G->far_col); free(G->near_ptr); free(G->near_col);
    free(G->far.t); free(G->far.s); free(G->near.t); free(G->near.s);
    free(T->perm); free(T->begin); free(T->end); free(T->child0); free(T->child1); free(T->parent);
    free(T->level); free(T->bmin); free(T->bmax);
    free(G->xyz); free(G->tri);
    free(G);
}

/* counts: clusters, farfield blocks, nearfield blocks, largest rank, points k */
void or_gca_sizes(const or_gca* G, int64_t* out) {
    out[0] = G->T.count;
    out[1] = G->far.n;
    out[2] = G->near.n;
    int mx = 0;
    for (int64_t c = 0; c < G->T.count; ++c)
        if (G->rank[c] > mx) mx = G->rank[c];
    out[3] = mx;
    out[4] = 6 * G->q * G->q;
}
void or_gca_ranks(const or_gca* G, int32_t* rank) {
    for (int64_t c = 0; c < G->T.count; ++c) rank[c] = G->rank[c];
}
void or_gca_pivots(const or_gca* G, int64_t c, int64_t* piv) {
    memcpy(piv, G->piv[c], G->rank[c] * sizeof(int64_t));
}
/* V_t of a leaf (|t| x rank) or E_c (rank_c x rank_parent); -1 otherwise */
int or_gca_basis(const or_gca* G, int64_t c, double* out) {
    if (c < 0 || c >= G->T.count) return -1;
    if (G->T.child0[c] < 0) {
        memcpy(out, G->V[c], (size_t)(G->T.end[c] - G->T.begin[c]) * G->rank[c] * sizeof(double));
        return 0;
    }
    return -1;
}
int or_gca_transfer(const or_gca* G, int64_t c, double* out) {
    if (c <= 0 || c >= G->T.count) return -1;
    const int64_t p = G->T.parent[c];
    memcpy(out, G->E[c], (size_t)G->rank[c] * G->rank[p] * sizeof(double));
    return 0;
}
/* L of cluster c and its row set (user indices); returns the row count. */
int64_t or_gca_L(const or_gca* G, int64_t c, int64_t* rows, double* L) { return gca_L(G, c, rows, L); }
int64_t or_gca_rowcount(const or_gca* G, int64_t c) {
    const tree_t* T = &G->T;
    if (T->child0[c] < 0) return T->end[c] - T->begin[c];
    return G->rank[T->child0[c]] + G->rank[T->child1[c]];
}

/* y = G~ x (x, y column-major n x nrhs, user order): step 6 and the passes of
 * section 2 with the GCA bases; parts selects farfield / nearfield. */
void or_gca_matvec(const or_gca* G, const double* x, int nrhs, double* y, int parts) {
    const tree_t* T = &G->T;
    const int64_t n = T->n, nc = T->count;
    const int K = G->kmax;
    double* xh = calloc((size_t)nc * K * nrhs, sizeof(double));
    double* yh = calloc((size_t)nc * K * nrhs, sizeof(double));
    for (int64_t i = 0; i < n * nrhs; ++i) y[i] = 0.0;
    if (parts & OR_PART_FAR) {
        /* leaves: xh_t = V_t^T x|_t */
        for (int64_t c = 0; c < nc; ++c) {
            if (T->child0[c] >= 0) continue;
            const int rk = G->rank[c];
            for (int64_t a = T->begin[c]; a < T->end[c]; ++a)
                for (int nu = 0; nu < rk; ++nu)
                    for (int r = 0; r < nrhs; ++r)
                        xh[(c * K + nu) * nrhs + r] += G->V[c][(a - T->begin[c]) * rk + nu] * x[T->perm[a] + r * n];
        }
        /* upward, children after their parents in pre-order: reverse order */
        for (int64_t c = nc - 1; c >= 1; --c) {
            const int64_t p = T->parent[c];
            const int kc = G->rank[c], kp = G->rank[p];
            for (int nu = 0; nu < kp; ++nu)
                for (int r = 0; r < nrhs; ++r) {
                    double s = 0.0;
                    for (int a = 0; a < kc; ++a) s += G->E[c][a * kp + nu] * xh[(c * K + a) * nrhs + r];
                    xh[(p * K + nu) * nrhs + r] += s;
                }
        }
        /* coupling S_ts = G|_{t^ x s^} */
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t t = 0; t < nc; ++t)
            for (int64_t b = G->far_ptr[t]; b < G->far_ptr[t + 1]; ++b) {
                const int64_t s = G->far_col[b];
                for (int nu = 0; nu < G->rank[t]; ++nu)
                    for (int mu = 0; mu < G->rank[s]; ++mu) {
                        const double e = or_entry(OR_SLP, &G->mesh, G->piv[t][nu], G->piv[s][mu], G->q_ss);
                        for (int r = 0; r < nrhs; ++r) yh[(t * K + nu) * nrhs + r] += e * xh[(s * K + mu) * nrhs + r];
                    }
            }
        /* downward: parents before children */
        for (int64_t c = 1; c < nc; ++c) {
            const int64_t p = T->parent[c];
            const int kc = G->rank[c], kp = G->rank[p];
            for (int a = 0; a < kc; ++a)
                for (int r = 0; r < nrhs; ++r) {
                    double s = 0.0;
                    for (int nu = 0; nu < kp; ++nu) s += G->E[c][a * kp + nu] * yh[(p * K + nu) * nrhs + r];
                    yh[(c * K + a) * nrhs + r] += s;
                }
        }
        /* leaves: y|_t += V_t yh_t */
        for (int64_t c = 0; c < nc; ++c) {
            if (T->child0[c] >= 0) continue;
            const int rk = G->rank[c];
            for (int64_t a = T->begin[c]; a < T->end[c]; ++a)
                for (int r = 0; r < nrhs; ++r) {
                    double s = 0.0;
                    for (int nu = 0; nu < rk; ++nu) s += G->V[c][(a - T->begin[c]) * rk + nu] * yh[(c * K + nu) * nrhs + r];
                    y[T->perm[a] + r * n] += s;
                }
        }
    }
    if (parts & OR_PART_NEAR) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t t = 0; t < nc; ++t)
            for (int64_t b = G->near_ptr[t]; b < G->near_ptr[t + 1]; ++b) {
                const int64_t s = G->near_col[b];
                for (int64_t a = T->begin[t]; a < T->end[t]; ++a) {
                    const int64_t i = T->perm[a];
                    for (int64_t bb = T->begin[s]; bb < T->end[s]; ++bb) {
                        const int64_t j = T->perm[bb];
                        const double e = or_entry(OR_SLP, &G->mesh, i, j, G->q_ss);
                        for (int r = 0; r < nrhs; ++r) y[i + r * n] += e * x[j + r * n];
                    }
                }
            }
    }
    free(xh);
    free(yh);
}

/* The rows of y = A x (forward, A = G or K in its H^2 form) for the triangles
 * of cluster c0 only: the leaf forward transformation and the upward pass run
 * in full; the coupling, downward pass, leaf backward transformation and
 * nearfield only where they reach the rows of c0 (c0's ancestors and
 * descendants).  The other rows of y are 0.  Used as a bounded sample of the
 * full product. */
/* The leaf forward transformation and the upward pass of the forward product
 * (x-hat of every cluster, [nc][k][nrhs]). */
void or_h2_upward(const or_h2* H, const double* x, int nrhs, double* xh) {
    const tree_t* T = &H->T;
    const int64_t n = T->n, nc = T->count;
    const int k = H->k;
    for (size_t e = 0; e < (size_t)nc * k * nrhs; ++e) xh[e] = 0.0;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] >= 0) continue;
        int64_t b = T->begin[c], sz = T->end[c] - b;
        for (int nu = 0; nu < k; ++nu)
            for (int r = 0; r < nrhs; ++r) {
                double s = 0.0;
                for (int64_t a = 0; a < sz; ++a) s += H->W[c][a * k + nu] * x[T->perm[b + a] + r * n];
                xh[(c * k + nu) * nrhs + r] = s;
            }
    }
    for (int64_t c = nc - 1; c >= 0; --c) {
        if (T->child0[c] < 0) continue;
        const int64_t ch[2] = {T->child0[c], T->child1[c]};
        for (int q = 0; q < 2; ++q) {
            const double* E = H->E[ch[q]];
            for (int nu = 0; nu < k; ++nu)
                for (int r = 0; r < nrhs; ++r) {
                    double s = 0.0;
                    for (int nup = 0; nup < k; ++nup) s += E[nup * k + nu] * xh[(ch[q] * k + nup) * nrhs + r];
                    xh[(c * k + nu) * nrhs + r] += s;
                }
        }
    }
}

/* The rows for cluster c0 from x-hat of or_h2_upward (xh != NULL), else
 * computing x-hat first. */
void or_h2_matvec_subtree_from(const or_h2* H, int64_t c0, const double* xh_in, const double* x, int nrhs, double* y) {
    const tree_t* T = &H->T;
    const int64_t n = T->n, nc = T->count;
    const int k = H->k;
    double* xh_own = NULL;
    if (!xh_in) {
        xh_own = malloc((size_t)nc * k * nrhs * sizeof(double));
        or_h2_upward(H, x, nrhs, xh_own);
        xh_in = xh_own;
    }
    const double* xh = xh_in;
    double* yh = calloc((size_t)nc * k * nrhs, sizeof(double));
    char* act = calloc(nc, 1);
    for (int64_t c = 0; c < nc; ++c) {
        const int anc = T->begin[c] <= T->begin[c0] && T->end[c] >= T->end[c0];
        const int des = T->begin[c] >= T->begin[c0] && T->end[c] <= T->end[c0];
        act[c] = (char)(anc || des);
    }
#pragma omp parallel
    {
        double* S = malloc((size_t)k * k * sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < nc; ++t) {
            if (!act[t]) continue;
            for (int64_t b = H->far_ptr[t]; b < H->far_ptr[t + 1]; ++b) {
                const int64_t s = H->far_col[b];
                coupling_matrix(H, t, s, S);
                for (int nu = 0; nu < k; ++nu)
                    for (int r = 0; r < nrhs; ++r) {
                        double acc = 0.0;
                        for (int mu = 0; mu < k; ++mu) acc += S[nu * k + mu] * xh[(s * k + mu) * nrhs + r];
                        yh[(t * k + nu) * nrhs + r] += acc;
                    }
            }
        }
        free(S);
    }
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] < 0 || !act[c]) continue;
        const int64_t ch[2] = {T->child0[c], T->child1[c]};
        for (int q = 0; q < 2; ++q) {
            if (!act[ch[q]]) continue;
            const double* E = H->E[ch[q]];
            for (int nup = 0; nup < k; ++nup)
                for (int r = 0; r < nrhs; ++r) {
                    double s = 0.0;
                    for (int nu = 0; nu < k; ++nu) s += E[nup * k + nu] * yh[(c * k + nu) * nrhs + r];
                    yh[(ch[q] * k + nup) * nrhs + r] += s;
                }
        }
    }
    for (int64_t i = 0; i < n * nrhs; ++i) y[i] = 0.0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < nc; ++c) {
        if (T->child0[c] >= 0 || !act[c] || T->begin[c] < T->begin[c0] || T->end[c] > T->end[c0]) continue;
        const int64_t b = T->begin[c], sz = T->end[c] - b;
        for (int64_t a = 0; a < sz; ++a) {
            const int64_t i = T->perm[b + a];
            for (int r = 0; r < nrhs; ++r) {
                double s = 0.0;
                for (int nu = 0; nu < k; ++nu) s += H->V[c][a * k + nu] * yh[(c * k + nu) * nrhs + r];
                y[i + r * n] += s;
            }
        }
        for (int64_t q = H->near_ptr[c]; q < H->near_ptr[c + 1]; ++q) {
            const int64_t s = H->near_col[q];
            for (int64_t a = 0; a < sz; ++a) {
                const int64_t i = T->perm[b + a];
                for (int64_t bb = T->begin[s]; bb < T->end[s]; ++bb) {
                    const int64_t j = T->perm[bb];
                    const double e = or_entry(H->kernel, &H->mesh, i, j, H->q_ss);
                    for (int r = 0; r < nrhs; ++r) y[i + r * n] += e * x[j + r * n];
                }
            }
        }
    }
    free(act);
    free(xh_own);
    free(yh);
}

void or_h2_matvec_subtree(const or_h2* H, int64_t c0, const double* x, int nrhs, double* y) {
    or_h2_matvec_subtree_from(H, c0, NULL, x, nrhs, y);
}

/* ========================================================================= */
/* Hybrid cross approximation, HCA (section 3), single layer G, and its     */
/* hierarchical compression into an H^2-matrix (end of section 3)           */
/* ========================================================================= */
/* Per farfield block b = (t, s):                                            */
/*  1. S[nu,mu] = g(xi_{t,nu}, xi_{s,mu}) with the tensor Chebyshev nodes of */
/*     the H^2 specification (k = m^3 per cluster).                          */
/*  2. Cross approximation of S with full pivoting (the pivoted LU of       */
/*     section 3; the pivot and stop rules of or_gca_aca) with tolerance     */
/*     eps_aca and at most kaca steps: row pivots tau, column pivots sigma,  */
/*     rank r_b.                                                             */
/*  3. C_b = (S|_{tau x sigma})^{-1}, so that S ~ S|_{: x sigma} C_b         */
/*     S|_{tau x :}; C_b is indexed [sigma position][tau position].          */
/*  4. Take-back (eq. hca_discrete): A_b[i,kappa] = int_{tau_i}              */
/*     g(x, xi_{s,sigma_kappa}) dx (i in t), B_b[j,lambda] = int_{tau_j}     */
/*     g(xi_{t,tau_lambda}, y) dy (j in s), both by the 7-point rule (the    */
/*     nodes lie in the partner's box, away from the triangle);              */
/*     G|_{t x s} ~ A_b C_b B_b^T.                                           */
/* Hierarchical compression (the paper cites it and leaves it open; this is  */
/* the reading): orthonormal nested cluster bases from the HCA blocks,       */
/* bottom-up over the cluster tree.                                          */
/*  5. F_t = the farfield blocks (t*, s) with t* = t or an ancestor of t.   */
/*     With B_b = Q R (thin QR) every block contributes the columns          */
/*     A_b|_t W_b, W_b = C_b R^T: A_b|_t C_b B_b^T = (A_b|_t W_b) Q^T and Q^T */
/*     has orthonormal rows, so Z_t = [A_b|_t W_b]_{b in F_t} has the left   */
/*     singular vectors and values of the block row of t in the HCA matrix.  */
/*  6. Leaf t: Q_t = the left singular vectors of Z_t whose singular values  */
/*     exceed eps_c sigma_1(Z_t), at most kmax of them.  Parent t (children  */
/*     t1, t2): P_t = the same for [Q_t1^T Z_t|_t1 ; Q_t2^T Z_t|_t2];        */
/*     (E_t1 ; E_t2) = P_t split by rows, Q_t = [Q_t1 E_t1 ; Q_t2 E_t2].     */
/*     Singular vectors: Householder QR of Z^T, then one-sided Jacobi        */
/*     (Hestenes) on the triangular factor.                                  */
/*  7. Coupling S_ts = (Q_t^T A_b) C_b (Q_s^T B_b)^T.                        */
/* The H^2 product runs the passes of section 2 with V_t = Q_t (leaves),     */
/* the transfers E and the couplings S; the nearfield as in the H^2 form.    */

struct or_hca {
    or_mesh mesh;
    double* xyz;
    int32_t* tri;
    int m, k, kaca, kmax, q_ss;
    double eta, eps_aca, eps_c;
    tree_t T;
    blist far, near;
    int64_t *far_ptr, *far_col, *near_ptr, *near_col;
    double* nodes;  /* per cluster 3 m Chebyshev nodes */
    int* brank;     /* r_b per farfield block (far list order) */
    int** btau;     /* row pivots (node indices of t) */
    int** bsig;     /* column pivots (node indices of s) */
    double** bC;    /* r_b x r_b, [sigma pos][tau pos] */
    double** bW;    /* r_b x r_b, C_b R^T */
    int* rank;      /* k_t */
    double** Q;     /* every cluster: |t| x k_t, rows in tree order */
    double** E;     /* non-root clusters: k_c x k_parent */
    double** S;     /* farfield blocks: k_t x k_s */
};

/* node nu of cluster c */
static void hca_node(const or_hca* H, int64_t c, int nu, double* x) {
    const int m = H->m;
    const double* z = H->nodes + c * 3 * m;
    x[0] = z[nu % m];
    x[1] = z[m + (nu / m) % m];
    x[2] = z[2 * m + nu / (m * m)];
}

/* int_{tau_i} g(x, p) dx by the 7-point rule */
static double hca_panel_potential(const or_mesh* M, int64_t i, const double* p) {
    double X[9], area, nrm[3], uv[14], rw[7];
    tri_vertices(M, i, X);
    or_tri_geom(X, X + 3, X + 6, &area, nrm);
    or_radon7(uv, rw);
    double s = 0.0;
    for (int q = 0; q < 7; ++q) {
        double xq[3];
        for (int d = 0; d < 3; ++d) xq[d] = X[d] + uv[2 * q] * (X[3 + d] - X[d]) + uv[2 * q + 1] * (X[6 + d] - X[d]);
        s += rw[q] * kernel_slp(xq, p);
    }
    return area * s;
}

/* A_b (|t| x r, rows in tree order) of step 4 */
static void hca_A(const or_hca* H, int64_t b, double* A) {
    const int64_t t = H->far.t[b], s = H->far.s[b];
    const int r = H->brank[b];
    for (int64_t a = H->T.begin[t]; a < H->T.end[t]; ++a)
        for (int kap = 0; kap < r; ++kap) {
            double p[3];
            hca_node(H, s, H->bsig[b][kap], p);
            A[(a - H->T.begin[t]) * r + kap] = hca_panel_potential(&H->mesh, H->T.perm[a], p);
        }
}
/* B_b (|s| x r) of step 4 */
static void hca_B(const or_hca* H, int64_t b, double* B) {
    const int64_t t = H->far.t[b], s = H->far.s[b];
    const int r = H->brank[b];
    for (int64_t a = H->T.begin[s]; a < H->T.end[s]; ++a)
        for (int lam = 0; lam < r; ++lam) {
            double p[3];
            hca_node(H, t, H->btau[b][lam], p);
            B[(a - H->T.begin[s]) * r + lam] = hca_panel_potential(&H->mesh, H->T.perm[a], p);
        }
}

/* Inverse of the r x r matrix M (row-major) by Gauss-Jordan elimination with
 * partial pivoting; returns -1 if a pivot is 0. */
static int hca_inverse(const double* M, int r, double* Inv) {
    double* W = malloc((size_t)r * 2 * r * sizeof(double) + 1);
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < 2 * r; ++j) W[i * 2 * r + j] = j < r ? M[i * r + j] : (j - r == i ? 1.0 : 0.0);
    int bad = 0;
    for (int c = 0; c < r; ++c) {
        int p = c;
        for (int i = c + 1; i < r; ++i)
            if (fabs(W[i * 2 * r + c]) > fabs(W[p * 2 * r + c])) p = i;
        if (W[p * 2 * r + c] == 0.0) { bad = 1; break; }
        if (p != c)
            for (int j = 0; j < 2 * r; ++j) {
                double tmp = W[c * 2 * r + j];
                W[c * 2 * r + j] = W[p * 2 * r + j];
                W[p * 2 * r + j] = tmp;
            }
        const double d = W[c * 2 * r + c];
        for (int j = 0; j < 2 * r; ++j) W[c * 2 * r + j] /= d;
        for (int i = 0; i < r; ++i) {
            if (i == c) continue;
            const double f = W[i * 2 * r + c];
            if (f != 0.0)
                for (int j = 0; j < 2 * r; ++j) W[i * 2 * r + j] -= f * W[c * 2 * r + j];
        }
    }
    for (int i = 0; i < r && !bad; ++i)
        for (int j = 0; j < r; ++j) Inv[i * r + j] = W[i * 2 * r + r + j];
    free(W);
    return bad ? -1 : 0;
}

/* R of the thin Householder QR of the rows x cols matrix X (row-major),
 * p = min(rows, cols): R is p x cols upper trapezoidal (row-major). */
static void hca_qr_r(const double* X, int rows, int cols, double* R) {
    double* A = malloc((size_t)rows * cols * sizeof(double) + 1);
    double* v = malloc((size_t)rows * sizeof(double) + 1);
    memcpy(A, X, (size_t)rows * cols * sizeof(double));
    const int p = rows < cols ? rows : cols;
    for (int j = 0; j < p; ++j) {
        double nrm = 0.0;
        for (int i = j; i < rows; ++i) nrm += A[(size_t)i * cols + j] * A[(size_t)i * cols + j];
        nrm = sqrt(nrm);
        if (nrm == 0.0) continue;
        const double alpha = A[(size_t)j * cols + j] > 0 ? -nrm : nrm;
        for (int i = j; i < rows; ++i) v[i] = A[(size_t)i * cols + j];
        v[j] -= alpha;
        double vv = 0.0;
        for (int i = j; i < rows; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        for (int c = j; c < cols; ++c) {
            double d = 0.0;
            for (int i = j; i < rows; ++i) d += v[i] * A[(size_t)i * cols + c];
            d = 2.0 * d / vv;
            for (int i = j; i < rows; ++i) A[(size_t)i * cols + c] -= d * v[i];
        }
    }
    for (int i = 0; i < p; ++i)
        for (int c = 0; c < cols; ++c) R[(size_t)i * cols + c] = c < i ? 0.0 : A[(size_t)i * cols + c];
    free(A);
    free(v);
}

/* Left singular vectors and values of Z (r x cols, row-major): Householder
 * QR of Z^T = Q R (R p x r), one-sided Jacobi on R: R V = U Sigma, so Z =
 * V Sigma (Q U)^T.  U_out: r x r (column j = j-th left singular vector),
 * sv: r values, in decreasing order. */
static void hca_left_svd(const double* Z, int r, int cols, double* U_out, double* sv) {
    const int p = r < cols ? r : cols;
    double* Zt = malloc((size_t)cols * r * sizeof(double) + 1);
    for (int i = 0; i < r; ++i)
        for (int c = 0; c < cols; ++c) Zt[(size_t)c * r + i] = Z[(size_t)i * cols + c];
    double* R = malloc((size_t)p * r * sizeof(double) + 1);
    hca_qr_r(Zt, cols, r, R);
    free(Zt);
    double* V = calloc((size_t)r * r, sizeof(double));
    for (int i = 0; i < r; ++i) V[i * r + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        int rotated = 0;
        for (int i = 0; i < r - 1; ++i)
            for (int j = i + 1; j < r; ++j) {
                double a = 0.0, bq = 0.0, g = 0.0;
                for (int q = 0; q < p; ++q) {
                    a += R[q * r + i] * R[q * r + i];
                    bq += R[q * r + j] * R[q * r + j];
                    g += R[q * r + i] * R[q * r + j];
                }
                if (g == 0.0 || fabs(g) <= 1e-15 * sqrt(a * bq)) continue;
                rotated = 1;
                const double zeta = (bq - a) / (2.0 * g);
                const double tn = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + tn * tn), sn = cs * tn;
                for (int q = 0; q < p; ++q) {
                    const double xi = R[q * r + i], xj = R[q * r + j];
                    R[q * r + i] = cs * xi - sn * xj;
                    R[q * r + j] = sn * xi + cs * xj;
                }
                for (int q = 0; q < r; ++q) {
                    const double xi = V[q * r + i], xj = V[q * r + j];
                    V[q * r + i] = cs * xi - sn * xj;
                    V[q * r + j] = sn * xi + cs * xj;
                }
            }
        if (!rotated) break;
    }
    double* nrm = malloc((size_t)r * sizeof(double) + 1);
    int* ord = malloc((size_t)r * sizeof(int) + 1);
    for (int j = 0; j < r; ++j) {
        double s = 0.0;
        for (int q = 0; q < p; ++q) s += R[q * r + j] * R[q * r + j];
        nrm[j] = sqrt(s);
        ord[j] = j;
    }
    for (int a = 1; a < r; ++a)  /* insertion sort, decreasing, stable */
        for (int b = a; b > 0 && nrm[ord[b]] > nrm[ord[b - 1]]; --b) {
            int tmp = ord[b];
            ord[b] = ord[b - 1];
            ord[b - 1] = tmp;
        }
    for (int j = 0; j < r; ++j) {
        sv[j] = nrm[ord[j]];
        for (int q = 0; q < r; ++q) U_out[q * r + j] = V[q * r + ord[j]];
    }
    free(R); free(V); free(nrm); free(ord);
}

/* Steps 1-3 for farfield block b. */
static void hca_block_aca(or_hca* H, int64_t b) {
    const int k = H->k;
    const int64_t t = H->far.t[b], s = H->far.s[b];
    double* S = malloc((size_t)k * k * sizeof(double));
    for (int nu = 0; nu < k; ++nu) {
        double xt[3];
        hca_node(H, t, nu, xt);
        for (int mu = 0; mu < k; ++mu) {
            double xs[3];
            hca_node(H, s, mu, xs);
            S[nu * k + mu] = kernel_slp(xt, xs);
        }
    }
    int* tau = malloc((k + 1) * sizeof(int));
    int* sig = malloc((k + 1) * sizeof(int));
    int r = or_gca_aca(S, k, k, H->eps_aca, H->kaca, tau, sig);
    double* M = malloc(((size_t)r * r + 1) * sizeof(double));
    double* C = malloc(((size_t)r * r + 1) * sizeof(double));
    for (int a = 0; a < r; ++a)
        for (int c = 0; c < r; ++c) M[a * r + c] = S[tau[a] * k + sig[c]]; /* [tau pos][sigma pos] */
    if (hca_inverse(M, r, C)) r = 0;                                       /* C: [sigma pos][tau pos] */
    H->brank[b] = r;
    H->btau[b] = tau;
    H->bsig[b] = sig;
    H->bC[b] = C;
    free(M);
    free(S);
}

/* W_b = C_b R^T with B_b = Q R (step 5). */
static void hca_block_weight(or_hca* H, int64_t b) {
    const int r = H->brank[b];
    const int64_t s = H->far.s[b];
    const int64_t ns = H->T.end[s] - H->T.begin[s];
    double* W = calloc((size_t)r * r + 1, sizeof(double));
    if (r > 0) {
        double* B = malloc((size_t)ns * r * sizeof(double));
        hca_B(H, b, B);
        const int p = ns < r ? (int)ns : r;
        double* R = malloc((size_t)p * r * sizeof(double));
        hca_qr_r(B, (int)ns, r, R);
        for (int a = 0; a < r; ++a)
            for (int c = 0; c < p; ++c) { /* (C R^T)[a][c]; columns c >= p stay 0 */
                double acc = 0.0;
                for (int l = 0; l < r; ++l) acc += H->bC[b][a * r + l] * R[c * r + l];
                W[a * r + c] = acc;
            }
        free(B);
        free(R);
    }
    H->bW[b] = W;
}

/* Q_c^T A_b|_c (k_c x r) for a cluster c inside the row cluster of b. */
static void hca_project_A(const or_hca* H, int64_t b, int64_t c, double* out) {
    const int r = H->brank[b], kc = H->rank[c];
    const int64_t s = H->far.s[b];
    const int64_t nc_ = H->T.end[c] - H->T.begin[c];
    for (int e = 0; e < kc * r; ++e) out[e] = 0.0;
    for (int64_t a = 0; a < nc_; ++a)
        for (int kap = 0; kap < r; ++kap) {
            double p[3];
            hca_node(H, s, H->bsig[b][kap], p);
            const double v = hca_panel_potential(&H->mesh, H->T.perm[H->T.begin[c] + a], p);
            for (int nu = 0; nu < kc; ++nu) out[nu * r + kap] += H->Q[c][a * kc + nu] * v;
        }
}

/* Step 6 for cluster c (children done). */
static void hca_compress_cluster(or_hca* H, int64_t c) {
    const tree_t* T = &H->T;
    const int leaf = T->child0[c] < 0;
    const int64_t nct = T->end[c] - T->begin[c];
    const int k1 = leaf ? 0 : H->rank[T->child0[c]];
    const int rows = leaf ? (int)nct : k1 + H->rank[T->child1[c]];
    /* F_c: the farfield blocks of c and of its ancestors */
    int64_t nb = 0, cols = 0;
    for (int64_t a = c; a >= 0; a = T->parent[a])
        for (int64_t q = H->far_ptr[a]; q < H->far_ptr[a + 1]; ++q) {
            ++nb;
            cols += H->brank[H->far_col[q]];
        }
    double* Z = calloc((size_t)rows * cols + 1, sizeof(double));
    int64_t off = 0;
    for (int64_t a = c; a >= 0; a = T->parent[a])
        for (int64_t q = H->far_ptr[a]; q < H->far_ptr[a + 1]; ++q) {
            const int64_t b = H->far_col[q];
            const int r = H->brank[b];
            if (r == 0) continue;
            double* Ah = malloc((size_t)rows * r * sizeof(double));
            if (leaf) {
                const int64_t s = H->far.s[b];
                for (int64_t i = 0; i < nct; ++i)
                    for (int kap = 0; kap < r; ++kap) {
                        double p[3];
                        hca_node(H, s, H->bsig[b][kap], p);
                        Ah[i * r + kap] = hca_panel_potential(&H->mesh, T->perm[T->begin[c] + i], p);
                    }
            } else {
                hca_project_A(H, b, T->child0[c], Ah);
                hca_project_A(H, b, T->child1[c], Ah + (size_t)k1 * r);
            }
            for (int i = 0; i < rows; ++i)
                for (int j = 0; j < r; ++j) {
                    double acc = 0.0;
                    for (int l = 0; l < r; ++l) acc += Ah[i * r + l] * H->bW[b][l * r + j];
                    Z[(size_t)i * cols + off + j] = acc;
                }
            off += r;
            free(Ah);
        }
    (void)nb;
    int kt = 0;
    double* U = malloc(((size_t)rows * rows + 1) * sizeof(double));
    if (rows > 0 && cols > 0) {
        double* sv = malloc((size_t)rows * sizeof(double));
        hca_left_svd(Z, rows, (int)cols, U, sv);
        const int lim = rows < cols ? rows : (int)cols;
        if (sv[0] > 0.0)
            while (kt < lim && kt < H->kmax && sv[kt] > H->eps_c * sv[0]) ++kt;
        free(sv);
    }
    free(Z);
    H->rank[c] = kt;
    H->Q[c] = malloc(((size_t)nct * kt + 1) * sizeof(double));
    if (leaf) {
        for (int64_t i = 0; i < nct; ++i)
            for (int j = 0; j < kt; ++j) H->Q[c][i * kt + j] = U[i * rows + j];
    } else {
        const int64_t ch[2] = {T->child0[c], T->child1[c]};
        int roff = 0;
        for (int h = 0; h < 2; ++h) {
            const int kc = H->rank[ch[h]];
            H->E[ch[h]] = malloc(((size_t)kc * kt + 1) * sizeof(double));
            for (int a = 0; a < kc; ++a)
                for (int j = 0; j < kt; ++j) H->E[ch[h]][a * kt + j] = U[(roff + a) * rows + j];
            /* Q_c restricted to the child: Q_child E_child */
            const int64_t b0 = T->begin[ch[h]] - T->begin[c], nch = T->end[ch[h]] - T->begin[ch[h]];
            for (int64_t i = 0; i < nch; ++i)
                for (int j = 0; j < kt; ++j) {
                    double acc = 0.0;
                    for (int a = 0; a < kc; ++a) acc += H->Q[ch[h]][i * kc + a] * H->E[ch[h]][a * kt + j];
                    H->Q[c][(b0 + i) * kt + j] = acc;
                }
            roff += kc;
        }
    }
    free(U);
}

/* Step 7 for farfield block b. */
static void hca_coupling(or_hca* H, int64_t b) {
    const int64_t t = H->far.t[b], s = H->far.s[b];
    const int r = H->brank[b], kt = H->rank[t], ks = H->rank[s];
    const int64_t nt_ = H->T.end[t] - H->T.begin[t], ns = H->T.end[s] - H->T.begin[s];
    double* Sb = calloc((size_t)kt * ks + 1, sizeof(double));
    if (r > 0 && kt > 0 && ks > 0) {
        double* A = malloc((size_t)nt_ * r * sizeof(double));
        double* B = malloc((size_t)ns * r * sizeof(double));
        hca_A(H, b, A);
        hca_B(H, b, B);
        double* QA = calloc((size_t)kt * r, sizeof(double));
        double* QB = calloc((size_t)ks * r, sizeof(double));
        for (int64_t i = 0; i < nt_; ++i)
            for (int nu = 0; nu < kt; ++nu)
                for (int l = 0; l < r; ++l) QA[nu * r + l] += H->Q[t][i * kt + nu] * A[i * r + l];
        for (int64_t j = 0; j < ns; ++j)
            for (int mu = 0; mu < ks; ++mu)
                for (int l = 0; l < r; ++l) QB[mu * r + l] += H->Q[s][j * ks + mu] * B[j * r + l];
        for (int nu = 0; nu < kt; ++nu)
            for (int mu = 0; mu < ks; ++mu) {
                double acc = 0.0;
                for (int kap = 0; kap < r; ++kap)
                    for (int lam = 0; lam < r; ++lam) acc += QA[nu * r + kap] * H->bC[b][kap * r + lam] * QB[mu * r + lam];
                Sb[nu * ks + mu] = acc;
            }
        free(A); free(B); free(QA); free(QB);
    }
    H->S[b] = Sb;
}

or_hca* or_hca_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, int m, double eta, int leaf,
                      double eps_aca, int kaca, double eps_c, int kmax, int q_ss) {
    if (m < 1 || m > 8 || leaf < 1 || nt < 1 || kmax < 1 || kaca < 1 || !(eps_aca >= 0.0) || !(eps_c >= 0.0))
        return NULL;
    or_hca* H = calloc(1, sizeof(or_hca));
    H->xyz = malloc(3 * nv * sizeof(double));
    H->tri = malloc(3 * nt * sizeof(int32_t));
    memcpy(H->xyz, xyz, 3 * nv * sizeof(double));
    memcpy(H->tri, tri, 3 * nt * sizeof(int32_t));
    H->mesh.xyz = H->xyz;
    H->mesh.tri = H->tri;
    H->mesh.nv = nv;
    H->mesh.nt = nt;
    H->m = m;
    H->k = m * m * m;
    H->kaca = kaca < H->k ? kaca : H->k;
    H->kmax = kmax;
    H->q_ss = q_ss;
    H->eta = eta;
    H->eps_aca = eps_aca;
    H->eps_c = eps_c;
    tree_t* T = &H->T;
    T->n = nt;
    T->perm = malloc(nt * sizeof(int64_t));
    for (int64_t i = 0; i < nt; ++i) T->perm[i] = i;
    int64_t* tmp = malloc(nt * sizeof(int64_t));
    tree_split(&H->mesh, T, 0, nt, -1, 0, leaf, tmp);
    free(tmp);
    block_build(T, eta, 0, 0, &H->far, &H->near);
    const int64_t nc = T->count, nf = H->far.n;
    int64_t* ids = malloc((nf ? nf : 1) * sizeof(int64_t));
    for (int64_t b = 0; b < nf; ++b) ids[b] = b;
    H->far_ptr = csr_from(nc, H->far.t, ids, nf, &H->far_col); /* block ids by row cluster */
    free(ids);
    H->near_ptr = csr_from(nc, H->near.t, H->near.s, H->near.n, &H->near_col);
    H->nodes = malloc((size_t)nc * 3 * m * sizeof(double));
    for (int64_t c = 0; c < nc; ++c) cluster_nodes(T->bmin + 3 * c, T->bmax + 3 * c, m, H->nodes + c * 3 * m);
    H->brank = calloc(nf + 1, sizeof(int));
    H->btau = calloc(nf + 1, sizeof(int*));
    H->bsig = calloc(nf + 1, sizeof(int*));
    H->bC = calloc(nf + 1, sizeof(double*));
    H->bW = calloc(nf + 1, sizeof(double*));
    H->S = calloc(nf + 1, sizeof(double*));
    H->rank = calloc(nc, sizeof(int));
    H->Q = calloc(nc, sizeof(double*));
    H->E = calloc(nc, sizeof(double*));
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < nf; ++b) {
        hca_block_aca(H, b);
        hca_block_weight(H, b);
    }
    int maxlev = 0;
    for (int64_t c = 0; c < nc; ++c)
        if (T->level[c] > maxlev) maxlev = T->level[c];
    for (int lev = maxlev; lev >= 0; --lev) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t c = 0; c < nc; ++c)
            if (T->level[c] == lev) hca_compress_cluster(H, c);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < nf; ++b) hca_coupling(H, b);
    return H;
}

void or_hca_destroy(or_hca* H) {
    if (!H) return;
    tree_t* T = &H->T;
    for (int64_t b = 0; b < H->far.n; ++b) {
        free(H->btau[b]); free(H->bsig[b]); free(H->bC[b]); free(H->bW[b]); free(H->S[b]);
    }
    for (int64_t c = 0; c < T->count; ++c) {
        free(H->Q[c]);
        free(H->E[c]);
    }
    free(H->btau); free(H->bsig); free(H->bC); free(H->bW); free(H->S); free(H->brank);
    free(H->Q); free(H->E); free(H->rank); free(H->nodes);
    free(H->far_ptr); free(H->far_col); free(H->near_ptr); free(H->near_col);
    free(H->far.t); free(H->far.s); free(H->near.t); free(H->near.s);
    free(T->perm); free(T->begin); free(T->end); free(T->child0); free(T->child1); free(T->parent);
    free(T->level); free(T->bmin); free(T->bmax);
    free(H->xyz); free(H->tri);
    free(H);
}

/* counts: clusters, farfield blocks, nearfield blocks, largest cluster rank,
 * k = m^3, largest block rank */
void or_hca_sizes(const or_hca* H, int64_t* out) {
    out[0] = H->T.count;
    out[1] = H->far.n;
    out[2] = H->near.n;
    int mx = 0, mb = 0;
    for (int64_t c = 0; c < H->T.count; ++c)
        if (H->rank[c] > mx) mx = H->rank[c];
    for (int64_t b = 0; b < H->far.n; ++b)
        if (H->brank[b] > mb) mb = H->brank[b];
    out[3] = mx;
    out[4] = H->k;
    out[5] = mb;
}
void or_hca_ranks(const or_hca* H, int32_t* rank, int32_t* brank) {
    if (rank)
        for (int64_t c = 0; c < H->T.count; ++c) rank[c] = H->rank[c];
    if (brank)
        for (int64_t b = 0; b < H->far.n; ++b) brank[b] = H->brank[b];
}
/* farfield block list (row and column clusters) and the user triangle
 * indices of cluster c in tree order (returns |c|) */
void or_hca_blocks(const or_hca* H, int64_t* far_t, int64_t* far_s) {
    for (int64_t b = 0; b < H->far.n; ++b) {
        far_t[b] = H->far.t[b];
        far_s[b] = H->far.s[b];
    }
}
int64_t or_hca_cluster(const or_hca* H, int64_t c, int64_t* idx) {
    for (int64_t a = H->T.begin[c]; a < H->T.end[c]; ++a) idx[a - H->T.begin[c]] = H->T.perm[a];
    return H->T.end[c] - H->T.begin[c];
}
/* pivots (node indices) and C_b of block b; returns r_b */
int or_hca_block(const or_hca* H, int64_t b, int32_t* tau, int32_t* sigma, double* C) {
    const int r = H->brank[b];
    for (int a = 0; a < r; ++a) {
        if (tau) tau[a] = H->btau[b][a];
        if (sigma) sigma[a] = H->bsig[b][a];
    }
    if (C) memcpy(C, H->bC[b], (size_t)r * r * sizeof(double));
    return r;
}
/* the interpolation node nu of cluster c */
void or_hca_node(const or_hca* H, int64_t c, int nu, double* x) { hca_node(H, c, nu, x); }
/* g~_hca(x, y) of block b: sum over kappa, lambda of g(x, xi_{s,sigma_kappa})
 * c_{kappa lambda} g(xi_{t,tau_lambda}, y) */
double or_hca_kernel(const or_hca* H, int64_t b, const double* x, const double* y) {
    const int r = H->brank[b];
    double s = 0.0;
    for (int kap = 0; kap < r; ++kap) {
        double p[3];
        hca_node(H, H->far.s[b], H->bsig[b][kap], p);
        const double gx = kernel_slp(x, p);
        for (int lam = 0; lam < r; ++lam) {
            double q[3];
            hca_node(H, H->far.t[b], H->btau[b][lam], q);
            s += gx * H->bC[b][kap * r + lam] * kernel_slp(q, y);
        }
    }
    return s;
}
/* A_b C_b B_b^T (|t| x |s|, tree order of both clusters) */
void or_hca_block_matrix(const or_hca* H, int64_t b, double* out) {
    const int64_t t = H->far.t[b], s = H->far.s[b];
    const int r = H->brank[b];
    const int64_t nt_ = H->T.end[t] - H->T.begin[t], ns = H->T.end[s] - H->T.begin[s];
    double* A = malloc(((size_t)nt_ * r + 1) * sizeof(double));
    double* B = malloc(((size_t)ns * r + 1) * sizeof(double));
    hca_A(H, b, A);
    hca_B(H, b, B);
    for (int64_t i = 0; i < nt_; ++i)
        for (int64_t j = 0; j < ns; ++j) {
            double acc = 0.0;
            for (int kap = 0; kap < r; ++kap)
                for (int lam = 0; lam < r; ++lam) acc += A[i * r + kap] * H->bC[b][kap * r + lam] * B[j * r + lam];
            out[i * ns + j] = acc;
        }
    free(A);
    free(B);
}
/* Q_c (|c| x k_c), E_c (k_c x k_parent), S_b (k_t x k_s); -1 where absent */
int or_hca_basis(const or_hca* H, int64_t c, double* out) {
    if (c < 0 || c >= H->T.count) return -1;
    memcpy(out, H->Q[c], (size_t)(H->T.end[c] - H->T.begin[c]) * H->rank[c] * sizeof(double));
    return 0;
}
int or_hca_transfer(const or_hca* H, int64_t c, double* out) {
    if (c <= 0 || c >= H->T.count) return -1;
    memcpy(out, H->E[c], (size_t)H->rank[c] * H->rank[H->T.parent[c]] * sizeof(double));
    return 0;
}
int or_hca_coupling(const or_hca* H, int64_t b, double* out) {
    if (b < 0 || b >= H->far.n) return -1;
    memcpy(out, H->S[b], (size_t)H->rank[H->far.t[b]] * H->rank[H->far.s[b]] * sizeof(double));
    return 0;
}

/* y = G~ x (x, y column-major n x nrhs, user order).  hmatrix = 0: the
 * compressed H^2 form (leaf forward x-hat_t = Q_t^T x|_t, upward through E,
 * coupling S, downward, leaf backward y|_t += Q_t y-hat_t); hmatrix = 1: the
 * HCA blocks themselves, y|_t += A_b C_b B_b^T x|_s.  parts selects the
 * farfield / nearfield (nearfield: the Galerkin entries of the H^2 form). */
void or_hca_matvec(const or_hca* H, const double* x, int nrhs, double* y, int parts, int hmatrix) {
    const tree_t* T = &H->T;
    const int64_t n = T->n, nc = T->count;
    for (int64_t i = 0; i < n * nrhs; ++i) y[i] = 0.0;
    if ((parts & OR_PART_FAR) && hmatrix) {
        /* row clusters in parallel: every block of row t writes rows of t only */
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t t = 0; t < nc; ++t)
            for (int64_t q = H->far_ptr[t]; q < H->far_ptr[t + 1]; ++q) {
                const int64_t b = H->far_col[q], s = H->far.s[b];
                const int r = H->brank[b];
                const int64_t nt_ = T->end[t] - T->begin[t], ns = T->end[s] - T->begin[s];
                double* A = malloc(((size_t)nt_ * r + 1) * sizeof(double));
                double* B = malloc(((size_t)ns * r + 1) * sizeof(double));
                double* u = calloc((size_t)r * nrhs + 1, sizeof(double));
                double* v = calloc((size_t)r * nrhs + 1, sizeof(double));
                hca_A(H, b, A);
                hca_B(H, b, B);
                for (int64_t j = 0; j < ns; ++j)
                    for (int lam = 0; lam < r; ++lam)
                        for (int rr = 0; rr < nrhs; ++rr) u[lam * nrhs + rr] += B[j * r + lam] * x[T->perm[T->begin[s] + j] + rr * n];
                for (int kap = 0; kap < r; ++kap)
                    for (int lam = 0; lam < r; ++lam)
                        for (int rr = 0; rr < nrhs; ++rr) v[kap * nrhs + rr] += H->bC[b][kap * r + lam] * u[lam * nrhs + rr];
                for (int64_t i = 0; i < nt_; ++i)
                    for (int kap = 0; kap < r; ++kap)
                        for (int rr = 0; rr < nrhs; ++rr) y[T->perm[T->begin[t] + i] + rr * n] += A[i * r + kap] * v[kap * nrhs + rr];
                free(A); free(B); free(u); free(v);
            }
    }
    if ((parts & OR_PART_FAR) && !hmatrix) {
        int K = 1;
        for (int64_t c = 0; c < nc; ++c)
            if (H->rank[c] > K) K = H->rank[c];
        double* xh = calloc((size_t)nc * K * nrhs, sizeof(double));
        double* yh = calloc((size_t)nc * K * nrhs, sizeof(double));
        for (int64_t c = 0; c < nc; ++c) {
            if (T->child0[c] >= 0) continue;
            const int kc = H->rank[c];
            for (int64_t a = T->begin[c]; a < T->end[c]; ++a)
                for (int nu = 0; nu < kc; ++nu)
                    for (int r = 0; r < nrhs; ++r)
                        xh[(c * K + nu) * nrhs + r] += H->Q[c][(a - T->begin[c]) * kc + nu] * x[T->perm[a] + r * n];
        }
        for (int64_t c = nc - 1; c >= 1; --c) {
            const int64_t p = T->parent[c];
            const int kc = H->rank[c], kp = H->rank[p];
            for (int nu = 0; nu < kp; ++nu)
                for (int r = 0; r < nrhs; ++r) {
                    double s = 0.0;
                    for (int a = 0; a < kc; ++a) s += H->E[c][a * kp + nu] * xh[(c * K + a) * nrhs + r];
                    xh[(p * K + nu) * nrhs + r] += s;
                }
        }
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t t = 0; t < nc; ++t)
            for (int64_t q = H->far_ptr[t]; q < H->far_ptr[t + 1]; ++q) {
                const int64_t b = H->far_col[q], s = H->far.s[b];
                const int kt = H->rank[t], ks = H->rank[s];
                for (int nu = 0; nu < kt; ++nu)
                    for (int mu = 0; mu < ks; ++mu)
                        for (int r = 0; r < nrhs; ++r)
                            yh[(t * K + nu) * nrhs + r] += H->S[b][nu * ks + mu] * xh[(s * K + mu) * nrhs + r];
            }
        for (int64_t c = 1; c < nc; ++c) {
            const int64_t p = T->parent[c];
            const int kc = H->rank[c], kp = H->rank[p];
            for (int a = 0; a < kc; ++a)
                for (int r = 0; r < nrhs; ++r) {
                    double s = 0.0;
                    for (int nu = 0; nu < kp; ++nu) s += H->E[c][a * kp + nu] * yh[(p * K + nu) * nrhs + r];
                    yh[(c * K + a) * nrhs + r] += s;
                }
        }
        for (int64_t c = 0; c < nc; ++c) {
            if (T->child0[c] >= 0) continue;
            const int kc = H->rank[c];
            for (int64_t a = T->begin[c]; a < T->end[c]; ++a)
                for (int r = 0; r < nrhs; ++r) {
                    double s = 0.0;
                    for (int nu = 0; nu < kc; ++nu) s += H->Q[c][(a - T->begin[c]) * kc + nu] * yh[(c * K + nu) * nrhs + r];
                    y[T->perm[a] + r * n] += s;
                }
        }
        free(xh);
        free(yh);
    }
    if (parts & OR_PART_NEAR) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t t = 0; t < nc; ++t)
            for (int64_t b = H->near_ptr[t]; b < H->near_ptr[t + 1]; ++b) {
                const int64_t s = H->near_col[b];
                for (int64_t a = T->begin[t]; a < T->end[t]; ++a) {
                    const int64_t i = T->perm[a];
                    for (int64_t bb = T->begin[s]; bb < T->end[s]; ++bb) {
                        const int64_t j = T->perm[bb];
                        const double e = or_entry(OR_SLP, &H->mesh, i, j, H->q_ss);
                        for (int r = 0; r < nrhs; ++r) y[i + r * n] += e * x[j + r * n];
                    }
                }
            }
    }
}
