/*
 * FP64 CPU oracle — TEST INFRASTRUCTURE ONLY (see h2oracle.c).
 *
 * Conventions
 *   Mesh: xyz[nv*3] doubles, tri[nt*3] int32 vertex indices, triangles
 *   counter-clockwise seen from outside.  psi_i = 1 on triangle tau_i.
 *   Vectors: column-major n x nrhs, leading dimension n, user triangle order.
 *
 * Quadrature specification (shared with the CUDA path by specification only)
 *   Regular pairs (no shared vertex): Radon's 7-point degree-5 rule on each
 *     triangle, 49 kernel evaluations per pair.
 *   Singular pairs (shared vertex indices): Sauter-Schwab relative-coordinate
 *     rules, tensor Gauss-Legendre with q points per direction on [0,1]^4,
 *     reference triangle T = {0 <= x2 <= x1 <= 1},
 *     chi(x) = P0 + x1 (P1-P0) + x2 (P2-P1):
 *     identical (6 regions, Jacobian xi^3 a^2 b), with (xi,a,b,c) in [0,1]^4:
 *       R1: x = (xi, xi(1-a+ab)),        y = (xi(1-abc), xi(1-a))
 *       R3: x = (xi, xi a(1-b+bc)),      y = (xi(1-ab), xi a(1-b))
 *       R5: x = (xi(1-abc), xi a(1-bc)), y = (xi, xi a(1-b))
 *       R2, R4, R6: R1, R3, R5 with x and y exchanged.
 *     common edge P0P1 (5 regions):
 *       R1 (xi^3 a^2):   x = (xi, xi a c),               y = (xi(1-ab), xi a(1-b))
 *       R2 (xi^3 a^2 b): x = (xi, xi a),                 y = (xi(1-abc), xi a b(1-c))
 *       R3 (xi^3 a^2 b): x = (xi(1-ab), xi a(1-b)),      y = (xi, xi a b c)
 *       R4 (xi^3 a^2 b): x = (xi(1-abc), xi a b(1-c)),   y = (xi, xi a)
 *       R5 (xi^3 a^2 b): x = (xi(1-abc), xi a(1-bc)),    y = (xi, xi a b)
 *     common vertex P0 (2 regions, Jacobian xi^3 b):
 *       R1: x = (xi, xi a), y = (xi b, xi b c);  R2: x and y exchanged.
 *     int_tau int_sigma k = 4 |tau||sigma| sum_R int_[0,1]^4 J_R k(chi_P(x), chi_Q(y)).
 *   Canonical orientation of a singular pair {i, j}, i != j: the outer panel P
 *     is the triangle with the lower user index; shared vertices are listed
 *     first and in the same order in P and Q (edge: P = rotation of tau_lo with
 *     its unshared vertex last; vertex: both rotated to start at the shared
 *     vertex).  g_ij = g_ji; k_ij, k_ji come from the same points.
 *   Double-layer entry of a triangle with itself: 0.
 *
 * H^2 specification
 *   Cluster tree: box = bounding box of all vertices of the cluster's
 *     triangles; split while |t| > leaf along the longest box axis (lowest
 *     axis wins ties) at the box midpoint 0.5*(lo+hi); triangles whose
 *     centroid ((a+b)+c)/3 along that axis is < midpoint go to child 0, in
 *     their current order, the rest to child 1; if one side would be empty,
 *     a stable sort by centroid coordinate and a split at floor(|t|/2).
 *     Clusters are numbered in depth-first pre-order.
 *   Block tree: from (root, root); farfield if dist > 0 and
 *     max(diam B_t, diam B_s) <= eta dist(B_t, B_s) (diam: box diagonal,
 *     dist: Euclidean box distance); nearfield if both are leaves; otherwise
 *     split s if t is a leaf, t if s is a leaf, else both.
 *   Interpolation: per axis, m Chebyshev nodes of the first kind
 *     c + h cos((2a+1) pi / (2m)), a = 0..m-1, on the cluster box with every
 *     half-width h raised to at least 1e-2 times the largest half-width;
 *     tensor index nu = a + m (b + m c).
 *   Leaf bases: V_t[i,nu] = int_{tau_i} L_{t,nu}; W_s = V_s (single layer) or
 *     W_s[j,mu] = int_{tau_j} n_j . grad L_{s,mu} (double layer), by a
 *     collapsed Gauss rule exact for degree 3(m-1).
 *   Transfer: E_{t'}[nu',nu] = L_{t,nu}(xi_{t',nu'}).
 *   Coupling: S_ts[nu,mu] = g(xi_{t,nu}, xi_{s,mu}).
 *
 * Parity status: every function here is pinned by tests that do not call the
 * function's own formula (tests/test_oracle_*.py); none is "parity unpinned".
 */
#ifndef H2ORACLE_H
#define H2ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_SLP = 0, OR_DLP = 1, OR_TEST_POLY = 2 };
enum { OR_PART_FAR = 1, OR_PART_NEAR = 2, OR_PART_ALL = 3 };
enum { OR_IDENTICAL = 3, OR_EDGE = 2, OR_VERTEX = 1 };

typedef struct {
    const double* xyz;
    const int32_t* tri;
    int64_t nv, nt;
} or_mesh;

typedef struct or_h2 or_h2;

int or_gauss_legendre01(int q, double* x, double* w);
void or_radon7(double* uv, double* w);
int or_collapsed_rule(int q, double* uv, double* w);
void or_tri_geom(const double* a, const double* b, const double* c, double* area, double* normal);

double or_pair_regular(int kernel, const double* X, const double* Y);
double or_ss_pair(int kernel, int type, const double* P, const double* Q, const double* nrm, double sgn, int q);
int or_shared_vertices(const or_mesh* M, int64_t i, int64_t j);
void or_orient_pair(const or_mesh* M, int64_t lo, int64_t hi, int* type_out, double* P, double* Q);
double or_entry(int kernel, const or_mesh* M, int64_t i, int64_t j, int q_ss);

void or_dense_matvec(int kernel, const or_mesh* M, int q_ss, const double* x, int nrhs, double* y, int transpose);
void or_dense_rows(int kernel, const or_mesh* M, int q_ss, const int64_t* rows, int64_t nrows, const double* x,
                   int nrhs, double* y);
void or_dense_matrix(int kernel, const or_mesh* M, int q_ss, double* A);

/* Double layer with continuous piecewise-linear trial functions (section 1,
 * eq. (dlp), phi_j the hat functions of the vertices).
 *   or_ss_pair3: or_ss_pair with the barycentric coordinate of each corner of
 *     panel `side` (0: P, 1: Q; lambda = (1 - z1, z1 - z2, z2) in chi's
 *     coordinates) as a factor: out[3].
 *   or_entry_dlp_p1: out[c] = int_{tau_i} int_{tau_j} dg/dn_y lambda_{j,c}(y),
 *     c the corners of tau_j in the caller's order.
 *   or_dense_dlp_p1: K1 (nt x nv, row-major), K1[i, v] = sum over the
 *     triangles j at vertex v of the corner values. */
void or_ss_pair3(int kernel, int type, const double* P, const double* Q, const double* nrm, double sgn, int q,
                 int side, double* out);
void or_entry_dlp_p1(const or_mesh* M, int64_t i, int64_t j, int q_ss, double* out);
void or_dense_dlp_p1(const or_mesh* M, int q_ss, double* A);

or_h2* or_h2_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, int kernel, int m, double eta,
                    int leaf, int q_ss);
void or_h2_destroy(or_h2* H);
void or_h2_sizes(const or_h2* H, int64_t* out);
void or_h2_tree(const or_h2* H, int64_t* perm, int64_t* begin, int64_t* end, int64_t* child0, int64_t* child1,
                double* bmin, double* bmax);
void or_h2_blocks(const or_h2* H, int64_t* far_t, int64_t* far_s, int64_t* near_t, int64_t* near_s);
int or_h2_leaf_basis(const or_h2* H, int64_t c, double* V, double* W);
int or_h2_transfer(const or_h2* H, int64_t c, double* E);
void or_h2_nodes(const or_h2* H, double* nodes);
void or_h2_matvec(const or_h2* H, const double* x, int nrhs, double* y, int transpose, int parts);
/* K1 x (transpose = 0: x nv x nrhs, y nt x nrhs) or K1^T x (transpose = 1:
 * x nt x nrhs, y nv x nrhs), the double layer with piecewise-linear trial
 * functions in the same H^2 form (per-corner basis W1 on the vertex side, V on
 * the triangle side, the passes of or_h2_matvec, the nearfield by
 * or_entry_dlp_p1). */
void or_h2_matvec_dlp_p1(const or_h2* H, const double* x, int nrhs, double* y, int transpose, int parts);
double or_ss_moment(int type, int q, int a, int b, int c, int d);
double or_test_poly_P(const double* x);
double or_test_poly_Q(const double* y);
void or_h2_rows(const or_h2* H, const int64_t* rows, int64_t nrows, const double* x, int nrhs, double* y);
/* rows of the forward product for the triangles of cluster c0 only (others 0) */
void or_h2_matvec_subtree(const or_h2* H, int64_t c0, const double* x, int nrhs, double* y);
/* its two parts: x-hat of every cluster ([nc][k][nrhs]), and the rows from it */
void or_h2_upward(const or_h2* H, const double* x, int nrhs, double* xh);
void or_h2_matvec_subtree_from(const or_h2* H, int64_t c0, const double* xh, const double* x, int nrhs, double* y);
void or_h2_update_geometry(or_h2* H, const double* xyz);
int or_h2_grad(const or_h2* H, const double* w, const double* x, int nrhs, double* gX, int parts);
int or_num_threads(void);
void or_set_threads(int n);

/* Green cross approximation of the single layer G (section 4); the
 * specification is written out before or_gca_create in h2oracle.c. */
typedef struct or_gca or_gca;
int or_gca_boundary_rule(const double* lo, const double* hi, int q, double* z, double* w, double* nz);
double or_gca_green(const double* lo, const double* hi, int q, const double* x, const double* y);
int or_gca_aca(const double* L, int rows, int cols, double eps, int kmax, int* tau, int* sigma);
or_gca* or_gca_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, int q, double eta, int leaf,
                      double eps, int kmax, int q_ss);
void or_gca_destroy(or_gca* G);
void or_gca_sizes(const or_gca* G, int64_t* out);
void or_gca_ranks(const or_gca* G, int32_t* rank);
void or_gca_pivots(const or_gca* G, int64_t c, int64_t* piv);
int or_gca_basis(const or_gca* G, int64_t c, double* out);
int or_gca_transfer(const or_gca* G, int64_t c, double* out);
int64_t or_gca_L(const or_gca* G, int64_t c, int64_t* rows, double* L);
int64_t or_gca_rowcount(const or_gca* G, int64_t c);
void or_gca_matvec(const or_gca* G, const double* x, int nrhs, double* y, int parts);

/* Hybrid cross approximation of the single layer G (section 3) and its
 * hierarchical compression into an H^2-matrix; the specification is written
 * out before struct or_hca in h2oracle.c. */
typedef struct or_hca or_hca;
or_hca* or_hca_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, int m, double eta, int leaf,
                      double eps_aca, int kaca, double eps_c, int kmax, int q_ss);
void or_hca_destroy(or_hca* H);
void or_hca_sizes(const or_hca* H, int64_t* out);
void or_hca_ranks(const or_hca* H, int32_t* rank, int32_t* brank);
void or_hca_blocks(const or_hca* H, int64_t* far_t, int64_t* far_s);
int64_t or_hca_cluster(const or_hca* H, int64_t c, int64_t* idx);
int or_hca_block(const or_hca* H, int64_t b, int32_t* tau, int32_t* sigma, double* C);
void or_hca_node(const or_hca* H, int64_t c, int nu, double* x);
double or_hca_kernel(const or_hca* H, int64_t b, const double* x, const double* y);
void or_hca_block_matrix(const or_hca* H, int64_t b, double* out);
int or_hca_basis(const or_hca* H, int64_t c, double* out);
int or_hca_transfer(const or_hca* H, int64_t c, double* out);
int or_hca_coupling(const or_hca* H, int64_t b, double* out);
void or_hca_matvec(const or_hca* H, const double* x, int nrhs, double* y, int parts, int hmatrix);

#ifdef __cplusplus
}
#endif
#endif
