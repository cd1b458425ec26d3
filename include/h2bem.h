/*
 * h2bem — H^2-matrix-vector products for the Galerkin boundary element
 * discretisation of the 3-D Laplace single-layer (G) and double-layer (K)
 * operators on one NVIDIA GB300 GPU (sm_103a).
 *
 * Problem (S. Boerm, "Fast large-scale boundary element algorithms"):
 *   section 1, eq. (slp):  g_ij = int_{tau_i} int_{tau_j} g(x,y) dy dx,
 *   section 1, eq. (dlp):  k_ij = int_{tau_i} int_{tau_j} dg/dn_y(x,y) dy dx,
 *   with g(x,y) = 1/(4 pi |x-y|), piecewise-constant basis functions
 *   psi_i = 1 on triangle tau_i (the Dirichlet basis of eq. (dlp) is taken
 *   piecewise constant as well).
 *   The matrix is approximated by an H^2-matrix (section 2, eq. (vsw)):
 *   farfield blocks G|_{t x s} ~ V_t S_ts W_s^T with tensor Chebyshev cluster
 *   bases of order m (k = m^3, section 3), nested through transfer matrices
 *   (section 2, eq. (transfer)); nearfield blocks are evaluated on the fly by
 *   a 7 x 7-point Gauss rule (regular pairs) and Sauter-Schwab quadrature
 *   (pairs sharing a vertex, sections 1 and 5), or once and stored
 *   (opts.store_near).  The hypersingular operator on continuous piecewise-
 *   linear functions is applied through its single-layer representation
 *   (h2bem_apply_hypersingular), and the Dirichlet-to-Neumann system of
 *   section 1 is solved by conjugate gradients (h2bem_apply_mass, h2bem_cg).
 *
 * Conventions (all entry points):
 *   - Every function returns an int status: H2BEM_OK (0) or one of the
 *     H2BEM_ERR_* codes.  On error nothing is written to the outputs and a
 *     message is kept for the calling thread (h2bem_last_error).
 *   - Handles are opaque.  The library copies what it needs from the caller's
 *     buffers; the caller keeps ownership of every buffer it passes.  The
 *     library owns (allocates and frees) the device memory of its handles.
 *   - Triangles are int32 vertex indices, oriented counter-clockwise seen
 *     from outside, so (b-a)x(c-a) is the outward normal (section 1).
 *   - Vectors are column-major n x nrhs with a leading dimension >= n, in the
 *     caller's triangle order (vertex order, nv x nrhs, for the hypersingular
 *     operator).
 *   - Functions that take a `stream` (a cudaStream_t, NULL = legacy default
 *     stream) enqueue their GPU work on it; unless stated otherwise they
 *     return once the work is enqueued.
 *   - Nothing runs on a CPU fallback: without a usable CUDA device every GPU
 *     entry point returns H2BEM_ERR_CUDA.
 */
#ifndef H2BEM_H
#define H2BEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define H2BEM_OK 0
#define H2BEM_ERR_ARG 1     /* invalid argument (null pointer, range, size)  */
#define H2BEM_ERR_MESH 2    /* degenerate triangle or inward orientation     */
#define H2BEM_ERR_OOM 3     /* host or device allocation failed              */
#define H2BEM_ERR_CUDA 4    /* CUDA runtime error or no usable device        */
#define H2BEM_ERR_TIMEOUT 5 /* a bounded device-side wait expired            */
#define H2BEM_ERR_STATE 6   /* handle used in a state that does not allow it */

/* ---- operator kinds and precision tiers -------------------------------- */
#define H2BEM_SLP 0 /* single layer G, eq. (slp) */
#define H2BEM_DLP 1 /* double layer K, eq. (dlp) */

#define H2BEM_FP64 0       /* every step at FP64 accuracy: FP64, or double-float    */
                           /* arithmetic on the FP32 pipe (relative error about    */
                           /* 1e-14) for the nearfield, the coupling and the       */
                           /* Sauter-Schwab points                                  */
#define H2BEM_MIXED_FP32 1 /* FP32 farfield, regular and Sauter-Schwab pairs (FP64- */
                           /* class points with opts.singular_fp64); the double    */
                           /* layer's differentiated-basis side and the            */
                           /* accumulation into y in FP64                          */
#define H2BEM_MIXED_TF32 2 /* as MIXED_FP32, coupling contraction on tensor cores  */
                           /* in TF32 with FP32 accumulation                        */
#define H2BEM_MIXED_BF16 3 /* as MIXED_TF32 with BF16 operands                      */

/* cluster bases of the farfield (h2bem_opts.basis) */
#define H2BEM_BASIS_CHEBYSHEV 0 /* tensor Chebyshev interpolation of order m (section 3) */
#define H2BEM_BASIS_GCA 1       /* Green cross approximation (section 4)                 */
#define H2BEM_BASIS_HCA 2       /* hybrid cross approximation, compressed to H^2 (section 3) */

typedef struct h2bem_mesh h2bem_mesh;
typedef struct h2bem_tree h2bem_tree;
typedef struct h2bem_op h2bem_op;

/* Options of an operator.  Obtain defaults with h2bem_opts_default. */
typedef struct {
    int q_ss;           /* Gauss points per direction of the Sauter-Schwab rules (1..16, default 5) */
    int precision;      /* H2BEM_FP64 (default) or a MIXED tier                                    */
    int cache_singular; /* 1: evaluate the x-independent singular entries once at set-up and       */
                        /*    keep them in device memory (about 13 doubles per triangle); 0: on    */
                        /*    the fly in every apply (default)                                     */
    int use_graph;      /* 1: h2bem_apply / h2bem_apply_transpose with device buffers on a         */
                        /*    non-default stream replay a captured CUDA graph of their launch      */
                        /*    sequence when called again with the same buffers, sizes and          */
                        /*    direction (the second such call captures it); 0: plain launches     */
    int autotune;       /* 1: the first apply with a given right-hand-side width and direction    */
                        /*    times the launch variants of the regular nearfield (one CTA per     */
                        /*    row leaf, or persistent CTAs taking rows from a work counter; the  */
                        /*    register budget) and                                                 */
                        /*    of the SIMT coupling (2, 4 or 8 slices per CTA, one CTA per row or  */
                        /*    persistent) on the operator's own data and keeps the fastest; the   */
                        /*    variants sum in different orders, so results differ by rounding.    */
                        /*    No tuning while the stream is being captured.  0: defaults (one     */
                        /*    CTA per row, 4 slices).  2 + v (v = 0..35) fixes a variant:         */
                        /*    v = nearfield persistent + 2 coupling persistent + 4 i + 12 j,     */
                        /*    where i = 0, 1, 2 selects 2, 4, 8 slices and j = 0, 1, 2 a          */
                        /*    nearfield register budget for 4, 3, 2 CTAs per SM (FP32 single     */
                        /*    layer)                                                               */
    int singular_fp64;  /* 1: Sauter-Schwab quadrature points of pairs sharing a vertex at FP64-    */
                        /*    class accuracy in every tier (double-float arithmetic on the FP32   */
                        /*    pipe, relative error about 1e-14 per point; the area scale and the  */
                        /*    accumulation into y in FP64), as the FP64 tier always does; 0       */
                        /*    (default): FP32 points and sums in the MIXED tiers, FP64 area scale */
                        /*    and accumulation                                                      */
    int recompute_basis; /* 1: no stored leaf bases; every apply re-evaluates the cluster-basis   */
                        /*    values by quadrature (saves n k values of device memory); 0         */
                        /*    (default): V (and W) evaluated once at set-up and stored             */
    int store_near;     /* 1: evaluate every nearfield entry once at set-up (regular pairs and     */
                        /*    Sauter-Schwab pairs, in the tier's working precision: FP32 in the    */
                        /*    MIXED tiers, FP64 in H2BEM_FP64) and keep the nearfield blocks in    */
                        /*    device memory (stats.near_stored_bytes, about near_pairs values);    */
                        /*    every apply then streams them instead of evaluating the quadrature. */
                        /*    The nearfield sum of each row is formed by one CTA without atomics. */
                        /*    0 (default): nearfield on the fly in every apply                     */
    int basis;          /* H2BEM_BASIS_CHEBYSHEV (default) or H2BEM_BASIS_GCA: cluster bases by   */
                        /*    Green cross approximation (section 4) for the single layer in the   */
                        /*    FP64 and MIXED_FP32 tiers.  For every cluster t, Green's             */
                        /*    representation formula on the box omega_t (B_t grown by its largest  */
                        /*    side on every side, section 5) is discretised by gca_q x gca_q       */
                        /*    Gauss points on each face; adaptive cross approximation of the       */
                        /*    matrix L = (A C) of the potentials of the rows (the triangles of a   */
                        /*    leaf, the children's pivot triangles otherwise) picks pivot          */
                        /*    triangles t^ and gives V^_t = L|sigma (L|tau,sigma)^-1: the leaf     */
                        /*    basis of a leaf, the transfer matrices of the children otherwise     */
                        /*    (eq. (transfer)).  The coupling matrices are the Galerkin entries    */
                        /*    G|_{t^ x s^} (7 x 7-point rule), evaluated once at set-up and stored */
                        /*    in the tier's precision; the interpolation order m is then unused    */
                        /*    for the farfield.  The construction runs on the host (OpenMP).       */
    int gca_q;          /* GCA: Gauss points per face axis (1..16, default 4; 6 q^2 points)        */
    int gca_kmax;       /* GCA: largest rank of a cluster (1..64, default 64)                      */
    int tc_wait_test;   /* 0 (default).  1, for tests of the fault path only: in the tensor-core   */
                        /*    coupling the first pipeline wait of every CTA with three or more     */
                        /*    blocks waits on a barrier that nothing signals, with a bound of      */
                        /*    about 50 us, so that it expires; the CTA then drains what it issued */
                        /*    (normal bound), frees its tensor memory and returns, and the apply   */
                        /*    reports H2BEM_ERR_TIMEOUT (its result is invalid)                   */
    double gca_eps;     /* GCA: ACA stops when a pivot falls to gca_eps times the first            */
                        /*    (>= 0, default 1e-6)                                                 */
    /* basis = H2BEM_BASIS_HCA (single layer; FP64 and MIXED_FP32 tiers): for every farfield   */
    /* block (t, s) the coupling matrix S = g(xi_t, xi_s) of the order-m Chebyshev nodes is     */
    /* cross-approximated with full pivoting, S ~ S|sigma C S|tau with C = (S|tau,sigma)^-1,  */
    /* and the interpolation "taken back": G|t x s ~ A C B^T with A = int g(x, xi_s,sigma),    */
    /* B = int g(xi_t,tau, y) (eq. (hca_discrete), 7-point rule).  The blocks are then         */
    /* compressed into orthonormal nested cluster bases Q_t (truncated singular vectors of    */
    /* the block rows of t and its ancestors, from the leaves up) with couplings               */
    /* Q_t^T A C B^T Q_s, stored in the tier's precision; the transposed apply uses stored     */
    /* transposed couplings (the HCA matrix is not exactly symmetric).  Host construction    */
    /* (OpenMP); its cost grows as n log n times the blocks per cluster row.                 */
    int hca_kaca;       /* HCA: most cross-approximation steps per block (>= 1, at most m^3 are   */
                        /*    taken; default 64)                                                   */
    int hca_kmax;       /* HCA: largest rank of a compressed cluster basis (1..64, default 64)     */
    double hca_eps_aca; /* HCA: a block's cross approximation stops when a pivot falls to          */
                        /*    hca_eps_aca times the first (>= 0, default 1e-6)                     */
    double hca_eps;     /* HCA: compression keeps the singular values above hca_eps times the      */
                        /*    largest of each cluster's block row (>= 0, default 1e-6)             */
} h2bem_opts;

/* Statistics of an operator (counts are exact, from its own block lists). */
typedef struct {
    int64_t n;                 /* triangles                                   */
    int64_t nclusters, nleaves, depth;
    int64_t nfar, nnear;       /* farfield / nearfield blocks                 */
    int64_t near_pairs;        /* triangle pairs in nearfield blocks          */
    int64_t regular_pairs;     /* of which share no vertex (7 x 7 rule)       */
    int64_t singular_pairs[3]; /* canonical pairs: identical, edge, vertex    */
    int64_t k;                 /* interpolation points per cluster, m^3       */
    int64_t launches;          /* kernels launched by the last apply          */
    double last_apply_ms;      /* device time of the last timed apply         */
    double stage_ms[8];        /* per stage of the last timed apply, see      */
                               /* h2bem_apply_timed                            */
    int64_t launch_variant[5]; /* of the last apply: regular nearfield         */
                               /* persistent (0/1), regular nearfield CTAs per */
                               /* SM of its register budget (4, 3, 2), SIMT    */
                               /* coupling slices per CTA, SIMT coupling       */
                               /* persistent (0/1), 1 if chosen by the         */
                               /* autotuner or fixed through opts.autotune     */
    int64_t regular_evals;     /* pairs the regular nearfield kernel          */
                               /* evaluates per apply (49 kernel evaluations   */
                               /* each): every pair of the blocks (t, s >= t)  */
                               /* sharing no vertex, both orders when s = t;   */
                               /* its result serves (t, s) and (s, t)          */
    int64_t near_stored_bytes; /* device bytes of the stored nearfield blocks */
                               /* (opts.store_near), else 0                    */
    int64_t far_stored_bytes;  /* device bytes of stored farfield matrices     */
                               /* (GCA: coupling and transfer matrices; HCA:   */
                               /* also the transposed couplings)               */
    double mean_rank;          /* GCA, HCA: mean rank over the clusters; else k */
} h2bem_stats;

/* Message of the last failed call on the calling thread (empty if none).
 * Writes at most len bytes including the terminating zero; returns H2BEM_OK. */
int h2bem_last_error(char* buf, size_t len);

/* ---- mesh (host only) ---------------------------------------------------- */
/* Copies a surface mesh (section 1: index set of panels tau_i).
 *   xyz: nv x 3 doubles (row per vertex); tri: nt x 3 int32 vertex indices.
 * Errors: H2BEM_ERR_ARG for null pointers, nv < 3, nt < 1 or an index out of
 * range; H2BEM_ERR_MESH if a triangle has zero area or the signed enclosed
 * volume sum_i a_i.(b_i x c_i)/6 is not positive (triangles inward). */
int h2bem_mesh_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, h2bem_mesh** out);
int h2bem_mesh_destroy(h2bem_mesh* mesh);

/* ---- cluster tree (host only; section 2, Definition "cluster tree") ------ */
/* Builds the cluster tree by bounding-box bisection: box = bounding box of
 * the vertices of the cluster's triangles (section 3: supp psi_i in B_t);
 * split while |t| > leaf_size along the longest axis (lowest axis on ties) at
 * the box midpoint, by triangle centroid (< midpoint to the first child, in
 * the current order); a stable median split if one side would be empty.
 * Clusters are numbered in depth-first pre-order.  leaf_size >= 1. */
int h2bem_tree_build(const h2bem_mesh* mesh, int leaf_size, h2bem_tree** out);
/* Takes a caller-made cluster tree: perm[n] (tree position -> triangle),
 * begin/end[nclusters] (ranges of tree positions), child0/child1[nclusters]
 * (-1 = none; a cluster has no child or two).  Cluster 0 is the root; each
 * child's range is the matching half of its parent's.  Boxes are recomputed.
 * Errors: H2BEM_ERR_ARG if the arrays do not describe such a tree. */
int h2bem_tree_upload(const h2bem_mesh* mesh, int64_t nclusters, const int64_t* perm, const int64_t* begin,
                      const int64_t* end, const int64_t* child0, const int64_t* child1, h2bem_tree** out);
/* Counts; any output pointer may be NULL. */
int h2bem_tree_info(const h2bem_tree* tree, int64_t* nclusters, int64_t* nleaves, int64_t* depth);
/* Copies the tree out (arrays sized as in h2bem_tree_upload; bmin/bmax are
 * nclusters x 3).  Any pointer may be NULL. */
int h2bem_tree_export(const h2bem_tree* tree, int64_t* perm, int64_t* begin, int64_t* end, int64_t* child0,
                      int64_t* child1, double* bmin, double* bmax);
int h2bem_tree_destroy(h2bem_tree* tree);

/* ---- block tree (host only; section 2, Definition "block tree") ---------- */
/* Farfield and nearfield leaves from (root, root): farfield if dist > 0 and
 * max(diam B_t, diam B_s) <= eta dist(B_t, B_s) (section 3,
 * eq. (admissibility) with the factor 2 folded into eta); nearfield if both
 * clusters are leaves; else subdivide per the block-tree definition.
 * Call with NULL arrays to get the counts, then with arrays of those sizes.
 * eta >= 0 (eta = 0: everything nearfield). */
int h2bem_blocks(const h2bem_tree* tree, double eta, int64_t* nfar, int64_t* nnear, int64_t* far_t, int64_t* far_s,
                 int64_t* near_t, int64_t* near_s);

/* ---- Green cross approximation (host only; section 4) -------------------- */
/* The GCA cluster bases that h2bem_operator_create builds with opts->basis =
 * H2BEM_BASIS_GCA (gca_q, gca_kmax, gca_eps of opts; the other fields are
 * ignored), for inspection: rank[c] for every cluster (nclusters values) and
 * the pivot triangles of every cluster as tree positions, cluster by cluster
 * in pivot order (npiv = the sum of the ranks).  Any output may be NULL; call
 * with piv = NULL to get npiv first.  Errors: ARG (NULL mesh, tree or opts,
 * sizes, gca_q, gca_kmax, gca_eps). */
int h2bem_gca_bases(const h2bem_mesh* mesh, const h2bem_tree* tree, const h2bem_opts* opts, int64_t* rank,
                    int64_t* npiv, int64_t* piv);

/* ---- hybrid cross approximation (host only; section 3) -------------------- */
/* The ranks of the HCA construction that h2bem_operator_create builds with
 * opts->basis = H2BEM_BASIS_HCA for the single layer with interpolation order
 * m and admissibility eta (hca_* fields of opts; the others are ignored):
 * rank[c] of the compressed basis of every cluster (nclusters values) and
 * brank[b] of the cross approximation of every farfield block, in the order
 * of h2bem_blocks (nfar values).  Any output may be NULL.  Errors: ARG (NULL
 * mesh, tree or opts, sizes, m, eta, hca_* fields). */
int h2bem_hca_ranks(const h2bem_mesh* mesh, const h2bem_tree* tree, int m, double eta, const h2bem_opts* opts,
                    int64_t* rank, int64_t* nfar, int64_t* brank);

/* ---- operator -------------------------------------------------------------- */
int h2bem_opts_default(h2bem_opts* opts);
/* Selects G (H2BEM_SLP) or K (H2BEM_DLP), interpolation order m (1..6,
 * k = m^3, section 3) and admissibility eta; builds the block lists and
 * uploads mesh, tree and lists to the current CUDA device.  opts may be NULL
 * (defaults).  Synchronous.  Errors: ARG (kernel, m, eta, opts; GCA or HCA
 * bases with the double layer, a tensor-core tier or recompute_basis), OOM,
 * CUDA. */
int h2bem_operator_create(const h2bem_mesh* mesh, const h2bem_tree* tree, int kernel, int m, double eta,
                          const h2bem_opts* opts, h2bem_op** out);
/* Many meshes as one operator (batching).  Builds the block-diagonal operator
 * diag(A_1, ..., A_B) over the concatenation of the meshes, in the order given:
 * triangle i of mesh b is index off_b + i with off_b = sum of the earlier
 * meshes' triangle counts.  Each mesh gets its own cluster tree (as
 * h2bem_tree_build with leaf_size) and its own block tree from its own root
 * (section 2, Definitions "cluster tree" and "block tree"; no block couples two
 * meshes), so A_b equals the operator h2bem_operator_create builds for mesh b
 * alone.  Every stage of h2bem_apply on the result is then a single launch
 * over all meshes.  The meshes are copied; the caller keeps ownership.
 * Errors: as h2bem_operator_create; ARG if nmeshes < 1 or a mesh is NULL. */
int h2bem_batch_create(int nmeshes, const h2bem_mesh* const* meshes, int leaf_size, int kernel, int m, double eta,
                       const h2bem_opts* opts, h2bem_op** out);
int h2bem_operator_destroy(h2bem_op* op);
/* Counts and the launch variants of the last apply; after h2bem_apply_timed
 * waits for its events and adds their stage times.  Errors: ARG (NULL),
 * CUDA, TIMEOUT (see h2bem_apply_timed). */
int h2bem_stats_get(const h2bem_op* op, h2bem_stats* stats);

/* y = A x (A = G or K in its H^2 approximation; section 2, eq. (vsw) for the
 * farfield, eq. (slp)/(dlp) quadrature for the nearfield).
 *   x: n x nrhs, leading dimension ldx >= n; y: n x nrhs, ldy >= n; both in
 *   the caller's triangle order; 1 <= nrhs <= 64.  x and y may each be
 *   device or host memory (detected per pointer); they must not overlap.
 *   With device buffers the call is asynchronous on `stream`; with a host
 *   buffer it synchronises the stream before returning.  Page-locked host
 *   memory that is mapped into the device's address space (cudaHostAlloc,
 *   cudaHostRegister) is read and written in place by the kernels, in the
 *   caller's order; other host memory is copied through device scratch.
 * Scratch device memory is allocated on the first call and grown when nrhs
 * grows; concurrent applies of one operator on different streams race on it
 * and on the operator's per-cluster arrival counts of the upward pass, so
 * order the applies of one operator (one stream, or events between them).
 * Errors: ARG (null, nrhs, ld), CUDA, OOM. */
int h2bem_apply(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy, void* stream);
/* y = A^T x, same conventions (transposed blocks, V and W exchanged). */
int h2bem_apply_transpose(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy,
                          void* stream);
/* Shape gradient of the single or double layer (section 1, eq. (slp) /
 * eq. (dlp), in their H^2 form of section 2, eq. (vsw)): dxyz[3 v + d] =
 * d/dX_{v,d} sum_r <w_r, A(X) x_r>, A = G or K, the derivative with respect
 * to vertex coordinate d of vertex v with the cluster tree and the block
 * lists held fixed.  It runs through the nearfield quadrature (7-point rule
 * and Sauter-Schwab, areas included; for K also the source triangles' normals
 * through their area-normals), the leaf bases (for K the column basis
 * W = int n . grad L through the Hessian of the Lagrange polynomials), the
 * transfer and coupling matrices and, through the Chebyshev nodes, the
 * cluster boxes (centre and floored half-width, section 3) down to the
 * vertices realising the box extremes.  FP64 in every precision tier.
 *   w, x: n x nrhs (leading dimension ld >= n), 1 <= nrhs <= 64;
 *   dxyz: nv x 3 output (overwritten);
 *   dx: optional (NULL to skip) n x nrhs output (ld) = A^T w = d/dx, by
 *   h2bem_apply_transpose in the operator's tier.
 * All buffers device memory; asynchronous on `stream`.  Work vectors are
 * allocated on the first call.  Errors: ARG (NULL, GCA or HCA bases, nrhs,
 * ld, host pointers), CUDA, OOM. */
int h2bem_grad(h2bem_op* op, const double* w, const double* x, int64_t ld, int nrhs, double* dxyz, double* dx,
               void* stream);
/* y = W x, the hypersingular operator on continuous piecewise-linear
 * functions (section 1: w_ij = -int phi_i d/dn_x int dg/dn_y phi_j, hat
 * functions phi_j of the mesh vertices), through its single-layer
 * representation, which section 1 uses to set W up:
 *   W = sum_{d=1..3} C_d^T G C_d,  (C_d)_{tau j} = (curl phi_j |_tau)_d,
 * curl phi = n x grad phi, constant on each triangle tau = (a, b, c):
 * curl phi_a = (b - c) / (2 |tau|) and cyclically.  G is this operator, which
 * must be a single layer (H2BEM_SLP); one call applies it to 3 nrhs columns
 * in its own tier.  x, y: device, nv x nrhs, leading dimensions ldx, ldy >= nv,
 * the caller's vertex order (the vertices of h2bem_mesh_create; for a batch
 * operator the concatenated vertices).  W annihilates constants.
 * Asynchronous on `stream`; work vectors (2 x 3 n nrhs doubles) are kept by
 * the operator.  Errors: ARG (NULL, double-layer operator, nrhs < 0, ld, host
 * pointers), CUDA, OOM. */
int h2bem_apply_hypersingular(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy,
                              void* stream);
/* The double layer with continuous piecewise-linear trial functions (section 1,
 * eq. (dlp) with phi_v the hat functions of the vertices; the Dirichlet basis
 * of the paper's experiments, section 5):
 *   (K1)_{i v} = int_{tau_i} int dg/dn_y(x, y) phi_v(y) dy dx,
 * rows the triangles, columns the vertices.  Per pair of triangles the trial
 * function is the barycentric coordinate of a corner of the source panel, so
 * the H^2 form keeps the operator's tree, blocks, transfers, coupling and
 * output basis V and takes per-corner source bases W1_c = int n . grad L
 * lambda_c; regular nearfield pairs use the 7 x 7-point rule with lambda_c at
 * the source points, pairs sharing a vertex the full Sauter-Schwab tensor
 * rule (q_ss points per direction) with the same factors.  op must be a
 * double-layer operator (H2BEM_DLP) with stored leaf bases.  The K1-specific
 * parts (corner bases, nearfield and singular values) are FP64 in every tier;
 * the passes follow the operator's tier.  The first call evaluates the corner
 * bases and the singular values (synchronous); later calls are asynchronous.
 *   transpose = 0: y = K1 x + alpha M1 x, x on the vertices (nv x nrhs,
 *                  ldx >= nv, the vertex order of h2bem_mesh_create), y on the
 *                  triangles (n x nrhs, ldy >= n, the caller's triangle order);
 *   transpose = 1: y = K1^T x + alpha M1^T x, x on the triangles, y on the
 *                  vertices;
 * M1 is the P0 x P1 mass matrix, (M1)_{i v} = int_{tau_i} phi_v = |tau_i| / 3
 * for the corners v of tau_i (alpha = -1/2 with x = -b gives the right-hand
 * side (M1^T/2 - K1^T) b of the Neumann-to-Dirichlet system of section 1).
 * 1 <= nrhs <= 64; device buffers.  Errors: ARG (NULL, kernel, recompute_basis,
 * nrhs, ld, host pointers), CUDA, OOM. */
int h2bem_apply_dlp_p1(h2bem_op* op, double alpha, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy,
                       int transpose, void* stream);
/* y = A x + alpha M x with the P0 mass matrix M = diag(|tau_i|) (section 1,
 * the mass matrix m_ij of eq. (matrix_dtn) with piecewise-constant columns).
 * With A = K and alpha = 1/2 this is the right-hand side (M/2 + K) b of the
 * Dirichlet-to-Neumann system G x = (M/2 + K) b.  x, y: device, n x nrhs,
 * leading dimensions ldx, ldy >= n, caller's triangle order; asynchronous on
 * `stream`.  Errors: as h2bem_apply; ARG for host pointers. */
int h2bem_apply_mass(h2bem_op* op, double alpha, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy,
                     void* stream);
/* Conjugate gradients for G x = b (G the single layer, symmetric positive
 * definite; section 1, eq. (matrix_dtn) for the Dirichlet-to-Neumann
 * problem), every column an independent system: x0 = 0, stop when
 * |b - G x| <= rtol |b| for every column or after maxit iterations.  G is
 * applied in the operator's tier; the iteration runs in FP64.
 *   b: device n x nrhs (ldb >= n); x: device n x nrhs output (ldx >= n);
 *   iters (host, may be NULL): iterations done; relres (host, may be NULL,
 *   nrhs values): final |r| / |b| per column (the recurrence residual).
 * Synchronises `stream` in every iteration (the step lengths are host
 * scalars).  Work vectors are allocated on the first call.
 * Errors: ARG (NULL, double-layer operator, nrhs, ld, rtol <= 0, maxit < 0,
 * host pointers), CUDA, OOM. */
int h2bem_cg(h2bem_op* op, const double* b, int64_t ldb, int nrhs, double* x, int64_t ldx, double rtol, int maxit,
             int* iters, double* relres, void* stream);
/* Conjugate gradients for (W + m m^T) x = b, W the hypersingular operator on
 * continuous piecewise-linear functions applied through this single layer
 * (h2bem_apply_hypersingular; section 1), m a vector on the vertices (for
 * example the integrals of the hat functions) or NULL.  W is symmetric
 * positive semi-definite and annihilates constants (on a closed surface); the
 * rank-one term m m^T with m . 1 != 0 makes the system definite.  Summing the
 * equations gives (m . 1)(m . x) = 1 . b, so for data b = c + mu m with
 * 1 . c = 0 (the right-hand side of a compatible system plus a multiple of m)
 * the solution has m . x = mu: the constant that W leaves free (the
 * Neumann-to-Dirichlet system W x = (M1^T/2 - K1^T) b of section 1 needs such
 * a condition).  Every column is an independent system; x0 = 0; stop when
 * |b - A x| <= rtol |b| or after maxit iterations.
 *   m: device, nv values (or NULL); b, x: device, nv x nrhs (ldb, ldx >= nv);
 *   iters, relres as for h2bem_cg.
 * Synchronises `stream` in every iteration.  Errors: ARG (NULL, double-layer
 * operator, nrhs, ld, rtol, maxit, host pointers), CUDA, OOM. */
int h2bem_cg_hypersingular(h2bem_op* op, const double* m, const double* b, int64_t ldb, int nrhs, double* x,
                           int64_t ldx, double rtol, int maxit, int* iters, double* relres, void* stream);
/* As h2bem_apply with device buffers only, and records CUDA events around
 * each stage on `stream` (asynchronous: no host wait, so timed applies can run
 * back to back).  The next h2bem_stats_get waits for the last of them and
 * fills stage_ms and last_apply_ms of that apply:
 * [0] permute in, [1] leaf forward, [2] upward, [3] coupling, [4] downward,
 * [5] leaf backward, [6] nearfield regular (with opts.store_near: the stored
 * nearfield, which runs right after [0]), [7] nearfield singular.
 * h2bem_stats_get then also reports an expired bounded wait of the
 * tensor-core coupling (TIMEOUT); for operators of the tensor-core tiers it
 * reports one of any completed apply. */
int h2bem_apply_timed(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy, void* stream);

/* Allocation-free y = A x (the paper has no counterpart: this is a service
 * for callers of this library).  Same arguments and result as h2bem_apply,
 * for callers that cannot let the library allocate device memory when they
 * apply the operator: h2bem_apply allocates its work vectors with cudaMalloc
 * on its first call, which fails or stalls for a caller whose device memory
 * is all held by its own pool allocator, or who must not trigger the device
 * synchronisation a cudaMalloc/cudaFree may imply.  This call allocates
 * nothing: its work vectors live in a fixed 64 MiB array inside the library,
 * present on every GPU that loads the library until the process exits.
 *   - x and y must be device memory of the current device (no host
 *     staging); they must not overlap.  The operator must have been created
 *     with that device current.
 *   - The work space needed is 2 n NRp 8 + 2 nclusters k NRp e + n nx b
 *     bytes, every term rounded up to a multiple of 256.  NRp is min(nrhs,16)
 *     rounded up to 1, 4, 8 or 16; e = 8 for the FP64 tier or the double
 *     layer, else 4.  The last term is x in the stored nearfield's precision
 *     or in FP32 for the regular nearfield and the singular row gather:
 *     b = 4, nx = max(NRp, 4) in the MIXED tiers (for the double layer
 *     without opts.store_near only unless opts.singular_fp64 is set);
 *     b = 8, nx = 2 in the FP64 tier with opts.store_near and NRp = 1; else
 *     0.  An operator that needs more than 64 MiB is rejected with
 *     H2BEM_ERR_ARG (use h2bem_apply).
 *   - The first call on a device looks up the array's device address (once,
 *     with that device current); make that first call before any stream
 *     capture.
 *   - All calls share the one array and the work vectors it holds are
 *     overwritten by every call: calls that may overlap on the GPU (on
 *     different streams, or from different threads without ordering) race
 *     and give wrong results.  Calls on one stream are ordered and safe.
 *   - Enqueued on `stream`; returns once the work is enqueued.  The launch
 *     sequence is h2bem_apply's (without autotuning: the launch variants are
 *     those an earlier h2bem_apply tuned, else the defaults).  An expired
 *     bounded wait of the tensor-core coupling is reported, as for
 *     h2bem_apply_timed, by the next h2bem_stats_get (H2BEM_ERR_TIMEOUT).
 * Errors: ARG (null, nrhs, ld, host pointers or another device's memory,
 * work space too large), CUDA. */
int h2bem_apply_noalloc(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy, void* stream);

#ifdef __cplusplus
}
#endif
#endif
