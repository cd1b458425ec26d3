// Internal declarations shared by the host set-up (api.cpp) and the CUDA
// kernels of libh2bem.  Not part of the public C ABI (include/h2bem.h).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace h2 {

constexpr int kMaxM = 6;             // interpolation order (k = m^3 <= 216)
constexpr int kMaxK = kMaxM * kMaxM * kMaxM;
constexpr int kMaxLeaf = 64;         // largest leaf cluster the kernels stage
constexpr int kMaxBasisPts = 128;    // points of the leaf-basis triangle rule
constexpr int kMaxQss = 8;           // Gauss points per singular direction

enum Kernel { SLP = 0, DLP = 1, DLP_T = 2 };  // DLP_T: rows of K^T (normal at the row triangle)
enum SingType { IDENTICAL = 3, EDGE = 2, VERTEX = 1 };

// Triangles in tree order, structure of arrays.
struct Geom {
    int n;
    const double* v;     // [9][n]: coordinate d of corner c at v[(3c+d)*n + i]
    const double* area;  // [n]
    const double* nrm;   // [3][n] outward unit normal
    const double* ctr;   // [3][n] centroid
    const int* vid;      // [3][n] vertex indices (singular-pair test)
    // nearfield quadrature data (x-independent, computed with the geometry):
    const float* qo;     // [3][n][7] FP32 offsets y_q - c of the 7-point rule's points
    const double* qa;    // [3][n][7] FP64 points y_q
    const float* chl;    // [6][n] centroid split: hi = fl(c) (rows 0..2), lo = fl(c - hi) (rows 3..5)
    const double* plane; // [n] c . n (offset of the triangle's plane)
    const float* nef;    // [18][n] FP32: normal hi (0..2) and lo = fl(n - hi) (3..5), edges E1 = b - a (6..8),
                         // E2 = c - a (9..11), each rounded from FP64, and their low parts fl(E - hi)
                         // (12..14, 15..17)
    const float* areaf;  // [n] area rounded to FP32
};

// Cluster tree on the device.
struct Tree {
    int nc;
    const int* begin;    // [nc] first tree position
    const int* end;      // [nc] one past the last
    const int* child0;   // [nc] -1 for leaves
    const int* child1;
    const double* box;   // [9][nc]: centre x,y,z, (floored) half-width x,y,z, 1/half-width x,y,z
    const float2* zhl;   // [nc][3][m] interpolation node coordinates c_d + h_d cheb[a] as FP32 (hi, lo):
                         // hi = fl(z), lo = fl(z - hi)
    const float* etr;    // [nc][3][m][m] FP32 transfer factors of each non-root cluster c to its parent p:
                         // E[d][a'][a] = L_{p,a}^{(d)}(z_{c,d}[a']), evaluated in FP64 and rounded once
};

// Quadrature and interpolation constants passed by value.
struct Consts {
    int m, k;
    double cheb[kMaxM];          // cos((2a+1) pi / (2m)), a = 0..m-1
    double bary[kMaxM];          // 1 / prod_{b != a} (cheb[a] - cheb[b]) (reference-interval Lagrange weights)
    float cheb_hi[kMaxM];        // float split of cheb: cheb = hi + lo
    float cheb_lo[kMaxM];
    double ru[7], rv[7], rw[7];  // Radon 7-point rule on the unit simplex, weights sum to 1
    float rwf[7], ruf[7], rvf[7];  // the same in FP32: weights, u - 1/3, v - 1/3
    int nb;                      // points of the leaf-basis rule
};

// Launch variant of a row-parallel kernel: work != nullptr runs persistent
// CTAs (as many as fit on the GPU) that take rows from the counter *work
// (reset by the launcher); nsl = slices of the SIMT coupling (2, 4 or 8).
struct LaunchCfg {
    int nsl = 4;
    int* work = nullptr;
    int nb = 0;  // regular nearfield (FP32 single layer): CTAs per SM of the register budget (0: 4)
};
// CTAs of `func` resident on the whole GPU at once (occupancy x SMs)
int resident_ctas(const void* func, int threads, size_t smem);

// ---- Green cross approximation (gca.cpp, k_gca.cu) -----------------------
// Inputs of the host construction of the GCA cluster bases: mesh, cluster
// tree (tree positions; boxes nc x 3), the Gauss-Legendre rule on [0, 1] with
// q points for the faces of d omega_t, the 7-point rule (u, v, weight), the
// ACA tolerance and the largest rank.
struct GcaSetup {
    const double* xyz;
    const int32_t* tri;
    int64_t n, nc;
    const int64_t *perm, *begin, *end, *child0, *child1, *level;
    const double *bmin, *bmax;
    int q, kmax;
    double eps;
    const double *gl_x, *gl_w;
    const double *ru, *rv, *rw;
};
// Result: rank per cluster; pivot tree positions (CSR piv_off / piv, pivot
// order); leaf bases V (|t| x rank_t row-major, rows in tree order) at voff[t];
// transfer matrices E_c (rank_c x rank_parent row-major) at eoff[c]; -1 where
// absent.
struct GcaResult {
    std::vector<int> rank, piv_off, piv;
    std::vector<int64_t> voff, eoff;
    std::vector<double> V, E;
};
int gca_build(const GcaSetup& setup, GcaResult& result);
constexpr int kGcaMaxRank = 64;  // largest GCA rank the kernels stage
// full-pivot cross approximation of the rows x cols matrix A (row-major,
// destroyed): the pivot is the first entry in row-major order within a
// relative 2^-40 of the largest residual entry; stop at rank kmax, at a zero
// residual or when the pivot falls to eps times the first; row pivots tau,
// column pivots sigma; returns the rank (gca.cpp)
int cross_approx(std::vector<double>& A, int rows, int cols, double eps, int kmax, std::vector<int>& tau,
                 std::vector<int>& sigma);
// Hybrid cross approximation (section 3) of the single layer and its
// compression into an H^2-matrix (hca.cpp): the tree as for GcaSetup, the
// interpolation order m of the blocks' node grids, the farfield blocks
// (far_t, far_s) in the order the coupling matrices are returned, the cross
// approximation tolerance / step limit, the compression tolerance / rank cap
// and the 7-point rule
struct HcaSetup {
    const double* xyz;
    const int32_t* tri;
    int64_t n, nc;
    const int64_t *perm, *begin, *end, *child0, *child1, *level;
    const double *bmin, *bmax;
    int m, kaca, kmax;
    double eps_aca, eps_c;
    const double *ru, *rv, *rw;
    int64_t nfar;
    const int *far_t, *far_s;
};
// Result: rank per cluster and per block; leaf bases Q (|t| x rank_t
// row-major, rows in tree order) at voff[t]; transfers E_c (rank_c x
// rank_parent) at eoff[c] (-1 where absent); coupling S_b (rank_t x rank_s)
// at soff[b]
struct HcaResult {
    std::vector<int> rank, brank;
    std::vector<int64_t> voff, eoff, soff;
    std::vector<double> V, E, S;
};
int hca_build(const HcaSetup& setup, HcaResult& result);
// coupling matrices S_b = G|_{t^ x s^} of the farfield CSR (rows / ptr / col)
// at element offsets soff[b], FP64 quadrature stored as FP32 (f32) or FP64
void launch_gca_assemble(const Geom& g, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                         const int* rank, const int* piv_off, const int* piv, const int64_t* soff, bool f32, void* S,
                         cudaStream_t s);
// one tree level: x-hat_p = sum_c E_c^T x-hat_c (up) or y-hat_c += E_c y-hat_p
void launch_gca_updown(bool up, bool f32, int NR, int np, const int* parents, const int* child0, const int* child1,
                       const int* rank, const int64_t* eoff, const void* E, int K, void* v, cudaStream_t s);
// y-hat_t = sum_b S_b x-hat_s over the farfield blocks of every row t
void launch_gca_coupling(bool f32, int NR, int nrows, const int* rows, const int* ptr, const int* col,
                         const int* rank, const int64_t* soff, const void* S, int K, const void* xh, void* yh,
                         cudaStream_t s);

// ---- double layer with piecewise-linear trial functions (k_p1.cu) --------
// corner gather x3[(c n + pos) NR + r] = x[vid_c(pos) + r ldx]; vertex sum of
// y3 (same layout) into y; regular nearfield over the ordered blocks (forward:
// y += K1 x from x3; transposed: y3 += from x in tree order); Sauter-Schwab
// values (6 per canonical edge / vertex pair) and their application
void launch_p1_gather(int n, int NR, int nrhs, const int* vid, const double* x, int64_t ldx, double* x3,
                      cudaStream_t s);
void launch_p1_scatter(int nv, int n, int NR, int nrhs, const int* vptr, const int* inc, const int* iperm,
                       const double* y3, double* y, int64_t ldy, cudaStream_t s);
// fp32: the mixed tiers' FP32 kernel (off unused), else double-float (FP64 tier)
void launch_p1_near(bool transpose, bool fp32, int NR, const Geom& g, const Tree& t, const Consts& c, int nrows,
                    const int* rows, const int* ptr, const int* col, const float* off, const double* xin,
                    double* yout, cudaStream_t s);
// point offsets from the centroid as float pairs ([6][n][7]: hi, then lo) for launch_p1_near
void launch_p1_offsets(int n, const double* qa, const double* ctr, float* off, cudaStream_t s);
void launch_p1_sing_eval(const Geom& g, int np, const int* lo, const int* hi, const int* code, const double* tab,
                         int npts, double* vals, cudaStream_t s);
void launch_p1_sing_apply(bool transpose, int n, int np, int NR, const int* lo, const int* hi, const int* code,
                          const double* vals, const double* xin, double* yout, cudaStream_t s);
void launch_p1_mass(bool transpose, int n, int NR, double alpha, const double* area, const double* xin, double* yout,
                    cudaStream_t s);
void launch_leaf_forward_stored_acc(const Tree& t, int k, int max_leaf, int nleaves, const int* leaves, bool xh64,
                                    int NR, const double* B, const double* xp, void* xh, cudaStream_t s);

// ---- launchers (stream-ordered; no synchronisation) -----------------------
void launch_geom(const double* xyz, const int* tri, const int* perm, int n, const Consts& c, double* v, double* area,
                 double* nrm, double* ctr, int* vid, float* qo, double* qa, float* chl, double* plane, float* nef,
                 float* areaf, cudaStream_t s);
void launch_permute_in(const double* x, int64_t ldx, int nrhs, int NR, const int* perm, int n, double* xp,
                       cudaStream_t s);
// the same, reading x in the caller's order and scattering through iperm
// (for x in mapped host memory: coalesced reads over the host link)
void launch_permute_in_scatter(const double* x, int64_t ldx, int nrhs, int NR, const int* iperm, int n, double* xp,
                               cudaStream_t s);
void launch_permute_out(const double* yp, int NR, int nrhs, const int* iperm, int n, double* y, int64_t ldy,
                        cudaStream_t s);

// nearfield, regular pairs, each unordered pair of leaves {t, s} once: one
// CTA per row leaf t in `rows`, columns s >= t from CSR (the first column of
// a row is t itself).  ker: SLP or DLP; transpose applies K^T (double layer).
// xs: x in FP32, rows of near_store_nx(true, NR) values (launch_store_x); read
// by the FP32 single layer, which takes x from it instead of xp.
// coupling by double-float arithmetic on the FP32 pipe (k_coupling_df.cu):
// the FP64 tier's single layer and the mixed tiers' double layer (its FP64
// side), for m = 4, 5 and up to 8 right-hand sides; xh64 / yh64: x-hat /
// y-hat stored as double (else float)
bool coupling_df_supported(int m, int NR);
void launch_coupling_df(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                        int NR, bool xh64, bool yh64, const void* xh, void* yh, cudaStream_t s);
// the FP64 tier's regular nearfield by double-float arithmetic on the FP32
// pipe (k_near_df.cu): the operation of launch_near_sym (single or double
// layer; transpose: K^T for the double layer)
void launch_near_df(const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                    const int* col, bool dlp, bool transpose, int NR, const double* xp, double* yp, cudaStream_t s);
void launch_near_sym(const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                     const int* col, int ker, bool transpose, bool fp32, int NR, const double* xp, const float* xs,
                     double* yp, const LaunchCfg& cfg, cudaStream_t s);
// Stored nearfield (k_nearstore.cu).  Block (t, s) of the ordered list at
// element offset off[b], column by column with leading dimension |t| | 1
// (FP32 if f32, else FP64).  NearStore: destination of the storing variant of
// the regular kernel (entries a / (4 pi); off_ts / off_st: offsets of (t, s)
// and (s, t) for block b of the unordered list).
struct NearStore {
    void* N = nullptr;
    const int64_t* off_ts = nullptr;
    const int64_t* off_st = nullptr;
};
void launch_near_sym_store(const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                           const int* col, int ker, bool fp32, const NearStore& ns, cudaStream_t s);
// x in the stored precision, rows of near_store_nx(f32, NR) values
int near_store_nx(bool f32, int NR);
void launch_store_x(bool f32, int n, int NR, const double* xp, void* xs, cudaStream_t s);
// One row leaf t of the ordered list: positions [rb, rb + R), blocks [b0, b1).
struct alignas(16) NearRow {
    int rb, R, b0, b1;
};
// One block (t, s): element offset of its stored values (of block (s, t) for
// the transposed apply), first position and size of s.
struct alignas(16) NearBlock {
    long long off;
    int cb, C;
};
// y|_t = sum N_ts x|_s over the ordered list (transpose: block (s, t) read
// transposed); writes every row of y (the farfield adds afterwards)
int near_stored_warps(bool f32, int max_leaf, int NR);
void launch_near_stored(bool f32, bool transpose, int NR, int nrows, const NearRow* rows, const NearBlock* blocks,
                        const void* nst, const void* xs, int max_leaf, double* yp, cudaStream_t s);
void launch_sing_scatter(bool f32, int np, const int64_t* pos0, const int64_t* pos1, const double* v0,
                         const double* v1, void* nst, cudaStream_t s);

// nearfield, singular pairs of one type (canonical orientation, see api.cpp)
//   mode 0: evaluate and scatter into yp;  mode 1: evaluate and store the
//   values (val0 = a_{lo,hi}, val1 = a_{hi,lo});  mode 2: scatter stored values.
void launch_singular(const Geom& g, int type, int ker, int npairs, const int* lo, const int* hi, const int* code,
                     const double* tab, int npts, int mode, bool fp32, bool transpose, int NR, const double* xp,
                     double* yp, double* val0, double* val1, cudaStream_t s);
// FP64-class evaluation of modes 0 and 1 (double-float arithmetic, k_sing_df.cu)
void launch_singular_df(const Geom& g, int type, int ker, int npairs, const int* lo, const int* hi, const int* code,
                        const double* tab, int npts, int mode, bool transpose, int NR, const double* xp, double* yp,
                        double* val0, double* val1, cudaStream_t s);
// mode 3 of launch_singular (FP32 evaluation only): the pair's entries
// a_{lo,hi}, a_{hi,lo} (swapped if transpose) as floats at the places
// ((int2*)val1)[pid] = (position in row lo, position in row hi or -1) of
// (float*)val0, the row order of launch_sing_gather.
// launch_sing_gather: y_i += sum_{e in [ptr[i], ptr[i+1])} vals[e] x_{other[e]},
// x in FP32 rows of max(NR, 4) values (launch_store_x).
void launch_sing_gather(int NR, int n, const int* ptr, const int* other, const float* vals, const float* xs,
                        double* yp, cudaStream_t s);

// farfield.  basis32: basis values in FP32 (else FP64); xh64 / yh64: the
// cluster vectors xh / yh are double (else float).
void launch_leaf_forward(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nleaves,
                         const int* leaves, bool dlp_basis, bool basis32, bool xh64, int NR, const double* xp,
                         void* xh, cudaStream_t s);
void launch_leaf_backward(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nleaves,
                          const int* leaves, bool dlp_basis, bool basis32, bool yh64, int NR, const void* yh,
                          double* yp, cudaStream_t s);
// stored leaf bases B[pos * k + nu] (FP32 if basis32, else FP64), evaluated
// once; the transforms of an apply read them (max_leaf: largest leaf)
void launch_leaf_basis(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nleaves,
                       const int* leaves, bool dlp_basis, bool basis32, void* B, cudaStream_t s);
void launch_leaf_forward_stored(const Tree& t, int k, int max_leaf, int nleaves, const int* leaves, bool basis32,
                                bool xh64, int NR, const void* B, const double* xp, void* xh, cudaStream_t s);
void launch_leaf_backward_stored(const Tree& t, int k, int max_leaf, int nleaves, const int* leaves, bool basis32,
                                 bool yh64, int NR, const void* B, const void* yh, double* yp, cudaStream_t s);
// The transfers over the top levels of the tree in one launch (FP32 vectors,
// m = 4, up to 8 right-hand sides; returns false otherwise: launch per level).
// start: the clusters of the first per-level launch's level and the leaves
// above it.  Upward (up = true): their x-hat is complete, the launch forms
// every ancestor's (cnt: per-cluster arrival counts, zero at set-up).
// Downward: adds to their y-hat what their ancestors pass down.
bool launch_tree_updown(bool up, const Tree& t, const Consts& c, int n, const int* start, const int* parent,
                        unsigned* cnt, bool v64, int NR, void* v, cudaStream_t s);
void launch_upward(const Tree& t, const Consts& c, int nparents, const int* parents, bool xh64, int NR, void* xh,
                   cudaStream_t s);
void launch_downward(const Tree& t, const Consts& c, int nparents, const int* parents, bool yh64, int NR, void* yh,
                     cudaStream_t s);


// precision: 0 FP64 (xh, yh double), 1 FP32 SIMT arithmetic (xh / yh double
// if xh64 / yh64, else float)
void launch_coupling(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                     int precision, bool xh64, bool yh64, int NR, const void* xh, void* yh, const LaunchCfg& cfg,
                     cudaStream_t s);
// coupling on the tensor cores (k_coupling_tc.cu), float x-hat / y-hat;
// kind 0 TF32, 1 TF32x3, 2 BF16.  coupling_tc_status reads (and optionally
// clears) the device flag an expired wait sets (H2BEM_ERR_TIMEOUT, else 0).
bool coupling_tc_supported(int m, int kind);
void launch_coupling_tc(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                        int kind, int NR, const float* xh, float* yh, int stall_test, cudaStream_t s);
int coupling_tc_status(bool reset);

}  // namespace h2

namespace h2 {
// shape gradient (single layer, FP64), k_grad.cu
void launch_grad_coupling(const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr, const int* col,
                          int NR, const double* wh, const double* xh, double* dbox, cudaStream_t s);
void launch_grad_transfer(const Tree& t, const Consts& c, int nch, const int* children, const int* parent, int NR,
                          const double* xh, const double* wh, const double* yh, const double* zh, double* dbox,
                          cudaStream_t s);
void launch_grad_leaf(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nl, const int* leaves,
                      int NR, const double* xp, const double* wp, const double* yh, const double* zh, double* dbox,
                      double* dX, cudaStream_t s);
void launch_grad_near(const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                      const int* col, int NR, const double* xp, const double* wp, double* dX, cudaStream_t s);
void launch_grad_singular(const Geom& g, int type, int npairs, const int* lo, const int* hi, const int* code,
                          const double* tab, int npts, int NR, const double* xp, const double* wp, double* dX,
                          cudaStream_t s);
void launch_grad_box(int nc, const int* cext, const int* cflag, const double* dbox, double* dX, cudaStream_t s);
// the double layer's terms (k_grad_dlp.cu): column-side leaf basis W (beta =
// x z-hat), regular nearfield (both sides of every ordered pair), Sauter-Schwab
// edge / vertex pairs by the full tensor rule (x1, x2, y1, y2, weight x
// Jacobian per point)
void launch_grad_leaf_w(const Geom& g, const Tree& t, const Consts& c, const double* rule, int nl, const int* leaves,
                        int NR, const double* xp, const double* zh, double* dbox, double* dX, cudaStream_t s);
void launch_grad_near_dlp(const Geom& g, const Tree& t, const Consts& c, int nrows, const int* rows, const int* ptr,
                          const int* col, int NR, const double* xp, const double* wp, double* dX, cudaStream_t s);
void launch_grad_singular_dlp(const Geom& g, int npairs, const int* lo, const int* hi, const int* code,
                              const double* tab, int npts, int NR, const double* xp, const double* wp, double* dX,
                              cudaStream_t s);

}  // namespace h2

namespace h2 {
// conjugate gradients and mass term (k_cg.cu); vectors column-major n x nrhs
void launch_dots(int n, int nrhs, const double* a, int64_t lda, const double* b, int64_t ldb, double* out,
                 cudaStream_t s);
void launch_cg_step(int n, int nrhs, const double* alpha, const double* p, int64_t ldp, const double* q, int64_t ldq,
                    double* x, int64_t ldx, double* res, int64_t ldr, cudaStream_t s);
void launch_cg_dir(int n, int nrhs, const double* beta, const double* res, int64_t ldr, double* p, int64_t ldp,
                   cudaStream_t s);
void launch_rank1_add(int n, int nrhs, const double* m, const double* d, double* q, int64_t ldq, cudaStream_t s);
void launch_mass_add(int n, int nrhs, double alpha, const double* area_user, const double* x, int64_t ldx, double* y,
                     int64_t ldy, cudaStream_t s);
void launch_area_user(int n, const int* perm, const double* area, double* out, cudaStream_t s);
// hypersingular operator through the single layer (k_hyper.cu): z = C_d x
// (n x 3 nrhs, column d nrhs + r) and y = sum_d C_d^T w
void launch_curl_fwd(int n, int nrhs, const double* xyz, const int* tri, const double* x, int64_t ldx, double* z,
                     cudaStream_t s);
void launch_curl_bwd(int nv, int n, int nrhs, const int* vptr, const int* inc, const double* xyz, const int* tri,
                     const double* w, double* y, int64_t ldy, cudaStream_t s);
}  // namespace h2

struct h2bem_op;
namespace h2 {
// Used by the allocation-free entry point (noalloc.cu).
int set_error(int code, const char* msg);
int64_t op_size(const h2bem_op* op);
size_t work_bytes(const h2bem_op* op, int NR);
int apply_with_work(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy, cudaStream_t s,
                    unsigned char* work);
}  // namespace h2
