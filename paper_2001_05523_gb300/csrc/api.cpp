// libh2bem host side: validation, cluster tree, block tree, singular-pair
// lists, quadrature tables, device upload and the apply sequence.
// The C ABI is declared and documented in include/h2bem.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/h2bem.h"
#include "internal.h"

using h2::kMaxLeaf;
using h2::kMaxM;

// ===========================================================================
// errors
// ===========================================================================
static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? H2BEM_ERR_OOM : H2BEM_ERR_CUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                           \
    } while (0)

extern "C" int h2bem_last_error(char* buf, size_t len) {
    if (buf && len) {
        size_t n = std::min(len - 1, g_err.size());
        memcpy(buf, g_err.data(), n);
        buf[n] = 0;
    }
    return H2BEM_OK;
}

// ===========================================================================
// mesh
// ===========================================================================
struct h2bem_mesh {
    std::vector<double> xyz;
    std::vector<int32_t> tri;
    int64_t nv = 0, nt = 0;
};

extern "C" int h2bem_mesh_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, h2bem_mesh** out) {
    if (!out) return fail(H2BEM_ERR_ARG, "mesh_create: out is NULL");
    *out = nullptr;
    if (!xyz || !tri) return fail(H2BEM_ERR_ARG, "mesh_create: NULL array");
    if (nv < 3 || nt < 1) return fail(H2BEM_ERR_ARG, "mesh_create: need nv >= 3 and nt >= 1 (got %lld, %lld)",
                                      (long long)nv, (long long)nt);
    if (nt > (int64_t)1 << 30 || nv > (int64_t)1 << 30) return fail(H2BEM_ERR_ARG, "mesh_create: mesh too large");
    for (int64_t i = 0; i < 3 * nt; ++i)
        if (tri[i] < 0 || tri[i] >= nv)
            return fail(H2BEM_ERR_ARG, "mesh_create: triangle %lld has vertex index %d out of range",
                        (long long)(i / 3), (int)tri[i]);
    double vol = 0.0;
    for (int64_t i = 0; i < nt; ++i) {
        const double* a = xyz + 3 * (int64_t)tri[3 * i];
        const double* b = xyz + 3 * (int64_t)tri[3 * i + 1];
        const double* c = xyz + 3 * (int64_t)tri[3 * i + 2];
        double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double len = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        if (!(len > 0.0)) return fail(H2BEM_ERR_MESH, "mesh_create: triangle %lld is degenerate", (long long)i);
        vol += a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    if (!(vol > 0.0))
        return fail(H2BEM_ERR_MESH, "mesh_create: signed volume %.3e <= 0 (triangles must be counter-clockwise "
                    "seen from outside)", vol / 6.0);
    auto* m = new (std::nothrow) h2bem_mesh;
    if (!m) return fail(H2BEM_ERR_OOM, "mesh_create: out of host memory");
    m->xyz.assign(xyz, xyz + 3 * nv);
    m->tri.assign(tri, tri + 3 * nt);
    m->nv = nv;
    m->nt = nt;
    *out = m;
    return H2BEM_OK;
}

extern "C" int h2bem_mesh_destroy(h2bem_mesh* mesh) {
    delete mesh;
    return H2BEM_OK;
}

// ===========================================================================
// cluster tree
// ===========================================================================
struct h2bem_tree {
    int64_t n = 0, nc = 0, depth = 0;
    std::vector<int64_t> perm, begin, end, child0, child1, parent, level;
    std::vector<double> bmin, bmax;  // nc x 3
};

namespace {

void cluster_box(const h2bem_mesh& M, const int64_t* idx, int64_t cnt, double* lo, double* hi) {
    for (int d = 0; d < 3; ++d) {
        lo[d] = INFINITY;
        hi[d] = -INFINITY;
    }
    for (int64_t a = 0; a < cnt; ++a)
        for (int c = 0; c < 3; ++c) {
            const double* p = &M.xyz[3 * (int64_t)M.tri[3 * idx[a] + c]];
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], p[d]);
                hi[d] = std::max(hi[d], p[d]);
            }
        }
}

double centroid(const h2bem_mesh& M, int64_t t, int d) {
    const int32_t* v = &M.tri[3 * t];
    return ((M.xyz[3 * (int64_t)v[0] + d] + M.xyz[3 * (int64_t)v[1] + d]) + M.xyz[3 * (int64_t)v[2] + d]) / 3.0;
}

struct TreeBuilder {
    const h2bem_mesh& M;
    h2bem_tree& T;
    int leaf;
    std::vector<int64_t> scratch;

    int64_t add(int64_t b, int64_t e, int64_t parent, int64_t level) {
        int64_t c = T.nc++;
        T.begin.push_back(b);
        T.end.push_back(e);
        T.parent.push_back(parent);
        T.level.push_back(level);
        T.child0.push_back(-1);
        T.child1.push_back(-1);
        T.bmin.resize(3 * T.nc);
        T.bmax.resize(3 * T.nc);
        cluster_box(M, &T.perm[b], e - b, &T.bmin[3 * c], &T.bmax[3 * c]);
        T.depth = std::max(T.depth, level);
        return c;
    }

    // iterative depth-first pre-order construction
    void build() {
        struct Item { int64_t b, e, parent, level; int which; };
        std::vector<Item> stack;
        stack.push_back({0, T.n, -1, 0, -1});
        while (!stack.empty()) {
            Item it = stack.back();
            stack.pop_back();
            int64_t c = add(it.b, it.e, it.parent, it.level);
            if (it.parent >= 0) (it.which == 0 ? T.child0 : T.child1)[it.parent] = c;
            if (it.e - it.b <= leaf) continue;
            const double* lo = &T.bmin[3 * c];
            const double* hi = &T.bmax[3 * c];
            int axis = 0;
            for (int d = 1; d < 3; ++d)
                if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
            const double mid = 0.5 * (lo[axis] + hi[axis]);
            int64_t* p = &T.perm[it.b];
            const int64_t cnt = it.e - it.b;
            scratch.resize(cnt);
            int64_t n0 = 0, n1 = 0;
            for (int64_t a = 0; a < cnt; ++a) {
                if (centroid(M, p[a], axis) < mid) p[n0++] = p[a];
                else scratch[n1++] = p[a];
            }
            std::copy(scratch.begin(), scratch.begin() + n1, p + n0);
            int64_t split = n0;
            if (n0 == 0 || n1 == 0) {
                std::vector<std::pair<double, int64_t>> key(cnt);
                for (int64_t a = 0; a < cnt; ++a) key[a] = {centroid(M, p[a], axis), a};
                std::stable_sort(key.begin(), key.end(),
                                 [](const std::pair<double, int64_t>& x, const std::pair<double, int64_t>& y) {
                                     return x.first < y.first;
                                 });
                std::vector<int64_t> tmp(cnt);
                for (int64_t a = 0; a < cnt; ++a) tmp[a] = p[key[a].second];
                std::copy(tmp.begin(), tmp.end(), p);
                split = cnt / 2;
            }
            // push the second child first so the first child is numbered next
            stack.push_back({it.b + split, it.e, c, it.level + 1, 1});
            stack.push_back({it.b, it.b + split, c, it.level + 1, 0});
        }
    }
};

}  // namespace

extern "C" int h2bem_tree_build(const h2bem_mesh* mesh, int leaf_size, h2bem_tree** out) {
    if (!out) return fail(H2BEM_ERR_ARG, "tree_build: out is NULL");
    *out = nullptr;
    if (!mesh) return fail(H2BEM_ERR_ARG, "tree_build: mesh is NULL");
    if (leaf_size < 1) return fail(H2BEM_ERR_ARG, "tree_build: leaf_size must be >= 1");
    std::unique_ptr<h2bem_tree> T(new (std::nothrow) h2bem_tree);
    if (!T) return fail(H2BEM_ERR_OOM, "tree_build: out of host memory");
    T->n = mesh->nt;
    T->perm.resize(T->n);
    for (int64_t i = 0; i < T->n; ++i) T->perm[i] = i;
    TreeBuilder B{*mesh, *T, leaf_size, {}};
    B.build();
    *out = T.release();
    return H2BEM_OK;
}

extern "C" int h2bem_tree_upload(const h2bem_mesh* mesh, int64_t nclusters, const int64_t* perm, const int64_t* begin,
                                 const int64_t* end, const int64_t* child0, const int64_t* child1, h2bem_tree** out) {
    if (!out) return fail(H2BEM_ERR_ARG, "tree_upload: out is NULL");
    *out = nullptr;
    if (!mesh || !perm || !begin || !end || !child0 || !child1 || nclusters < 1)
        return fail(H2BEM_ERR_ARG, "tree_upload: NULL array or nclusters < 1");
    const int64_t n = mesh->nt;
    std::vector<char> seen(n, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (perm[i] < 0 || perm[i] >= n || seen[perm[i]]) return fail(H2BEM_ERR_ARG, "tree_upload: perm is not a permutation");
        seen[perm[i]] = 1;
    }
    if (begin[0] != 0 || end[0] != n) return fail(H2BEM_ERR_ARG, "tree_upload: root must span [0, n)");
    std::unique_ptr<h2bem_tree> T(new (std::nothrow) h2bem_tree);
    if (!T) return fail(H2BEM_ERR_OOM, "tree_upload: out of host memory");
    T->n = n;
    T->nc = nclusters;
    T->perm.assign(perm, perm + n);
    T->begin.assign(begin, begin + nclusters);
    T->end.assign(end, end + nclusters);
    T->child0.assign(child0, child0 + nclusters);
    T->child1.assign(child1, child1 + nclusters);
    T->parent.assign(nclusters, -1);
    T->level.assign(nclusters, -1);
    T->level[0] = 0;
    int64_t reached = 1;
    for (int64_t c = 0; c < nclusters; ++c) {
        if (begin[c] < 0 || end[c] > n || begin[c] >= end[c])
            return fail(H2BEM_ERR_ARG, "tree_upload: cluster %lld has an empty or invalid range", (long long)c);
        const int64_t a = child0[c], b = child1[c];
        if ((a < 0) != (b < 0)) return fail(H2BEM_ERR_ARG, "tree_upload: cluster %lld has one child", (long long)c);
        if (a < 0) continue;
        if (a >= nclusters || b >= nclusters || a == 0 || b == 0 || T->parent[a] >= 0 || T->parent[b] >= 0 || a == b)
            return fail(H2BEM_ERR_ARG, "tree_upload: bad child index at cluster %lld", (long long)c);
        if (begin[a] != begin[c] || end[a] != begin[b] || end[b] != end[c])
            return fail(H2BEM_ERR_ARG, "tree_upload: children of %lld do not split its range", (long long)c);
        T->parent[a] = T->parent[b] = c;
        reached += 2;
    }
    if (reached != nclusters) return fail(H2BEM_ERR_ARG, "tree_upload: clusters unreachable from the root");
    // levels top-down (parents need not precede children in the numbering)
    std::vector<int64_t> st{0};
    while (!st.empty()) {
        int64_t c = st.back();
        st.pop_back();
        if (T->child0[c] >= 0) {
            T->level[T->child0[c]] = T->level[T->child1[c]] = T->level[c] + 1;
            st.push_back(T->child0[c]);
            st.push_back(T->child1[c]);
        }
    }
    T->bmin.resize(3 * nclusters);
    T->bmax.resize(3 * nclusters);
    for (int64_t c = 0; c < nclusters; ++c) {
        T->depth = std::max(T->depth, T->level[c]);
        cluster_box(*mesh, &T->perm[T->begin[c]], T->end[c] - T->begin[c], &T->bmin[3 * c], &T->bmax[3 * c]);
    }
    *out = T.release();
    return H2BEM_OK;
}

extern "C" int h2bem_tree_info(const h2bem_tree* tree, int64_t* nclusters, int64_t* nleaves, int64_t* depth) {
    if (!tree) return fail(H2BEM_ERR_ARG, "tree_info: tree is NULL");
    if (nclusters) *nclusters = tree->nc;
    if (nleaves) {
        int64_t l = 0;
        for (int64_t c = 0; c < tree->nc; ++c) l += tree->child0[c] < 0;
        *nleaves = l;
    }
    if (depth) *depth = tree->depth;
    return H2BEM_OK;
}

extern "C" int h2bem_tree_export(const h2bem_tree* tree, int64_t* perm, int64_t* begin, int64_t* end, int64_t* child0,
                                 int64_t* child1, double* bmin, double* bmax) {
    if (!tree) return fail(H2BEM_ERR_ARG, "tree_export: tree is NULL");
    if (perm) std::copy(tree->perm.begin(), tree->perm.end(), perm);
    if (begin) std::copy(tree->begin.begin(), tree->begin.end(), begin);
    if (end) std::copy(tree->end.begin(), tree->end.end(), end);
    if (child0) std::copy(tree->child0.begin(), tree->child0.end(), child0);
    if (child1) std::copy(tree->child1.begin(), tree->child1.end(), child1);
    if (bmin) std::copy(tree->bmin.begin(), tree->bmin.end(), bmin);
    if (bmax) std::copy(tree->bmax.begin(), tree->bmax.end(), bmax);
    return H2BEM_OK;
}

extern "C" int h2bem_tree_destroy(h2bem_tree* tree) {
    delete tree;
    return H2BEM_OK;
}

// ===========================================================================
// block tree
// ===========================================================================
namespace {

struct Blocks {
    std::vector<int64_t> ft, fs, nt, ns;
};

double diam(const h2bem_tree& T, int64_t c) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
        double e = T.bmax[3 * c + d] - T.bmin[3 * c + d];
        s += e * e;
    }
    return std::sqrt(s);
}

double dist(const h2bem_tree& T, int64_t a, int64_t b) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
        double g = 0.0;
        if (T.bmin[3 * b + d] > T.bmax[3 * a + d]) g = T.bmin[3 * b + d] - T.bmax[3 * a + d];
        else if (T.bmin[3 * a + d] > T.bmax[3 * b + d]) g = T.bmin[3 * a + d] - T.bmax[3 * b + d];
        s += g * g;
    }
    return std::sqrt(s);
}

void build_blocks(const h2bem_tree& T, double eta, Blocks& B) {
    std::vector<std::pair<int64_t, int64_t>> st{{0, 0}};
    while (!st.empty()) {
        auto [t, s] = st.back();
        st.pop_back();
        const double dd = dist(T, t, s);
        if (dd > 0.0 && std::max(diam(T, t), diam(T, s)) <= eta * dd) {
            B.ft.push_back(t);
            B.fs.push_back(s);
            continue;
        }
        const bool tl = T.child0[t] < 0, sl = T.child0[s] < 0;
        if (tl && sl) {
            B.nt.push_back(t);
            B.ns.push_back(s);
        } else if (tl) {
            st.push_back({t, T.child1[s]});
            st.push_back({t, T.child0[s]});
        } else if (sl) {
            st.push_back({T.child1[t], s});
            st.push_back({T.child0[t], s});
        } else {
            st.push_back({T.child1[t], T.child1[s]});
            st.push_back({T.child1[t], T.child0[s]});
            st.push_back({T.child0[t], T.child1[s]});
            st.push_back({T.child0[t], T.child0[s]});
        }
    }
}

}  // namespace

extern "C" int h2bem_blocks(const h2bem_tree* tree, double eta, int64_t* nfar, int64_t* nnear, int64_t* far_t,
                            int64_t* far_s, int64_t* near_t, int64_t* near_s) {
    if (!tree) return fail(H2BEM_ERR_ARG, "blocks: tree is NULL");
    if (!(eta >= 0.0) || !std::isfinite(eta)) return fail(H2BEM_ERR_ARG, "blocks: eta must be finite and >= 0");
    Blocks B;
    build_blocks(*tree, eta, B);
    if (nfar) *nfar = (int64_t)B.ft.size();
    if (nnear) *nnear = (int64_t)B.nt.size();
    if (far_t) std::copy(B.ft.begin(), B.ft.end(), far_t);
    if (far_s) std::copy(B.fs.begin(), B.fs.end(), far_s);
    if (near_t) std::copy(B.nt.begin(), B.nt.end(), near_t);
    if (near_s) std::copy(B.ns.begin(), B.ns.end(), near_s);
    return H2BEM_OK;
}

// ===========================================================================
// quadrature (library's own construction)
// ===========================================================================
namespace {

// Gauss-Legendre on [0,1] by the Golub-Welsch method: the nodes are the
// eigenvalues of the symmetric tridiagonal Jacobi matrix of the Legendre
// recurrence (off-diagonal k / sqrt(4k^2 - 1)), the weights the squared first
// components of its normalised eigenvectors.  Eigen-decomposition by cyclic
// Jacobi rotations (q <= 32).
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
    std::vector<double> A(q * q, 0.0), V(q * q, 0.0);
    for (int i = 0; i < q; ++i) V[i * q + i] = 1.0;
    for (int k = 1; k < q; ++k) {
        double b = k / std::sqrt(4.0 * k * k - 1.0);
        A[(k - 1) * q + k] = A[k * q + k - 1] = b;
    }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < q; ++i)
            for (int j = i + 1; j < q; ++j) off += A[i * q + j] * A[i * q + j];
        if (off < 1e-40) break;
        for (int p = 0; p < q; ++p)
            for (int r = p + 1; r < q; ++r) {
                double apr = A[p * q + r];
                if (apr == 0.0) continue;
                double theta = (A[r * q + r] - A[p * q + p]) / (2.0 * apr);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < q; ++k) {  // A <- A J
                    double akp = A[k * q + p], akr = A[k * q + r];
                    A[k * q + p] = c * akp - s * akr;
                    A[k * q + r] = s * akp + c * akr;
                }
                for (int k = 0; k < q; ++k) {  // A <- J^T A
                    double apk = A[p * q + k], ark = A[r * q + k];
                    A[p * q + k] = c * apk - s * ark;
                    A[r * q + k] = s * apk + c * ark;
                }
                for (int k = 0; k < q; ++k) {  // V <- V J
                    double vkp = V[k * q + p], vkr = V[k * q + r];
                    V[k * q + p] = c * vkp - s * vkr;
                    V[k * q + r] = s * vkp + c * vkr;
                }
            }
    }
    std::vector<std::pair<double, double>> nw(q);
    for (int i = 0; i < q; ++i) nw[i] = {0.5 * (1.0 + A[i * q + i]), V[0 * q + i] * V[0 * q + i]};
    std::sort(nw.begin(), nw.end());
    x.resize(q);
    w.resize(q);
    for (int i = 0; i < q; ++i) {
        x[i] = nw[i].first;
        w[i] = nw[i].second;
    }
}

// Collapsed Gauss rule on the unit simplex, (u, v, weight) per point, exact
// for total degree 3(m - 1): the leaf bases' rule.
void basis_rule_host(int m, std::vector<double>& rule) {
    const int qb = (3 * (m - 1) + 3) / 2;
    std::vector<double> x, w;
    gauss_legendre(std::max(qb, 1), x, w);
    rule.clear();
    for (size_t i = 0; i < x.size(); ++i)
        for (size_t j = 0; j < x.size(); ++j) rule.insert(rule.end(), {x[i], (1.0 - x[i]) * x[j], 2.0 * w[i] * w[j] * (1.0 - x[i])});
}

// The full Sauter-Schwab tensor rule for pairs sharing an edge (type 1) or a
// vertex (type 2), q Gauss points per direction: per point the reference
// coordinates (x1, x2) on P and (y1, y2) on Q of T = {0 <= x2 <= x1 <= 1} and
// the weight times the region's Jacobian (relative-coordinate Duffy maps with
// (xi, a, b, c) in [0, 1]^4; the shared vertices are the first corners):
//   edge, R1 (xi^3 a^2):   x = (xi, xi a c),             y = (xi (1-ab), xi a (1-b))
//         R2 (xi^3 a^2 b): x = (xi, xi a),               y = (xi (1-abc), xi a b (1-c))
//         R3 (xi^3 a^2 b): x = (xi (1-ab), xi a (1-b)),  y = (xi, xi a b c)
//         R4 (xi^3 a^2 b): x = (xi (1-abc), xi a b (1-c)), y = (xi, xi a)
//         R5 (xi^3 a^2 b): x = (xi (1-abc), xi a (1-bc)), y = (xi, xi a b)
//   vertex (xi^3 b):       x = (xi, xi a), y = (xi b, xi b c), and x, y exchanged.
void ss_full_table(int type, int q, std::vector<double>& tab) {
    std::vector<double> g, w;
    gauss_legendre(q, g, w);
    tab.clear();
    for (int i0 = 0; i0 < q; ++i0)
        for (int i1 = 0; i1 < q; ++i1)
            for (int i2 = 0; i2 < q; ++i2)
                for (int i3 = 0; i3 < q; ++i3) {
                    const double xi = g[i0], a = g[i1], b = g[i2], c = g[i3];
                    const double wt = w[i0] * w[i1] * w[i2] * w[i3];
                    const double x3 = xi * xi * xi;
                    if (type == 1) {
                        const double j1 = x3 * a * a, j2 = j1 * b;
                        tab.insert(tab.end(), {xi, xi * a * c, xi * (1 - a * b), xi * a * (1 - b), wt * j1});
                        tab.insert(tab.end(), {xi, xi * a, xi * (1 - a * b * c), xi * a * b * (1 - c), wt * j2});
                        tab.insert(tab.end(), {xi * (1 - a * b), xi * a * (1 - b), xi, xi * a * b * c, wt * j2});
                        tab.insert(tab.end(), {xi * (1 - a * b * c), xi * a * b * (1 - c), xi, xi * a, wt * j2});
                        tab.insert(tab.end(), {xi * (1 - a * b * c), xi * a * (1 - b * c), xi, xi * a * b, wt * j2});
                    } else {
                        const double j = x3 * b;
                        tab.insert(tab.end(), {xi, xi * a, xi * b, xi * b * c, wt * j});
                        tab.insert(tab.end(), {xi * b, xi * b * c, xi, xi * a, wt * j});
                    }
                }
}

// Sauter-Schwab point tables after the exact integration of the monomial
// factors (see k_sing.cu).  Rows: identical [aa, 2ab, bb, W]; edge [6 Gram
// monomials, alpha, beta, gamma, W_g, W_dg]; vertex: the 1-D Gauss rule
// [x_k, w_k] (the kernel forms the factorised triple sum).
void ss_tables(int q, std::vector<double>& ti, std::vector<double>& te, std::vector<double>& tv,
               std::vector<double>& tvg, std::vector<double>& te1) {
    std::vector<double> x, w;
    gauss_legendre(q, x, w);
    ti.clear();
    te.clear();
    tv.clear();
    // identical: regions R1, R3, R5 (R2, R4, R6 mirror them); int xi^2 a = 1/6, times 2 mirrors
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < q; ++k) {
            const double e = x[k];
            double al, be;
            if (r == 0) { al = e; be = 1.0; }
            else if (r == 1) { al = 1.0; be = e; }
            else { al = -e; be = 1.0 - e; }
            ti.insert(ti.end(), {al * al, 2.0 * al * be, be * be, w[k] / 3.0});
        }
    // edge: (alpha, beta, gamma) for vectors (P1-P0, P2-P1, Q2-Q1)
    for (int r = 0; r < 5; ++r)
        for (int k = 0; k < q; ++k)
            for (int l = 0; l < q; ++l) {
                const double e2 = x[k], e3 = x[l], ww = w[k] * w[l];
                double al, be, ga, f;
                switch (r) {
                    case 0: al = e2; be = e3; ga = -(1.0 - e2); f = 1.0; break;
                    case 1: al = e2 * e3; be = 1.0; ga = -e2 * (1.0 - e3); f = e2; break;
                    case 2: al = -e2; be = 1.0 - e2; ga = -e2 * e3; f = e2; break;
                    case 3: al = -e2 * e3; be = e2 * (1.0 - e3); ga = -1.0; f = e2; break;
                    default: al = -e2 * e3; be = 1.0 - e2 * e3; ga = -e2; f = e2; break;
                }
                te.insert(te.end(), {al * al, be * be, ga * ga, 2 * al * be, 2 * al * ga, 2 * be * ga, al, be, ga,
                                     ww * f / 6.0, ww * f / 2.0});
            }
    // vertex: the 1-D rule (x_k, w_k, w_k x_k / 2); the kernel forms the factorised sums
    for (int k = 0; k < q; ++k) tv.insert(tv.end(), {x[k], w[k], 0.5 * w[k] * x[k]});
    // edge: the 1-D rule (x_k, w_k, w_k / 2, w_k x_k / 2) for the factorised sums
    te1.clear();
    for (int k = 0; k < q; ++k) te1.insert(te1.end(), {x[k], w[k], 0.5 * w[k], 0.5 * w[k] * x[k]});
    // vertex, Gram form for the shape gradient: (alpha, beta, gamma, delta) for
    // vectors (P1-P0, P2-P1, Q1-Q0, Q2-Q1); rows [10 Gram monomials, W_g]
    tvg.clear();
    for (int r = 0; r < 2; ++r)
        for (int i = 0; i < q; ++i)
            for (int k = 0; k < q; ++k)
                for (int l = 0; l < q; ++l) {
                    const double e1 = x[i], e2 = x[k], e3 = x[l], ww = w[i] * w[k] * w[l];
                    double al, be, ga, de;
                    if (r == 0) { al = 1.0; be = e1; ga = -e2; de = -e2 * e3; }
                    else { al = e2; be = e2 * e3; ga = -1.0; de = -e1; }
                    tvg.insert(tvg.end(), {al * al, be * be, ga * ga, de * de, 2 * al * be, 2 * al * ga, 2 * al * de,
                                           2 * be * ga, 2 * be * de, 2 * ga * de, ww * e2 / 3.0});
                }
}

}  // namespace

// ===========================================================================
// operator
// ===========================================================================
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    ~DevBuf() { if (p) cudaFree(p); }
    int alloc(size_t b) {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (b == 0) return H2BEM_OK;
        cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            p = nullptr;
            return fail(e == cudaErrorMemoryAllocation ? H2BEM_ERR_OOM : H2BEM_ERR_CUDA, "cudaMalloc(%zu): %s", b,
                        cudaGetErrorString(e));
        }
        bytes = b;
        return H2BEM_OK;
    }
    template <typename T>
    T* as() const { return reinterpret_cast<T*>(p); }
};

template <typename T>
static int upload(DevBuf& d, const std::vector<T>& h) {
    int rc = d.alloc(h.size() * sizeof(T));
    if (rc) return rc;
    if (!h.empty()) CU(cudaMemcpy(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return H2BEM_OK;
}

struct Csr {
    std::vector<int> rows, ptr, col;  // compacted rows with >= 1 entry
    DevBuf drows, dptr, dcol;
    int upload_all() {
        int rc;
        if ((rc = upload(drows, rows)) || (rc = upload(dptr, ptr)) || (rc = upload(dcol, col))) return rc;
        return H2BEM_OK;
    }
    int nrows() const { return (int)rows.size(); }
};

static void make_csr(int64_t nkeys, const std::vector<int64_t>& key, const std::vector<int64_t>& val, Csr& C,
                     const std::vector<int>* remap_rows = nullptr) {
    std::vector<int64_t> cnt(nkeys + 1, 0);
    for (int64_t k : key) cnt[k + 1]++;
    for (int64_t r = 0; r < nkeys; ++r) cnt[r + 1] += cnt[r];
    std::vector<int> colall(key.size());
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (size_t b = 0; b < key.size(); ++b) colall[fill[key[b]]++] = (int)val[b];
    C.rows.clear();
    C.ptr.assign(1, 0);
    C.col.clear();
    for (int64_t r = 0; r < nkeys; ++r) {
        if (cnt[r + 1] == cnt[r]) continue;
        C.rows.push_back(remap_rows ? (*remap_rows)[r] : (int)r);
        // columns of a row in increasing cluster order
        std::vector<int> cs(colall.begin() + cnt[r], colall.begin() + cnt[r + 1]);
        std::sort(cs.begin(), cs.end());
        C.col.insert(C.col.end(), cs.begin(), cs.end());
        C.ptr.push_back((int)C.col.size());
    }
}

struct h2bem_op {
    int kernel = 0, m = 0, k = 0, precision = 0, q_ss = 5, cache_singular = 0;
    double eta = 0;
    int64_t n = 0, nv = 0, nc = 0, nleaves = 0, depth = 0;
    int64_t nfar = 0, nnear = 0, near_pairs = 0, sing[3] = {0, 0, 0};
    int64_t regular_evals = 0;  // pairs evaluated by the regular nearfield kernel
    h2::Consts consts{};
    // device geometry and tree
    DevBuf xyz, tri, perm, iperm, v, area, nrm, ctr, vid, qo, qa, chl, plane, nef, areaf;
    DevBuf cbegin, cend, cchild0, cchild1, cbox, czhl, cetr, leaves, basis_rule;
    std::vector<int> leaves_h;
    int max_leaf = 0;               // largest leaf cluster
    DevBuf basisV, basisW;          // stored leaf bases [pos][nu]: V (FP32 in the mixed tier), W (double layer, FP64)
    std::vector<std::vector<int>> level_parents;  // non-leaf clusters per level
    std::vector<DevBuf> dlevel;
    // one launch each way for the top levels of the transfers (levels <
    // tree_L0, each with at most kTreeTopParents parents): the clusters of level
    // tree_L0 and the leaves above it, per-cluster arrival counts (upward)
    int tree_L0 = 0, tree_nstart = 0;
    DevBuf tree_start, tree_cnt;
    Csr far, far_t, near, near_u;  // near_u: the blocks (t, s) of near with s >= t
    // singular pairs by type (index 0: identical, 1: edge, 2: vertex)
    DevBuf sp_lo[3], sp_hi[3], sp_code[3], sp_tab[3], sp_v0[3], sp_v1[3], sp_gtab, sp_gtab_edge;
    int sp_gnpts = 0, sp_gnpts_edge = 0;
    // shape gradient: per-cluster extreme vertices and floor flags, child list
    DevBuf cext, cflag, children, parent;
    int nchildren = 0;
    DevBuf g_xp, g_wp, g_xh, g_wh, g_yh, g_zh, g_dbox;
    int g_NR = 0;
    int sp_npts[3] = {0, 0, 0};
    int64_t sp_count[3] = {0, 0, 0};
    // workspace
    int ws_NR = 0;
    DevBuf xp, yp, xh, yh, xstage, ystage;
    size_t stage_elems = 0;
    cudaEvent_t ev[10] = {};
    double last_ms = 0.0, stage_ms[8] = {0};
    bool timing_pending = false;  // a timed apply recorded events not read yet (h2bem_stats_get reads them)
    int64_t launches = 0;
    // launch variants (autotune): per right-hand-side width slot and direction
    int autotune = 0;
    int singular_fp64 = 0, recompute_basis = 0;
    struct Tuned {
        bool done = false;
        h2::LaunchCfg near, coup;  // work pointers filled in at launch
        bool near_persist = false, coup_persist = false;
        int near_nb = 0;
    } tuned[4][2];
    int64_t last_variant[5] = {0, 4, 4, 0, 0};
    DevBuf work;  // row counters of persistent launches (2 ints)
    DevBuf area_user;              // |tau_i| in the caller's order (mass term), made on first use
    DevBuf cg_r, cg_p, cg_q, cg_s, cg_d; // conjugate-gradient vectors and scalars
    int64_t cg_cap = 0;
    // stored nearfield (store_near): the blocks of `near` and their offsets
    // (boff: block (t, s); boff_t: block (s, t) of the same list entry)
    int store_near = 0;
    DevBuf nst, nrow, nblk, nblk_t, xs;  // values, NearRow per row, NearBlock per block (and for A^T)
    int64_t nst_bytes = 0;
    int stage_order = 0;  // 1: the last apply ran the stored nearfield first
    // singular entries applied by rows (FP32 Sauter-Schwab points): CSR of the
    // entries of each tree position (partner positions sg_other), the values in
    // that order (sg_vals; sg_vals_t for the cached transposed double layer),
    // and per canonical pair its two places (types in order at sg_off);
    // evaluated per apply or once (cache_singular)
    int sing_gather = 0;
    DevBuf sg_ptr, sg_other, sg_pos, sg_vals, sg_vals_t;
    int64_t sg_off[3] = {0, 0, 0};
    // hypersingular operator: triangles at each vertex (3 tau + corner), work vectors
    DevBuf vptr, vinc, hyp_z, hyp_w;
    int64_t hyp_cap = 0;
    // double layer with piecewise-linear trial functions (h2bem_apply_dlp_p1),
    // made on first use: per-corner leaf bases W1_c [pos][k] (FP64), the
    // Sauter-Schwab values of the edge / vertex pairs (6 per pair), and corner
    // work vectors x3 / y3 [3][n][NR]
    int p1_ready = 0;
    DevBuf p1_W1[3], p1_vals[2], p1_tab, p1_x3, p1_y3, p1_off;
    int64_t p1_cap = 0;
    // Green cross approximation (opts.basis = GCA): rank and pivot tree
    // positions per cluster, transfer matrices E_c and coupling matrices S_b
    // stored compactly at eoff[c] / soff[b] (FP64, or FP32 in MIXED_FP32); the
    // leaf bases are basisV, zero-padded to k columns
    int gca = 0;
    // hybrid cross approximation (opts.basis = HCA): the same stored passes as
    // GCA (gca = 1), couplings from the host; the transposed apply runs the
    // column-ordered blocks (far_t) with the transposed couplings at g_soff_t
    int hca = 0;
    DevBuf g_soff_t, g_St;
    // double-layer shape gradient: full Sauter-Schwab tables (edge, vertex)
    int gd_ready = 0, gd_npts[2] = {0, 0};
    DevBuf gd_tab[2];
    int tc_wait_test = 0;  // opts.tc_wait_test (tests of the tensor-core timeout path)
    DevBuf g_rank, g_pivoff, g_piv, g_eoff, g_E, g_soff, g_S;
    int64_t gca_bytes = 0;
    double gca_mean_rank = 0.0;
    // CUDA graph of the launch sequence (use_graph)
    int use_graph = 0;
    int64_t ws_gen = 0;
    cudaGraphExec_t gexec = nullptr;
    struct GKey {
        const void* x = nullptr;
        void* y = nullptr;
        int64_t ldx = 0, ldy = 0, ws_gen = -1, launches = 0;
        int nrhs = 0;
        bool tr = false;
        cudaStream_t s = nullptr;
        bool operator==(const GKey& o) const {
            return x == o.x && y == o.y && ldx == o.ldx && ldy == o.ldy && ws_gen == o.ws_gen && nrhs == o.nrhs &&
                   tr == o.tr && s == o.s;
        }
    } gkey_seen, gkey_graph;

    h2::Geom geom() const {
        return h2::Geom{(int)n, v.as<const double>(), area.as<const double>(), nrm.as<const double>(),
                        ctr.as<const double>(), vid.as<const int>(), qo.as<const float>(), qa.as<const double>(),
                        chl.as<const float>(), plane.as<const double>(), nef.as<const float>(),
                        areaf.as<const float>()};
    }
    h2::Tree tree() const {
        return h2::Tree{(int)nc, cbegin.as<const int>(), cend.as<const int>(), cchild0.as<const int>(),
                        cchild1.as<const int>(), cbox.as<const double>(), czhl.as<const float2>(),
                        cetr.as<const float>()};
    }
    // a second stream for the farfield passes, which run concurrently with the
    // nearfield (fork and join events, no timing)
    cudaStream_t s_far = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ~h2bem_op() {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (s_far) cudaStreamDestroy(s_far);
        if (gexec) cudaGraphExecDestroy(gexec);
    }
};

extern "C" int h2bem_opts_default(h2bem_opts* opts) {
    if (!opts) return fail(H2BEM_ERR_ARG, "opts_default: NULL");
    memset(opts, 0, sizeof *opts);
    opts->q_ss = 5;
    opts->precision = H2BEM_FP64;
    opts->cache_singular = 0;
    opts->basis = H2BEM_BASIS_CHEBYSHEV;
    opts->gca_q = 4;
    opts->gca_kmax = h2::kGcaMaxRank;
    opts->gca_eps = 1e-6;
    opts->hca_kaca = 64;
    opts->hca_kmax = h2::kGcaMaxRank;
    opts->hca_eps_aca = 1e-6;
    opts->hca_eps = 1e-6;
    return H2BEM_OK;
}

namespace {

// Singular pairs in the canonical orientation: outer panel = lower user index.
// code bits: [1:0] rotation of the outer panel, [3:2],[5:4],[7:6] corners of
// the inner panel listed as Q0, Q1, Q2.
void singular_pairs(const h2bem_mesh& M, std::vector<int64_t> lo[3], std::vector<int64_t> hi[3],
                    std::vector<int> code[3]) {
    const int64_t nt = M.nt, nv = M.nv;
    std::vector<int64_t> vptr(nv + 1, 0);
    for (int64_t i = 0; i < 3 * nt; ++i) vptr[M.tri[i] + 1]++;
    for (int64_t v = 0; v < nv; ++v) vptr[v + 1] += vptr[v];
    std::vector<int64_t> vtri(3 * nt), fill(vptr.begin(), vptr.end() - 1);
    for (int64_t t = 0; t < nt; ++t)
        for (int c = 0; c < 3; ++c) vtri[fill[M.tri[3 * t + c]]++] = t;
    std::vector<int64_t> nb;
    for (int64_t i = 0; i < nt; ++i) {
        const int32_t* ti = &M.tri[3 * i];
        nb.clear();
        for (int c = 0; c < 3; ++c)
            for (int64_t e = vptr[ti[c]]; e < vptr[ti[c] + 1]; ++e)
                if (vtri[e] >= i) nb.push_back(vtri[e]);
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        for (int64_t j : nb) {
            const int32_t* tj = &M.tri[3 * j];
            int shared = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) shared += ti[a] == tj[b];
            int cd = 0, slot;
            if (j == i) {
                slot = 0;
                cd = 0 | (0 << 2) | (1 << 4) | (2 << 6);
            } else if (shared == 2) {
                slot = 1;
                int un = 0;
                for (int a = 0; a < 3; ++a) {
                    bool f = false;
                    for (int b = 0; b < 3; ++b) f |= ti[a] == tj[b];
                    if (!f) un = a;
                }
                const int rP = (un + 1) % 3;
                const int32_t p0 = ti[rP], p1 = ti[(rP + 1) % 3];
                int q0 = 0, q1 = 0, q2 = 0;
                for (int b = 0; b < 3; ++b) {
                    if (tj[b] == p0) q0 = b;
                    else if (tj[b] == p1) q1 = b;
                    else q2 = b;
                }
                cd = rP | (q0 << 2) | (q1 << 4) | (q2 << 6);
            } else if (shared == 1) {
                slot = 2;
                int a0 = 0, b0 = 0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        if (ti[a] == tj[b]) { a0 = a; b0 = b; }
                cd = a0 | (b0 << 2) | (((b0 + 1) % 3) << 4) | (((b0 + 2) % 3) << 6);
            } else {
                continue;  // duplicate triangles sharing three vertices are not supported
            }
            lo[slot].push_back(i);
            hi[slot].push_back(j);
            code[slot].push_back(cd);
        }
    }
}

}  // namespace

// Stored nearfield (opts.store_near): offsets of the ordered blocks (t, s)
// of `near` (|s| columns of |t| | 1 values, each block on a 16-byte
// boundary), the regular entries written by the storing variant of the
// nearfield kernel, then the Sauter-Schwab entries of the canonical pairs
// scattered to (lo, hi) and (hi, lo).
static int build_near_store(h2bem_op* op, const h2bem_tree& tree, const std::vector<int>& iperm,
                            const std::vector<int64_t> (&slo)[3], const std::vector<int64_t> (&shi)[3]) {
    const bool f32 = op->precision != H2BEM_FP64;
    const int es = f32 ? (int)sizeof(float) : (int)sizeof(double), vec = 16 / es;
    const Csr& N = op->near;
    const int64_t nc = op->nc;
    auto size_of = [&](int64_t c) { return (int)(tree.end[c] - tree.begin[c]); };
    std::vector<int> rowpos(nc, -1);
    for (int r = 0; r < N.nrows(); ++r) rowpos[N.rows[r]] = r;
    // index of block (t, s) in the ordered list (columns of a row are sorted)
    auto find = [&](int t, int s) -> int64_t {
        const int r = rowpos[t];
        if (r < 0) return -1;
        const auto b = std::lower_bound(N.col.begin() + N.ptr[r], N.col.begin() + N.ptr[r + 1], s);
        if (b == N.col.begin() + N.ptr[r + 1] || *b != s) return -1;
        return b - N.col.begin();
    };
    std::vector<int64_t> boff(N.col.size()), boff_t(N.col.size());
    int64_t tot = 0;
    for (int r = 0; r < N.nrows(); ++r) {
        const int ld = size_of(N.rows[r]) | 1;
        for (int b = N.ptr[r]; b < N.ptr[r + 1]; ++b) {
            boff[b] = tot;
            tot += ((int64_t)size_of(N.col[b]) * ld + vec - 1) / vec * vec;
        }
    }
    for (int r = 0; r < N.nrows(); ++r)
        for (int b = N.ptr[r]; b < N.ptr[r + 1]; ++b) {
            const int64_t bt = find(N.col[b], N.rows[r]);
            if (bt < 0) return fail(H2BEM_ERR_ARG, "operator_create: nearfield block list is not symmetric");
            boff_t[b] = boff[bt];
        }
    const Csr& U = op->near_u;
    std::vector<int64_t> ots(U.col.size()), ost(U.col.size());
    for (int r = 0; r < U.nrows(); ++r)
        for (int b = U.ptr[r]; b < U.ptr[r + 1]; ++b) {
            const int64_t b1 = find(U.rows[r], U.col[b]), b2 = find(U.col[b], U.rows[r]);
            if (b1 < 0 || b2 < 0) return fail(H2BEM_ERR_ARG, "operator_create: nearfield block list is not symmetric");
            ots[b] = boff[b1];
            ost[b] = boff[b2];
        }
    std::vector<int> leaf_of(op->n, -1);
    for (int l : op->leaves_h)
        for (int64_t p = tree.begin[l]; p < tree.end[l]; ++p) leaf_of[p] = l;
    int rc;
    op->nst_bytes = tot * es;
    std::vector<h2::NearRow> nrow(N.nrows());
    std::vector<h2::NearBlock> nblk(N.col.size()), nblk_t(N.col.size());
    for (int r = 0; r < N.nrows(); ++r) {
        nrow[r] = h2::NearRow{(int)tree.begin[N.rows[r]], size_of(N.rows[r]), N.ptr[r], N.ptr[r + 1]};
        for (int b = N.ptr[r]; b < N.ptr[r + 1]; ++b) {
            nblk[b] = h2::NearBlock{(long long)boff[b], (int)tree.begin[N.col[b]], size_of(N.col[b])};
            nblk_t[b] = h2::NearBlock{(long long)boff_t[b], (int)tree.begin[N.col[b]], size_of(N.col[b])};
        }
    }
    if ((rc = op->nst.alloc((size_t)op->nst_bytes)) || (rc = upload(op->nrow, nrow)) || (rc = upload(op->nblk, nblk)) ||
        (rc = upload(op->nblk_t, nblk_t)))
        return rc;
    CU(cudaMemset(op->nst.p, 0, (size_t)op->nst_bytes));
    {
        DevBuf dts, dst;
        if ((rc = upload(dts, ots)) || (rc = upload(dst, ost))) return rc;
        h2::NearStore ns;
        ns.N = op->nst.p;
        ns.off_ts = dts.as<int64_t>();
        ns.off_st = dst.as<int64_t>();
        h2::launch_near_sym_store(op->geom(), op->tree(), op->consts, U.nrows(), U.drows.as<int>(), U.dptr.as<int>(),
                                  U.dcol.as<int>(), op->kernel == H2BEM_DLP ? h2::DLP : h2::SLP, f32, ns, 0);
        CU(cudaGetLastError());
        CU(cudaDeviceSynchronize());
    }
    for (int ty = 0; ty < 3; ++ty) {
        if (ty == 0 && op->kernel == H2BEM_DLP) continue;  // k_ii = 0, written by the regular pass
        const int np = (int)op->sp_count[ty];
        if (np == 0) continue;
        std::vector<int64_t> p0(np), p1(np);
        for (int p = 0; p < np; ++p) {
            const int lo = iperm[slo[ty][p]], hi = iperm[shi[ty][p]];
            const int lt = leaf_of[lo], ls = leaf_of[hi];
            const int il = lo - (int)tree.begin[lt], jl = hi - (int)tree.begin[ls];
            const int64_t b1 = find(lt, ls), b2 = find(ls, lt);
            if (b1 < 0 || b2 < 0) return fail(H2BEM_ERR_ARG, "operator_create: a singular pair outside the nearfield");
            p0[p] = boff[b1] + (int64_t)jl * (size_of(lt) | 1) + il;
            p1[p] = boff[b2] + (int64_t)il * (size_of(ls) | 1) + jl;
        }
        DevBuf dp0, dp1, v0, v1;
        if ((rc = upload(dp0, p0)) || (rc = upload(dp1, p1))) return rc;
        const double *pv0 = op->sp_v0[ty].as<double>(), *pv1 = op->sp_v1[ty].as<double>();
        if (!pv0 || !pv1) {  // no FP64 cache (not requested, or kept as float pairs for the row gather)
            if ((rc = v0.alloc(np * sizeof(double))) || (rc = v1.alloc(np * sizeof(double)))) return rc;
            h2::launch_singular(op->geom(), h2::IDENTICAL - ty, op->kernel, np, op->sp_lo[ty].as<int>(),
                                op->sp_hi[ty].as<int>(), op->sp_code[ty].as<int>(), op->sp_tab[ty].as<double>(),
                                op->sp_npts[ty], 1, f32 && !op->singular_fp64, false, 1, nullptr, nullptr,
                                v0.as<double>(), v1.as<double>(), 0);
            pv0 = v0.as<double>();
            pv1 = v1.as<double>();
        }
        h2::launch_sing_scatter(f32, np, dp0.as<int64_t>(), dp1.as<int64_t>(), pv0, pv1, op->nst.p, 0);
        CU(cudaGetLastError());
        CU(cudaDeviceSynchronize());
    }
    return H2BEM_OK;
}

// GCA cluster bases (gca.cpp on the host), uploaded compactly; the leaf bases
// into basisV zero-padded to op->k = the largest rank rounded up to 4; the
// coupling matrices of the farfield CSR evaluated on the GPU (k_gca.cu).
static int gca_setup(h2bem_op* op, const h2bem_mesh* mesh, const h2bem_tree* tree, const h2bem_opts& opts) {
    const int64_t n = op->n, nc = op->nc;
    std::vector<double> glx, glw;
    gauss_legendre(opts.gca_q, glx, glw);
    h2::GcaSetup S{};
    S.xyz = mesh->xyz.data();
    S.tri = mesh->tri.data();
    S.n = n;
    S.nc = nc;
    S.perm = tree->perm.data();
    S.begin = tree->begin.data();
    S.end = tree->end.data();
    S.child0 = tree->child0.data();
    S.child1 = tree->child1.data();
    S.level = tree->level.data();
    S.bmin = tree->bmin.data();
    S.bmax = tree->bmax.data();
    S.q = opts.gca_q;
    S.kmax = opts.gca_kmax;
    S.eps = opts.gca_eps;
    S.gl_x = glx.data();
    S.gl_w = glw.data();
    S.ru = op->consts.ru;
    S.rv = op->consts.rv;
    S.rw = op->consts.rw;
    h2::GcaResult R;
    h2::gca_build(S, R);
    int kmax = 1;
    double rsum = 0.0;
    for (int64_t c = 0; c < nc; ++c) {
        kmax = std::max(kmax, R.rank[c]);
        rsum += R.rank[c];
    }
    op->gca = 1;
    op->gca_mean_rank = nc ? rsum / nc : 0.0;
    const int K = (kmax + 3) / 4 * 4;
    op->k = K;
    const bool f32 = op->precision != H2BEM_FP64;
    const size_t es = f32 ? sizeof(float) : sizeof(double);
    // leaf bases [pos][K]
    std::vector<double> B((size_t)n * K, 0.0);
    for (int64_t c = 0; c < nc; ++c) {
        if (tree->child0[c] >= 0) continue;
        const int rk = R.rank[c];
        for (int64_t a = tree->begin[c]; a < tree->end[c]; ++a)
            for (int nu = 0; nu < rk; ++nu)
                B[(size_t)a * K + nu] = R.V[R.voff[c] + (a - tree->begin[c]) * rk + nu];
    }
    std::vector<int64_t> eoff(nc, 0);
    for (int64_t c = 0; c < nc; ++c) eoff[c] = R.eoff[c] < 0 ? 0 : R.eoff[c];
    // coupling offsets in the order of the farfield CSR, every block on a
    // 16-byte boundary (sizes rounded up to 4 elements) for the asynchronous copies
    std::vector<int64_t> soff(op->far.col.size() + 1, 0);
    for (int r = 0; r < op->far.nrows(); ++r) {
        const int t = op->far.rows[r];
        for (int b = op->far.ptr[r]; b < op->far.ptr[r + 1]; ++b)
            soff[b + 1] = soff[b] + ((int64_t)R.rank[t] * R.rank[op->far.col[b]] + 3) / 4 * 4;
    }
    int rc;
    if (f32) {
        std::vector<float> Bf(B.begin(), B.end()), Ef(R.E.begin(), R.E.end());
        if ((rc = upload(op->basisV, Bf)) || (rc = upload(op->g_E, Ef))) return rc;
    } else {
        if ((rc = upload(op->basisV, B)) || (rc = upload(op->g_E, R.E))) return rc;
    }
    if ((rc = upload(op->g_rank, R.rank)) || (rc = upload(op->g_pivoff, R.piv_off)) || (rc = upload(op->g_piv, R.piv)) ||
        (rc = upload(op->g_eoff, eoff)) || (rc = upload(op->g_soff, soff)))
        return rc;
    const int64_t ns = soff.back();
    if ((rc = op->g_S.alloc((size_t)std::max<int64_t>(ns, 1) * es))) return rc;
    h2::launch_gca_assemble(op->geom(), op->consts, op->far.nrows(), op->far.drows.as<int>(), op->far.dptr.as<int>(),
                            op->far.dcol.as<int>(), op->g_rank.as<int>(), op->g_pivoff.as<int>(), op->g_piv.as<int>(),
                            op->g_soff.as<int64_t>(), f32, op->g_S.p, 0);
    CU(cudaGetLastError());
    op->gca_bytes = (int64_t)((size_t)ns * es + R.E.size() * es);
    return H2BEM_OK;
}

extern "C" int h2bem_gca_bases(const h2bem_mesh* mesh, const h2bem_tree* tree, const h2bem_opts* opts_in,
                               int64_t* rank, int64_t* npiv, int64_t* piv) {
    if (!mesh || !tree || !opts_in) return fail(H2BEM_ERR_ARG, "gca_bases: NULL argument");
    if (tree->n != mesh->nt) return fail(H2BEM_ERR_ARG, "gca_bases: tree and mesh differ in size");
    const h2bem_opts& opts = *opts_in;
    if (opts.gca_q < 1 || opts.gca_q > 16 || opts.gca_kmax < 1 || opts.gca_kmax > h2::kGcaMaxRank ||
        !(opts.gca_eps >= 0.0) || !std::isfinite(opts.gca_eps))
        return fail(H2BEM_ERR_ARG, "gca_bases: gca_q in 1..16, gca_kmax in 1..%d, gca_eps >= 0", h2::kGcaMaxRank);
    std::vector<double> glx, glw;
    gauss_legendre(opts.gca_q, glx, glw);
    const double r15 = std::sqrt(15.0);
    const double a = (6.0 - r15) / 21.0, b = (6.0 + r15) / 21.0;
    const double wa = (155.0 - r15) / 1200.0, wb = (155.0 + r15) / 1200.0;
    const double u[7] = {1.0 / 3.0, a, 1.0 - 2.0 * a, a, b, 1.0 - 2.0 * b, b};
    const double v[7] = {1.0 / 3.0, a, a, 1.0 - 2.0 * a, b, b, 1.0 - 2.0 * b};
    const double w[7] = {9.0 / 40.0, wa, wa, wa, wb, wb, wb};
    h2::GcaSetup S{};
    S.xyz = mesh->xyz.data();
    S.tri = mesh->tri.data();
    S.n = tree->n;
    S.nc = tree->nc;
    S.perm = tree->perm.data();
    S.begin = tree->begin.data();
    S.end = tree->end.data();
    S.child0 = tree->child0.data();
    S.child1 = tree->child1.data();
    S.level = tree->level.data();
    S.bmin = tree->bmin.data();
    S.bmax = tree->bmax.data();
    S.q = opts.gca_q;
    S.kmax = opts.gca_kmax;
    S.eps = opts.gca_eps;
    S.gl_x = glx.data();
    S.gl_w = glw.data();
    S.ru = u;
    S.rv = v;
    S.rw = w;
    h2::GcaResult R;
    h2::gca_build(S, R);
    if (rank)
        for (int64_t c = 0; c < tree->nc; ++c) rank[c] = R.rank[c];
    if (npiv) *npiv = (int64_t)R.piv.size();
    if (piv)
        for (size_t e = 0; e < R.piv.size(); ++e) piv[e] = R.piv[e];
    return H2BEM_OK;
}

// Radon's 7-point rule on the unit simplex (degree 5; weights sum to 1)
static void radon7_rule(double* u, double* v, double* w) {
    const double r15 = std::sqrt(15.0);
    const double a = (6.0 - r15) / 21.0, b = (6.0 + r15) / 21.0;
    const double wa = (155.0 - r15) / 1200.0, wb = (155.0 + r15) / 1200.0;
    const double uu[7] = {1.0 / 3.0, a, 1.0 - 2.0 * a, a, b, 1.0 - 2.0 * b, b};
    const double vv[7] = {1.0 / 3.0, a, a, 1.0 - 2.0 * a, b, b, 1.0 - 2.0 * b};
    const double ww[7] = {9.0 / 40.0, wa, wa, wa, wb, wb, wb};
    for (int q = 0; q < 7; ++q) {
        u[q] = uu[q];
        v[q] = vv[q];
        w[q] = ww[q];
    }
}

static int check_hca_opts(const h2bem_opts& o, int m, const char* who) {
    (void)m;
    if (o.hca_kaca < 1) return fail(H2BEM_ERR_ARG, "%s: hca_kaca must be >= 1", who);
    if (o.hca_kmax < 1 || o.hca_kmax > h2::kGcaMaxRank)
        return fail(H2BEM_ERR_ARG, "%s: hca_kmax must be in 1..%d", who, h2::kGcaMaxRank);
    if (!(o.hca_eps_aca >= 0.0) || !std::isfinite(o.hca_eps_aca) || !(o.hca_eps >= 0.0) || !std::isfinite(o.hca_eps))
        return fail(H2BEM_ERR_ARG, "%s: hca_eps_aca and hca_eps must be finite and >= 0", who);
    return H2BEM_OK;
}

static void hca_setup_fill(h2::HcaSetup& S, const h2bem_mesh* mesh, const h2bem_tree* tree, int m,
                           const h2bem_opts& opts, const double* ru, const double* rv, const double* rw) {
    S.xyz = mesh->xyz.data();
    S.tri = mesh->tri.data();
    S.n = tree->n;
    S.nc = tree->nc;
    S.perm = tree->perm.data();
    S.begin = tree->begin.data();
    S.end = tree->end.data();
    S.child0 = tree->child0.data();
    S.child1 = tree->child1.data();
    S.level = tree->level.data();
    S.bmin = tree->bmin.data();
    S.bmax = tree->bmax.data();
    S.m = m;
    S.kaca = opts.hca_kaca;
    S.kmax = opts.hca_kmax;
    S.eps_aca = opts.hca_eps_aca;
    S.eps_c = opts.hca_eps;
    S.ru = ru;
    S.rv = rv;
    S.rw = rw;
}

// HCA bases of the operator: construction on the host for the blocks of the
// farfield CSR, then leaf bases [pos][K] (zero-padded), transfers, couplings
// in CSR order and transposed couplings in the order of far_t (column-major,
// every block on a 16-byte boundary), uploaded in the tier's precision.
static int hca_setup(h2bem_op* op, const h2bem_mesh* mesh, const h2bem_tree* tree, const h2bem_opts& opts) {
    const int64_t n = op->n, nc = op->nc;
    std::vector<int> bt, bs;
    for (int r = 0; r < op->far.nrows(); ++r)
        for (int b = op->far.ptr[r]; b < op->far.ptr[r + 1]; ++b) {
            bt.push_back(op->far.rows[r]);
            bs.push_back(op->far.col[b]);
        }
    double ru[7], rv[7], rw[7];
    radon7_rule(ru, rv, rw);
    h2::HcaSetup S{};
    hca_setup_fill(S, mesh, tree, op->m, opts, ru, rv, rw);
    S.nfar = (int64_t)bt.size();
    S.far_t = bt.data();
    S.far_s = bs.data();
    h2::HcaResult R;
    h2::hca_build(S, R);
    int kmax = 1;
    double rsum = 0.0;
    for (int64_t c = 0; c < nc; ++c) {
        kmax = std::max(kmax, R.rank[c]);
        rsum += R.rank[c];
    }
    op->gca = 1;
    op->hca = 1;
    op->gca_mean_rank = nc ? rsum / nc : 0.0;
    const int K = (kmax + 3) / 4 * 4;
    op->k = K;
    const bool f32 = op->precision != H2BEM_FP64;
    const size_t es = f32 ? sizeof(float) : sizeof(double);
    std::vector<double> B((size_t)n * K, 0.0);
    for (int64_t c = 0; c < nc; ++c) {
        if (tree->child0[c] >= 0) continue;
        const int rk = R.rank[c];
        for (int64_t a = tree->begin[c]; a < tree->end[c]; ++a)
            for (int nu = 0; nu < rk; ++nu) B[(size_t)a * K + nu] = R.V[R.voff[c] + (a - tree->begin[c]) * rk + nu];
    }
    std::vector<int64_t> eoff(nc, 0);
    for (int64_t c = 0; c < nc; ++c) eoff[c] = R.eoff[c] < 0 ? 0 : R.eoff[c];
    auto pad4 = [](int64_t e) { return (e + 3) / 4 * 4; };
    // forward couplings in CSR order
    const int64_t nf = (int64_t)bt.size();
    std::vector<int64_t> soff(nf + 1, 0);
    for (int64_t b = 0; b < nf; ++b) soff[b + 1] = soff[b] + pad4((int64_t)R.rank[bt[b]] * R.rank[bs[b]]);
    // the coupling kernel streams every block column-major (entry (nu, mu) of
    // a kt x ks block at mu kt + nu); hca_build returns them row-major
    std::vector<double> Sf(std::max<int64_t>(soff[nf], 1), 0.0);
    for (int64_t b = 0; b < nf; ++b) {
        const int kt = R.rank[bt[b]], ks = R.rank[bs[b]];
        for (int nu = 0; nu < kt; ++nu)
            for (int mu = 0; mu < ks; ++mu) Sf[soff[b] + (int64_t)mu * kt + nu] = R.S[R.soff[b] + (int64_t)nu * ks + mu];
    }
    // transposed couplings in the order of far_t (row s, column t: S_(t,s)^T)
    std::vector<int64_t> first(nc + 1, 0);  // forward blocks of row t: [first[t], first[t+1]) in CSR order
    for (int64_t b = 0; b < nf; ++b) first[bt[b] + 1]++;
    for (int64_t c = 0; c < nc; ++c) first[c + 1] += first[c];
    const int64_t nft = (int64_t)op->far_t.col.size();
    std::vector<int64_t> sofft(nft + 1, 0);
    std::vector<int64_t> fwd(nft, -1);
    for (int r = 0; r < op->far_t.nrows(); ++r) {
        const int sc = op->far_t.rows[r];
        for (int q = op->far_t.ptr[r]; q < op->far_t.ptr[r + 1]; ++q) {
            const int tc = op->far_t.col[q];
            for (int64_t b = first[tc]; b < first[tc + 1]; ++b)
                if (bs[b] == sc) {
                    fwd[q] = b;
                    break;
                }
            if (fwd[q] < 0) return fail(H2BEM_ERR_STATE, "operator_create: HCA transposed block list is inconsistent");
            sofft[q + 1] = sofft[q] + pad4((int64_t)R.rank[sc] * R.rank[tc]);
        }
    }
    // S_b^T (ks x kt) column-major is S_b row-major
    std::vector<double> St(std::max<int64_t>(sofft[nft], 1), 0.0);
    for (int64_t q = 0; q < nft; ++q) {
        const int64_t b = fwd[q];
        std::copy(R.S.begin() + R.soff[b], R.S.begin() + R.soff[b + 1], St.begin() + sofft[q]);
    }
    int rc;
    if (f32) {
        std::vector<float> Bf(B.begin(), B.end()), Ef(R.E.begin(), R.E.end()), Sff(Sf.begin(), Sf.end()),
            Stf(St.begin(), St.end());
        if ((rc = upload(op->basisV, Bf)) || (rc = upload(op->g_E, Ef)) || (rc = upload(op->g_S, Sff)) ||
            (rc = upload(op->g_St, Stf)))
            return rc;
    } else {
        if ((rc = upload(op->basisV, B)) || (rc = upload(op->g_E, R.E)) || (rc = upload(op->g_S, Sf)) ||
            (rc = upload(op->g_St, St)))
            return rc;
    }
    if ((rc = upload(op->g_rank, R.rank)) || (rc = upload(op->g_eoff, eoff)) || (rc = upload(op->g_soff, soff)) ||
        (rc = upload(op->g_soff_t, sofft)))
        return rc;
    op->gca_bytes = (int64_t)((soff[nf] + sofft[nft] + (int64_t)R.E.size()) * es);
    return H2BEM_OK;
}

extern "C" int h2bem_hca_ranks(const h2bem_mesh* mesh, const h2bem_tree* tree, int m, double eta,
                               const h2bem_opts* opts_in, int64_t* rank, int64_t* nfar, int64_t* brank) {
    if (!mesh || !tree || !opts_in) return fail(H2BEM_ERR_ARG, "hca_ranks: NULL argument");
    if (tree->n != mesh->nt) return fail(H2BEM_ERR_ARG, "hca_ranks: tree and mesh differ in size");
    if (m < 1 || m > kMaxM) return fail(H2BEM_ERR_ARG, "hca_ranks: m must be in 1..%d", kMaxM);
    if (!(eta >= 0.0) || !std::isfinite(eta)) return fail(H2BEM_ERR_ARG, "hca_ranks: eta must be finite and >= 0");
    int rc;
    if ((rc = check_hca_opts(*opts_in, m, "hca_ranks"))) return rc;
    Blocks Bl;
    build_blocks(*tree, eta, Bl);
    std::vector<int> bt(Bl.ft.begin(), Bl.ft.end()), bs(Bl.fs.begin(), Bl.fs.end());
    double ru[7], rv[7], rw[7];
    radon7_rule(ru, rv, rw);
    h2::HcaSetup S{};
    hca_setup_fill(S, mesh, tree, m, *opts_in, ru, rv, rw);
    S.nfar = (int64_t)bt.size();
    S.far_t = bt.data();
    S.far_s = bs.data();
    h2::HcaResult R;
    h2::hca_build(S, R);
    if (rank)
        for (int64_t c = 0; c < tree->nc; ++c) rank[c] = R.rank[c];
    if (nfar) *nfar = S.nfar;
    if (brank)
        for (int64_t b = 0; b < S.nfar; ++b) brank[b] = R.brank[b];
    return H2BEM_OK;
}

static int create_impl(const h2bem_mesh* mesh, const h2bem_tree* tree, const Blocks* prebuilt, int kernel, int m,
                       double eta, const h2bem_opts* opts_in, h2bem_op** out) {
    if (!out) return fail(H2BEM_ERR_ARG, "operator_create: out is NULL");
    *out = nullptr;
    if (!mesh || !tree) return fail(H2BEM_ERR_ARG, "operator_create: NULL mesh or tree");
    if (tree->n != mesh->nt) return fail(H2BEM_ERR_ARG, "operator_create: tree is for %lld triangles, mesh has %lld",
                                         (long long)tree->n, (long long)mesh->nt);
    if (kernel != H2BEM_SLP && kernel != H2BEM_DLP) return fail(H2BEM_ERR_ARG, "operator_create: kernel must be SLP or DLP");
    if (m < 1 || m > kMaxM) return fail(H2BEM_ERR_ARG, "operator_create: m must be in 1..%d", kMaxM);
    if (!(eta >= 0.0) || !std::isfinite(eta)) return fail(H2BEM_ERR_ARG, "operator_create: eta must be finite and >= 0");
    h2bem_opts opts;
    h2bem_opts_default(&opts);
    if (opts_in) opts = *opts_in;
    if (opts.q_ss < 1 || opts.q_ss > h2::kMaxQss) return fail(H2BEM_ERR_ARG, "operator_create: q_ss must be in 1..%d", h2::kMaxQss);
    if (opts.precision < H2BEM_FP64 || opts.precision > H2BEM_MIXED_BF16)
        return fail(H2BEM_ERR_ARG, "operator_create: unknown precision tier %d", opts.precision);
    if ((opts.precision == H2BEM_MIXED_TF32 && !h2::coupling_tc_supported(m, 0)) ||
        (opts.precision == H2BEM_MIXED_BF16 && !h2::coupling_tc_supported(m, 2)))
        return fail(H2BEM_ERR_ARG, "operator_create: the tensor-core tiers need m <= 5 (k <= 128), got m = %d", m);
    if (opts.tc_wait_test != 0 && opts.tc_wait_test != 1)
        return fail(H2BEM_ERR_ARG, "operator_create: tc_wait_test must be 0 or 1");
    if (opts.basis != H2BEM_BASIS_CHEBYSHEV && opts.basis != H2BEM_BASIS_GCA && opts.basis != H2BEM_BASIS_HCA)
        return fail(H2BEM_ERR_ARG, "operator_create: unknown basis %d", opts.basis);
    if (opts.basis == H2BEM_BASIS_HCA) {
        if (kernel != H2BEM_SLP) return fail(H2BEM_ERR_ARG, "operator_create: HCA bases are built for the single layer");
        if (opts.precision != H2BEM_FP64 && opts.precision != H2BEM_MIXED_FP32)
            return fail(H2BEM_ERR_ARG, "operator_create: HCA bases run in the FP64 and MIXED_FP32 tiers");
        if (opts.recompute_basis) return fail(H2BEM_ERR_ARG, "operator_create: HCA bases are stored (recompute_basis = 0)");
        int rc;
        if ((rc = check_hca_opts(opts, m, "operator_create"))) return rc;
    }
    if (opts.basis == H2BEM_BASIS_GCA) {
        if (kernel != H2BEM_SLP) return fail(H2BEM_ERR_ARG, "operator_create: GCA bases are built for the single layer");
        if (opts.precision != H2BEM_FP64 && opts.precision != H2BEM_MIXED_FP32)
            return fail(H2BEM_ERR_ARG, "operator_create: GCA bases run in the FP64 and MIXED_FP32 tiers");
        if (opts.recompute_basis) return fail(H2BEM_ERR_ARG, "operator_create: GCA bases are stored (recompute_basis = 0)");
        if (opts.gca_q < 1 || opts.gca_q > 16) return fail(H2BEM_ERR_ARG, "operator_create: gca_q must be in 1..16");
        if (opts.gca_kmax < 1 || opts.gca_kmax > h2::kGcaMaxRank)
            return fail(H2BEM_ERR_ARG, "operator_create: gca_kmax must be in 1..%d", h2::kGcaMaxRank);
        if (!(opts.gca_eps >= 0.0) || !std::isfinite(opts.gca_eps))
            return fail(H2BEM_ERR_ARG, "operator_create: gca_eps must be finite and >= 0");
    }
    for (int64_t c = 0; c < tree->nc; ++c)
        if (tree->child0[c] < 0 && tree->end[c] - tree->begin[c] > kMaxLeaf)
            return fail(H2BEM_ERR_ARG, "operator_create: leaf clusters may hold at most %d triangles", kMaxLeaf);
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1)
        return fail(H2BEM_ERR_CUDA, "operator_create: no CUDA device");

    std::unique_ptr<h2bem_op> op(new (std::nothrow) h2bem_op);
    if (!op) return fail(H2BEM_ERR_OOM, "operator_create: out of host memory");
    op->kernel = kernel;
    op->m = m;
    op->k = m * m * m;
    op->eta = eta;
    op->precision = opts.precision;
    op->q_ss = opts.q_ss;
    op->cache_singular = opts.cache_singular ? 1 : 0;
    op->use_graph = opts.use_graph ? 1 : 0;
    if (opts.autotune < 0 || opts.autotune > 37)
        return fail(H2BEM_ERR_ARG, "operator_create: autotune must be 0, 1 or 2..37, got %d", opts.autotune);
    op->autotune = opts.autotune == 1 ? 1 : 0;
    op->singular_fp64 = opts.singular_fp64 ? 1 : 0;
    op->recompute_basis = opts.recompute_basis ? 1 : 0;
    op->store_near = opts.store_near ? 1 : 0;
    op->tc_wait_test = opts.tc_wait_test;
    if (opts.autotune >= 2) {  // a fixed launch variant for every width and direction
        const int v = opts.autotune - 2;
        for (auto& slot : op->tuned)
            for (auto& tu : slot) {
                tu.done = true;
                tu.near_persist = (v & 1) != 0;
                tu.coup_persist = (v & 2) != 0;
                tu.coup.nsl = (v / 4) % 3 == 0 ? 2 : (v / 4) % 3 == 1 ? 4 : 8;
                tu.near_nb = v / 12 == 0 ? 0 : v / 12 == 1 ? 3 : 2;
            }
    }
    op->n = mesh->nt;
    op->nv = mesh->nv;
    op->nc = tree->nc;
    op->depth = tree->depth;
    const int64_t n = op->n, nc = op->nc;

    // constants
    h2::Consts& C = op->consts;
    C.m = m;
    C.k = m * m * m;
    for (int a = 0; a < m; ++a) C.cheb[a] = std::cos((2.0 * a + 1.0) * M_PI / (2.0 * m));
    for (int a = 0; a < m; ++a) {
        C.cheb_hi[a] = (float)C.cheb[a];
        C.cheb_lo[a] = (float)(C.cheb[a] - (double)C.cheb_hi[a]);
    }
    for (int a = 0; a < m; ++a) {
        double pr = 1.0;
        for (int b = 0; b < m; ++b)
            if (b != a) pr *= C.cheb[a] - C.cheb[b];
        C.bary[a] = 1.0 / pr;
    }
    {
        const double r = std::sqrt(15.0);
        const double a = (6.0 - r) / 21.0, b = (6.0 + r) / 21.0;
        const double wa = (155.0 - r) / 1200.0, wb = (155.0 + r) / 1200.0;
        const double u[7] = {1.0 / 3.0, a, 1.0 - 2.0 * a, a, b, 1.0 - 2.0 * b, b};
        const double v[7] = {1.0 / 3.0, a, a, 1.0 - 2.0 * a, b, b, 1.0 - 2.0 * b};
        const double w[7] = {9.0 / 40.0, wa, wa, wa, wb, wb, wb};
        for (int p = 0; p < 7; ++p) {
            C.ru[p] = u[p];
            C.rv[p] = v[p];
            C.rw[p] = w[p];
            C.rwf[p] = (float)w[p];
            C.ruf[p] = (float)(u[p] - 1.0 / 3.0);
            C.rvf[p] = (float)(v[p] - 1.0 / 3.0);
        }
    }
    // leaf-basis rule: collapsed Gauss, exact for total degree 3(m-1)
    {
        std::vector<double> rule;
        basis_rule_host(m, rule);
        C.nb = (int)(rule.size() / 3);
        if (C.nb > h2::kMaxBasisPts) return fail(H2BEM_ERR_ARG, "operator_create: basis rule too large");
        int rc = upload(op->basis_rule, rule);
        if (rc) return rc;
    }

    // tree arrays, interpolation boxes (half-widths floored at 1e-2 of the largest)
    std::vector<int> iperm(n), permv(n), cb(nc), ce(nc), c0(nc), c1(nc);
    std::vector<double> box(9 * nc);
    for (int64_t i = 0; i < n; ++i) {
        permv[i] = (int)tree->perm[i];
        iperm[tree->perm[i]] = (int)i;
    }
    for (int64_t c = 0; c < nc; ++c) {
        cb[c] = (int)tree->begin[c];
        ce[c] = (int)tree->end[c];
        c0[c] = (int)tree->child0[c];
        c1[c] = (int)tree->child1[c];
        double h[3], hmax = 0.0;
        for (int d = 0; d < 3; ++d) {
            box[d * nc + c] = 0.5 * (tree->bmin[3 * c + d] + tree->bmax[3 * c + d]);
            h[d] = 0.5 * (tree->bmax[3 * c + d] - tree->bmin[3 * c + d]);
            hmax = std::max(hmax, h[d]);
        }
        for (int d = 0; d < 3; ++d) {
            box[(3 + d) * nc + c] = std::max(h[d], 1e-2 * hmax);
            box[(6 + d) * nc + c] = 1.0 / box[(3 + d) * nc + c];
        }
        if (c0[c] < 0) op->leaves_h.push_back((int)c);
        else {
            if ((int64_t)op->level_parents.size() <= tree->level[c]) op->level_parents.resize(tree->level[c] + 1);
            op->level_parents[tree->level[c]].push_back((int)c);
        }
    }
    // interpolation nodes z = c + h cheb[a] of every cluster and axis as FP32 (hi, lo)
    std::vector<float> zhl((size_t)nc * 3 * m * 2);
    for (int64_t c = 0; c < nc; ++c)
        for (int d = 0; d < 3; ++d)
            for (int a = 0; a < m; ++a) {
                const double z = box[d * nc + c] + box[(3 + d) * nc + c] * op->consts.cheb[a];
                const float hi = (float)z;
                const size_t e = (((size_t)c * 3 + d) * m + a) * 2;
                zhl[e] = hi;
                zhl[e + 1] = (float)(z - (double)hi);
            }
    // FP32 transfer factors of every child to its parent: L_{p,a}(z_{c}[a']) with
    // yhat = (z - c_p) / h_p, by barycentric products in FP64, rounded once
    std::vector<float> etr((size_t)nc * 3 * m * m, 0.0f);
    for (int64_t p = 0; p < nc; ++p) {
        if (c0[p] < 0) continue;
        for (int ch : {c0[p], c1[p]})
            for (int d = 0; d < 3; ++d)
                for (int ap = 0; ap < m; ++ap) {
                    const double z = box[d * nc + ch] + box[(3 + d) * nc + ch] * op->consts.cheb[ap];
                    const double yh = (z - box[d * nc + p]) * box[(6 + d) * nc + p];
                    for (int a = 0; a < m; ++a) {
                        double pr = op->consts.bary[a];
                        for (int b = 0; b < m; ++b)
                            if (b != a) pr *= yh - op->consts.cheb[b];
                        etr[(((size_t)ch * 3 + d) * m + ap) * m + a] = (float)pr;
                    }
                }
    }
    op->nleaves = (int64_t)op->leaves_h.size();
    std::vector<int> leaf_index(nc, -1);
    for (size_t l = 0; l < op->leaves_h.size(); ++l) leaf_index[op->leaves_h[l]] = (int)l;

    // block lists
    Blocks B;
    if (prebuilt) B = *prebuilt;
    else build_blocks(*tree, eta, B);
    op->nfar = (int64_t)B.ft.size();
    op->nnear = (int64_t)B.nt.size();
    op->near_pairs = 0;
    for (size_t b = 0; b < B.nt.size(); ++b)
        op->near_pairs += (tree->end[B.nt[b]] - tree->begin[B.nt[b]]) * (tree->end[B.ns[b]] - tree->begin[B.ns[b]]);
    make_csr(nc, B.ft, B.fs, op->far);
    make_csr(nc, B.fs, B.ft, op->far_t);
    make_csr(nc, B.nt, B.ns, op->near);
    {
        // The nearfield is applied by unordered pairs of leaves; the block
        // tree of one cluster tree with a symmetric admissibility condition
        // contains (s, t) with every (t, s).
        std::vector<std::pair<int64_t, int64_t>> fwd(B.nt.size()), bwd(B.nt.size());
        std::vector<int64_t> ut, us;
        for (size_t b = 0; b < B.nt.size(); ++b) {
            fwd[b] = {B.nt[b], B.ns[b]};
            bwd[b] = {B.ns[b], B.nt[b]};
            if (B.ns[b] >= B.nt[b]) {
                ut.push_back(B.nt[b]);
                us.push_back(B.ns[b]);
            }
        }
        std::sort(fwd.begin(), fwd.end());
        std::sort(bwd.begin(), bwd.end());
        if (fwd != bwd) return fail(H2BEM_ERR_ARG, "operator_create: nearfield block list is not symmetric");
        make_csr(nc, ut, us, op->near_u);
    }

    // singular pairs (tree positions), sorted by outer position
    std::vector<int64_t> slo[3], shi[3];
    std::vector<int> scode[3];
    singular_pairs(*mesh, slo, shi, scode);
    std::vector<double> tabs[3], tvg, tgram_edge, te1;
    ss_tables(op->q_ss, tabs[0], tgram_edge, tabs[2], tvg, te1);
    tabs[1] = te1;
    const int widths[3] = {4, 4, 3};

    int rc;
    if ((rc = upload(op->xyz, mesh->xyz)) || (rc = upload(op->tri, std::vector<int>(mesh->tri.begin(), mesh->tri.end()))) ||
        (rc = upload(op->perm, permv)) || (rc = upload(op->iperm, iperm)) || (rc = upload(op->cbegin, cb)) ||
        (rc = upload(op->cend, ce)) || (rc = upload(op->cchild0, c0)) || (rc = upload(op->cchild1, c1)) ||
        (rc = upload(op->cbox, box)) || (rc = upload(op->czhl, zhl)) || (rc = upload(op->cetr, etr)) || (rc = upload(op->leaves, op->leaves_h)))
        return rc;
    if ((rc = op->far.upload_all()) || (rc = op->far_t.upload_all()) || (rc = op->near.upload_all()) ||
        (rc = op->near_u.upload_all()) || (rc = op->work.alloc(4 * sizeof(int))))
        return rc;
    {
        // triangles at each vertex (caller's order), for the hypersingular operator
        std::vector<int> vp(op->nv + 1, 0), vi(3 * n);
        for (int64_t e = 0; e < 3 * n; ++e) vp[mesh->tri[e] + 1]++;
        for (int64_t v = 0; v < op->nv; ++v) vp[v + 1] += vp[v];
        std::vector<int> fill(vp.begin(), vp.end() - 1);
        for (int64_t e = 0; e < 3 * n; ++e) vi[fill[mesh->tri[e]]++] = (int)e;
        if ((rc = upload(op->vptr, vp)) || (rc = upload(op->vinc, vi))) return rc;
    }
    op->dlevel.resize(op->level_parents.size());
    for (size_t L = 0; L < op->level_parents.size(); ++L)
        if ((rc = upload(op->dlevel[L], op->level_parents[L]))) return rc;
    {
        // the top levels: up to the first level with more than kTreeTopParents
        // parents, at most kTreeTopLevels (the downward walk holds the path)
        constexpr size_t kTreeTopParents = 1024;
        constexpr int kTreeTopLevels = 32;
        int L0 = 0;
        while (L0 < (int)op->level_parents.size() && L0 < kTreeTopLevels &&
               op->level_parents[L0].size() <= kTreeTopParents)
            ++L0;
        op->tree_L0 = L0;
        std::vector<int> start;
        for (int64_t cl = 0; cl < nc; ++cl)
            if (tree->level[cl] == L0 || (c0[cl] < 0 && tree->level[cl] < L0)) start.push_back((int)cl);
        op->tree_nstart = (int)start.size();
        if ((rc = upload(op->tree_start, start)) || (rc = op->tree_cnt.alloc(nc * sizeof(unsigned)))) return rc;
        CU(cudaMemset(op->tree_cnt.p, 0, nc * sizeof(unsigned)));
    }
    {
        // pairs the regular nearfield kernel evaluates: all pairs of the
        // blocks (t, s >= t) that share no vertex, both orders in s = t
        std::vector<int> leaf_of(n);
        for (int l : op->leaves_h)
            for (int64_t p = tree->begin[l]; p < tree->end[l]; ++p) leaf_of[p] = l;
        int64_t ev = 0;
        for (size_t r = 0; r < op->near_u.rows.size(); ++r) {
            const int t0 = op->near_u.rows[r];
            for (int b = op->near_u.ptr[r]; b < op->near_u.ptr[r + 1]; ++b) {
                const int s0 = op->near_u.col[b];
                ev += (tree->end[t0] - tree->begin[t0]) * (tree->end[s0] - tree->begin[s0]);
            }
        }
        for (int t = 0; t < 3; ++t)
            for (size_t p = 0; p < slo[t].size(); ++p)
                ev -= t == 0 ? 1 : leaf_of[iperm[slo[t][p]]] == leaf_of[iperm[shi[t][p]]] ? 2 : 1;
        op->regular_evals = ev;
    }
    for (int t = 0; t < 3; ++t) {
        const size_t np = slo[t].size();
        op->sing[t] = (int64_t)np;
        op->sp_count[t] = (int64_t)np;
        std::vector<int> lo(np), hi(np);
        for (size_t p = 0; p < np; ++p) {
            lo[p] = iperm[slo[t][p]];
            hi[p] = iperm[shi[t][p]];
        }
        op->sp_npts[t] = (int)(tabs[t].size() / widths[t]);
        if ((rc = upload(op->sp_lo[t], lo)) || (rc = upload(op->sp_hi[t], hi)) || (rc = upload(op->sp_code[t], scode[t])) ||
            (rc = upload(op->sp_tab[t], tabs[t])))
            return rc;
    }
    op->sing_gather = op->precision != H2BEM_FP64 && !op->singular_fp64;
    if (op->sing_gather) {
        // entries by row: (2 pid, other) in row lo, (2 pid + 1, lo) in row hi (once if lo = hi);
        // the double layer has no identical-pair entries (k_ii = 0)
        int64_t tot = 0;
        for (int t = 0; t < 3; ++t) {
            op->sg_off[t] = tot;
            tot += (int64_t)slo[t].size();
        }
        std::vector<int> ptr(n + 1, 0);
        for (int t = (kernel == H2BEM_DLP ? 1 : 0); t < 3; ++t)
            for (size_t p = 0; p < slo[t].size(); ++p) {
                const int lo = iperm[slo[t][p]], hi = iperm[shi[t][p]];
                ptr[lo + 1]++;
                if (hi != lo) ptr[hi + 1]++;
            }
        for (int64_t i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
        std::vector<int> fill(ptr.begin(), ptr.end() - 1);
        std::vector<int> other(ptr[n]);
        std::vector<int2> pos(std::max<int64_t>(tot, 1), make_int2(0, -1));
        for (int t = (kernel == H2BEM_DLP ? 1 : 0); t < 3; ++t)
            for (size_t p = 0; p < slo[t].size(); ++p) {
                const int lo = iperm[slo[t][p]], hi = iperm[shi[t][p]];
                int2& ps = pos[op->sg_off[t] + (int64_t)p];
                ps.x = fill[lo];
                other[fill[lo]++] = hi;
                if (hi != lo) {
                    ps.y = fill[hi];
                    other[fill[hi]++] = lo;
                }
            }
        const size_t nv = (size_t)std::max<int64_t>(ptr[n], 1);
        if ((rc = upload(op->sg_ptr, ptr)) || (rc = upload(op->sg_other, other)) || (rc = upload(op->sg_pos, pos)) ||
            (rc = op->sg_vals.alloc(nv * sizeof(float))))
            return rc;
        if (op->cache_singular && kernel == H2BEM_DLP && (rc = op->sg_vals_t.alloc(nv * sizeof(float)))) return rc;
    }
    // shape-gradient data: vertex realising each bounding-box extreme (first in
    // the cluster's triangle order, corners in order), floored axes, the axis
    // of the largest half-width, children and parents
    {
        std::vector<int> cext(6 * nc), cflag(nc), ch, par(nc, -1);
        for (int64_t c = 0; c < nc; ++c) {
            double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            int vlo[3] = {0, 0, 0}, vhi[3] = {0, 0, 0};
            for (int64_t a = tree->begin[c]; a < tree->end[c]; ++a)
                for (int q = 0; q < 3; ++q) {
                    const int32_t v = mesh->tri[3 * tree->perm[a] + q];
                    for (int d = 0; d < 3; ++d) {
                        const double val = mesh->xyz[3 * (int64_t)v + d];
                        if (val < lo[d]) { lo[d] = val; vlo[d] = v; }
                        if (val > hi[d]) { hi[d] = val; vhi[d] = v; }
                    }
                }
            double h[3], hmax = 0.0;
            int am = 0;
            for (int d = 0; d < 3; ++d) {
                cext[d * nc + c] = vlo[d];
                cext[(3 + d) * nc + c] = vhi[d];
                h[d] = 0.5 * (tree->bmax[3 * c + d] - tree->bmin[3 * c + d]);
                if (h[d] > hmax) { hmax = h[d]; am = d; }
            }
            int fl = am << 3;
            for (int d = 0; d < 3; ++d)
                if (h[d] < 1e-2 * hmax) fl |= 1 << d;
            cflag[c] = fl;
            if (tree->child0[c] >= 0) {
                ch.push_back((int)tree->child0[c]);
                ch.push_back((int)tree->child1[c]);
                par[tree->child0[c]] = par[tree->child1[c]] = (int)c;
            }
        }
        op->nchildren = (int)ch.size();
        int rc2;
        if ((rc2 = upload(op->cext, cext)) || (rc2 = upload(op->cflag, cflag)) || (rc2 = upload(op->children, ch)) ||
            (rc2 = upload(op->parent, par)) || (rc2 = upload(op->sp_gtab, tvg)) ||
            (rc2 = upload(op->sp_gtab_edge, tgram_edge)))
            return rc2;
        op->sp_gnpts = (int)(tvg.size() / 11);
        op->sp_gnpts_edge = (int)(tgram_edge.size() / 11);
    }
    // geometry in tree order
    if ((rc = op->v.alloc(9 * n * sizeof(double))) || (rc = op->area.alloc(n * sizeof(double))) ||
        (rc = op->nrm.alloc(3 * n * sizeof(double))) || (rc = op->ctr.alloc(3 * n * sizeof(double))) ||
        (rc = op->vid.alloc(3 * n * sizeof(int))) || (rc = op->qo.alloc(21 * n * sizeof(float))) ||
        (rc = op->qa.alloc(21 * n * sizeof(double))) || (rc = op->chl.alloc(6 * n * sizeof(float))) ||
        (rc = op->plane.alloc(n * sizeof(double))) || (rc = op->nef.alloc(18 * n * sizeof(float))) ||
        (rc = op->areaf.alloc(n * sizeof(float))))
        return rc;
    h2::launch_geom(op->xyz.as<double>(), op->tri.as<int>(), op->perm.as<int>(), (int)n, op->consts, op->v.as<double>(),
                    op->area.as<double>(), op->nrm.as<double>(), op->ctr.as<double>(), op->vid.as<int>(),
                    op->qo.as<float>(), op->qa.as<double>(), op->chl.as<float>(), op->plane.as<double>(),
                    op->nef.as<float>(), op->areaf.as<float>(), 0);
    CU(cudaGetLastError());
    // leaf bases: V_t[i, nu] = int L_nu; for the double layer also W_s[j, nu] = int n_j . grad L_nu
    for (int l : op->leaves_h) op->max_leaf = std::max(op->max_leaf, (int)(tree->end[l] - tree->begin[l]));
    if (opts.basis == H2BEM_BASIS_GCA) {
        if ((rc = gca_setup(op.get(), mesh, tree, opts))) return rc;
    } else if (opts.basis == H2BEM_BASIS_HCA) {
        if ((rc = hca_setup(op.get(), mesh, tree, opts))) return rc;
    } else if (!op->recompute_basis) {
        const bool v32 = op->precision != H2BEM_FP64;
        if ((rc = op->basisV.alloc((size_t)n * op->k * (v32 ? sizeof(float) : sizeof(double))))) return rc;
        h2::launch_leaf_basis(op->geom(), op->tree(), op->consts, op->basis_rule.as<double>(), (int)op->nleaves,
                              op->leaves.as<int>(), false, v32, op->basisV.p, 0);
        CU(cudaGetLastError());
        if (kernel == H2BEM_DLP) {
            if ((rc = op->basisW.alloc((size_t)n * op->k * sizeof(double)))) return rc;
            h2::launch_leaf_basis(op->geom(), op->tree(), op->consts, op->basis_rule.as<double>(), (int)op->nleaves,
                                  op->leaves.as<int>(), true, false, op->basisW.p, 0);
            CU(cudaGetLastError());
        }
    }
    // x-independent singular entries, evaluated once if requested: float pairs
    // for the row gather (FP32 points), else FP64 values for the scatter
    if (op->cache_singular && op->sing_gather) {
        // both orders for the double layer (A and A^T); the single layer is symmetric
        for (int tr = 0; tr < (kernel == H2BEM_DLP ? 2 : 1); ++tr)
            for (int t = (kernel == H2BEM_DLP ? 1 : 0); t < 3; ++t)
                h2::launch_singular(op->geom(), h2::IDENTICAL - t, kernel, (int)op->sp_count[t], op->sp_lo[t].as<int>(),
                                    op->sp_hi[t].as<int>(), op->sp_code[t].as<int>(), op->sp_tab[t].as<double>(),
                                    op->sp_npts[t], 3, true, tr == 1, 1, nullptr, nullptr,
                                    reinterpret_cast<double*>((tr ? op->sg_vals_t : op->sg_vals).as<float>()),
                                    reinterpret_cast<double*>(op->sg_pos.as<int2>() + op->sg_off[t]), 0);
        CU(cudaGetLastError());
    } else if (op->cache_singular) {
        for (int t = 0; t < 3; ++t) {
            const int np = (int)op->sp_count[t];
            if ((rc = op->sp_v0[t].alloc(np * sizeof(double))) || (rc = op->sp_v1[t].alloc(np * sizeof(double)))) return rc;
            if (t == 0 && kernel == H2BEM_DLP) {
                if (np) {
                    CU(cudaMemset(op->sp_v0[t].p, 0, np * sizeof(double)));
                    CU(cudaMemset(op->sp_v1[t].p, 0, np * sizeof(double)));
                }
                continue;
            }
            h2::launch_singular(op->geom(), h2::IDENTICAL - t, kernel, np, op->sp_lo[t].as<int>(), op->sp_hi[t].as<int>(),
                                op->sp_code[t].as<int>(), op->sp_tab[t].as<double>(), op->sp_npts[t], 1,
                                op->precision != H2BEM_FP64 && !op->singular_fp64, false, 1,
                                nullptr, nullptr, op->sp_v0[t].as<double>(), op->sp_v1[t].as<double>(), 0);
            CU(cudaGetLastError());
        }
    }
    if (op->store_near && (rc = build_near_store(op.get(), *tree, iperm, slo, shi))) return rc;
    CU(cudaDeviceSynchronize());
    for (auto& e : op->ev) CU(cudaEventCreate(&e));
    {
        int lo = 0, hi = 0;  // the farfield stream at the highest priority: its short
        CU(cudaDeviceGetStreamPriorityRange(&lo, &hi));  // dependent launches then start promptly
        CU(cudaStreamCreateWithPriority(&op->s_far, cudaStreamNonBlocking, hi));
        CU(cudaEventCreateWithFlags(&op->ev_fork, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&op->ev_join, cudaEventDisableTiming));
    }
    *out = op.release();
    return H2BEM_OK;
}

extern "C" int h2bem_operator_create(const h2bem_mesh* mesh, const h2bem_tree* tree, int kernel, int m, double eta,
                                     const h2bem_opts* opts, h2bem_op** out) {
    return create_impl(mesh, tree, nullptr, kernel, m, eta, opts, out);
}

// Block-diagonal operator over several meshes: the meshes are concatenated
// (vertex and triangle indices offset), their cluster trees form a forest
// (each built as by h2bem_tree_build), and block lists are built per mesh
// from its own root, so no block couples two meshes.
extern "C" int h2bem_batch_create(int nmeshes, const h2bem_mesh* const* meshes, int leaf_size, int kernel, int m,
                                  double eta, const h2bem_opts* opts, h2bem_op** out) {
    if (!out) return fail(H2BEM_ERR_ARG, "batch_create: out is NULL");
    *out = nullptr;
    if (nmeshes < 1 || !meshes) return fail(H2BEM_ERR_ARG, "batch_create: need at least one mesh");
    if (leaf_size < 1) return fail(H2BEM_ERR_ARG, "batch_create: leaf_size must be >= 1");
    if (!(eta >= 0.0) || !std::isfinite(eta)) return fail(H2BEM_ERR_ARG, "batch_create: eta must be finite and >= 0");
    h2bem_mesh U;
    h2bem_tree F;
    Blocks B;
    int64_t voff = 0, toff = 0, coff = 0;
    for (int b = 0; b < nmeshes; ++b) {
        const h2bem_mesh* M = meshes[b];
        if (!M) return fail(H2BEM_ERR_ARG, "batch_create: mesh %d is NULL", b);
        if (toff + M->nt > ((int64_t)1 << 30)) return fail(H2BEM_ERR_ARG, "batch_create: batch too large");
        h2bem_tree* T = nullptr;
        int rc = h2bem_tree_build(M, leaf_size, &T);
        if (rc) return rc;
        std::unique_ptr<h2bem_tree> Tp(T);
        U.xyz.insert(U.xyz.end(), M->xyz.begin(), M->xyz.end());
        for (int32_t v : M->tri) U.tri.push_back((int32_t)(v + voff));
        for (int64_t i = 0; i < T->n; ++i) F.perm.push_back(T->perm[i] + toff);
        for (int64_t c = 0; c < T->nc; ++c) {
            F.begin.push_back(T->begin[c] + toff);
            F.end.push_back(T->end[c] + toff);
            F.child0.push_back(T->child0[c] < 0 ? -1 : T->child0[c] + coff);
            F.child1.push_back(T->child1[c] < 0 ? -1 : T->child1[c] + coff);
            F.parent.push_back(T->parent[c] < 0 ? -1 : T->parent[c] + coff);
            F.level.push_back(T->level[c]);
        }
        F.bmin.insert(F.bmin.end(), T->bmin.begin(), T->bmin.end());
        F.bmax.insert(F.bmax.end(), T->bmax.begin(), T->bmax.end());
        F.depth = std::max(F.depth, T->depth);
        Blocks Bm;
        build_blocks(*T, eta, Bm);
        for (size_t q = 0; q < Bm.ft.size(); ++q) {
            B.ft.push_back(Bm.ft[q] + coff);
            B.fs.push_back(Bm.fs[q] + coff);
        }
        for (size_t q = 0; q < Bm.nt.size(); ++q) {
            B.nt.push_back(Bm.nt[q] + coff);
            B.ns.push_back(Bm.ns[q] + coff);
        }
        voff += M->nv;
        toff += M->nt;
        coff += T->nc;
    }
    U.nv = voff;
    U.nt = toff;
    F.n = toff;
    F.nc = coff;
    return create_impl(&U, &F, &B, kernel, m, eta, opts, out);
}

extern "C" int h2bem_operator_destroy(h2bem_op* op) {
    if (op) cudaDeviceSynchronize();
    delete op;
    return H2BEM_OK;
}

static int resolve_timing(h2bem_op* op);

extern "C" int h2bem_stats_get(const h2bem_op* op, h2bem_stats* st) {
    if (!op || !st) return fail(H2BEM_ERR_ARG, "stats_get: NULL argument");
    // the stage times of a timed apply are read here (the operator's own
    // event buffer; the counts are unchanged)
    const int trc = resolve_timing(const_cast<h2bem_op*>(op));
    memset(st, 0, sizeof *st);
    st->n = op->n;
    st->nclusters = op->nc;
    st->nleaves = op->nleaves;
    st->depth = op->depth;
    st->nfar = op->nfar;
    st->nnear = op->nnear;
    st->near_pairs = op->near_pairs;
    st->singular_pairs[0] = op->sing[0];
    st->singular_pairs[1] = op->sing[1];
    st->singular_pairs[2] = op->sing[2];
    st->regular_pairs = op->near_pairs - op->sing[0] - 2 * (op->sing[1] + op->sing[2]);
    st->regular_evals = op->regular_evals;
    st->near_stored_bytes = op->nst_bytes;
    st->far_stored_bytes = op->gca_bytes;
    st->mean_rank = op->gca ? op->gca_mean_rank : (double)op->k;
    for (int i = 0; i < 5; ++i) st->launch_variant[i] = op->last_variant[i];
    st->k = op->k;
    st->launches = op->launches;
    st->last_apply_ms = op->last_ms;
    for (int i = 0; i < 8; ++i) st->stage_ms[i] = op->stage_ms[i];
    return trc;
}

// ===========================================================================
// apply
// ===========================================================================
static int pad_nr(int nrhs) { return nrhs <= 1 ? 1 : nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : 16; }

// Precision of the farfield vectors: FP64 tier everything double; mixed
// tier float, except on the side of the double layer's differentiated
// Lagrange basis W (input side of K, output side of K^T): W has large entries
// on thin boxes, and an FP32 x-hat (or y-hat) there loses ~1e-6, so that side
// keeps its basis, transfers and accumulations in double (for K x also the
// coupling entries, whose rounding the cancelling x-hat amplifies).
static bool xh_is64(const h2bem_op* op, bool tr) {
    return op->precision == H2BEM_FP64 || (op->kernel == H2BEM_DLP && !tr);
}
static bool yh_is64(const h2bem_op* op, bool tr) {
    return op->precision == H2BEM_FP64 || (op->kernel == H2BEM_DLP && tr);
}

// The regular nearfield of the FP32 single layer reads x in FP32 (xs).
static bool near_reads_xs(const h2bem_op* op) {
    return !op->store_near && op->precision != H2BEM_FP64 && op->kernel == H2BEM_SLP;
}

// x in the stored nearfield's precision (FP32 tiers, or a single FP64 column
// padded to 16 bytes), or in FP32 for the singular row gather and the FP32
// single layer's regular nearfield; 0 where none needs it (the stored FP64
// apply reads x directly)
static size_t store_x_bytes(const h2bem_op* op, int NR) {
    const bool f32 = op->precision != H2BEM_FP64;
    if (!op->store_near)
        return (op->sing_gather || near_reads_xs(op)) ? (size_t)op->n * h2::near_store_nx(true, NR) * sizeof(float) : 0;
    if (!f32 && NR > 1) return 0;
    return (size_t)op->n * h2::near_store_nx(f32, NR) * (f32 ? sizeof(float) : sizeof(double));
}

// Singular entries of an apply by rows: the float pairs of every canonical
// pair (evaluated here unless cached), x in FP32, and one gather launch;
// returns the number of launches.
static int64_t sing_gather_apply(const h2bem_op* op, int NR, bool transpose, const double* xp, double* yp, void* xs,
                                 bool xs_ready, cudaStream_t s) {
    const h2::Geom g = op->geom();
    const bool dlp = op->kernel == H2BEM_DLP;
    int64_t nl = 0;
    const bool tr = transpose && dlp;
    if (!op->cache_singular)
        for (int ty = (dlp ? 1 : 0); ty < 3; ++ty) {
            const int np = (int)op->sp_count[ty];
            h2::launch_singular(g, h2::IDENTICAL - ty, dlp ? h2::DLP : h2::SLP, np, op->sp_lo[ty].as<int>(),
                                op->sp_hi[ty].as<int>(), op->sp_code[ty].as<int>(), op->sp_tab[ty].as<double>(),
                                op->sp_npts[ty], 3, true, tr, 1, nullptr, nullptr,
                                reinterpret_cast<double*>(op->sg_vals.as<float>()),
                                reinterpret_cast<double*>(op->sg_pos.as<int2>() + op->sg_off[ty]), s);
            nl += np > 0 ? 1 : 0;
        }
    const float* vals = (op->cache_singular && tr) ? op->sg_vals_t.as<float>() : op->sg_vals.as<float>();
    if (!xs_ready) h2::launch_store_x(true, (int)op->n, NR, xp, xs, s);
    h2::launch_sing_gather(NR, (int)op->n, op->sg_ptr.as<int>(), op->sg_other.as<int>(), vals, (const float*)xs, yp, s);
    return nl + (xs_ready ? 1 : 2);
}

// Nearfield of an apply from the stored blocks (x converted first where
// needed): writes every row of yp; returns the number of launches.
static int64_t near_stored_apply(const h2bem_op* op, int NR, bool transpose, const double* xp, double* yp, void* xs,
                                 cudaStream_t s) {
    const bool f32 = op->precision != H2BEM_FP64;
    const bool tr = transpose && op->kernel == H2BEM_DLP;  // the stored single layer is symmetric
    int64_t nl = 0;
    const void* xsrc = xp;
    if (store_x_bytes(op, NR)) {
        h2::launch_store_x(f32, (int)op->n, NR, xp, xs, s);
        xsrc = xs;
        ++nl;
    }
    h2::launch_near_stored(f32, tr, NR, op->near.nrows(), op->nrow.as<h2::NearRow>(),
                           (tr ? op->nblk_t : op->nblk).as<h2::NearBlock>(), op->nst.p, xsrc, op->max_leaf, yp, s);
    return nl + (op->near.nrows() > 0 ? 1 : 0);
}

static int ensure_workspace(h2bem_op* op, int NR) {
    if (op->ws_NR >= NR) return H2BEM_OK;
    const bool wide = op->precision == H2BEM_FP64 || op->kernel == H2BEM_DLP;  // either direction
    const size_t xsz = wide ? sizeof(double) : sizeof(float);
    const size_t ysz = xsz;
    int rc;
    if ((rc = op->xp.alloc(op->n * NR * sizeof(double))) || (rc = op->yp.alloc(op->n * NR * sizeof(double))) ||
        (rc = op->xh.alloc((size_t)op->nc * op->k * NR * xsz)) || (rc = op->yh.alloc((size_t)op->nc * op->k * NR * ysz)) ||
        (rc = op->xs.alloc(store_x_bytes(op, NR))))
        return rc;
    op->ws_NR = NR;
    op->ws_gen++;
    return H2BEM_OK;
}

// Coupling stage: on the tensor cores in the TF32 / BF16 tiers where both
// cluster vectors are FP32, else the SIMT kernels.
static int tc_kind(const h2bem_op* op, bool xh64, bool yh64) {
    if (xh64 || yh64) return -1;
    if (op->precision == H2BEM_MIXED_TF32) return 0;
    if (op->precision == H2BEM_MIXED_BF16) return 2;
    return -1;
}

// Upward / downward pass of the Chebyshev bases: the wide levels (tree_L0 and
// below) one launch per level, the levels above in one launch each way (FP32,
// m = 4, up to 8 right-hand sides; else per level too).  Returns the launches
// issued.
static int64_t run_upward(h2bem_op* op, const h2::Tree& t, const h2::Consts& c, bool xh64, int NR, void* xh,
                          cudaStream_t s) {
    const int nlev = (int)op->level_parents.size();
    int64_t nl = 0;
    for (int L = nlev - 1; L >= op->tree_L0; --L, ++nl)
        h2::launch_upward(t, c, (int)op->level_parents[L].size(), op->dlevel[L].as<int>(), xh64, NR, xh, s);
    if (op->tree_L0 > 0 && h2::launch_tree_updown(true, t, c, op->tree_nstart, op->tree_start.as<int>(),
                                                  op->parent.as<int>(), op->tree_cnt.as<unsigned>(), xh64, NR, xh, s))
        return nl + 1;
    for (int L = op->tree_L0 - 1; L >= 0; --L, ++nl)
        h2::launch_upward(t, c, (int)op->level_parents[L].size(), op->dlevel[L].as<int>(), xh64, NR, xh, s);
    return nl;
}
static int64_t run_downward(h2bem_op* op, const h2::Tree& t, const h2::Consts& c, bool yh64, int NR, void* yh,
                            cudaStream_t s) {
    const int nlev = (int)op->level_parents.size();
    int64_t nl = 0;
    if (op->tree_L0 > 0 && h2::launch_tree_updown(false, t, c, op->tree_nstart, op->tree_start.as<int>(),
                                                  op->parent.as<int>(), nullptr, yh64, NR, yh, s)) {
        nl = 1;
    } else {
        for (int L = 0; L < op->tree_L0; ++L, ++nl)
            h2::launch_downward(t, c, (int)op->level_parents[L].size(), op->dlevel[L].as<int>(), yh64, NR, yh, s);
    }
    for (int L = op->tree_L0; L < nlev; ++L, ++nl)
        h2::launch_downward(t, c, (int)op->level_parents[L].size(), op->dlevel[L].as<int>(), yh64, NR, yh, s);
    return nl;
}

static void run_coupling(const h2bem_op* op, const h2::Tree& t, const h2::Consts& c, const Csr& far, bool xh64,
                         bool yh64, int NR, void* xh, void* yh, const h2::LaunchCfg& cfg, cudaStream_t s) {
    const int kind = tc_kind(op, xh64, yh64);
    // double-float entries and sums on the FP32 pipe: the FP64 tier, and the
    // double layer's FP64 side in the mixed tiers
    const bool df = op->precision == H2BEM_FP64 ||
                    (op->precision != H2BEM_FP64 && op->kernel == H2BEM_DLP && (xh64 || yh64));
    if (df && h2::coupling_df_supported(op->m, NR)) {
        h2::launch_coupling_df(t, c, far.nrows(), far.drows.as<int>(), far.dptr.as<int>(), far.dcol.as<int>(), NR,
                               xh64, yh64, xh, yh, s);
        return;
    }
    if (kind >= 0)
        h2::launch_coupling_tc(t, c, far.nrows(), far.drows.as<int>(), far.dptr.as<int>(), far.dcol.as<int>(), kind, NR,
                               (const float*)xh, (float*)yh, op->tc_wait_test, s);
    else
        h2::launch_coupling(t, c, far.nrows(), far.drows.as<int>(), far.dptr.as<int>(), far.dcol.as<int>(),
                            op->precision == H2BEM_FP64 ? 0 : 1, xh64, yh64, NR, xh, yh, cfg, s);
}

static int nr_slot(int NR) { return NR == 1 ? 0 : NR == 4 ? 1 : NR == 8 ? 2 : 3; }

// device time of f() on stream s: best of two after one warm-up (synchronises)
template <typename F>
static float time_on(cudaStream_t s, F f) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    f();
    float best = 1e30f;
    for (int r = 0; r < 2; ++r) {
        cudaEventRecord(a, s);
        f();
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// the launch variants an apply uses (tuned ones once the autotuner has run)
static void launch_cfgs(h2bem_op* op, int NR, bool transpose, h2::LaunchCfg& near, h2::LaunchCfg& coup) {
    const auto& tu = op->tuned[nr_slot(NR)][transpose ? 1 : 0];
    int* w = op->work.as<int>();
    near = h2::LaunchCfg{};
    coup = h2::LaunchCfg{};
    if (tu.done) {
        near.work = tu.near_persist ? w : nullptr;
        near.nb = tu.near_nb;
        coup.nsl = tu.coup.nsl;
        coup.work = tu.coup_persist ? w + 1 : nullptr;
    }
    op->last_variant[0] = near.work != nullptr;
    // register budget in effect: variants exist for the FP32 single layer, the others use 2 CTAs per SM
    const bool budgets = op->precision != H2BEM_FP64 && op->kernel == H2BEM_SLP;
    op->last_variant[1] = budgets ? (near.nb == 0 ? 4 : near.nb) : 2;
    op->last_variant[2] = coup.nsl;
    op->last_variant[3] = coup.work != nullptr;
    op->last_variant[4] = tu.done ? 1 : 0;
}

// Work vectors of one chunk: tree-ordered x and y (FP64, RHS-interleaved),
// the cluster vectors x-hat and y-hat, and x in FP32 for the singular row
// gather / the stored nearfield (store_x_bytes).
struct Work {
    double* xp;
    double* yp;
    void* xh;
    void* yh;
    void* xs;
};

// One chunk of at most 16 right-hand sides, device buffers, tree order work.
// ext = NULL: the operator's own work vectors (allocated or grown here);
// otherwise caller-provided ones of work_bytes() (no allocation, no tuning).
static int apply_chunk(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy, cudaStream_t s,
                       bool transpose, bool timed, bool xmapped = false, const Work* ext = nullptr) {
    const int NR = pad_nr(nrhs);
    Work w;
    if (ext) {
        w = *ext;
    } else {
        int rc = ensure_workspace(op, NR);
        if (rc) return rc;
        w = Work{op->xp.as<double>(), op->yp.as<double>(), op->xh.p, op->yh.p, op->xs.p};
    }
    const bool fp32 = op->precision != H2BEM_FP64;
    const bool xh64 = xh_is64(op, transpose), yh64 = yh_is64(op, transpose);
    const size_t ysz = yh64 ? sizeof(double) : sizeof(float);
    const h2::Geom g = op->geom();
    const h2::Tree t = op->tree();
    const h2::Consts& c = op->consts;
    const int n = (int)op->n;
    // forward basis and kernel variants: A = V S W^T + N;  A^T = W S^T V^T + N^T
    const bool dlp = op->kernel == H2BEM_DLP;
    const bool in_dlp = dlp && !transpose;   // W_s on the input side
    const bool out_dlp = dlp && transpose;   // W_s on the output side
    const int near_ker = !dlp ? h2::SLP : transpose ? h2::DLP_T : h2::DLP;
    // GCA: the single layer is symmetric and its coupling matrices are stored
    // for the blocks of `far`, so A^T x runs the forward farfield; HCA keeps
    // transposed couplings for the blocks of `far_t`
    const bool col_order = transpose && (!op->gca || op->hca);
    const Csr& far = col_order ? op->far_t : op->far;
    const DevBuf& g_soff = (transpose && op->hca) ? op->g_soff_t : op->g_soff;
    const DevBuf& g_S = (transpose && op->hca) ? op->g_St : op->g_S;
    auto mark = [&](int i) {
        if (timed) cudaEventRecord(op->ev[i], s);
    };
    int64_t nl = 0;  // kernels launched by this chunk
    // autotuning on the first apply of this width and direction (not under capture)
    auto& tu = op->tuned[nr_slot(NR)][transpose ? 1 : 0];
    bool tune_now = false;
    if (op->autotune && !tu.done && !ext) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        tune_now = cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
    }
    auto near_launch = [&](const h2::LaunchCfg& cf) {
        h2::launch_near_sym(g, t, c, op->near_u.nrows(), op->near_u.drows.as<int>(), op->near_u.dptr.as<int>(),
                            op->near_u.dcol.as<int>(), dlp ? h2::DLP : h2::SLP, transpose, fp32, NR,
                            w.xp, (const float*)w.xs, w.yp, cf, s);
    };
    mark(0);
    if (xmapped)  // x in mapped host memory: read in the caller's order
        h2::launch_permute_in_scatter(x, ldx, nrhs, NR, op->iperm.as<int>(), n, w.xp, s);
    else
        h2::launch_permute_in(x, ldx, nrhs, NR, op->perm.as<int>(), n, w.xp, s);
    // the stored nearfield writes every row of y first; otherwise the stages add to zero
    if (!op->store_near) CU(cudaMemsetAsync(w.yp, 0, op->n * NR * sizeof(double), s));
    // x in FP32 for the regular nearfield (and then the singular row gather)
    const bool xs_ready = near_reads_xs(op) && op->near_u.nrows() > 0;
    if (xs_ready) {
        h2::launch_store_x(true, n, NR, w.xp, w.xs, s);
        nl += 1;
    }
    if (tune_now && op->near_u.nrows() > 0 && !op->store_near) {
        float best = 1e30f;
        const bool budgets = fp32 && !dlp;  // register-budget variants exist for the FP32 single layer
        for (int nb : {0, 3, 2}) {
            if (nb && !budgets) continue;
            for (int pers = 0; pers < 2; ++pers) {
                h2::LaunchCfg cf;
                cf.nb = nb;
                cf.work = pers ? op->work.as<int>() : nullptr;
                const float ms = time_on(s, [&] { near_launch(cf); });
                if (ms < best) {
                    best = ms;
                    tu.near_persist = pers != 0;
                    tu.near_nb = nb;
                }
            }
        }
        CU(cudaMemsetAsync(w.yp, 0, op->n * NR * sizeof(double), s));
    }
    if (tune_now && op->nfar > 0 && !op->gca && tc_kind(op, xh64, yh64) < 0 && (op->m == 4 || op->m == 5)) {
        tu.coup.nsl = -1;  // tuned below, once x-hat is ready
    }
    nl += 1;
    mark(1);
    // the farfield passes up to the downward pass run on the operator's second
    // stream, concurrently with the nearfield, which adds to y atomically; the
    // leaf backward transformation (a plain add into y) follows both.  Timed
    // and tuning applies stay on one stream, so that stage times mean what
    // they say.
    const bool overlap = !timed && !tune_now && !op->store_near && op->nfar > 0 && op->s_far;
    cudaStream_t fs = s;
    if (overlap) {
        CU(cudaEventRecord(op->ev_fork, s));
        CU(cudaStreamWaitEvent(op->s_far, op->ev_fork, 0));
        fs = op->s_far;
    }
    auto leaf_backward = [&]() {
        if (op->recompute_basis)
            h2::launch_leaf_backward(g, t, c, op->basis_rule.as<double>(), (int)op->nleaves, op->leaves.as<int>(),
                                     out_dlp, fp32 && !out_dlp, yh64, NR, w.yh, w.yp, s);
        else
            h2::launch_leaf_backward_stored(t, (int)op->k, op->max_leaf, (int)op->nleaves, op->leaves.as<int>(),
                                            fp32 && !out_dlp, yh64, NR, out_dlp ? op->basisW.p : op->basisV.p,
                                            w.yh, w.yp, s);
    };
    // stored nearfield first (stage times are then mapped by the order of the events)
    const int fo = op->store_near ? 1 : 0;
    op->stage_order = fo;
    if (op->store_near) {
        nl += near_stored_apply(op, NR, transpose, w.xp, w.yp, w.xs, s);
        mark(2);
    }
    if (op->nfar > 0) {
        CU(cudaMemsetAsync(w.yh, 0, (size_t)op->nc * op->k * NR * ysz, fs));
        // the double layer's differentiated basis is evaluated in FP64 in every tier
        if (op->recompute_basis)
            h2::launch_leaf_forward(g, t, c, op->basis_rule.as<double>(), (int)op->nleaves, op->leaves.as<int>(),
                                    in_dlp, fp32 && !in_dlp, xh64, NR, w.xp, w.xh, fs);
        else
            h2::launch_leaf_forward_stored(t, (int)op->k, op->max_leaf, (int)op->nleaves, op->leaves.as<int>(),
                                           fp32 && !in_dlp, xh64, NR, in_dlp ? op->basisW.p : op->basisV.p,
                                           w.xp, w.xh, fs);
        nl += 1 + (far.nrows() > 0 ? 1 : 0) + 1;
        mark(2 + fo);
        if (op->gca) {
            for (int L = (int)op->level_parents.size() - 1; L >= 0; --L)
                h2::launch_gca_updown(true, fp32, NR, (int)op->level_parents[L].size(), op->dlevel[L].as<int>(),
                                      op->cchild0.as<int>(), op->cchild1.as<int>(), op->g_rank.as<int>(),
                                      op->g_eoff.as<int64_t>(), op->g_E.p, (int)op->k, w.xh, fs);
            nl += (int64_t)op->level_parents.size();
        } else {
            nl += run_upward(op, t, c, xh64, NR, w.xh, fs);
        }
        mark(3 + fo);
        if (tune_now && tu.coup.nsl == -1) {
            float best = 1e30f;
            for (int nsl : {2, 4, 8})
                for (int pers = 0; pers < 2; ++pers) {
                    h2::LaunchCfg cf;
                    cf.nsl = nsl;
                    cf.work = pers ? op->work.as<int>() + 1 : nullptr;
                    const float ms = time_on(s, [&] { run_coupling(op, t, c, far, xh64, yh64, NR, w.xh, w.yh, cf, s); });
                    if (ms < best) {
                        best = ms;
                        tu.coup.nsl = nsl;
                        tu.coup_persist = pers != 0;
                    }
                }
        }
        if (tune_now) {
            if (tu.coup.nsl < 0) tu.coup.nsl = 4;
            tu.done = true;
        }
        h2::LaunchCfg cfg_near, cfg_coup;
        launch_cfgs(op, NR, transpose, cfg_near, cfg_coup);
        if (op->gca)
            h2::launch_gca_coupling(fp32, NR, far.nrows(), far.drows.as<int>(), far.dptr.as<int>(), far.dcol.as<int>(),
                                    op->g_rank.as<int>(), g_soff.as<int64_t>(), g_S.p, (int)op->k, w.xh, w.yh, fs);
        else
            run_coupling(op, t, c, far, xh64, yh64, NR, w.xh, w.yh, cfg_coup, fs);
        mark(4 + fo);
        if (op->gca) {
            for (size_t L = 0; L < op->level_parents.size(); ++L)
                h2::launch_gca_updown(false, fp32, NR, (int)op->level_parents[L].size(), op->dlevel[L].as<int>(),
                                      op->cchild0.as<int>(), op->cchild1.as<int>(), op->g_rank.as<int>(),
                                      op->g_eoff.as<int64_t>(), op->g_E.p, (int)op->k, w.yh, fs);
            nl += (int64_t)op->level_parents.size();
        } else {
            nl += run_downward(op, t, c, yh64, NR, w.yh, fs);
        }
        mark(5 + fo);
        if (overlap) CU(cudaEventRecord(op->ev_join, fs));
        else leaf_backward();
    } else {
        for (int i = 2 + fo; i <= 5 + fo; ++i) mark(i);
    }
    if (tune_now) tu.done = true;  // operators without farfield
    if (op->store_near) {
        mark(7);
        mark(8);
        h2::launch_permute_out(w.yp, NR, nrhs, op->iperm.as<int>(), n, y, ldy, s);
        nl += 1;
        op->launches += nl;
        mark(9);
        CU(cudaGetLastError());
        return H2BEM_OK;
    }
    mark(6);
    // nearfield, regular pairs: each unordered pair of leaves once, both directions
    {
        h2::LaunchCfg cfg_near, cfg_coup;
        launch_cfgs(op, NR, transpose, cfg_near, cfg_coup);
        near_launch(cfg_near);
    }
    nl += op->near_u.nrows() > 0 ? 1 : 0;
    mark(7);
    if (op->sing_gather) nl += sing_gather_apply(op, NR, transpose, w.xp, w.yp, w.xs, xs_ready, s);
    for (int ty = 0; ty < 3 && !op->sing_gather; ++ty) {
        if (ty == 0 && dlp) continue;  // the double-layer entry of a triangle with itself vanishes
        const int np = (int)op->sp_count[ty];
        nl += np > 0 ? 1 : 0;
        if (op->cache_singular)
            h2::launch_singular(g, h2::IDENTICAL - ty, near_ker, np, op->sp_lo[ty].as<int>(), op->sp_hi[ty].as<int>(),
                                nullptr, nullptr, 0, 2, false, transpose, NR, w.xp, w.yp,
                                op->sp_v0[ty].as<double>(), op->sp_v1[ty].as<double>(), s);
        else
            h2::launch_singular(g, h2::IDENTICAL - ty, near_ker, np, op->sp_lo[ty].as<int>(), op->sp_hi[ty].as<int>(),
                                op->sp_code[ty].as<int>(), op->sp_tab[ty].as<double>(), op->sp_npts[ty], 0,
                                fp32 && !op->singular_fp64, transpose,
                                NR, w.xp, w.yp, nullptr, nullptr, s);
    }
    mark(8);
    if (overlap) {  // join the farfield stream, then its leaf backward transformation
        CU(cudaStreamWaitEvent(s, op->ev_join, 0));
        leaf_backward();
    }
    h2::launch_permute_out(w.yp, NR, nrhs, op->iperm.as<int>(), n, y, ldy, s);
    nl += 1;
    op->launches += nl;
    mark(9);
    CU(cudaGetLastError());
    return H2BEM_OK;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Page-locked host memory with a device address (UVA maps it; on this
// platform the device reads and writes it coherently over the host link).
static bool mapped_host(const void* p, void** dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    *dev = a.devicePointer;
    return true;
}

static int apply_impl(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy, void* stream,
                      bool transpose, bool timed) {
    if (!op) return fail(H2BEM_ERR_ARG, "apply: op is NULL");
    if (!x || !y) return fail(H2BEM_ERR_ARG, "apply: NULL vector");
    if (nrhs < 1 || nrhs > 64) return fail(H2BEM_ERR_ARG, "apply: nrhs must be in 1..64");
    if (ldx < op->n || ldy < op->n) return fail(H2BEM_ERR_ARG, "apply: leading dimensions must be >= n");
    {
        const char* xb = (const char*)x;
        const char* xe = (const char*)(x + (nrhs - 1) * ldx + op->n);
        const char* yb = (const char*)y;
        const char* ye = (const char*)(y + (nrhs - 1) * ldy + op->n);
        if (xb < ye && yb < xe) return fail(H2BEM_ERR_ARG, "apply: x and y overlap");
    }
    cudaStream_t s = (cudaStream_t)stream;
    op->launches = 0;
    const bool xdev = is_device_ptr(x), ydev = is_device_ptr(y);
    if (timed && (!xdev || !ydev)) return fail(H2BEM_ERR_ARG, "apply_timed: x and y must be device memory");
    const double* xd = x;
    double* yd = y;
    int64_t lx = ldx, ly = ldy;
    // page-locked host memory mapped into the device's address space: the
    // permute kernels read x and write y through it (over the host link, in
    // the caller's order); other host memory goes through staging copies
    void *xmap = nullptr, *ymap = nullptr;
    const bool xm = !xdev && mapped_host(x, &xmap), ym = !ydev && mapped_host(y, &ymap);
    if (xm) xd = (const double*)xmap;
    if (ym) yd = (double*)ymap;
    if ((!xdev && !xm) || (!ydev && !ym)) {
        const size_t need = (size_t)op->n * nrhs;
        if (op->stage_elems < need) {
            int rc;
            if ((rc = op->xstage.alloc(need * sizeof(double))) || (rc = op->ystage.alloc(need * sizeof(double)))) return rc;
            op->stage_elems = need;
        }
        if (!xdev && !xm) {
            CU(cudaMemcpy2DAsync(op->xstage.p, op->n * sizeof(double), x, ldx * sizeof(double), op->n * sizeof(double),
                                 nrhs, cudaMemcpyHostToDevice, s));
            xd = op->xstage.as<double>();
            lx = op->n;
        }
        if (!ydev && !ym) {
            yd = op->ystage.as<double>();
            ly = op->n;
        }
    }
    // CUDA graph replay: device buffers, a non-default stream, same arguments as
    // the previous call (the first repeat captures, later repeats replay)
    const bool graphable = op->use_graph && xdev && ydev && !timed && s != nullptr;
    if (graphable) {
        int rc = ensure_workspace(op, pad_nr(std::min(nrhs, 16)));
        if (rc) return rc;
        h2bem_op::GKey key;
        key.x = x;
        key.y = y;
        key.ldx = ldx;
        key.ldy = ldy;
        key.nrhs = nrhs;
        key.tr = transpose;
        key.s = s;
        key.ws_gen = op->ws_gen;
        if (op->gexec && key == op->gkey_graph) {
            CU(cudaGraphLaunch(op->gexec, s));
            op->launches = op->gkey_graph.launches;
            return H2BEM_OK;
        }
        if (key == op->gkey_seen) {
            cudaGraph_t graph = nullptr;
            CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            op->launches = 0;
            for (int c0 = 0; c0 < nrhs && rc == 0; c0 += 16)
                rc = apply_chunk(op, xd + c0 * lx, lx, std::min(16, nrhs - c0), yd + c0 * ly, ly, s, transpose, false);
            cudaError_t ce = cudaStreamEndCapture(s, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (ce != cudaSuccess) return fail(H2BEM_ERR_CUDA, "apply: graph capture failed: %s", cudaGetErrorString(ce));
            if (op->gexec) cudaGraphExecDestroy(op->gexec);
            op->gexec = nullptr;
            ce = cudaGraphInstantiate(&op->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return fail(H2BEM_ERR_CUDA, "apply: graph instantiation failed: %s", cudaGetErrorString(ce));
            key.launches = op->launches;
            op->gkey_graph = key;
            CU(cudaGraphLaunch(op->gexec, s));
            return H2BEM_OK;
        }
        op->gkey_seen = key;
    }
    for (int c0 = 0; c0 < nrhs; c0 += 16) {
        const int nr = std::min(16, nrhs - c0);
        int rc = apply_chunk(op, xd + c0 * lx, lx, nr, yd + c0 * ly, ly, s, transpose, timed, xm);
        if (rc) return rc;
    }
    if (!ydev && !ym) {
        CU(cudaMemcpy2DAsync(y, ldy * sizeof(double), yd, ly * sizeof(double), op->n * sizeof(double), nrhs,
                             cudaMemcpyDeviceToHost, s));
    }
    if (!xdev || !ydev) {
        CU(cudaStreamSynchronize(s));
        if (h2::coupling_tc_status(true))
            return fail(H2BEM_ERR_TIMEOUT, "apply: a bounded wait of the tensor-core coupling expired");
    }
    if (timed) op->timing_pending = true;  // read by h2bem_stats_get: no host wait here
    return H2BEM_OK;
}

// Stage times of the last timed apply: waits for its last event.  Operators of
// the tensor-core tiers also read the timeout flag of the coupling kernels
// (synchronous), so an expired wait of any completed apply is reported here.
static int resolve_timing(h2bem_op* op) {
    if (!op->timing_pending) {
        if (op->precision == H2BEM_MIXED_TF32 || op->precision == H2BEM_MIXED_BF16) {
            if (h2::coupling_tc_status(true))
                return fail(H2BEM_ERR_TIMEOUT, "stats_get: a bounded wait of the tensor-core coupling expired");
        }
        return H2BEM_OK;
    }
    op->timing_pending = false;
    CU(cudaEventSynchronize(op->ev[9]));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, op->ev[0], op->ev[9]);
    op->last_ms = ms;
    // events in launch order; the stored nearfield runs right after permute_in
    const int map[2][8][2] = {{{0, 1}, {1, 2}, {2, 3}, {3, 4}, {4, 5}, {5, 6}, {6, 7}, {7, 8}},
                              {{0, 1}, {2, 3}, {3, 4}, {4, 5}, {5, 6}, {6, 7}, {1, 2}, {7, 8}}};
    for (int i = 0; i < 8; ++i) {
        cudaEventElapsedTime(&ms, op->ev[map[op->stage_order][i][0]], op->ev[map[op->stage_order][i][1]]);
        op->stage_ms[i] = ms;
    }
    if (h2::coupling_tc_status(true))
        return fail(H2BEM_ERR_TIMEOUT, "apply_timed: a bounded wait of the tensor-core coupling expired");
    return H2BEM_OK;
}

extern "C" int h2bem_apply(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy, void* stream) {
    return apply_impl(op, x, ldx, nrhs, y, ldy, stream, false, false);
}

extern "C" int h2bem_apply_transpose(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy,
                                     void* stream) {
    return apply_impl(op, x, ldx, nrhs, y, ldy, stream, true, false);
}

extern "C" int h2bem_apply_timed(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy,
                                 void* stream) {
    return apply_impl(op, x, ldx, nrhs, y, ldy, stream, false, true);
}

// ===========================================================================
// mass term and conjugate gradients (section 1, eq. (matrix_dtn))
// ===========================================================================
static int ensure_area_user(h2bem_op* op, cudaStream_t s) {
    if (op->area_user.p) return H2BEM_OK;
    int rc = op->area_user.alloc(op->n * sizeof(double));
    if (rc) return rc;
    h2::launch_area_user((int)op->n, op->perm.as<int>(), op->area.as<double>(), op->area_user.as<double>(), s);
    CU(cudaGetLastError());
    return H2BEM_OK;
}

extern "C" int h2bem_apply_mass(h2bem_op* op, double alpha, const double* x, int64_t ldx, int nrhs, double* y,
                                int64_t ldy, void* stream) {
    if (!op || !x || !y) return fail(H2BEM_ERR_ARG, "apply_mass: NULL argument");
    if (!is_device_ptr(x) || !is_device_ptr(y)) return fail(H2BEM_ERR_ARG, "apply_mass: x and y must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = apply_impl(op, x, ldx, nrhs, y, ldy, stream, false, false);
    if (rc) return rc;
    if ((rc = ensure_area_user(op, s))) return rc;
    h2::launch_mass_add((int)op->n, nrhs, alpha, op->area_user.as<double>(), x, ldx, y, ldy, s);
    CU(cudaGetLastError());
    return H2BEM_OK;
}

extern "C" int h2bem_apply_hypersingular(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y,
                                         int64_t ldy, void* stream) {
    if (!op || !x || !y) return fail(H2BEM_ERR_ARG, "apply_hypersingular: NULL argument");
    if (op->kernel != H2BEM_SLP) return fail(H2BEM_ERR_ARG, "apply_hypersingular: needs a single-layer operator");
    if (nrhs < 0) return fail(H2BEM_ERR_ARG, "apply_hypersingular: nrhs must be >= 0");
    if (ldx < op->nv || ldy < op->nv) return fail(H2BEM_ERR_ARG, "apply_hypersingular: leading dimensions must be >= nv");
    if (!is_device_ptr(x) || !is_device_ptr(y))
        return fail(H2BEM_ERR_ARG, "apply_hypersingular: x and y must be device memory");
    if (nrhs == 0) return H2BEM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)op->n;
    const int64_t need = 3 * (int64_t)n * nrhs;
    int rc;
    if (op->hyp_cap < need) {
        if ((rc = op->hyp_z.alloc(need * sizeof(double))) || (rc = op->hyp_w.alloc(need * sizeof(double)))) return rc;
        op->hyp_cap = need;
    }
    double *z = op->hyp_z.as<double>(), *w = op->hyp_w.as<double>();
    h2::launch_curl_fwd(n, nrhs, op->xyz.as<double>(), op->tri.as<int>(), x, ldx, z, s);
    CU(cudaGetLastError());
    if ((rc = apply_impl(op, z, n, 3 * nrhs, w, n, stream, false, false))) return rc;
    h2::launch_curl_bwd((int)op->nv, n, nrhs, op->vptr.as<int>(), op->vinc.as<int>(), op->xyz.as<double>(),
                        op->tri.as<int>(), w, y, ldy, s);
    CU(cudaGetLastError());
    return H2BEM_OK;
}

// ===========================================================================
// double layer with piecewise-linear trial functions K1 (h2bem_apply_dlp_p1)
// ===========================================================================
// First use: the per-corner leaf bases W1_c[pos][nu] = int_{tau} n . grad
// L_nu lambda_c (the leaf-basis kernel with the rule's weights scaled by the
// barycentric coordinate lambda_c = (1 - u - v, u, v) of its points; the
// integrand's degree stays within the rule's exactness), and the Sauter-Schwab
// values of the edge- and vertex-adjacent pairs (full tensor rule, q_ss
// points per direction, FP64).  The double layer's identical pairs vanish.
static int p1_setup(h2bem_op* op) {
    if (op->p1_ready) return H2BEM_OK;
    const int64_t n = op->n;
    const h2::Geom g = op->geom();
    const h2::Tree t = op->tree();
    int rc;
    std::vector<double> rule;
    basis_rule_host(op->m, rule);
    for (int c = 0; c < 3; ++c) {
        std::vector<double> rc_ = rule;
        for (size_t p = 0; p < rule.size() / 3; ++p) {
            const double u = rule[3 * p], v = rule[3 * p + 1];
            rc_[3 * p + 2] *= c == 0 ? 1.0 - u - v : c == 1 ? u : v;
        }
        DevBuf dr;
        if ((rc = upload(dr, rc_))) return rc;
        if ((rc = op->p1_W1[c].alloc((size_t)n * op->k * sizeof(double)))) return rc;
        if (op->nfar > 0)
            h2::launch_leaf_basis(g, t, op->consts, dr.as<double>(), (int)op->nleaves, op->leaves.as<int>(), true, false,
                                  op->p1_W1[c].p, 0);
        CU(cudaDeviceSynchronize());
    }
    for (int ty = 1; ty <= 2; ++ty) {
        std::vector<double> tab;
        ss_full_table(ty, op->q_ss, tab);
        if ((rc = upload(op->p1_tab, tab))) return rc;
        const int np = (int)op->sp_count[ty];
        if ((rc = op->p1_vals[ty - 1].alloc((size_t)std::max(np, 1) * 6 * sizeof(double)))) return rc;
        h2::launch_p1_sing_eval(g, np, op->sp_lo[ty].as<int>(), op->sp_hi[ty].as<int>(), op->sp_code[ty].as<int>(),
                                op->p1_tab.as<double>(), (int)(tab.size() / 5), op->p1_vals[ty - 1].as<double>(), 0);
        CU(cudaDeviceSynchronize());
    }
    // point offsets from the centroids as float pairs, for the regular nearfield
    if ((rc = op->p1_off.alloc((size_t)6 * n * 7 * sizeof(float)))) return rc;
    h2::launch_p1_offsets((int)n, g.qa, g.ctr, op->p1_off.as<float>(), 0);
    CU(cudaDeviceSynchronize());
    op->p1_ready = 1;
    return H2BEM_OK;
}

// One chunk of at most 16 right-hand sides, device buffers.
// forward:  x on vertices (ldx), y on triangles (ldy);  transpose: the reverse.
static int apply_p1_chunk(h2bem_op* op, double alpha, const double* x, int64_t ldx, int nrhs, double* y,
                          int64_t ldy, cudaStream_t s, bool transpose) {
    const int NR = pad_nr(nrhs);
    int rc;
    if ((rc = ensure_workspace(op, NR))) return rc;
    const int64_t need = 3 * op->n * NR;
    if (op->p1_cap < need) {
        if ((rc = op->p1_x3.alloc(need * sizeof(double))) || (rc = op->p1_y3.alloc(need * sizeof(double)))) return rc;
        op->p1_cap = need;
    }
    const bool fp32 = op->precision != H2BEM_FP64;
    const bool xh64 = xh_is64(op, transpose), yh64 = yh_is64(op, transpose);
    const size_t xsz = xh64 ? sizeof(double) : sizeof(float), ysz = yh64 ? sizeof(double) : sizeof(float);
    const h2::Geom g = op->geom();
    const h2::Tree t = op->tree();
    const h2::Consts& c = op->consts;
    const int n = (int)op->n;
    double* x3 = op->p1_x3.as<double>();
    double* y3 = op->p1_y3.as<double>();
    double* xp = op->xp.as<double>();
    double* yp = op->yp.as<double>();
    h2::LaunchCfg cfg_near, cfg_coup;
    launch_cfgs(op, NR, transpose, cfg_near, cfg_coup);
    if (!transpose) {
        h2::launch_p1_gather(n, NR, nrhs, op->vid.as<int>(), x, ldx, x3, s);
        CU(cudaMemsetAsync(yp, 0, (size_t)n * NR * sizeof(double), s));
        if (op->nfar > 0) {
            CU(cudaMemsetAsync(op->xh.p, 0, (size_t)op->nc * op->k * NR * xsz, s));
            CU(cudaMemsetAsync(op->yh.p, 0, (size_t)op->nc * op->k * NR * ysz, s));
            for (int cc = 0; cc < 3; ++cc)
                h2::launch_leaf_forward_stored_acc(t, (int)op->k, op->max_leaf, (int)op->nleaves, op->leaves.as<int>(),
                                                   xh64, NR, op->p1_W1[cc].as<double>(), x3 + (size_t)cc * n * NR,
                                                   op->xh.p, s);
            run_upward(op, t, c, xh64, NR, op->xh.p, s);
            run_coupling(op, t, c, op->far, xh64, yh64, NR, op->xh.p, op->yh.p, cfg_coup, s);
            run_downward(op, t, c, yh64, NR, op->yh.p, s);
            h2::launch_leaf_backward_stored(t, (int)op->k, op->max_leaf, (int)op->nleaves, op->leaves.as<int>(), fp32,
                                            yh64, NR, op->basisV.p, op->yh.p, yp, s);
        }
        h2::launch_p1_near(false, fp32, NR, g, t, c, op->near.nrows(), op->near.drows.as<int>(), op->near.dptr.as<int>(),
                           op->near.dcol.as<int>(), op->p1_off.as<float>(), x3, yp, s);
        for (int ty = 1; ty <= 2; ++ty)
            h2::launch_p1_sing_apply(false, n, (int)op->sp_count[ty], NR, op->sp_lo[ty].as<int>(),
                                     op->sp_hi[ty].as<int>(), op->sp_code[ty].as<int>(),
                                     op->p1_vals[ty - 1].as<double>(), x3, yp, s);
        h2::launch_p1_mass(false, n, NR, alpha, op->area.as<double>(), x3, yp, s);
        h2::launch_permute_out(yp, NR, nrhs, op->iperm.as<int>(), n, y, ldy, s);
    } else {
        h2::launch_permute_in(x, ldx, nrhs, NR, op->perm.as<int>(), n, xp, s);
        CU(cudaMemsetAsync(y3, 0, (size_t)need * sizeof(double), s));
        if (op->nfar > 0) {
            CU(cudaMemsetAsync(op->yh.p, 0, (size_t)op->nc * op->k * NR * ysz, s));
            h2::launch_leaf_forward_stored(t, (int)op->k, op->max_leaf, (int)op->nleaves, op->leaves.as<int>(), fp32,
                                           xh64, NR, op->basisV.p, xp, op->xh.p, s);
            run_upward(op, t, c, xh64, NR, op->xh.p, s);
            run_coupling(op, t, c, op->far_t, xh64, yh64, NR, op->xh.p, op->yh.p, cfg_coup, s);
            run_downward(op, t, c, yh64, NR, op->yh.p, s);
            for (int cc = 0; cc < 3; ++cc)
                h2::launch_leaf_backward_stored(t, (int)op->k, op->max_leaf, (int)op->nleaves, op->leaves.as<int>(),
                                                false, yh64, NR, op->p1_W1[cc].p, op->yh.p, y3 + (size_t)cc * n * NR,
                                                s);
        }
        h2::launch_p1_near(true, fp32, NR, g, t, c, op->near.nrows(), op->near.drows.as<int>(), op->near.dptr.as<int>(),
                           op->near.dcol.as<int>(), op->p1_off.as<float>(), xp, y3, s);
        for (int ty = 1; ty <= 2; ++ty)
            h2::launch_p1_sing_apply(true, n, (int)op->sp_count[ty], NR, op->sp_lo[ty].as<int>(),
                                     op->sp_hi[ty].as<int>(), op->sp_code[ty].as<int>(),
                                     op->p1_vals[ty - 1].as<double>(), xp, y3, s);
        h2::launch_p1_mass(true, n, NR, alpha, op->area.as<double>(), xp, y3, s);
        h2::launch_p1_scatter((int)op->nv, n, NR, nrhs, op->vptr.as<int>(), op->vinc.as<int>(), op->iperm.as<int>(),
                              y3, y, ldy, s);
    }
    CU(cudaGetLastError());
    return H2BEM_OK;
}

extern "C" int h2bem_apply_dlp_p1(h2bem_op* op, double alpha, const double* x, int64_t ldx, int nrhs, double* y,
                                  int64_t ldy, int transpose, void* stream) {
    if (!op || !x || !y) return fail(H2BEM_ERR_ARG, "apply_dlp_p1: NULL argument");
    if (op->kernel != H2BEM_DLP) return fail(H2BEM_ERR_ARG, "apply_dlp_p1: needs a double-layer operator");
    if (op->recompute_basis) return fail(H2BEM_ERR_ARG, "apply_dlp_p1: needs stored leaf bases (recompute_basis = 0)");
    if (nrhs < 1 || nrhs > 64) return fail(H2BEM_ERR_ARG, "apply_dlp_p1: nrhs must be in 1..64");
    const int64_t nin = transpose ? op->n : op->nv, nout = transpose ? op->nv : op->n;
    if (ldx < nin || ldy < nout) return fail(H2BEM_ERR_ARG, "apply_dlp_p1: leading dimensions too small");
    if (!is_device_ptr(x) || !is_device_ptr(y)) return fail(H2BEM_ERR_ARG, "apply_dlp_p1: x and y must be device memory");
    int rc;
    if ((rc = p1_setup(op))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    for (int c0 = 0; c0 < nrhs; c0 += 16) {
        const int nr = std::min(16, nrhs - c0);
        if ((rc = apply_p1_chunk(op, alpha, x + c0 * ldx, ldx, nr, y + c0 * ldy, ldy, s, transpose != 0))) return rc;
    }
    return H2BEM_OK;
}

// Conjugate gradients on n-vectors with the operator q = A p (apply(p, q),
// n x nrhs blocks with leading dimension n), every column its own system;
// x0 = 0; the step lengths are host scalars.
template <typename F>
static int cg_run(h2bem_op* op, int n, F apply, const double* b, int64_t ldb, int nrhs, double* x, int64_t ldx,
                  double rtol, int maxit, int* iters, double* relres, cudaStream_t s) {
    const int64_t need = (int64_t)n * nrhs;
    int rc;
    if (op->cg_cap < need) {
        if ((rc = op->cg_r.alloc(need * sizeof(double))) || (rc = op->cg_p.alloc(need * sizeof(double))) ||
            (rc = op->cg_q.alloc(need * sizeof(double))) || (rc = op->cg_s.alloc(6 * 64 * sizeof(double))))
            return rc;
        op->cg_cap = need;
    }
    double *r = op->cg_r.as<double>(), *p = op->cg_p.as<double>(), *q = op->cg_q.as<double>();
    double* sc = op->cg_s.as<double>();  // [0..63] dots, [64..127] alpha, [128..191] beta
    // x0 = 0, r = p = b
    for (int c = 0; c < nrhs; ++c) CU(cudaMemsetAsync(x + c * ldx, 0, n * sizeof(double), s));
    CU(cudaMemcpy2DAsync(r, n * sizeof(double), b, ldb * sizeof(double), n * sizeof(double), nrhs,
                         cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(p, r, need * sizeof(double), cudaMemcpyDeviceToDevice, s));
    std::vector<double> bb(nrhs), rr(nrhs), pq(nrhs), al(nrhs), be(nrhs);
    h2::launch_dots(n, nrhs, b, ldb, b, ldb, sc, s);
    CU(cudaMemcpyAsync(bb.data(), sc, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    rr = bb;
    std::vector<char> done(nrhs);
    int it = 0;
    auto converged = [&](int c) { return bb[c] == 0.0 || rr[c] <= rtol * rtol * bb[c]; };
    for (int c = 0; c < nrhs; ++c) done[c] = converged(c);
    while (it < maxit && std::find(done.begin(), done.end(), 0) != done.end()) {
        if ((rc = apply(p, q))) return rc;
        h2::launch_dots(n, nrhs, p, n, q, n, sc, s);
        CU(cudaMemcpyAsync(pq.data(), sc, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        for (int c = 0; c < nrhs; ++c) al[c] = (done[c] || pq[c] <= 0.0) ? 0.0 : rr[c] / pq[c];
        CU(cudaMemcpyAsync(sc + 64, al.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
        h2::launch_cg_step(n, nrhs, sc + 64, p, n, q, n, x, ldx, r, n, s);
        h2::launch_dots(n, nrhs, r, n, r, n, sc, s);
        std::vector<double> rn(nrhs);
        CU(cudaMemcpyAsync(rn.data(), sc, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        ++it;
        for (int c = 0; c < nrhs; ++c) {
            be[c] = (done[c] || rr[c] == 0.0) ? 0.0 : rn[c] / rr[c];
            if (!done[c]) rr[c] = rn[c];
            done[c] = done[c] || converged(c);
        }
        CU(cudaMemcpyAsync(sc + 128, be.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
        h2::launch_cg_dir(n, nrhs, sc + 128, r, n, p, n, s);
        CU(cudaGetLastError());
    }
    CU(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (relres)
        for (int c = 0; c < nrhs; ++c) relres[c] = bb[c] > 0.0 ? std::sqrt(rr[c] / bb[c]) : 0.0;
    return H2BEM_OK;
}

extern "C" int h2bem_cg(h2bem_op* op, const double* b, int64_t ldb, int nrhs, double* x, int64_t ldx, double rtol,
                        int maxit, int* iters, double* relres, void* stream) {
    if (!op || !b || !x) return fail(H2BEM_ERR_ARG, "cg: NULL argument");
    if (op->kernel != H2BEM_SLP) return fail(H2BEM_ERR_ARG, "cg: needs the (symmetric positive definite) single layer");
    if (nrhs < 1 || nrhs > 64) return fail(H2BEM_ERR_ARG, "cg: nrhs must be in 1..64");
    if (ldb < op->n || ldx < op->n) return fail(H2BEM_ERR_ARG, "cg: leading dimensions must be >= n");
    if (!(rtol > 0.0) || maxit < 0) return fail(H2BEM_ERR_ARG, "cg: rtol must be > 0 and maxit >= 0");
    if (!is_device_ptr(b) || !is_device_ptr(x)) return fail(H2BEM_ERR_ARG, "cg: b and x must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)op->n;
    return cg_run(op, n, [&](const double* p, double* q) { return apply_impl(op, p, n, nrhs, q, n, stream, false, false); },
                  b, ldb, nrhs, x, ldx, rtol, maxit, iters, relres, s);
}

extern "C" int h2bem_cg_hypersingular(h2bem_op* op, const double* mvec, const double* b, int64_t ldb, int nrhs,
                                      double* x, int64_t ldx, double rtol, int maxit, int* iters, double* relres,
                                      void* stream) {
    if (!op || !b || !x) return fail(H2BEM_ERR_ARG, "cg_hypersingular: NULL argument");
    if (op->kernel != H2BEM_SLP) return fail(H2BEM_ERR_ARG, "cg_hypersingular: needs a single-layer operator");
    if (nrhs < 1 || nrhs > 64) return fail(H2BEM_ERR_ARG, "cg_hypersingular: nrhs must be in 1..64");
    if (ldb < op->nv || ldx < op->nv) return fail(H2BEM_ERR_ARG, "cg_hypersingular: leading dimensions must be >= nv");
    if (!(rtol > 0.0) || maxit < 0) return fail(H2BEM_ERR_ARG, "cg_hypersingular: rtol must be > 0 and maxit >= 0");
    if (!is_device_ptr(b) || !is_device_ptr(x) || (mvec && !is_device_ptr(mvec)))
        return fail(H2BEM_ERR_ARG, "cg_hypersingular: b, x and m must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    const int nv = (int)op->nv;
    int rc;
    if (!op->cg_d.p && (rc = op->cg_d.alloc(64 * sizeof(double)))) return rc;
    double* d = op->cg_d.as<double>();
    return cg_run(op, nv, [&](const double* p, double* q) {
        int r2 = h2bem_apply_hypersingular(op, p, nv, nrhs, q, nv, stream);
        if (r2 || !mvec) return r2;
        CU(cudaMemsetAsync(d, 0, nrhs * sizeof(double), s));
        h2::launch_dots(nv, nrhs, mvec, 0, p, nv, d, s);
        h2::launch_rank1_add(nv, nrhs, mvec, d, q, nv, s);
        CU(cudaGetLastError());
        return (int)H2BEM_OK;
    }, b, ldb, nrhs, x, ldx, rtol, maxit, iters, relres, s);
}

// ===========================================================================
// shape gradient (single layer, FP64)
// ===========================================================================
extern "C" int h2bem_grad(h2bem_op* op, const double* w, const double* x, int64_t ld, int nrhs, double* dxyz,
                          double* dx, void* stream) {
    if (!op || !w || !x || !dxyz) return fail(H2BEM_ERR_ARG, "grad: NULL argument");
    if (op->gca) return fail(H2BEM_ERR_ARG, "grad: the shape gradient runs through Chebyshev bases, not GCA or HCA bases");
    const bool dlp = op->kernel == H2BEM_DLP;
    if (nrhs < 1 || nrhs > 64) return fail(H2BEM_ERR_ARG, "grad: nrhs must be in 1..64");
    if (ld < op->n) return fail(H2BEM_ERR_ARG, "grad: leading dimension must be >= n");
    if (!is_device_ptr(w) || !is_device_ptr(x) || !is_device_ptr(dxyz) || (dx && !is_device_ptr(dx)))
        return fail(H2BEM_ERR_ARG, "grad: all vectors must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)op->n, nc = (int)op->nc, k = op->k;
    const int NRmax = pad_nr(std::min(nrhs, 16));
    if (op->g_NR < NRmax) {
        int rc;
        const size_t hv = (size_t)nc * k * NRmax * sizeof(double);
        if ((rc = op->g_xp.alloc((size_t)n * NRmax * sizeof(double))) ||
            (rc = op->g_wp.alloc((size_t)n * NRmax * sizeof(double))) || (rc = op->g_xh.alloc(hv)) ||
            (rc = op->g_wh.alloc(hv)) || (rc = op->g_yh.alloc(hv)) || (rc = op->g_zh.alloc(hv)) ||
            (rc = op->g_dbox.alloc((size_t)6 * nc * sizeof(double))))
            return rc;
        op->g_NR = NRmax;
    }
    if (dlp && !op->gd_ready) {  // full Sauter-Schwab tables of the edge and vertex pairs
        int rc;
        for (int ty = 1; ty <= 2; ++ty) {
            std::vector<double> tab;
            ss_full_table(ty, op->q_ss, tab);
            if ((rc = upload(op->gd_tab[ty - 1], tab))) return rc;
            op->gd_npts[ty - 1] = (int)(tab.size() / 5);
        }
        op->gd_ready = 1;
    }
    CU(cudaMemsetAsync(dxyz, 0, op->nv * 3 * sizeof(double), s));
    const h2::Geom g = op->geom();
    const h2::Tree t = op->tree();
    const h2::Consts& c = op->consts;
    for (int c0 = 0; c0 < nrhs; c0 += 16) {
        const int nr = std::min(16, nrhs - c0), NR = pad_nr(nr);
        double *xp = op->g_xp.as<double>(), *wp = op->g_wp.as<double>();
        double *xh = op->g_xh.as<double>(), *wh = op->g_wh.as<double>();
        double *yh = op->g_yh.as<double>(), *zh = op->g_zh.as<double>(), *dbox = op->g_dbox.as<double>();
        h2::launch_permute_in(x + c0 * ld, ld, nr, NR, op->perm.as<int>(), n, xp, s);
        h2::launch_permute_in(w + c0 * ld, ld, nr, NR, op->perm.as<int>(), n, wp, s);
        if (op->nfar > 0) {
            const size_t hv = (size_t)nc * k * NR * sizeof(double);
            // x-hat = W^T x (W = V for the single layer), w-hat = V^T w
            h2::launch_leaf_forward(g, t, c, op->basis_rule.as<double>(), (int)op->nleaves, op->leaves.as<int>(), dlp,
                                    false, true, NR, xp, xh, s);
            h2::launch_leaf_forward(g, t, c, op->basis_rule.as<double>(), (int)op->nleaves, op->leaves.as<int>(), false,
                                    false, true, NR, wp, wh, s);
            for (int L = (int)op->level_parents.size() - 1; L >= 0; --L) {
                h2::launch_upward(t, c, (int)op->level_parents[L].size(), op->dlevel[L].as<int>(), true, NR, xh, s);
                h2::launch_upward(t, c, (int)op->level_parents[L].size(), op->dlevel[L].as<int>(), true, NR, wh, s);
            }
            CU(cudaMemsetAsync(yh, 0, hv, s));
            CU(cudaMemsetAsync(zh, 0, hv, s));
            h2::launch_coupling(t, c, op->far.nrows(), op->far.drows.as<int>(), op->far.dptr.as<int>(),
                                op->far.dcol.as<int>(), 0, true, true, NR, xh, yh, h2::LaunchCfg{}, s);
            h2::launch_coupling(t, c, op->far_t.nrows(), op->far_t.drows.as<int>(), op->far_t.dptr.as<int>(),
                                op->far_t.dcol.as<int>(), 0, true, true, NR, wh, zh, h2::LaunchCfg{}, s);
            for (size_t L = 0; L < op->level_parents.size(); ++L) {
                h2::launch_downward(t, c, (int)op->level_parents[L].size(), op->dlevel[L].as<int>(), true, NR, yh, s);
                h2::launch_downward(t, c, (int)op->level_parents[L].size(), op->dlevel[L].as<int>(), true, NR, zh, s);
            }
            CU(cudaMemsetAsync(dbox, 0, (size_t)6 * nc * sizeof(double), s));
            h2::launch_grad_coupling(t, c, op->far.nrows(), op->far.drows.as<int>(), op->far.dptr.as<int>(),
                                     op->far.dcol.as<int>(), NR, wh, xh, dbox, s);
            h2::launch_grad_transfer(t, c, op->nchildren, op->children.as<int>(), op->parent.as<int>(), NR, xh, wh, yh,
                                     zh, dbox, s);
            h2::launch_grad_leaf(g, t, c, op->basis_rule.as<double>(), (int)op->nleaves, op->leaves.as<int>(), NR, xp,
                                 wp, yh, dlp ? nullptr : zh, dbox, dxyz, s);
            if (dlp)
                h2::launch_grad_leaf_w(g, t, c, op->basis_rule.as<double>(), (int)op->nleaves, op->leaves.as<int>(), NR,
                                       xp, zh, dbox, dxyz, s);
            h2::launch_grad_box(nc, op->cext.as<int>(), op->cflag.as<int>(), dbox, dxyz, s);
        }
        if (dlp) {
            h2::launch_grad_near_dlp(g, t, c, op->near.nrows(), op->near.drows.as<int>(), op->near.dptr.as<int>(),
                                     op->near.dcol.as<int>(), NR, xp, wp, dxyz, s);
            for (int ty = 1; ty <= 2; ++ty)  // identical pairs of the double layer vanish
                h2::launch_grad_singular_dlp(g, (int)op->sp_count[ty], op->sp_lo[ty].as<int>(), op->sp_hi[ty].as<int>(),
                                             op->sp_code[ty].as<int>(), op->gd_tab[ty - 1].as<double>(),
                                             op->gd_npts[ty - 1], NR, xp, wp, dxyz, s);
            CU(cudaGetLastError());
            continue;
        }
        h2::launch_grad_near(g, t, c, op->near.nrows(), op->near.drows.as<int>(), op->near.dptr.as<int>(),
                             op->near.dcol.as<int>(), NR, xp, wp, dxyz, s);
        for (int ty = 0; ty < 3; ++ty) {
            const double* tab = ty == 2 ? op->sp_gtab.as<double>()
                                : ty == 1 ? op->sp_gtab_edge.as<double>() : op->sp_tab[ty].as<double>();
            const int npts = ty == 2 ? op->sp_gnpts : ty == 1 ? op->sp_gnpts_edge : op->sp_npts[ty];
            h2::launch_grad_singular(g, h2::IDENTICAL - ty, (int)op->sp_count[ty], op->sp_lo[ty].as<int>(),
                                     op->sp_hi[ty].as<int>(), op->sp_code[ty].as<int>(), tab, npts, NR, xp, wp, dxyz, s);
        }
        CU(cudaGetLastError());
    }
    if (dx) {
        int rc = apply_impl(op, w, ld, nrhs, dx, ld, stream, true, false);
        if (rc) return rc;
    }
    return H2BEM_OK;
}

// ===========================================================================
// apply into caller-provided work vectors (used by the allocation-free entry
// point in noalloc.cu): apply_chunk's launch sequence on those vectors
// ===========================================================================
namespace h2 {

int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

int64_t op_size(const h2bem_op* op) { return op->n; }

// Bytes of work vectors one chunk of NR (padded) right-hand sides needs: the
// tree-ordered x and y, and the cluster vectors x-hat and y-hat.
size_t work_bytes(const h2bem_op* op, int NR) {
    const bool wide = op->precision == H2BEM_FP64 || op->kernel == H2BEM_DLP;
    const size_t e = wide ? sizeof(double) : sizeof(float);
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    return 2 * up((size_t)op->n * NR * sizeof(double)) + 2 * up((size_t)op->nc * op->k * NR * e) +
           up(store_x_bytes(op, NR));
}

int apply_with_work(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy, cudaStream_t s,
                    unsigned char* work) {
    const int NR = pad_nr(nrhs);
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const bool wide = op->precision == H2BEM_FP64 || op->kernel == H2BEM_DLP;
    const size_t vb = up((size_t)op->n * NR * sizeof(double));
    const size_t hb = up((size_t)op->nc * op->k * NR * (wide ? sizeof(double) : sizeof(float)));
    const Work w{reinterpret_cast<double*>(work), reinterpret_cast<double*>(work + vb), work + 2 * vb,
                 work + 2 * vb + hb, store_x_bytes(op, NR) ? work + 2 * vb + 2 * hb : nullptr};
    return apply_chunk(op, x, ldx, nrhs, y, ldy, s, false, false, false, &w);
}

}  // namespace h2
