"""Host-side check of the identity the FP32 double-layer kernels use for the
height of a rule point of triangle i above the plane of triangle j (section
1, eq. (dlp): the kernel's numerator (x - y) . n_j):

  h_p = (x_p - c_j) . n_j = D . n_j + (u_p - 1/3) E1_i . delta + (v_p - 1/3) E2_i . delta,

D = c_i - c_j, delta = n_j - n_i, E1_i = b - a, E2_i = c - a, x_p = a + u_p E1_i
+ v_p E2_i.  It holds because x_p - c_i lies in the plane of i (E . n_i = 0).
On neighbouring, nearly coplanar triangles the height is O(h^2 kappa) while
the coordinates are O(h): the right-hand side evaluated in FP32 (D . n_j from
the centroids' float splits with exact products, the E . delta terms small
times small) keeps the height to ~1e-6 of itself, where the left-hand side in
FP32 loses it to cancellation.  Both are emulated here with numpy float32."""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

f32 = np.float32


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def _split(x):
    h = f32(x)
    return h, f32(x - np.float64(h))


def _height_fp32(ci, cj, ni, nj, e1, e2, u, v):
    """The kernels' FP32 evaluation of the right-hand side."""
    chi = [_split(c) for c in ci]
    chj = [_split(c) for c in cj]
    Dh = [f32(chi[d][0] - chj[d][0]) for d in range(3)]
    Dl = [f32(chi[d][1] - chj[d][1]) for d in range(3)]
    nhj = [_split(x) for x in nj]
    nhi = [_split(x) for x in ni]
    dl = [f32(f32(nhj[d][0] - nhi[d][0]) + f32(nhj[d][1] - nhi[d][1])) for d in range(3)]
    # D . n_j: exact hi products (float64 holds a float32 product exactly), TwoSum of the cancelling sum
    p = [f32(Dh[d] * nhj[d][0]) for d in range(3)]
    r = [f32(np.float64(Dh[d]) * np.float64(nhj[d][0]) - np.float64(p[d])) for d in range(3)]
    s1, t1 = _two_sum(p[0], p[1])
    s2, t2 = _two_sum(s1, p[2])
    cr = f32(f32(t1 + t2) + f32(f32(r[0] + r[1]) + r[2]))
    for d in range(3):
        cr = f32(Dh[d] * nhj[d][1] + f32(Dl[d] * nhj[d][0] + cr))
    H0 = f32(s2 + cr)
    E1 = [f32(x) for x in e1]
    E2 = [f32(x) for x in e2]
    a1 = f32(f32(E1[0] * dl[0] + E1[1] * dl[1]) + E1[2] * dl[2])
    a2 = f32(f32(E2[0] * dl[0] + E2[1] * dl[1]) + E2[2] * dl[2])
    return f32(f32(u - f32(1.0 / 3.0)) * a1 + f32(f32(v - f32(1.0 / 3.0)) * a2 + H0))


def _neighbour_pairs(mesh, count, seed):
    """Pairs of triangles that share an edge (the nearest regular-quadrature
    neighbours are one ring further out, but these are the flattest)."""
    rng = np.random.default_rng(seed)
    tri = mesh.triangles
    edges = {}
    for t, (a, b, c) in enumerate(tri):
        for e in ((a, b), (b, c), (c, a)):
            edges.setdefault(tuple(sorted(e)), []).append(t)
    pairs = [v for v in edges.values() if len(v) == 2]
    idx = rng.choice(len(pairs), size=min(count, len(pairs)), replace=False)
    return [pairs[i] for i in idx]


@pytest.mark.parametrize("name", ["sphere", "ellipsoid", "jitter"])
def test_height_identity_fp32_keeps_small_heights(name):
    mesh = {"sphere": lambda: I.sphere(96), "ellipsoid": lambda: I.ellipsoid(64),
            "jitter": lambda: I.jitter(I.sphere(64), 0.01, 3)}[name]()
    V = mesh.vertices
    # seven points of the triangle, centre and off-centre (the identity holds for any point of it)
    uv = [(1 / 3, 1 / 3), (0.1, 0.45), (0.45, 0.1), (0.45, 0.45), (0.8, 0.1), (0.1, 0.8), (0.1, 0.1)]
    worst_id, worst_direct = 0.0, 0.0
    for i, j in _neighbour_pairs(mesh, 300, 7):
        Pi, Pj = V[mesh.triangles[i]], V[mesh.triangles[j]]
        ci, cj = Pi.mean(axis=0), Pj.mean(axis=0)
        e1, e2 = Pi[1] - Pi[0], Pi[2] - Pi[0]
        ni = np.cross(e1, e2)
        ni /= np.linalg.norm(ni)
        nj = np.cross(Pj[1] - Pj[0], Pj[2] - Pj[0])
        nj /= np.linalg.norm(nj)
        for u, v in uv:
            xp = Pi[0] + u * e1 + v * e2
            ref = np.dot(xp - cj, nj)  # FP64, the definition
            rhs = np.dot(ci - cj, nj) + (u - 1 / 3) * np.dot(e1, nj - ni) + (v - 1 / 3) * np.dot(e2, nj - ni)
            assert abs(rhs - ref) <= 1e-12 * np.linalg.norm(xp - cj)  # the identity itself, in FP64
            if abs(ref) < 1e-12:
                continue
            h32 = _height_fp32(ci, cj, ni, nj, e1, e2, f32(u), f32(v))
            worst_id = max(worst_id, abs(float(h32) - ref) / abs(ref))
            # the left-hand side directly in FP32
            direct = f32(np.dot((xp.astype(np.float32) - cj.astype(np.float32)), nj.astype(np.float32)))
            worst_direct = max(worst_direct, abs(float(direct) - ref) / abs(ref))
    print(f"{name}: identity in FP32 {worst_id:.2e}, direct FP32 {worst_direct:.2e}")
    assert worst_id < 1e-5  # measured 0.9-1.3e-6
    assert worst_direct > 10 * worst_id  # the cancellation the identity avoids
