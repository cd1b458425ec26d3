"""Independent brute-force integrals used to pin the oracle (numpy only).

* Closed-form potentials of a flat triangle with unit density:
  single layer  int_sigma 1/|x-y| dy        (edge-sum formula obtained from the
                                              2-D divergence theorem in the plane)
  double layer  int_sigma (x-y).n/|x-y|^3 dy (signed solid angle, van Oosterom-
                                              Strackee formula)
* Outer integral over a triangle by uniform 4-way subdivision with a collapsed
  Gauss rule on every piece, plus Richardson extrapolation in the depth.
"""
import numpy as np


def slp_potential(x, Y):
    x = np.atleast_2d(x)
    y0, y1, y2 = (np.asarray(v, float) for v in Y)
    n = np.cross(y1 - y0, y2 - y0)
    n /= np.linalg.norm(n)
    h = (x - y0) @ n
    xp = x - h[:, None] * n
    ah = np.abs(h)
    tot = np.zeros(len(x))
    for a, b in ((y0, y1), (y1, y2), (y2, y0)):
        t = (b - a) / np.linalg.norm(b - a)
        m = np.cross(t, n)
        sm = (a - xp) @ t
        sp = (b - xp) @ t
        p = (a - xp) @ m
        Rm = np.linalg.norm(x - a, axis=1)
        Rp = np.linalg.norm(x - b, axis=1)
        R02 = p * p + h * h
        with np.errstate(divide="ignore", invalid="ignore"):
            lg = np.where(sm >= 0, np.log((Rp + sp) / (Rm + sm)), np.log((Rm - sm) / (Rp - sp)))
        tot += p * lg - ah * (np.arctan2(p * sp, R02 + ah * Rp) - np.arctan2(p * sm, R02 + ah * Rm))
    return tot


def dlp_potential(x, Y):
    x = np.atleast_2d(x)
    a, b, c = (np.asarray(v, float) - x for v in Y)
    la, lb, lc = (np.linalg.norm(v, axis=1) for v in (a, b, c))
    num = np.einsum("ij,ij->i", a, np.cross(b, c))
    den = (la * lb * lc + np.einsum("ij,ij->i", a, b) * lc + np.einsum("ij,ij->i", a, c) * lb
           + np.einsum("ij,ij->i", b, c) * la)
    return -2.0 * np.arctan2(num, den)


def tri_rule(q):
    x, w = np.polynomial.legendre.leggauss(q)
    x = (x + 1) / 2
    w = w / 2
    U = np.repeat(x, q)
    V = (1 - U) * np.tile(x, q)
    W = 2 * np.repeat(w, q) * np.tile(w, q) * (1 - U)
    return U, V, W


def tri_integral(T, f, q=10):
    """int_T f by the collapsed Gauss rule (exact for polynomials of degree 2q-2)."""
    a, b, c = (np.asarray(v, float) for v in T)
    U, V, W = tri_rule(q)
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
    pts = a + U[:, None] * (b - a) + V[:, None] * (c - a)
    return area * (W * f(pts)).sum()


def subdivide(T, L):
    tris = [np.asarray(T, float)]
    for _ in range(L):
        nt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nt += [np.array([a, ab, ca]), np.array([ab, b, bc]), np.array([ca, bc, c]), np.array([ab, bc, ca])]
        tris = nt
    return tris


def outer_integral(X, f, L, q=10):
    return sum(tri_integral(t, f, q) for t in subdivide(X, L))


def pair_brute(X, Y, kernel, L=5, q=10):
    """int_X int_Y k dy dx, k = 1/(4 pi r) (kernel 0) or (x-y).n_Y/(4 pi r^3)
    (kernel 1), Richardson-extrapolated over subdivision depths L-1, L."""
    pot = slp_potential if kernel == 0 else dlp_potential
    f = lambda p: pot(p, Y) / (4 * np.pi)  # noqa: E731
    a = outer_integral(X, f, L - 1, q)
    b = outer_integral(X, f, L, q)
    return b + (b - a) / 3.0
