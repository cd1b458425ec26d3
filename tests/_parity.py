"""Error measures shared by the GPU parity tests.

Arrays are (nrhs, n): right-hand sides by rows, triangles (or vertices) by
columns, as the binding lays them out.

rel      ||y - ref||_2 / ||ref||_2 over all entries (the tolerances' measure).
rowmax   max_i ||y_i - ref_i||_2 / rms_i ||ref_i||_2: the worst single row
         (2-norm over the right-hand sides) against a typical row's size.  On n
         rows the 2-norm dilutes one wrong row by sqrt(n); this measure does
         not, so a few wrong rows (one pair class on cube edges, one leaf's
         tile) fail it even when rel passes.
close    asserts rel < tol and rowmax < ROWFACTOR tol and returns both.  The
         factor 10 leaves room for rows whose own error is larger than the
         mean because their nearfield carries more singular pairs.
"""
import numpy as np

ROWFACTOR = 10.0


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rowmax(a, b) -> float:
    a = np.atleast_2d(np.asarray(a, dtype=np.float64))
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    num = np.linalg.norm(a - b, axis=0)
    rms = np.sqrt(np.mean(np.sum(b * b, axis=0)))
    return float(num.max() / rms)


def close(a, b, tol: float, what: str = ""):
    e, r = rel(a, b), rowmax(a, b)
    print(f"{what} rel {e:.3e} rowmax {r:.3e} (tol {tol:.0e})")
    assert e < tol, f"{what}: rel {e:.3e} >= {tol:.0e}"
    assert r < ROWFACTOR * tol, f"{what}: rowmax {r:.3e} >= {ROWFACTOR * tol:.0e}"
    return e, r
