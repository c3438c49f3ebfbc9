"""Error measures of the GPU parity tests (test helpers, no method arithmetic).

rel: relative L2 error over all entries. maxrow: the largest single-entry error relative to the RMS of the
reference, so that a localised error (a tail item, an edge cell) that the L2 norm would average away still
shows. close: both at once; independent FP32 rounding gives a max-row error of a few times the relative L2
error, so the max-row bar is 10 x the tolerance."""
import numpy as np

TOL = 1e-5


def _flat(a):
    """All entries in double precision, complex ones (spectra) kept complex."""
    a = np.asarray(a)
    return a.astype(np.complex128 if np.iscomplexobj(a) else np.float64).ravel()


def rel(a, b):
    a, b = _flat(a), _flat(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def maxrow(a, b):
    a, b = _flat(a), _flat(b)
    return float(np.abs(a - b).max() / (np.linalg.norm(b) / np.sqrt(b.size)))


def close(a, b, tol=TOL):
    return rel(a, b) < tol and maxrow(a, b) < 10 * tol
