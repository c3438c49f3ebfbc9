"""Pins for the oracle's direct sums (Sec. 3.3 definitions of K v and dK/d ell v).

Each check compares the C direct sum with something other than itself:
brute force, finite differences, symmetry, the kernel's limits and its
structure (additivity over windows, reduction of a window with a constant feature).
"""
import math

import numpy as np
import pytest

import workloads
from oracle import fastsum


def brute(points, windows, ell, sigma_f, v):
    N = points.shape[0]
    P = len(windows)
    Kv = [0.0] * N
    dK = [[0.0] * N for _ in range(P)]
    for i in range(N):
        for s, w in enumerate(windows):
            for j in range(N):
                r2 = sum((float(points[i, f]) - float(points[j, f])) ** 2 for f in w)
                k = math.exp(-r2 / (2 * ell[s] ** 2))
                Kv[i] += sigma_f ** 2 * k * v[j]
                dK[s][i] += sigma_f ** 2 * r2 / ell[s] ** 3 * k * v[j]
    return np.array(Kv), np.array(dK)


@pytest.fixture(scope="module")
def small():
    wl = workloads.tiny(N=30, d=5, windows=[(0, 1, 2), (3, 4)], ell=[0.3, 0.15])
    v = wl.vector().astype(np.float64)
    return wl, v


def test_brute_force_tiny(small):
    wl, v = small
    Kv, dK = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v)
    Kb, dKb = brute(wl.points, wl.windows, wl.ell, wl.sigma_f, v)
    np.testing.assert_allclose(Kv, Kb, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dK, dKb, rtol=1e-12, atol=1e-12)


def test_row_subset_matches_full(small):
    wl, v = small
    Kv, dK = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v)
    rows = np.array([3, 0, 29, 17])
    Kr, dKr = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v, rows=rows)
    np.testing.assert_array_equal(Kr, Kv[rows])
    np.testing.assert_array_equal(dKr, dK[:, rows])


def test_ell_derivative_is_finite_difference(small):
    """dK/d ell_s v against a central FP64 difference of K v in ell_s (h = 1e-5)."""
    wl, v = small
    _, dK = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v)
    h = 1e-5
    for s in range(wl.P):
        ep, em = wl.ell.copy(), wl.ell.copy()
        ep[s] += h
        em[s] -= h
        Kp, _ = fastsum.direct(wl.points, wl.windows, ep, wl.sigma_f, v)
        Km, _ = fastsum.direct(wl.points, wl.windows, em, wl.sigma_f, v)
        fd = (Kp - Km) / (2 * h)
        assert np.linalg.norm(fd - dK[s]) <= 1e-8 * np.linalg.norm(dK[s])


def test_sigma_f_scaling(small):
    """K is quadratic in sigma_f, so dK/d sigma_f v = (2/sigma_f) K v (Sec. 3.3)."""
    wl, v = small
    K1, _ = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v)
    h = 1e-6
    Kp, _ = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f + h, v)
    Km, _ = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f - h, v)
    np.testing.assert_allclose((Kp - Km) / (2 * h), 2.0 / wl.sigma_f * K1, rtol=1e-7, atol=1e-9)


def test_symmetry(small):
    wl, v = small
    w = wl.vector(which=2).astype(np.float64)
    Kv, dKv = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v)
    Kw, dKw = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, w)
    assert abs(w @ Kv - v @ Kw) <= 1e-12 * abs(w @ Kv) + 1e-12
    for s in range(wl.P):
        assert abs(w @ dKv[s] - v @ dKw[s]) <= 1e-12 * np.abs(dKv[s]).sum() + 1e-12


def test_unit_vector_columns(small):
    """K e_j has diagonal entry sigma_f^2 P, entries in (0, sigma_f^2 P], and equals row j (symmetry);
    dK/d ell e_j vanishes on the diagonal (zero distance)."""
    wl, _ = small
    N = wl.N
    for j in (0, 11, N - 1):
        e = np.zeros(N)
        e[j] = 1.0
        col, dcol = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, e)
        assert col[j] == pytest.approx(wl.sigma_f ** 2 * wl.P, rel=1e-15)
        assert np.all(col > 0) and np.all(col <= wl.sigma_f ** 2 * wl.P + 1e-15)
        assert np.all(dcol[:, j] == 0.0)
        row = np.array([fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f,
                                       np.eye(N)[i], rows=[j])[0][0] for i in range(N)])
        np.testing.assert_allclose(row, col, rtol=1e-14)


def test_limits(small):
    """ell -> 0: K -> sigma_f^2 P I; ell -> infinity: K -> sigma_f^2 P 1 1^T; dK -> 0 at both ends."""
    wl, v = small
    tiny = np.full(wl.P, 1e-5)
    Kv, dK = fastsum.direct(wl.points, wl.windows, tiny, wl.sigma_f, v)
    np.testing.assert_allclose(Kv, wl.sigma_f ** 2 * wl.P * v, rtol=1e-12, atol=1e-12)
    assert np.abs(dK).max() < 1e-12
    huge = np.full(wl.P, 1e5)
    Kv, dK = fastsum.direct(wl.points, wl.windows, huge, wl.sigma_f, v)
    np.testing.assert_allclose(Kv, wl.sigma_f ** 2 * wl.P * v.sum(), rtol=1e-9)
    assert np.abs(dK).max() < 1e-9


def test_additive_over_windows(small):
    wl, v = small
    Kv, dK = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v)
    parts = [fastsum.direct(wl.points, [w], wl.ell[s:s + 1], wl.sigma_f, v) for s, w in enumerate(wl.windows)]
    np.testing.assert_allclose(Kv, sum(p[0] for p in parts), rtol=1e-13)
    for s in range(wl.P):
        np.testing.assert_array_equal(dK[s], parts[s][1][0])


def test_constant_feature_drops_out(small):
    wl, v = small
    X = wl.points.copy()
    X[:, 2] = 0.01
    a, da = fastsum.direct(X, [(0, 1, 2)], wl.ell[:1], 1.0, v)
    b, db = fastsum.direct(X, [(0, 1)], wl.ell[:1], 1.0, v)
    np.testing.assert_allclose(a, b, rtol=1e-14)
    np.testing.assert_allclose(da, db, rtol=1e-14)
