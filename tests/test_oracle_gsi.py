"""Pins of oracle/gsi.py (Algorithm "Computation of GSI") against the ANOVA decomposition computed by
brute force: the window's trigonometric polynomial is evaluated on a full grid of the torus, its
variance and the variance of each ANOVA term (integrate the other coordinates out, subtract the lower
terms) are taken numerically and compared with theta_u."""
import itertools

import numpy as np

import workloads
from oracle import gsi


def poly_on_grid(spec):
    """Values of h~(x) = sum_k spec_k e^{2 pi i k.x} on the grid x = l/M, l in I_M^d (complex)."""
    M = spec.shape[0]
    return np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(spec))) * M ** spec.ndim


def anova_variances(f):
    """Variance of every ANOVA term of the grid function f (real part; axes = features), by the
    inclusion-exclusion definition of the classical ANOVA decomposition."""
    d = f.ndim
    f = f - f.mean()
    terms = {}
    for r in range(1, d + 1):
        for u in itertools.combinations(range(d), r):
            other = tuple(t for t in range(d) if t not in u)
            g = f.mean(axis=other, keepdims=True) if other else f
            for rr in range(1, r):
                for v in itertools.combinations(u, rr):
                    g = g - terms[v]
            terms[u] = g
    return {u: float(np.mean(np.abs(np.broadcast_to(t, f.shape)) ** 2)) for u, t in terms.items()}


def test_theta_equals_anova_term_variances():
    wl = workloads.tiny(N=300, d=4, windows=[(0, 1, 2), (3,)], seed=21, ell=[0.3, 0.2])
    v = wl.vector()
    M = 12
    rho, theta, total = gsi.gsi(wl.points, wl.windows, wl.ell, v, M)
    # window (0, 1, 2): brute-force ANOVA of its polynomial on the grid
    spec = gsi.window_spectrum(wl.points, (0, 1, 2), wl.ell[0], v, M)
    var = anova_variances(poly_on_grid(spec))
    for u, t in var.items():
        assert abs(theta[tuple(u)] - t) <= 1e-9 * total, u
    # window (3,): a 1-D window's only term
    spec3 = gsi.window_spectrum(wl.points, (3,), wl.ell[1], v, M)
    var3 = anova_variances(poly_on_grid(spec3))
    assert abs(theta[(3,)] - var3[(0,)]) <= 1e-9 * total
    assert abs(sum(rho.values()) - 1.0) < 1e-12
    # Parseval: the total is the variance of the sum of the window polynomials' non-constant parts
    assert abs(total - (sum(var.values()) + var3[(0,)])) <= 1e-9 * total


def test_shared_subsets_accumulate():
    """Two windows sharing features: theta of a shared subset is the sum of both windows' terms."""
    wl = workloads.tiny(N=200, d=4, windows=[(0, 1, 2), (1, 2, 3)], seed=22, ell=[0.35, 0.35])
    v = wl.vector()
    M = 8
    _, theta, _ = gsi.gsi(wl.points, wl.windows, wl.ell, v, M)
    _, th1, _ = gsi.gsi(wl.points, [(0, 1, 2)], wl.ell[:1], v, M)
    _, th2, _ = gsi.gsi(wl.points, [(1, 2, 3)], wl.ell[1:], v, M)
    for u in gsi.subsets_of(wl.windows):
        assert abs(theta[u] - th1.get(u, 0.0) - th2.get(u, 0.0)) <= 1e-12 * max(theta.values())
    assert set(theta) == set(gsi.subsets_of(wl.windows))


def test_transposed_pattern_is_caught():
    """The subset labelling has teeth: swapping two axes of the spectrum changes theta of the
    singletons (the window's points are not symmetric in its features)."""
    wl = workloads.tiny(N=300, d=3, seed=23, ell=[0.3])
    wl.points[:, 1] *= 0.3                                  # make feature 1 less spread than feature 0
    v = wl.vector()
    spec = gsi.window_spectrum(wl.points, (0, 1, 2), 0.3, v, 12)
    pat = gsi.support_pattern(12, 3)
    e = np.abs(spec) ** 2
    t0, t1 = e[pat == 1].sum(), e[pat == 2].sum()
    et = np.abs(np.swapaxes(spec, 0, 1)) ** 2
    assert abs(et[pat == 1].sum() - t0) > 1e-3 * abs(t0) and abs(t0 - t1) > 1e-3 * abs(t0)
