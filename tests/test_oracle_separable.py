"""Pins for the separable reading of the regularisation (Sec. 3.4's tensor-product coefficients with
each 1-D factor a least-squares Fourier extension on the data's coordinate extent).

Every pin compares against something the fit does not compute itself: a cosine polynomial that must be
reproduced exactly, the analytic Fourier coefficients of Sec. 3.1 (erf form) as a competing candidate
of the least-squares problem, the kernel itself evaluated on the coordinate box, the ell-derivative
identity of the derivative kernel, and the direct sums through the Hoelder bound."""
import numpy as np
import pytest

import workloads
from oracle import bounds, fastsum, kernels


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def cos_eval(c, x):
    """sum_{k in I_M} c_k e^{2 pi i k x} for a 1-D coefficient vector indexed k + M/2 (real part)."""
    M = len(c)
    k = np.arange(-M // 2, M // 2)
    return (np.exp(2j * np.pi * np.outer(x, k)) @ c).real


@pytest.mark.parametrize("M", [8, 16, 32, 64])
def test_fit_interval_rule(M):
    eps = 1 / 16
    lo = max(0.25, 0.5 - 4.0 / M)
    assert kernels.fit_interval(0.0, M, eps) == pytest.approx(min(lo, 0.5 - eps))
    assert kernels.fit_interval(0.21875, M, eps) == pytest.approx(0.4375)      # the ball's radius
    mid = 0.205
    assert kernels.fit_interval(mid, M, eps) == pytest.approx(min(0.4375, max(lo, 0.41)))


@pytest.mark.parametrize("M,a", [(16, 0.3), (32, 0.4), (64, 0.4375)])
def test_extension_reproduces_a_cosine_polynomial(M, a):
    """A function that already is an even trigonometric polynomial of degree < M/2 is its own best fit:
    the coefficients come back exactly, with the halving of c_{+-k} and c_{-M/2} = 0."""
    f = lambda x: 0.3 + 0.5 * np.cos(2 * np.pi * 3 * x) - 0.2 * np.cos(2 * np.pi * (M // 2 - 1) * x)
    c = kernels.cosine_extension(f(kernels.extension_nodes(a, M)), a, M)
    want = np.zeros(M)
    want[M // 2] = 0.3
    want[M // 2 + 3] = want[M // 2 - 3] = 0.25
    want[M - 1] = want[1] = -0.1
    np.testing.assert_allclose(c, want, atol=1e-9)
    assert c[0] == 0.0


@pytest.mark.parametrize("ell", [0.08, 0.12, 0.3, 1.0])
@pytest.mark.parametrize("M", [16, 32])
def test_extension_beats_every_other_candidate(ell, M):
    """Least-squares optimality on the nodes, against independent candidates from the same space: the
    truncated analytic Fourier series of the periodised Gaussian (Sec. 3.1, erf form), the trigonometric
    interpolant of plain periodic continuation (Lemma "aliasing error", p = 0), and random perturbations
    of the fit."""
    a = 0.4
    x = kernels.extension_nodes(a, M)
    f = kernels.kappa(x, ell)
    c = kernels.factor_coefficients(ell, a, M)
    res = np.linalg.norm(cos_eval(c, x) - f)
    k = np.arange(-M // 2 + 1, M // 2)
    ca = np.zeros(M)
    ca[1:] = bounds.analytic_coeff_gauss_1d(k, ell)
    assert res <= np.linalg.norm(cos_eval(ca, x) - f) * (1 + 1e-12) + 1e-15
    ci = kernels.coefficients(ell, 1, M, 0, 1 / 16)
    ci[0] = 0.0                                   # the -M/2 term is outside the fit's space
    assert res <= np.linalg.norm(cos_eval(ci, x) - f) * (1 + 1e-12) + 1e-15
    rng = np.random.default_rng(int(ell * 100) + M)
    for _ in range(20):
        dk = rng.standard_normal(M // 2) * 1e-6
        cp = c.copy()
        cp[M // 2] += dk[0]
        cp[M // 2 + 1:] += dk[1:] / 2
        cp[1:M // 2] += dk[:0:-1] / 2
        assert np.linalg.norm(cos_eval(cp, x) - f) >= res


def test_extension_converges_geometrically_in_M():
    """On a fixed interval the sup error of the extension of an entire function falls geometrically
    with M (Fourier extension theory), checked on a dense grid of [0, a] against the kernel."""
    a, ell = 0.4, 0.5
    xx = np.linspace(0.0, a, 4001)
    errs = []
    for M in (8, 16, 32):
        errs.append(np.abs(cos_eval(kernels.factor_coefficients(ell, a, M), xx) - kernels.kappa(xx, ell)).max())
    assert errs[0] > 30 * errs[1] > 900 * errs[2]
    assert errs[2] < 1e-6


@pytest.mark.parametrize("kind", ["gauss", "der"])
def test_tensor_assembly_against_the_kernel_on_the_box(kind):
    """The d = 3 coefficients (tensor product, or the three-term sum for the derivative kernel, Sec. 3.4)
    evaluated as a trigonometric polynomial match kappa(||r||) on the box prod_t [-a_t, a_t] with
    unequal a_t, within the 1-D fits' errors. A transposed axis or a dropped term of the sum fails:
    points near the long axis's end lie outside the short axes' intervals."""
    M, ell = 32, 0.5
    iv = [0.26, 0.38, 0.4375]
    c = kernels.coefficients_separable(ell, M, iv, kind)
    rng = np.random.default_rng(4)
    r = rng.uniform(-1, 1, (4000, 3)) * np.asarray(iv)
    r[:200, 2] = 0.43 * np.sign(r[:200, 2])
    xx = np.linspace(0, 0.4375, 2001)
    e1 = max(np.abs(cos_eval(kernels.factor_coefficients(ell, a, M, q), xx[xx <= a]) -
                    kernels.kappa(xx[xx <= a], ell, q)).max() for a in iv for q in ("gauss", "der"))
    got = kernels.trig_poly_eval(c, r)
    want = kernels.kappa(np.linalg.norm(r, axis=1), ell, kind)
    assert np.abs(got - want).max() <= 3 * e1 * (1 + e1) ** 2 * 1.01 + 1e-14
    # transposing the intervals moves the long axis's fit onto a short axis
    ct = kernels.coefficients_separable(ell, M, iv[::-1], kind)
    assert np.abs(kernels.trig_poly_eval(ct, r) - want).max() > 30 * (3 * e1)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_derivative_coefficients_are_the_ell_derivative(d):
    """kappa_der = (ell/2) d/d ell kappa and the fit is linear in the samples, so c_hat^der equals
    (ell/2) d c_hat / d ell coefficient by coefficient (central differences, FP64)."""
    M, ell, h = 16, 0.45, 1e-5
    iv = [0.3, 0.36, 0.4][:d]
    fd = (kernels.coefficients_separable(ell + h, M, iv) - kernels.coefficients_separable(ell - h, M, iv)) / (2 * h)
    cd = kernels.coefficients_separable(ell, M, iv, "der")
    assert np.abs(cd - ell / 2 * fd).max() < 1e-8 * np.abs(cd).max()


def test_coefficients_are_even_and_real():
    M = 16
    c = kernels.coefficients_separable(0.3, M, [0.3, 0.35, 0.4], "der")
    assert np.all(c[0, :, :] == 0) and np.all(c[:, 0, :] == 0) and np.all(c[:, :, 0] == 0)
    inner = c[1:, 1:, 1:]
    np.testing.assert_allclose(inner, inner[::-1, ::-1, ::-1], atol=1e-15)


def test_separable_fast_sum_within_hoelder_bound_of_direct():
    """Exact trigonometric sum with the separable coefficients against the direct sums on data shaped
    like the benchmark (a subsample of the N = 1e6 nine-feature workload): every output within
    ||v||_1 sup|kappa - kappa_F| (eq. "NFFT approx error"'s Hoelder step), the sup taken over the
    window's pairwise differences; and relative L2 far inside the 1e-4 bar (measured <= 3e-6)."""
    wl = workloads.make("c1", N=1_000_000)
    rng = np.random.default_rng(5)
    idx = rng.choice(wl.N, 1500, replace=False)
    X = wl.points[idx]
    v = rng.standard_normal(1500)
    Kd, Dd = fastsum.direct(X, wl.windows, wl.ell, 1.0, v)
    Kt, Dt = fastsum.matvec_all(X, wl.windows, wl.ell, 1.0, v, 32, 4, level="ndft", split=False)
    assert rel(Kt, Kd) < 1e-6
    for s, w in enumerate(wl.windows):
        assert rel(Dt[s], Dd[s]) < 1e-5
        xs = X[:, list(w)].astype(np.float64)
        cg, cd, _ = fastsum.coefficients_for(xs, wl.ell[s], 32, split=False)
        r = (xs[:300, None, :] - xs[None, :, :]).reshape(-1, 3)
        sup = np.abs(kernels.trig_poly_eval(cd, r) - kernels.kappa(np.linalg.norm(r, axis=1), wl.ell[s], "der")).max()
        one = fastsum.ndft_fastsum(xs, v, [cd])[0][:300]
        dd = fastsum.direct(X[:, list(w)], [(0, 1, 2)], [wl.ell[s]], 1.0, v, rows=np.arange(300))[1][0]
        assert np.all(np.abs(one - dd * wl.ell[s] / 2) <= np.abs(v).sum() * sup * 1.0001 + 1e-12)


def test_separable_beats_radial_against_direct():
    """The reason for the reading: against the direct sums the separable coefficients are at least ten
    times more accurate than the radial regularisation for every derivative product of the benchmark's
    windows at M = 32."""
    wl = workloads.make("c1", N=1_000_000)
    rng = np.random.default_rng(6)
    idx = rng.choice(wl.N, 1200, replace=False)
    X = wl.points[idx]
    v = rng.standard_normal(1200)
    _, Dd = fastsum.direct(X, wl.windows, wl.ell, 1.0, v)
    _, Ds = fastsum.matvec_all(X, wl.windows, wl.ell, 1.0, v, 32, 4, level="ndft", split=False)
    _, Dr = fastsum.matvec_all(X, wl.windows, wl.ell, 1.0, v, 32, 4, level="ndft", reg="radial")
    for s in range(wl.P):
        assert rel(Ds[s], Dd[s]) * 10 < rel(Dr[s], Dd[s])


def test_matern_rejects_the_separable_reading():
    xs = np.zeros((4, 2))
    with pytest.raises(ValueError):
        fastsum.coefficients_for(xs, 0.3, 16, kernel="matern", reg="separable")
    cg, _, q = fastsum.coefficients_for(xs, 0.3, 16, kernel="matern")
    assert q == 0.0
    np.testing.assert_array_equal(cg, kernels.coefficients(0.3, 2, 16, kernels.default_p(16, 1 / 16), 1 / 16, "matern"))


# --------------------------------------------------------------------- quadratic split ----

def test_quadratic_part_is_the_brute_force_sum():
    """sum_j ||x_i - x_j||^2 v_j through the moments equals the double loop (targets = sources and a
    separate target set)."""
    rng = np.random.default_rng(12)
    x = rng.uniform(-0.2, 0.2, (40, 3))
    t = rng.uniform(-0.2, 0.2, (7, 3))
    v = rng.standard_normal(40)
    for tg in (None, t):
        tt = x if tg is None else tg
        want = np.array([sum(float(np.sum((tt[i] - x[j]) ** 2)) * v[j] for j in range(40)) for i in range(len(tt))])
        np.testing.assert_allclose(kernels.quadratic_part(x, v, tg), want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_quadratic_coefficients_represent_the_quadratic(d):
    """c_hat^P (kind 'quad') evaluated as a trigonometric polynomial is ||r||^2/(2 ell^2) on the box of the
    fit intervals, within the 1-D fit's error."""
    M, ell = 32, 0.7
    iv = [0.3, 0.38, 0.42][:d]
    c = kernels.coefficients_separable(ell, M, iv, "quad")
    rng = np.random.default_rng(13)
    r = rng.uniform(-1, 1, (3000, d)) * np.asarray(iv)
    want = (r * r).sum(axis=1) / (2 * ell * ell)
    e1 = 0.0                                     # the 1-D fits' sup errors on their intervals, summed
    for a in iv:
        xx = np.linspace(0, a, 3001)
        ca = kernels.cosine_extension(kernels.extension_nodes(a, M) ** 2 / (2 * ell * ell), a, M)
        e1 += np.abs(cos_eval(ca, xx) - xx ** 2 / (2 * ell * ell)).max()
    assert np.abs(kernels.trig_poly_eval(c, r) - want).max() <= e1 * 1.01 + 1e-15
    assert e1 < 1e-5 * want.max()


def test_split_rule_on_the_benchmark_windows():
    """The quadratic part is split off for the wide kernels (ell = 0.5, 1.0) of the benchmark's windows and
    kept for the narrow one (ell = 0.3), where the remainder would carry a larger constant term."""
    wl = workloads.make("c1", N=200_000)
    got = [fastsum.coefficients_for(np.ascontiguousarray(wl.points[:, list(w)].astype(np.float64)), wl.ell[s], 32)[2]
           for s, w in enumerate(wl.windows)]
    assert got[0] == 0.0 and got[1] == pytest.approx(2.0) and got[2] == pytest.approx(0.5)


def test_split_product_equals_the_unsplit_one_within_the_fit_error():
    """Remainder-by-transform plus quadratic-by-moments is the same approximation of the derivative product
    up to the fit error of the quadratic's own extension (which the split no longer needs), and both meet
    the direct sums."""
    wl = workloads.make("c1", N=1_000_000)
    rng = np.random.default_rng(14)
    idx = rng.choice(wl.N, 1500, replace=False)
    X = wl.points[idx]
    v = rng.standard_normal(1500)
    _, Dd = fastsum.direct(X, wl.windows, wl.ell, 1.0, v)
    _, Ds = fastsum.matvec_all(X, wl.windows, wl.ell, 1.0, v, 32, 4, level="ndft")
    _, Du = fastsum.matvec_all(X, wl.windows, wl.ell, 1.0, v, 32, 4, level="ndft", split=False)
    for s in range(wl.P):
        assert rel(Ds[s], Du[s]) < 1e-5
        assert rel(Ds[s], Dd[s]) < 1e-5
    _, Dn = fastsum.matvec_all(X, wl.windows, wl.ell, 1.0, v, 32, 4)          # CPU NFFT, split
    for s in range(wl.P):
        assert rel(Dn[s], Ds[s]) < 1e-6
