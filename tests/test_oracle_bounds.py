"""Pins for the oracle's coefficient code against the error theorems of Sec. 3.4 and
the numbers the paper prints in their proofs (tests/golden/paper_constants.txt)."""
import os

import mpmath as mp
import numpy as np
import pytest
from scipy.special import erfc

from oracle import bounds, kernels

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, val, tol = line.split()[:3]
        out[name] = (float(val), float(tol))
    return out


def test_golden_thresholds():
    g = golden()
    v, t = g["ell_threshold_low"]
    assert bounds.ELL_STAR == pytest.approx(v, abs=t)
    v, t = g["ell_threshold_high"]
    assert 0.5 * np.sqrt(2 / (5 - np.sqrt(17))) == pytest.approx(v, abs=t)
    v, _ = g["const_102"]
    assert 2539 / 25 == pytest.approx(v, abs=0.005) and 2539 / 25 < 102


def test_golden_gprime_at_sign_changes():
    """g(x) = x^2/(2 ell^2) exp(-x^2/(2 ell^2)); g' at the sign changes x_1, x_2 of g''."""
    g = golden()
    for ell in (0.3, 1.0):
        x1 = ell * np.sqrt((5 - np.sqrt(17)) / 2)
        x2 = ell * np.sqrt((5 + np.sqrt(17)) / 2)
        gp = lambda x: float(mp.diff(lambda t: t * t / (2 * ell * ell) * mp.exp(-t * t / (2 * ell * ell)), x))
        assert gp(x1) * 2 * ell == pytest.approx(g["gprime_x1_times_2ell"][0], abs=g["gprime_x1_times_2ell"][1])
        assert gp(x2) * 2 * ell == pytest.approx(g["gprime_x2_times_2ell"][0], abs=g["gprime_x2_times_2ell"][1])


def test_golden_A_max():
    """A(eta, ell) over eta >= 1 peaks at eta = 1, ell >= 1/2 at about 0.377."""
    g = golden()
    vals = [bounds.A(e, ell) for e in np.linspace(1, 5, 41) for ell in np.linspace(0.02, 3, 150)]
    assert max(vals) == pytest.approx(g["A_max_eta_ge_1"][0], abs=g["A_max_eta_ge_1"][1])
    x = np.linspace(0.01, 5, 100001)
    assert (x ** -2 * np.exp(-1 / (8 * x * x))).max() == pytest.approx(g["max_x2_exp"][0], abs=g["max_x2_exp"][1])


def test_golden_coefficient_sums():
    """sum_{k=1}^{M/2} |c_k(f)| <= 3/4 and sum_{k=1}^{M/2} |c_k(g)| < 7/2 (proofs of the theorems),
    with c_k(f) from the analytic form and c_k(g) by quadrature."""
    g = golden()
    for ell in (0.05, 0.2, 0.5, 1.0, 3.0):
        k = np.arange(1, 33)
        assert np.abs(bounds.analytic_coeff_gauss_1d(k, ell)).sum() <= g["sum_ck_f_half"][0]
        cg = [abs(float(mp.quad(lambda x: x * x / (2 * ell * ell) * mp.exp(-x * x / (2 * ell * ell))
                                * mp.cos(2 * mp.pi * kk * x), [-0.5, 0, 0.5]))) for kk in range(1, 17)]
        assert sum(cg) < g["sum_ck_g_half"][0]


def test_analytic_coefficient_bound():
    """|c_k(f)| <= ell sqrt(2 pi) e^{-2 pi^2 ell^2 k^2} + (case term) (proof of Theorem "multi_gauss")."""
    for ell in (0.1, 0.4, 0.6, 2.0):
        k = np.arange(1, 200)
        c = np.abs(bounds.analytic_coeff_gauss_1d(k, ell))
        tail = (np.exp(-1 / (8 * ell * ell)) / (2 * ell * ell * np.pi ** 2 * k ** 2) if ell < 0.5
                else np.exp(-0.5) / (np.pi ** 2 * k ** 2 * ell))
        assert np.all(c <= ell * np.sqrt(2 * np.pi) * np.exp(-2 * np.pi ** 2 * ell ** 2 * k ** 2) + tail + 1e-15)


def test_S_uses_erfc():
    e, ell = 2.0, 0.9
    assert bounds.S(e, ell) > erfc(e) / 4


def _measured_sup_error(ell, M, d, kind, npts, seed=0):
    rng = np.random.default_rng(seed)
    r = rng.uniform(-0.5, 0.5, size=(npts, d))
    c = kernels.coefficients(ell, d, M, 0, 1 / 16, kind)
    exact = kernels.kappa(np.linalg.norm(r, axis=1), ell, kind)
    return np.abs(kernels.trig_poly_eval(c, r) - exact).max()


@pytest.mark.parametrize("M,npts", [(16, 10000), (32, 10000), (64, 1500)])
def test_E5_protocol_3d(M, npts):
    """Sec. 3.4.3: measured ||kappa_ERR||_inf on uniform r in [-1/2,1/2]^3 stays below the bounds of
    Theorems "multi_gauss" and "multi_deriv" (plain periodic continuation, eta >= 1)."""
    for ell in (0.05, 0.1, 0.2, 0.3, 0.5, 1.0, 2.0):
        if bounds.eta(ell, M) < 1:
            continue
        eg = _measured_sup_error(ell, M, 3, "gauss", npts)
        ed = _measured_sup_error(ell, M, 3, "der", npts)
        # 1e-14: the FP64 rounding floor of evaluating a 64^3-term sum; some bounds are far below it
        assert eg <= bounds.bound_gauss_3d(ell, M) + 1e-14, (ell, M, eg)
        assert ed <= bounds.bound_der_3d(ell, M) + 1e-14, (ell, M, ed)


@pytest.mark.parametrize("M", [16, 32, 64])
def test_E5_protocol_1d(M):
    """Remarks "gaussian1d" / "deriv1d": 2 gamma + 4 A and 2 xi + 4 S in one dimension."""
    for ell in (0.03, 0.1, 0.3, 1.0, 3.0):
        if bounds.eta(ell, M) < 1:
            continue
        assert _measured_sup_error(ell, M, 1, "gauss", 20000) <= bounds.bound_gauss_1d(ell, M) + 1e-14
        assert _measured_sup_error(ell, M, 1, "der", 20000) <= bounds.bound_der_1d(ell, M) + 1e-14


def test_error_decreases_with_M():
    for ell in (0.1, 0.5):
        errs = [_measured_sup_error(ell, M, 3, "gauss", 3000) for M in (16, 32)]
        assert errs[1] < errs[0]
