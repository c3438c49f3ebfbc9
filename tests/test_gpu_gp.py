"""The regression system and GP training on the GPU (addker_cg, addker_gp_grad) against the FP64
oracle (oracle/gp.py: dense solves, the exact Hutchinson estimator for the same probes).

The GPU solves with the fast-summation operator K~ in FP32 to a CG tolerance; the oracle uses the
exact dense K. So the solutions differ by at most about kappa (eps + tol) in relative terms, with
kappa the condition number of K + beta I (computed here from the dense matrix), eps the operator's
relative error (measured here: the oracle's FP64 NFFT products against the dense products) and tol the
CG tolerance; the gradient terms inherit that bound (twice: once through alpha, once through the
probe solves). The tests use these bounds, computed from the data, as tolerances."""
import numpy as np
import pytest

import workloads
from oracle import fastsum, gp

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def problem(N=1000, M=64, beta=20.0):
    wl = workloads.tiny(N=N, d=5, windows=[(0, 1, 2), (3, 4)], seed=5, ell=[0.3, 0.45])
    wl.bandwidth = [M, M]
    wl.cutoff = 4
    wl.sigma_f = 1.1
    K, dK = gp.dense_kernel(wl.points, wl.windows, wl.ell, wl.sigma_f)
    ev = np.linalg.eigvalsh(K + beta * np.eye(wl.N))
    v = np.random.default_rng(3).standard_normal(wl.N)
    Kn, dKn = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v, wl.bandwidth, wl.cutoff)
    eps = max([rel(Kn, K @ v)] + [rel(dKn[s], dK[s] @ v) for s in range(wl.P)])
    return wl, K, dK, beta, ev[-1] / ev[0], eps


def make_op(torch, wl):
    from paper_2404_17344_gb300 import AddKer
    return AddKer(torch.from_numpy(wl.points).cuda(), wl.windows, wl.ell, wl.sigma_f, wl.bandwidth, wl.cutoff)


def test_cg_residual_and_solution(torch_cuda):
    torch = torch_cuda
    wl, K, dK, beta, kappa, eps = problem()
    tol = 1e-6
    Y = np.random.default_rng(1).standard_normal((wl.N, 3)).astype(np.float32)
    Y[:, 2] = 0.0                                               # a zero column returns x = 0 at once
    op = make_op(torch, wl)
    op.set_precond(0)                                           # plain CG, as the paper and the oracle's cg
    X, iters, relres = op.cg(torch.from_numpy(Y).cuda(), beta, tol=tol, maxit=500)
    X = X.cpu().numpy().astype(np.float64)
    assert relres[0] <= tol and relres[1] <= tol and iters[2] == 0 and not X[:, 2].any()
    for j in range(2):
        y = Y[:, j].astype(np.float64)
        # residual under the oracle's FP64 fast-summation operator: tol plus the FP32 product error
        Kx, _ = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, X[:, j], wl.bandwidth, wl.cutoff)
        assert np.linalg.norm(y - Kx - beta * X[:, j]) <= (tol + 1e-5) * np.linalg.norm(y)
        xs = np.linalg.solve(K + beta * np.eye(wl.N), y)
        assert rel(X[:, j], xs) <= kappa * (eps + tol)
    # the oracle's own CG on the dense matrix takes a similar number of iterations
    _, it_o, _ = gp.cg(lambda V: K @ V + beta * V, Y[:, 0].astype(np.float64), tol, 500)
    assert abs(iters[0] - it_o) <= max(3, it_o // 5)


def test_cg_initial_guess_and_maxit(torch_cuda):
    torch = torch_cuda
    wl, K, dK, beta, kappa, eps = problem(N=800)
    y = np.random.default_rng(4).standard_normal(wl.N).astype(np.float32)
    op = make_op(torch, wl)
    x, it, r = op.cg(torch.from_numpy(y).cuda(), beta, tol=1e-6, maxit=500)
    # restarting from the solution needs (almost) no iterations
    x2, it2, r2 = op.cg(torch.from_numpy(y).cuda(), beta, tol=1e-5, maxit=500, x0=x)
    assert it2[0] <= 1 and r2[0] <= 1e-5
    # maxit stops early and reports the residual it reached
    x3, it3, r3 = op.cg(torch.from_numpy(y).cuda(), beta, tol=1e-12, maxit=3)
    assert it3[0] == 3 and r3[0] > 1e-12


def test_gp_grad_matches_dense_estimator(torch_cuda):
    torch = torch_cuda
    wl, K, dK, beta, kappa, eps = problem()
    tol = 1e-6
    y = np.random.default_rng(1).standard_normal(wl.N).astype(np.float32)
    Z = np.random.default_rng(2).choice([-1.0, 1.0], size=(wl.N, 4)).astype(np.float32)
    op = make_op(torch, wl)
    g, fit, alpha, iters = op.gp_grad(torch.from_numpy(y).cuda(), beta, torch.from_numpy(Z).cuda(), tol=tol, maxit=500)
    y64, Z64 = y.astype(np.float64), Z.astype(np.float64)
    gref = gp.lml_grad_hutchinson_dense(K, dK, wl.sigma_f, beta, y64, Z64)
    bound = 2 * kappa * (eps + tol)
    assert np.abs(g - gref).max() <= bound * np.abs(gref).max()
    xs = np.linalg.solve(K + beta * np.eye(wl.N), y64)
    assert abs(fit - y64 @ xs) <= kappa * (eps + tol) * abs(y64 @ xs)
    assert rel(alpha.cpu(), xs) <= kappa * (eps + tol)
    assert 0 < iters <= 500
    # without probes only the data term remains: 1/2 alpha^T (dA/dtheta) alpha
    g0, _, _, _ = op.gp_grad(torch.from_numpy(y).cuda(), beta, None, tol=tol, maxit=500)
    D = [dK[s] for s in range(wl.P)] + [(2.0 / wl.sigma_f) * K, np.eye(wl.N)]
    ref0 = np.array([0.5 * xs @ (Dq @ xs) for Dq in D])
    assert np.abs(g0 - ref0).max() <= bound * np.abs(ref0).max()


def test_gp_grad_identity_probes_give_exact_gradient(torch_cuda):
    """Z = sqrt(N) I (N probes): the estimator is the exact trace, so the GPU gradient approaches the
    exact gradient of the log marginal likelihood (pinned in the CPU tests by finite differences)."""
    torch = torch_cuda
    wl, K, dK, beta, kappa, eps = problem(N=200, beta=5.0)
    y = np.random.default_rng(6).standard_normal(wl.N).astype(np.float32)
    Z = (np.sqrt(wl.N) * np.eye(wl.N)).astype(np.float32)
    op = make_op(torch, wl)
    g, _, _, _ = op.gp_grad(torch.from_numpy(y).cuda(), beta, torch.from_numpy(Z).cuda(), tol=1e-6, maxit=500)
    gex = gp.lml_grad_exact(K, dK, wl.sigma_f, beta, y.astype(np.float64))
    assert np.abs(g - gex).max() <= 2 * kappa * (eps + 1e-6) * np.abs(gex).max()


def test_preconditioned_cg_at_the_gp_noise_level(torch_cuda):
    """The GP configuration's points (a 1500-point sample, 8 windows of 3, ell = 0.5) at its noise variance
    beta = 0.01: with the Fourier low-mode preconditioner (default band 1) the GPU solve takes a fraction of
    plain CG's iterations and the oracle's preconditioned CG on the dense kernel takes about as many; both
    GPU solutions agree with the dense solve to the level the FP32 operator allows at this conditioning
    (measured 4e-5)."""
    torch = torch_cuda
    wl = workloads.make("c4", N=2_000_000)
    idx = np.random.default_rng(23).choice(wl.N, 1500, replace=False)
    X = np.ascontiguousarray(wl.points[idx])
    y = wl.targets()[idx]
    beta = 0.01
    K, _ = gp.dense_kernel(X, wl.windows, wl.ell, wl.sigma_f)
    xref = np.linalg.solve(K + beta * np.eye(len(y)), y.astype(np.float64))
    from paper_2404_17344_gb300 import AddKer
    op = AddKer(torch.from_numpy(X).cuda(), wl.windows, wl.ell, wl.sigma_f, wl.bandwidth, wl.cutoff)
    res = {}
    for band in (0, 1):
        op.set_precond(band)
        x, it, rr = op.cg(torch.from_numpy(y).cuda(), beta, tol=1e-6, maxit=2000)
        res[band] = (x.cpu().numpy().astype(np.float64), it[0], rr[0])
        assert rr[0] <= 1e-6
        assert rel(res[band][0], xref) <= 1e-3
    assert res[1][1] * 4 <= res[0][1]
    # the oracle's preconditioned CG with the same modes on the dense matrix
    coefs = [fastsum.coefficients_for(np.ascontiguousarray(X[:, list(w)].astype(np.float64)), wl.ell[s], 32)[0]
             for s, w in enumerate(wl.windows)]
    modes, wmode = gp.fourier_modes(wl.windows, coefs, 1, beta, wl.sigma_f, len(y))
    U, owner = gp.fourier_basis(X, wl.windows, modes)
    _, it_o, _ = gp.pcg(lambda v: K @ v + beta * v, gp.woodbury_apply(U, wmode[owner], beta), y.astype(np.float64),
                        1e-6, 500)
    assert abs(res[1][1] - it_o) <= max(4, it_o // 3)


def test_preconditioner_setting_and_well_conditioned_solves(torch_cuda):
    """Bands 1 to 3 give the same solution as plain CG on a well-conditioned system; band 4 is refused."""
    torch = torch_cuda
    wl, K, dK, beta, kappa, eps = problem(N=900)
    y = np.random.default_rng(7).standard_normal(wl.N).astype(np.float32)
    op = make_op(torch, wl)
    xs = np.linalg.solve(K + beta * np.eye(wl.N), y.astype(np.float64))
    for band in (0, 1, 2, 3):
        op.set_precond(band)
        x, it, rr = op.cg(torch.from_numpy(y).cuda(), beta, tol=1e-6, maxit=500)
        assert rr[0] <= 1e-6 and rel(x.cpu(), xs) <= kappa * (eps + 1e-6)
    from paper_2404_17344_gb300 import AddkerError
    with pytest.raises(AddkerError):
        op.set_precond(4)
