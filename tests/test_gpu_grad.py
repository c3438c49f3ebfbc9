"""Gradients of f = w^T K(theta) v on the GPU (addker_vjp and the autograd Function) against the
FP64 oracle: the exact gradient of the same NFFT approximation, finite differences, and the direct
FP64 gradient at the method's error level.

Tolerances (relative L2): grad_v and the hyperparameter gradients 1e-5 as for the products; the
coordinate gradient 3e-5 (it contracts the grids with window derivatives, whose magnitude is about
2n times the weights, so its FP32 rounding is a few times larger)."""
import numpy as np
import pytest

import workloads
from oracle import gradients
from parity_metrics import close

pytestmark = pytest.mark.gpu

TOL = 1e-5
TOL_X = 3e-5


def rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def make_op(torch, wl):
    from paper_2404_17344_gb300 import AddKer
    return AddKer(torch.from_numpy(wl.points).cuda(), wl.windows, wl.ell, wl.sigma_f, wl.bandwidth, wl.cutoff)


@pytest.mark.parametrize("cfg,N", [("c2", 4000), ("c3", 3000), ("c0", 1500)])
def test_vjp_vs_oracle_nfft_gradients(torch_cuda, cfg, N):
    torch = torch_cuda
    wl = workloads.make(cfg, N=N)
    wl.sigma_f = 1.4
    v, w = wl.vector(), wl.vector(which=2)
    op = make_op(torch, wl)
    gv, gt, gx = op.vjp(torch.from_numpy(v).cuda(), torch.from_numpy(w).cuda())
    rv, rell, rsf, rx = gradients.nfft_grad(wl.points, wl.windows, wl.ell, wl.sigma_f, v, w, wl.bandwidth, wl.cutoff)
    gt = gt.cpu().numpy()
    assert close(gv.cpu(), rv)
    assert close(gt[:wl.P], rell)
    assert abs(gt[wl.P] - rsf) <= TOL * abs(rsf)
    assert close(gx.cpu(), rx, TOL_X)


def test_autograd_function_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2404_17344_gb300.autograd import additive_kernel_matvec
    wl = workloads.make("c2", N=3000)
    v, w = wl.vector(), wl.vector(which=2)
    X = torch.from_numpy(wl.points).cuda().requires_grad_(True)
    vt = torch.from_numpy(v).cuda().requires_grad_(True)
    ell = torch.tensor(wl.ell, dtype=torch.float32, device="cuda", requires_grad=True)
    sf = torch.tensor(1.2, dtype=torch.float32, device="cuda", requires_grad=True)
    y = additive_kernel_matvec(X, vt, ell, sf, wl.windows, wl.bandwidth, wl.cutoff)
    loss = (torch.from_numpy(w).cuda() * y).sum()
    loss.backward()
    rv, rell, rsf, rx = gradients.nfft_grad(wl.points, wl.windows, wl.ell, 1.2, v, w, wl.bandwidth, wl.cutoff)
    assert close(vt.grad.cpu(), rv)
    assert close(ell.grad.cpu(), rell)
    assert abs(float(sf.grad) - rsf) <= TOL * abs(rsf)
    assert close(X.grad.cpu(), rx, TOL_X)


def test_finite_differences_on_gpu(torch_cuda):
    """Central differences of w^T K v computed by the GPU product: h = 1e-3 on ell, 1e-4 on x."""
    torch = torch_cuda
    from paper_2404_17344_gb300 import AddKer
    wl = workloads.make("c2", N=300)
    v, w = wl.vector(), wl.vector(which=2)
    vd, wd = torch.from_numpy(v).cuda(), torch.from_numpy(w)
    op = make_op(torch, wl)
    _, gt, gx = op.vjp(vd, wd.cuda())
    gt, gx = gt.cpu().numpy(), gx.cpu().numpy()

    def f(points, ell):
        o = AddKer(torch.from_numpy(points).cuda(), wl.windows, ell, wl.sigma_f, wl.bandwidth, wl.cutoff)
        y = o.matvec(vd).cpu().numpy().astype(np.float64)
        o.close()
        return float(w.astype(np.float64) @ y), float(np.abs(w) @ np.abs(y))

    # each FP32 output carries a relative error of about 1e-6 (rounding and atomic order), so f is known
    # to 1e-6 sum |w_i y_i|; a central difference divides twice that by 2h
    h = 1e-3
    for s in range(wl.P):
        ep, em = wl.ell.copy(), wl.ell.copy()
        ep[s] += h
        em[s] -= h
        (fp, ap), (fm, am) = f(wl.points, ep), f(wl.points, em)
        noise = 1e-6 * (ap + am) / (2 * h)
        assert abs(gt[s] - (fp - fm) / (2 * h)) <= noise + 1e-4 * abs(gt[s])
    h = 1e-4
    for k, c in [(0, 0), (17, 4), (123, 8), (299, 11)]:
        Xp, Xm = wl.points.copy(), wl.points.copy()
        Xp[k, c] += h
        Xm[k, c] -= h
        (fp, ap), (fm, am) = f(Xp, wl.ell), f(Xm, wl.ell)
        noise = 1e-6 * (ap + am) / (2 * h)
        assert abs(gx[k, c] - (fp - fm) / (2 * h)) <= noise + 1e-3 * abs(gx[k, c])


def test_direct_fp64_gradient_on_a_subset(torch_cuda):
    """Against the FP64 direct-sum gradient on 4096 sampled rows: the GPU gradient of the approximation
    differs from it by the method's own error (measured by the oracle's NFFT gradient) plus FP32."""
    torch = torch_cuda
    wl = workloads.make("c2", N=20000)
    v, w = wl.vector(), wl.vector(which=2)
    op = make_op(torch, wl)
    gv, gt, gx = op.vjp(torch.from_numpy(v).cuda(), torch.from_numpy(w).cuda())
    rows = np.random.default_rng(3).choice(wl.N, 4096, replace=False)
    dv, dell, dsf, dx = gradients.direct_grad(wl.points, wl.windows, wl.ell, wl.sigma_f, v, w, rows=rows)
    nv, nell, nsf, nx = gradients.nfft_grad(wl.points, wl.windows, wl.ell, wl.sigma_f, v, w, wl.bandwidth, wl.cutoff)
    assert rel(gv.cpu().numpy()[rows], dv[rows]) <= rel(nv[rows], dv[rows]) + TOL
    assert rel(gt.cpu().numpy()[:wl.P], dell) <= rel(nell, dell) + TOL
    assert rel(gx.cpu().numpy()[rows], dx) <= rel(nx[rows], dx) + TOL_X


@pytest.mark.slow
def test_vjp_at_the_configuration_size(torch_cuda):
    """The differentiation configuration at its full size (N = 2e5, 12 features, 4 windows of 3): every
    gradient against the oracle's FP64 NFFT gradients (the direct-sum comparison, O(N^2) in the oracle,
    runs at N = 2e4 above)."""
    torch = torch_cuda
    wl = workloads.make("c2", N=200_000)
    v, w = wl.vector(), wl.vector(which=2)
    op = make_op(torch, wl)
    gv, gt, gx = op.vjp(torch.from_numpy(v).cuda(), torch.from_numpy(w).cuda())
    gv, gt, gx = gv.cpu().numpy(), gt.cpu().numpy(), gx.cpu().numpy()
    rv, rell, rsf, rx = gradients.nfft_grad(wl.points, wl.windows, wl.ell, wl.sigma_f, v, w, wl.bandwidth, wl.cutoff)
    assert close(gv, rv)
    assert close(gt[:wl.P], rell)
    assert abs(gt[wl.P] - rsf) <= TOL * abs(rsf)
    assert close(gx, rx, TOL_X)
