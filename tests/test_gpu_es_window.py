"""The exponential-of-semicircle NFFT window (addker_opts.window = ADDKER_WIN_ES) on the GPU against the
FP64 oracle with the same window: 1e-5 relative L2 for the fused products on 3-D and mixed windows,
the spread grid itself (stage 0) against the oracle's spreading, and both windows against the exact
trigonometric sum within the window error. The coordinate gradient is refused for this window."""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import _clib, fastsum, window
from parity_metrics import close

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def make_op(torch, wl, win="es", **kw):
    from paper_2404_17344_gb300 import AddKer
    return AddKer(torch.from_numpy(wl.points).cuda(), wl.windows, wl.ell, wl.sigma_f, wl.bandwidth, wl.cutoff,
                  window=win, **kw)


@pytest.mark.parametrize("cfg,N", [("c1", 5000), ("c3", 3000), ("c1", 1)])
def test_es_products_match_oracle(torch_cuda, cfg, N):
    from paper_2404_17344_gb300 import ADDKER_ELL
    torch = torch_cuda
    wl = workloads.make(cfg, N=N)
    v = wl.vector()
    op = make_op(torch, wl)
    Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
    Kr, dKr = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v.astype(np.float64), wl.bandwidth,
                                 wl.cutoff, win="es")
    assert close(Kv.cpu(), Kr)
    # with one point the derivative products vanish (kappa_der(0) = 0): measure against |K v| there
    den = lambda b: max(np.linalg.norm(b), np.linalg.norm(Kr) if N == 1 else 0.0)
    for s in range(wl.P):
        d1 = np.asarray(dK[s].cpu(), np.float64)
        d2 = np.asarray(op.dmatvec(ADDKER_ELL(s), torch.from_numpy(v).cuda()).cpu(), np.float64)
        assert np.linalg.norm(d1 - dKr[s]) < TOL * den(dKr[s]), s
        assert np.linalg.norm(d2 - dKr[s]) < TOL * den(dKr[s]), s


def test_es_spread_grid_matches_oracle(torch_cuda):
    """Stage 0 (the spread grid, in the window's own normalisation: peak 1) against the oracle's spreading
    with the same window."""
    torch = torch_cuda
    wl = workloads.make("c1", N=4000)
    v = wl.vector()
    op = make_op(torch, wl)
    g = op.debug_stage(0, 0, torch.from_numpy(v).cuda())
    x = np.ascontiguousarray(wl.points[:, list(wl.windows[0])].astype(np.float64))
    n = 2 * wl.bandwidth[0]
    gref = np.zeros((n,) * 3)
    v64 = v.astype(np.float64)                                  # kept alive across the call
    _clib.lib().orc_spread(len(x), 3, _clib.ptr(x), _clib.ptr(v64), n, wl.cutoff,
                           window.es_beta(wl.cutoff), window.KINDS["es"], _clib.ptr(gref))
    assert close(np.asarray(g).reshape(gref.shape), gref)


def test_es_and_kb_approach_the_same_sum(torch_cuda):
    """Both windows approximate the exact trigonometric sum (the NDFT level of the oracle); on the GPU
    each stays within its window error plus the FP32 tolerance."""
    torch = torch_cuda
    wl = workloads.make("c1", N=1500)
    v = wl.vector()
    ref, dref = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v.astype(np.float64), wl.bandwidth,
                                   wl.cutoff, level="ndft")
    for win in ("kb", "es"):
        Kv, dK = make_op(torch, wl, win).matvec_all(torch.from_numpy(v).cuda())
        assert rel(Kv.cpu(), ref) < 1e-6 + TOL, win
        assert max(rel(dK[s].cpu(), dref[s]) for s in range(wl.P)) < 1e-5 + TOL, win


def test_es_vjp_is_refused(torch_cuda):
    from paper_2404_17344_gb300 import native
    torch = torch_cuda
    wl = workloads.make("c1", N=200)
    op = make_op(torch, wl)
    v = torch.from_numpy(wl.vector()).cuda()
    with pytest.raises(native.AddkerError) as e:
        op.vjp(v, v)
    assert e.value.status == native.ADDKER_EINVAL


@pytest.mark.parametrize("kernel,comp", [("matern", False), ("gauss", True), ("matern", True)])
def test_es_window_with_other_options(torch_cuda, kernel, comp):
    """The window choice composes with the kernel family and compensated accumulation: each combination
    against the oracle with the same window and kernel."""
    torch = torch_cuda
    wl = workloads.make("c3", N=4000)
    v = wl.vector()
    op = make_op(torch, wl, kernel=kernel, compensated=comp)
    Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
    Kr, dKr = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v.astype(np.float64), wl.bandwidth,
                                 wl.cutoff, win="es", kernel=kernel)
    assert close(Kv.cpu(), Kr)
    for s in range(wl.P):
        assert close(dK[s].cpu(), dKr[s]), s
