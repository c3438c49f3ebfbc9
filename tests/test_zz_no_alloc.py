"""addker_fastsum_noalloc against the plan path (addker_setup + addker_matvec_all) and the oracle.

The no-allocation entry point serves callers that cannot call cudaMalloc (servers that fix their
device memory at start-up, hosts whose own allocator owns the device memory). It takes all working
memory from one fixed device array, so calls in a row must each agree with the plan path and with
the oracle: every call sees the previous call's leftovers (a larger layout, other sizes) and must
clear what has to start at zero. This file is collected last so a stop-at-first-failure run has
already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import fastsum
from parity_metrics import close

pytestmark = pytest.mark.gpu

TOL = 1e-5          # the parity tolerance of the other GPU tests


def rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def maxrow(a, b):
    """Largest single-row error relative to the RMS of the reference: a localised error that the
    relative L2 norm would average away shows up here."""
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.abs(a - b).max() / (np.linalg.norm(b) / np.sqrt(b.size)))


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2404_17344_gb300 import native
    return torch, native


def noalloc_status(torch, native, X, ell, sigma_f, M, m, v, Kv, dK):
    N, d = X.shape
    return native.lib().addker_fastsum_noalloc(
        ctypes.c_void_p(X.data_ptr()), N, d, float(ell), float(sigma_f), M, m, ctypes.c_void_p(v.data_ptr()),
        ctypes.c_void_p(Kv.data_ptr()), ctypes.c_void_p(dK.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def noalloc(torch, native, X, ell, sigma_f, M, m, v):
    N = X.shape[0]
    Kv = torch.empty(N, device="cuda")
    dK = torch.empty(N, device="cuda")
    st = noalloc_status(torch, native, X, ell, sigma_f, M, m, v, Kv, dK)
    assert st == native.ADDKER_OK, native.lib().addker_strerror(st)
    return Kv.cpu().numpy(), dK.cpu().numpy()


def test_noalloc_matches_plan_path_on_two_calls(env):
    torch, native = env
    from paper_2404_17344_gb300 import AddKer
    wl = workloads.make("c1", N=20000)
    X = torch.from_numpy(np.ascontiguousarray(wl.points[:, :3])).cuda()
    ell, sigma_f = 0.5, 1.3
    op = AddKer(X, [(0, 1, 2)], [ell], sigma_f, 32, 4)
    for which in (1, 2):                                   # two calls in a row, different right-hand sides
        v = torch.from_numpy(wl.vector(which=which)).cuda()
        Kp, dKp = op.matvec_all(v)
        Kn, dKn = noalloc(torch, native, X, ell, sigma_f, 32, 4, v)
        assert rel(Kn, Kp.cpu()) < TOL
        assert rel(dKn, dKp[0].cpu()) < TOL


def test_noalloc_matches_the_oracle_for_every_window_size(env):
    """d = 3, 1, 2 (in that order, so each call starts from a larger or different layout's leftovers)
    and bandwidths 32, 16, 20: each call against the oracle's CPU NFFT with the same settings."""
    torch, native = env
    wl = workloads.make("c3", N=15000)
    for d, M, cols, ell in [(3, 32, (0, 1, 2), 0.4), (1, 16, (13,), 0.25), (2, 20, (9, 10), 0.7),
                            (3, 16, (3, 4, 5), 0.9)]:
        pts = np.ascontiguousarray(wl.points[:, list(cols)])
        X = torch.from_numpy(pts).cuda()
        v = wl.vector()
        m = 4 if M >= 20 else 3
        Kn, dKn = noalloc(torch, native, X, ell, 1.1, M, m, torch.from_numpy(v).cuda())
        Kr, dKr = fastsum.matvec_all(pts, [tuple(range(d))], [ell], 1.1, v.astype(np.float64), M, m)
        assert close(Kn, Kr) and close(dKn, dKr[0]), (d, M)
        assert maxrow(Kn, Kr) < 10 * TOL and maxrow(dKn, dKr[0]) < 10 * TOL, (d, M)


def test_noalloc_reports_a_point_outside_the_ball(env):
    torch, native = env
    pts = np.zeros((64, 3), np.float32)
    pts[:, 0] = np.linspace(-0.2, 0.2, 64)
    pts[5] = [0.0, 0.3, 0.0]
    X = torch.from_numpy(pts).cuda()
    v = torch.ones(64, device="cuda")
    Kv, dK = torch.empty(64, device="cuda"), torch.empty(64, device="cuda")
    assert noalloc_status(torch, native, X, 0.5, 1.0, 32, 4, v, Kv, dK) == native.ADDKER_EDOMAIN
    pts[5] = [0.0, 0.1, 0.0]                 # the next call is unaffected by the failed one
    X = torch.from_numpy(pts).cuda()
    Kn, dKn = noalloc(torch, native, X, 0.5, 1.0, 32, 4, v)
    Kr, dKr = fastsum.matvec_all(pts, [(0, 1, 2)], [0.5], 1.0, np.ones(64), 32, 4)
    assert close(Kn, Kr) and close(dKn, dKr[0])


def test_noalloc_rejects_requests_beyond_its_limit(env):
    torch, native = env
    X = torch.zeros(10, 3, device="cuda")
    v = torch.zeros(10, device="cuda")
    out = torch.empty(10, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = native.lib().addker_fastsum_noalloc(p(X), 10, 3, 0.5, 1.0, 64, 4, p(v), p(out), None, None)
    assert st == native.ADDKER_ELIMIT
    assert b"fixed memory" in native.lib().addker_strerror(st)
