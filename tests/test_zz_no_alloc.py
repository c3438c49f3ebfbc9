"""addker_fastsum_noalloc against the plan path (addker_setup + addker_matvec_all).

The no-allocation entry point serves callers that cannot call cudaMalloc (code running during
stream capture, servers that fix their device memory at start-up, hosts whose allocator owns the
device memory). It takes all working memory from one fixed device array, so two calls in a row
must both agree with the plan path: the second call sees the first call's leftovers and must clear
what has to start at zero. This file is collected last so a stop-at-first-failure run has already
run every other test."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5          # the parity tolerance of the other GPU tests


def rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2404_17344_gb300 import native
    return torch, native


def noalloc(torch, native, X, ell, sigma_f, M, m, v):
    N, d = X.shape
    Kv = torch.empty(N, device="cuda")
    dK = torch.empty(N, device="cuda")
    st = native.lib().addker_fastsum_noalloc(
        ctypes.c_void_p(X.data_ptr()), N, d, float(ell), float(sigma_f), M, m, ctypes.c_void_p(v.data_ptr()),
        ctypes.c_void_p(Kv.data_ptr()), ctypes.c_void_p(dK.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
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


def test_noalloc_rejects_requests_beyond_its_limit(env):
    torch, native = env
    X = torch.zeros(10, 3, device="cuda")
    v = torch.zeros(10, device="cuda")
    out = torch.empty(10, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = native.lib().addker_fastsum_noalloc(p(X), 10, 3, 0.5, 1.0, 64, 4, p(v), p(out), None, None)
    assert st == native.ADDKER_ELIMIT
    assert b"fixed memory" in native.lib().addker_strerror(st)
