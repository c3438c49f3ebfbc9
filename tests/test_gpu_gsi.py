"""Global sensitivity indices on the GPU (addker_gsi) against the FP64 oracle (oracle/gsi.py, exact
trigonometric sums). The GPU's S(k, W_s) is the FP32 adjoint NFFT (relative L2 error ~1e-6 against the
exact sum, the stage test's 1e-5 bound), and theta is quadratic in S, so indices and the total variance
agree to 2e-5 relative."""
import numpy as np
import pytest

import workloads
from oracle import gsi

pytestmark = pytest.mark.gpu

TOL = 2e-5


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


@pytest.mark.parametrize("cfg,N", [("c3", 3000), ("c1", 4000)])
def test_gsi_matches_oracle(torch_cuda, cfg, N):
    torch = torch_cuda
    wl = workloads.make(cfg, N=N)
    v = wl.vector()
    op = make_op(torch, wl)
    rho, total = op.gsi(torch.from_numpy(v).cuda())
    rho_o, theta_o, total_o = gsi.gsi(wl.points, wl.windows, wl.ell, v, wl.bandwidth)
    assert set(rho) == set(rho_o) == set(gsi.subsets_of(wl.windows))
    assert abs(total - total_o) <= TOL * total_o
    for u, r in rho_o.items():
        assert abs(rho[u] - r) <= TOL * max(r, 1e-3), u
    vals = list(rho.values())
    assert all(a >= b for a, b in zip(vals, vals[1:])) and abs(sum(vals) - 1.0) < 1e-9


def test_gsi_shared_features(torch_cuda):
    torch = torch_cuda
    wl = workloads.tiny(N=800, d=4, windows=[(0, 1, 2), (1, 2, 3)], seed=22, ell=[0.35, 0.5])
    wl.bandwidth = [16, 16]
    wl.cutoff = 4
    v = wl.vector()
    op = make_op(torch, wl)
    rho, total = op.gsi(torch.from_numpy(v).cuda())
    rho_o, _, total_o = gsi.gsi(wl.points, wl.windows, wl.ell, v, wl.bandwidth)
    assert len(rho) == len(gsi.subsets_of(wl.windows)) == 11
    assert abs(total - total_o) <= TOL * total_o
    for u, r in rho_o.items():
        assert abs(rho[u] - r) <= TOL * max(r, 1e-3), u
    # the plan's products are unaffected by a GSI call (its grids are left cleared)
    Kv1, _ = op.matvec_all(torch.from_numpy(v).cuda())
    op2 = make_op(torch, wl)
    Kv2, _ = op2.matvec_all(torch.from_numpy(v).cuda())
    assert float(torch.linalg.norm(Kv1 - Kv2) / torch.linalg.norm(Kv2)) < 1e-5
