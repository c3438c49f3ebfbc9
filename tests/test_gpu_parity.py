"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative L2 over all outputs):
  - against the oracle's CPU NFFT fast sum with identical settings: 1e-5 (FP32 spreading, DFT and
    interpolation of sums of up to ~1e6 terms per grid value);
  - stage-wise: spread grid and adjoint NFFT 1e-5;
  - against the FP64 direct sum: the method's own Fourier error, measured on the same rows by the
    oracle's CPU NFFT, plus 1e-5.
"""
import numpy as np
import pytest

import workloads
from oracle import fastsum
from parity_metrics import close, maxrow, rel

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def make_op(torch, wl, **kw):
    from paper_2404_17344_gb300 import AddKer
    return AddKer(torch.from_numpy(wl.points).cuda(), wl.windows, wl.ell, wl.sigma_f, wl.bandwidth, wl.cutoff, **kw)


def oracle_all(wl, v, **kw):
    return fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, np.asarray(v, np.float64), wl.bandwidth,
                              wl.cutoff, **kw)


@pytest.mark.parametrize("cfg,N", [("c0", 2000), ("c1", 20000), ("c2", 5000)])
def test_matvec_all_vs_oracle_nfft(torch_cuda, cfg, N):
    torch = torch_cuda
    wl = workloads.make(cfg, N=N)
    v = wl.vector()
    op = make_op(torch, wl)
    Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
    Kr, dKr = oracle_all(wl, v)
    assert close(Kv.cpu(), Kr)
    for s in range(wl.P):
        assert close(dK[s].cpu(), dKr[s]), s


def test_stage_spread_and_adjoint(torch_cuda):
    torch = torch_cuda
    wl = workloads.make("c1", N=30000)
    v = wl.vector()
    op = make_op(torch, wl)
    vd = torch.from_numpy(v).cuda()
    from oracle import _clib, window
    v64 = v.astype(np.float64)
    for s, w in enumerate(wl.windows):
        x = np.ascontiguousarray(wl.points[:, list(w)].astype(np.float64))
        g = op.debug_stage(s, 0, vd)
        gref = np.zeros((64,) * 3)
        _clib.lib().orc_spread(len(x), 3, _clib.ptr(x), _clib.ptr(v64), 64, 4, window.shape(2.0), 0, _clib.ptr(gref))
        assert close(g, gref), s
        S = op.debug_stage(s, 1, vd)
        Sref = fastsum.nfft_adjoint(x, v64, 32, 64, 4)
        assert np.iscomplexobj(S) and rel(S, Sref) < TOL, s


def test_mixed_window_sizes_and_generic_kernels(torch_cuda):
    """Windows of 1, 2 and 3 features (generic kernels for d_s < 3) and bandwidths 16/32."""
    torch = torch_cuda
    wl = workloads.make("c3", N=20000)
    v = wl.vector()
    op = make_op(torch, wl)
    Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
    Kr, dKr = oracle_all(wl, v)
    assert close(Kv.cpu(), Kr)
    for s in range(wl.P):
        assert close(dK[s].cpu(), dKr[s]), s


@pytest.mark.parametrize("M", [12, 20, 64])
def test_bandwidths_not_multiple_of_8(torch_cuda, M):
    """Bandwidths whose M^2 is not a multiple of the 32-column tile of the x-axis transform."""
    torch = torch_cuda
    wl = workloads.make("c1", N=5000)
    wl.bandwidth = [M] * wl.P
    wl.cutoff = 3 if M < 20 else 4
    v = wl.vector()
    op = make_op(torch, wl)
    Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
    Kr, dKr = oracle_all(wl, v)
    assert close(Kv.cpu(), Kr) and close(dK.cpu(), dKr)


@pytest.mark.parametrize("m", [2, 3, 5])
def test_other_cutoffs(torch_cuda, m):
    torch = torch_cuda
    wl = workloads.make("c1", N=6000)
    wl.cutoff = m
    v = wl.vector()
    op = make_op(torch, wl)
    Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
    Kr, dKr = oracle_all(wl, v)
    assert close(Kv.cpu(), Kr) and close(dK.cpu(), dKr)


@pytest.mark.parametrize("p", [0, 1, 4])
def test_radial_regularisation_degrees(torch_cuda, p):
    torch = torch_cuda
    wl = workloads.make("c0", N=3000)
    v = wl.vector()
    op = make_op(torch, wl, p=p, reg="radial")
    Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
    Kr, dKr = oracle_all(wl, v, p=p, reg="radial")
    assert close(Kv.cpu(), Kr) and close(dK.cpu(), dKr)


@pytest.mark.parametrize("cfg,N", [("c1", 20000), ("c3", 20000)])
def test_separable_reading_against_the_direct_sums(torch_cuda, cfg, N):
    """The default reading end to end: the GPU products against the oracle's CPU NFFT with the same
    separable coefficients (1e-5), and against the FP64 direct sums on 1000 rows within the oracle's
    own Fourier error plus 1e-5 (windows of 1, 2 and 3 features, bandwidths 16 and 32)."""
    torch = torch_cuda
    wl = workloads.make(cfg, N=N)
    v = wl.vector()
    Kv, dK = make_op(torch, wl).matvec_all(torch.from_numpy(v).cuda())
    Kv, dK = Kv.cpu().numpy(), dK.cpu().numpy()
    Kr, dKr = oracle_all(wl, v)
    assert close(Kv, Kr) and all(close(dK[s], dKr[s]) for s in range(wl.P))
    rows = np.random.default_rng(3).choice(wl.N, 1000, replace=False)
    Kd, dKd = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v.astype(np.float64), rows=rows)
    assert rel(Kv[rows], Kd) < rel(Kr[rows], Kd) + TOL
    for s in range(wl.P):
        assert rel(dK[s, rows], dKd[s]) < rel(dKr[s, rows], dKd[s]) + TOL, s


def test_dmatvec_selectors_and_multi_rhs(torch_cuda):
    from paper_2404_17344_gb300 import ADDKER_ELL, ADDKER_ELL_SHARED, ADDKER_SIGMA_F
    torch = torch_cuda
    wl = workloads.make("c1", N=10000)
    wl.sigma_f = 1.7
    V = torch.from_numpy(wl.vector(nrhs=3)).cuda()
    op = make_op(torch, wl)
    Kv, dK = op.matvec_all(V)                    # (N, 3), (P, N, 3)
    # repeated products agree to FP32 rounding, not bitwise: grid sums use atomics in any order
    for j in range(3):
        k1, d1 = op.matvec_all(V[:, j].contiguous())
        assert rel(Kv[:, j].cpu(), k1.cpu()) < TOL
        assert rel(dK[:, :, j].cpu(), d1.cpu()) < TOL
    Kr, dKr = oracle_all(wl, V[:, 1].cpu().numpy())
    assert close(Kv[:, 1].cpu(), Kr) and close(dK[:, :, 1].cpu(), dKr)
    assert rel(op.matvec(V).cpu(), Kv.cpu()) < TOL
    for s in range(wl.P):
        assert rel(op.dmatvec(ADDKER_ELL(s), V).cpu(), dK[s].cpu()) < TOL
    assert rel(op.dmatvec(ADDKER_ELL_SHARED, V).cpu(), dK.sum(0).cpu()) < TOL
    assert rel(op.dmatvec(ADDKER_SIGMA_F, V).cpu(), (2.0 / wl.sigma_f) * Kv.cpu()) < TOL


def test_host_buffers_entry(torch_cuda):
    torch = torch_cuda
    wl = workloads.make("c1", N=8000)
    v = wl.vector()
    op = make_op(torch, wl)
    Kd, dKd = op.matvec_all(torch.from_numpy(v).cuda())
    vh = torch.from_numpy(v).pin_memory()
    Kh = torch.empty(wl.N).pin_memory()
    dKh = torch.empty(wl.N * wl.P).pin_memory()
    op.matvec_all_host(vh, Kh, dKh)
    assert rel(Kh, Kd.cpu()) < TOL and rel(dKh.reshape(wl.P, wl.N), dKd.cpu()) < TOL
    Kr, dKr = oracle_all(wl, v)
    assert close(Kh, Kr)
    for s in range(wl.P):
        assert close(dKh.reshape(wl.P, wl.N)[s], dKr[s]), s


@pytest.mark.slow
def test_host_buffers_entry_full_size_against_the_oracle(torch_cuda):
    """The host-buffer entry at one right-hand side and three windows (its own path: per-window gathers
    with each window's copy overlapped) at the benchmark's size, N = 1e6, against the oracle's CPU NFFT
    on 4096 sampled rows."""
    torch = torch_cuda
    wl = workloads.make("c1", N=1_000_000)
    v = wl.vector()
    op = make_op(torch, wl)
    vh = torch.from_numpy(v).pin_memory()
    Kh = torch.empty(wl.N).pin_memory()
    dKh = torch.empty(wl.N * wl.P).pin_memory()
    op.matvec_all_host(vh, Kh, dKh)
    op.matvec_all_host(vh, Kh, dKh)                   # the second call runs on the staging buffers the first made
    Kh, dKh = Kh.numpy(), dKh.numpy().reshape(wl.P, wl.N)
    rows = np.random.default_rng(11).choice(wl.N, 4096, replace=False)
    Kn, dKn = oracle_all(wl, v, rows=rows)
    assert close(Kh[rows], Kn)
    for s in range(wl.P):
        assert close(dKh[s, rows], dKn[s]), s


def test_set_params(torch_cuda):
    torch = torch_cuda
    wl = workloads.make("c1", N=6000)
    v = wl.vector()
    op = make_op(torch, wl)
    new_ell = np.array([0.45, 0.2, 0.8])
    op.set_params(ell=new_ell, sigma_f=0.7)
    Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
    wl.ell, wl.sigma_f = new_ell, 0.7
    Kr, dKr = oracle_all(wl, v)
    assert close(Kv.cpu(), Kr) and close(dK.cpu(), dKr)


def test_edge_cases(torch_cuda):
    """N = 1; all points in one cell; a point on the ball's edge; a single 1-D window."""
    torch = torch_cuda
    from paper_2404_17344_gb300 import AddKer
    one = workloads.tiny(N=1, d=3)
    one.bandwidth, one.cutoff = [32], 4
    op = make_op(torch, one)
    Kv, dK = op.matvec_all(torch.ones(1, device="cuda"))
    Kr, dKr = oracle_all(one, np.ones(1))
    assert close(Kv.cpu(), Kr) and abs(float(dK.cpu()[0, 0]) - dKr[0, 0]) < TOL * abs(Kr[0])
    rng = np.random.default_rng(4)
    pts = (0.001 + 0.01 / 64 * rng.uniform(0, 1, (700, 3))).astype(np.float32)     # one grid cell
    pts[0] = [0.21875 * 0.9999, 0.0, 0.0]                                             # and one on the edge
    wl = workloads.Workload("cell", pts, [(0, 1, 2)], np.array([0.3]), 1.0, [32], 4, 5)
    v = wl.vector()
    op = make_op(torch, wl)
    Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
    Kr, dKr = oracle_all(wl, v)
    assert close(Kv.cpu(), Kr) and close(dK.cpu(), dKr)
    spread = workloads.make("c0", N=700).points
    wl1 = workloads.Workload("1d", spread, [(2,)], np.array([0.2]), 1.0, [64], 4, 5)
    op = make_op(torch, wl1)
    Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
    Kr, dKr = oracle_all(wl1, v)
    assert close(Kv.cpu(), Kr) and close(dK.cpu(), dKr)


def test_points_on_grid_lines(torch_cuda):
    """Coordinates on the oversampled grid's lines (n x an integer: the window taken at the end of its
    polynomial pieces, the cell index exactly at a step of floor) and on cell centres, every third point
    repeated; a 3-D window (fast kernels) and a 1-D window (low-dimensional kernels) at M = 32, n = 64."""
    torch = torch_cuda
    rng = np.random.default_rng(11)
    k = rng.integers(-7, 8, size=(600, 4)).astype(np.float64)
    half = 0.5 * rng.integers(0, 2, size=(600, 4))
    X = ((k + half) / 64.0).astype(np.float32)
    X = np.concatenate([X, X[::3]])
    wl = workloads.Workload("lines", X, [(0, 1, 2), (3,)], np.array([0.3, 0.5]), 1.0, [32, 32], 4, 5)
    v = wl.vector()
    op = make_op(torch, wl)
    Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
    Kr, dKr = oracle_all(wl, v)
    assert close(Kv.cpu(), Kr)
    for s in range(wl.P):
        assert close(dK[s].cpu(), dKr[s]), s


def test_rejects_point_outside_ball(torch_cuda):
    torch = torch_cuda
    from paper_2404_17344_gb300 import AddKer, AddkerError
    pts = np.zeros((100, 3), np.float32)
    pts[7] = [0.3, 0.0, 0.0]
    with pytest.raises(AddkerError) as e:
        AddKer(torch.from_numpy(pts).cuda(), [(0, 1, 2)], [0.5])
    assert e.value.status == -2
    pts[7] = [np.nan, 0, 0]
    with pytest.raises(AddkerError):
        AddKer(torch.from_numpy(pts).cuda(), [(0, 1, 2)], [0.5])


def test_prescale_matches_recipe(torch_cuda):
    torch = torch_cuda
    from paper_2404_17344_gb300 import prescale
    rng = np.random.default_rng(8)
    X = rng.standard_normal((5000, 6)).astype(np.float32)
    wins = [(0, 1, 2), (3, 4)]
    Xs, f = prescale(torch.from_numpy(X).cuda(), wins)
    mx = max(np.sqrt((X[:, list(w)].astype(np.float64) ** 2).sum(1)).max() for w in wins)
    assert f == pytest.approx((0.25 - 1 / 32) * (1 - 4e-7) / mx, rel=1e-6)
    np.testing.assert_allclose(Xs.cpu().numpy(), X * np.float32(f), rtol=1e-6)


def test_prescale_cube_matches_paper_rule(torch_cuda):
    """Sec. 3.2 as stated: each feature mapped from its range onto [-r, r], then divided by sqrt(d_max);
    every windowed point inside the ball of radius r = 1/4 - eps_B/2; a constant feature maps to 0."""
    torch = torch_cuda
    from paper_2404_17344_gb300 import prescale
    rng = np.random.default_rng(9)
    X = (rng.standard_normal((4000, 7)) * rng.uniform(0.1, 5.0, 7) + rng.uniform(-3, 3, 7)).astype(np.float32)
    X[:, 5] = 2.5                                               # constant feature
    wins = [(0, 1, 2), (3, 4), (5, 6)]
    Xs, f = prescale(torch.from_numpy(X).cuda(), wins, rule="cube")
    Xs = Xs.cpu().numpy().astype(np.float64)
    r = (0.25 - 1 / 32) * (1 - 4e-7)
    X64 = X.astype(np.float64)
    lo, hi = X64.min(0), X64.max(0)
    span = np.where(hi > lo, hi - lo, 1.0)
    ref = np.where(hi > lo, (2 * (X64 - lo) / span - 1) * r, 0.0) / np.sqrt(3)
    np.testing.assert_allclose(Xs, ref, atol=1e-6 * r)
    assert f == pytest.approx(4 * r / np.sqrt(3), rel=1e-12)
    assert max(np.sqrt((Xs[:, list(w)] ** 2).sum(1)).max() for w in wins) <= 0.25 - 1 / 32
    Xn = X.copy()
    Xn[3, 2] = np.inf
    with pytest.raises(Exception):
        prescale(torch.from_numpy(Xn).cuda(), wins, rule="cube")


@pytest.mark.slow
def test_full_size_mixed_windows_sampled_rows(torch_cuda):
    """N = 1e6, 15 features in windows of 3, 3, 3, 2, 2, 1, 1 (M = 32 / 16): every kernel kind at the
    batched configuration's size, in one product, on 1024 sampled rows against the CPU NFFT (measured
    at most 1.7e-6)."""
    torch = torch_cuda
    wl = workloads.make("c3", N=1_000_000)
    v = wl.vector()
    Kv, dK = make_op(torch, wl).matvec_all(torch.from_numpy(v).cuda())
    Kv, dK = Kv.cpu().numpy(), dK.cpu().numpy()
    rows = np.random.default_rng(1).choice(wl.N, 1024, replace=False)
    Kn, dKn = oracle_all(wl, v, rows=rows)
    assert close(Kv[rows], Kn)
    for s in range(wl.P):
        assert close(dK[s, rows], dKn[s]), s


@pytest.mark.slow
def test_full_size_batched_sampled_rows(torch_cuda):
    """The batched benchmark's launch at its full size: N = 1e6, windows of 3, 3, 3, 2, 2, 1, 1, eight
    right-hand sides in one product (one chunk: every kernel launched once for all of them) with the work
    items of 512 points the autotuner picks there, the right-hand sides in a column-major view as the
    benchmark passes them. Right-hand sides 0 and 7 on 1024 sampled rows against the CPU NFFT."""
    torch = torch_cuda
    wl = workloads.make("c3", N=1_000_000)
    V = wl.vector(nrhs=8)
    op = make_op(torch, wl)
    op.set_schedule(512, 512)
    Vd = torch.from_numpy(np.ascontiguousarray(V.T)).cuda().t()
    Kv, dK = op.matvec_all(Vd)
    Kv, dK = Kv.cpu().numpy(), dK.cpu().numpy()
    rows = np.random.default_rng(3).choice(wl.N, 1024, replace=False)
    for j in (0, 7):
        Kn, dKn = oracle_all(wl, V[:, j], rows=rows)
        assert close(Kv[rows, j], Kn), j
        for s in range(wl.P):
            assert close(dK[s, rows, j], dKn[s]), (j, s)


@pytest.mark.slow
def test_gp_configuration_size_sampled_rows(torch_cuda):
    """The GP configuration's operator at its full size (N = 2e6, 24 correlated features, 8 windows of 3):
    the fused product on 512 sampled rows against the CPU NFFT (all 2e6 points spread in FP64)."""
    torch = torch_cuda
    wl = workloads.make("c4", N=2_000_000)
    v = wl.vector()
    Kv, dK = make_op(torch, wl).matvec_all(torch.from_numpy(v).cuda())
    Kv, dK = Kv.cpu().numpy(), dK.cpu().numpy()
    rows = np.random.default_rng(2).choice(wl.N, 512, replace=False)
    Kn, dKn = oracle_all(wl, v, rows=rows)
    assert close(Kv[rows], Kn)
    for s in range(wl.P):
        assert close(dK[s, rows], dKn[s]), s


@pytest.mark.slow
def test_full_size_sampled_rows(torch_cuda):
    """N = 1e6, d = 9, three windows of 3 (the benchmark workload): GPU outputs on 1500 sampled rows
    against the CPU NFFT (all 1e6 points spread in FP64) and against the direct FP64 sums, for the plain
    FP32 path (the one the benchmark times) and the compensated one, both at the 1e-5 bar.

    The wide windows (ell = 0.5, 1.0) have their quadratic part split off: as a trigonometric polynomial
    it carries a constant term 18 and 24 times the derivative product, which multiplied every FP32 rounding
    of the transforms (plain path before the split: up to 1.1e-5 over 24 runs at ell = 1.0)."""
    torch = torch_cuda
    wl = workloads.make("c1", N=1_000_000)
    v = wl.vector()
    rows = np.random.default_rng(0).choice(wl.N, 1500, replace=False)
    Kn, dKn = oracle_all(wl, v, rows=rows)
    for comp in (False, True):
        op = make_op(torch, wl, compensated=comp)
        Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
        Kv, dK = Kv.cpu().numpy(), dK.cpu().numpy()
        assert close(Kv[rows], Kn), comp
        for s in range(wl.P):
            assert close(dK[s, rows], dKn[s]), (comp, s)
        op.close()
    Kd, dKd = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v.astype(np.float64), rows=rows[:300])
    assert rel(Kv[rows[:300]], Kd) < rel(Kn[:300], Kd) + TOL
    for s in range(wl.P):
        assert rel(dK[s, rows[:300]], dKd[s]) < rel(dKn[s, :300], dKd[s]) + TOL
        assert rel(dK[s, rows[:300]], dKd[s]) < 1e-4
