"""Several right-hand sides per launch: every stage of the product processes up to eight right-hand
sides in one launch per kernel kind (each with its own grid slot), larger batches in chunks. Results
must match the single-right-hand-side path column by column and the FP64 oracle, for every kernel kind
(3-D fast, 1-D/2-D fast, generic) and every product selector, across chunk boundaries and slot growth.

Tolerance: relative L2 1e-5 as for the single products (grid sums use atomics, so repeated products
agree to FP32 rounding, not bitwise)."""
import numpy as np
import pytest

import workloads
from oracle import fastsum
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


def make_op(torch, wl, **kw):
    from paper_2404_17344_gb300 import AddKer
    return AddKer(torch.from_numpy(wl.points).cuda(), wl.windows, wl.ell, wl.sigma_f, wl.bandwidth, wl.cutoff, **kw)


def columns_one_by_one(op, V):
    Ks, Ds = [], []
    for j in range(V.shape[1]):
        k, d = op.matvec_all(V[:, j].contiguous())
        Ks.append(k.cpu().numpy())
        Ds.append(d.cpu().numpy())
    return np.stack(Ks, 1), np.stack(Ds, 2)


@pytest.mark.parametrize("cfg,N,nrhs", [("c3", 3000, 11), ("c1", 6000, 8), ("c2", 4000, 3)])
def test_batched_matches_single_and_oracle(torch_cuda, cfg, N, nrhs):
    torch = torch_cuda
    wl = workloads.make(cfg, N=N)
    wl.sigma_f = 1.3
    V = torch.from_numpy(wl.vector(nrhs=nrhs)).cuda()
    op = make_op(torch, wl)
    Kv, dK = op.matvec_all(V)
    K1, D1 = columns_one_by_one(op, V)
    assert rel(Kv.cpu(), K1) < TOL
    assert rel(dK.cpu(), D1) < TOL
    for j in (0, nrhs - 1):                      # first chunk and last (possibly partial) chunk
        Kr, dKr = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f,
                                     V[:, j].cpu().numpy().astype(np.float64), wl.bandwidth, wl.cutoff)
        assert close(Kv[:, j].cpu(), Kr)
        for s in range(wl.P):
            assert close(dK[s, :, j].cpu(), dKr[s]), (j, s)


def test_batched_selectors_mixed_windows(torch_cuda):
    from paper_2404_17344_gb300 import ADDKER_ELL, ADDKER_ELL_SHARED, ADDKER_SIGMA_F
    torch = torch_cuda
    wl = workloads.make("c3", N=2500)
    wl.sigma_f = 0.8
    nrhs = 10
    V = torch.from_numpy(wl.vector(nrhs=nrhs)).cuda()
    op = make_op(torch, wl)
    Kv, dK = op.matvec_all(V)
    assert rel(op.matvec(V).cpu(), Kv.cpu()) < TOL
    for s in range(wl.P):
        assert rel(op.dmatvec(ADDKER_ELL(s), V).cpu(), dK[s].cpu()) < TOL, s
    assert rel(op.dmatvec(ADDKER_ELL_SHARED, V).cpu(), dK.sum(0).cpu()) < TOL
    assert rel(op.dmatvec(ADDKER_SIGMA_F, V).cpu(), (2.0 / wl.sigma_f) * Kv.cpu()) < TOL


def test_slot_growth_keeps_results(torch_cuda):
    """Slots grow 1 -> 4 -> 8 as batches grow; products before and after agree."""
    torch = torch_cuda
    wl = workloads.make("c3", N=2000)
    V = torch.from_numpy(wl.vector(nrhs=9)).cuda()
    op = make_op(torch, wl)
    k_first, d_first = op.matvec_all(V[:, 0].contiguous())
    K3, D3 = op.matvec_all(V[:, :3].contiguous())
    K9, D9 = op.matvec_all(V)
    k_last, d_last = op.matvec_all(V[:, 0].contiguous())
    assert rel(K3[:, 0].cpu(), k_first.cpu()) < TOL and rel(D3[:, :, 0].cpu(), d_first.cpu()) < TOL
    assert rel(K9[:, :3].cpu(), K3.cpu()) < TOL and rel(D9[:, :, :3].cpu(), D3.cpu()) < TOL
    assert rel(k_last.cpu(), k_first.cpu()) < TOL and rel(d_last.cpu(), d_first.cpu()) < TOL


def test_batched_generic_cutoff(torch_cuda):
    """m = 3: the generic kernels of every dimension, batched."""
    torch = torch_cuda
    wl = workloads.make("c3", N=1500)
    wl.cutoff = 3
    V = torch.from_numpy(wl.vector(nrhs=5)).cuda()
    op = make_op(torch, wl)
    Kv, dK = op.matvec_all(V)
    K1, D1 = columns_one_by_one(op, V)
    assert rel(Kv.cpu(), K1) < TOL and rel(dK.cpu(), D1) < TOL
    Kr, dKr = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, V[:, 4].cpu().numpy().astype(np.float64),
                                 wl.bandwidth, wl.cutoff)
    assert close(Kv[:, 4].cpu(), Kr) and close(dK[:, :, 4].cpu(), dKr)


def test_largest_small_transform(torch_cuda):
    """1-D and 2-D windows at the largest bandwidth (M = 64): the single-block transform with its
    largest shared-memory footprint."""
    torch = torch_cuda
    wl = workloads.tiny(N=3000, d=3, windows=[(0, 1), (2,)], ell=[0.3, 0.2])
    wl.bandwidth = [64, 64]
    wl.cutoff = 4
    V = torch.from_numpy(wl.vector(nrhs=2)).cuda()
    op = make_op(torch, wl)
    Kv, dK = op.matvec_all(V)
    for j in range(2):
        Kr, dKr = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f,
                                     V[:, j].cpu().numpy().astype(np.float64), wl.bandwidth, wl.cutoff)
        assert close(Kv[:, j].cpu(), Kr) and close(dK[:, :, j].cpu(), dKr)


def test_products_on_a_side_stream(torch_cuda):
    """addker_set_stream: the binding hands the library torch's current stream before every call. Products
    issued on a side stream (three in a row, so the repeated ones run as replayed graphs there) equal those
    of the default stream, and are complete once that stream is synchronised."""
    torch = torch_cuda
    wl = workloads.make("c3", N=2500)
    V = torch.from_numpy(wl.vector(nrhs=3)).cuda()
    op = make_op(torch, wl)
    K0, D0 = op.matvec_all(V)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        outs = [op.matvec_all(V) for _ in range(3)]
    side.synchronize()
    for k, d in outs:
        assert rel(k.cpu(), K0.cpu()) < TOL and rel(d.cpu(), D0.cpu()) < TOL


def test_host_entry_pageable_buffers(torch_cuda):
    """addker_matvec_all_host with ordinary (pageable) host memory and three right-hand sides: the copies go
    through cudaMemcpyAsync instead of the copy kernels of page-locked buffers; results as on device
    buffers and against the oracle."""
    torch = torch_cuda
    wl = workloads.make("c1", N=3000)
    nrhs = 3
    v = wl.vector(nrhs=nrhs)
    op = make_op(torch, wl)
    Kd, dKd = op.matvec_all(torch.from_numpy(v).cuda())
    vh = torch.from_numpy(np.ascontiguousarray(v.T)).reshape(-1)
    Kh = torch.empty(wl.N * nrhs)
    dKh = torch.empty(wl.N * wl.P * nrhs)
    assert not vh.is_pinned() and not Kh.is_pinned()
    op.matvec_all_host(vh, Kh, dKh, nrhs)
    assert rel(Kh.reshape(nrhs, wl.N).t(), Kd.cpu()) < TOL
    assert rel(dKh.reshape(nrhs, wl.P, wl.N).permute(1, 2, 0), dKd.cpu()) < TOL
    Kr, dKr = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v[:, 2].astype(np.float64),
                                 wl.bandwidth, wl.cutoff)
    assert close(Kh.reshape(nrhs, wl.N)[2], Kr)
    for s in range(wl.P):
        assert close(dKh.reshape(nrhs, wl.P, wl.N)[2, s], dKr[s]), s


def test_host_entry_batched(torch_cuda):
    torch = torch_cuda
    wl = workloads.make("c3", N=2000)
    nrhs = 9
    v = wl.vector(nrhs=nrhs)                     # (N, nrhs)
    op = make_op(torch, wl)
    Kd, dKd = op.matvec_all(torch.from_numpy(v).cuda())
    vh = torch.from_numpy(np.ascontiguousarray(v.T)).reshape(-1).pin_memory()
    Kh = torch.empty(wl.N * nrhs).pin_memory()
    dKh = torch.empty(wl.N * wl.P * nrhs).pin_memory()
    op.matvec_all_host(vh, Kh, dKh, nrhs)
    assert rel(Kh.reshape(nrhs, wl.N).t(), Kd.cpu()) < TOL
    assert rel(dKh.reshape(nrhs, wl.P, wl.N).permute(1, 2, 0), dKd.cpu()) < TOL


def test_graph_replay_matches_eager(torch_cuda):
    """Repeated identical products are captured and replayed as CUDA graphs; results match the eager
    path, and set_params / slot growth invalidate the captured graphs."""
    torch = torch_cuda
    wl = workloads.make("c3", N=2500)
    # (N, 3) view of column-major storage: the binding passes it without a copy, so the pointer repeats
    V = torch.from_numpy(np.ascontiguousarray(wl.vector(nrhs=3).T)).cuda().t()
    op = make_op(torch, wl)
    op.set_graphs(False)
    K0, D0 = op.matvec_all(V)
    op.set_graphs(True)
    Kv = torch.empty_like(K0.t().contiguous()).reshape(-1)
    dK = torch.empty(wl.P * wl.N * 3, device="cuda")
    outs = []
    for _ in range(4):                           # eager, capture, replay, replay
        Kv.zero_(); dK.zero_()
        k, d = op.matvec_all(V, out_Kv=Kv, out_dK=dK)
        outs.append((k.cpu(), d.cpu()))
    for k, d in outs:
        assert rel(k, K0.cpu()) < TOL and rel(d, D0.cpu()) < TOL
    info = op.info()
    assert info["graphs"] == 1 and info["graph_replays"] == 2 and info["slots"] == 4
    # new hyperparameters: the replay must use them
    op.set_params(ell=[e * 1.3 for e in wl.ell], sigma_f=1.7)
    for _ in range(3):
        k, d = op.matvec_all(V, out_Kv=Kv, out_dK=dK)
    op.set_graphs(False)
    k2, d2 = op.matvec_all(V)
    assert rel(k.cpu(), k2.cpu()) < TOL and rel(d.cpu(), d2.cpu()) < TOL
    # growing the slots (9 right-hand sides) discards graphs that point at the old grids
    op.set_graphs(True)
    V9 = torch.from_numpy(wl.vector(nrhs=9)).cuda()
    for _ in range(3):
        k9, _ = op.matvec_all(V9)
    for _ in range(3):
        k, d = op.matvec_all(V, out_Kv=Kv, out_dK=dK)
    assert rel(k.cpu(), k2.cpu()) < TOL and rel(d.cpu(), d2.cpu()) < TOL
    op.set_graphs(False)
    assert rel(op.matvec(V9).cpu(), k9.cpu()) < TOL


@pytest.mark.parametrize("cfg,N,nrhs", [("c3", 3000, 1), ("c1", 5000, 3)])
def test_autotune_keeps_results(torch_cuda, cfg, N, nrhs):
    """The autotuner re-cuts the work items for every candidate size; the product afterwards (and its
    graph replays) matches the product before, and the chosen size is one of the candidates."""
    torch = torch_cuda
    wl = workloads.make(cfg, N=N)
    V = torch.from_numpy(wl.vector(nrhs=nrhs) if nrhs > 1 else wl.vector()).cuda()
    op = make_op(torch, wl)
    K0, D0 = op.matvec_all(V)
    chosen, times = op.autotune(V)
    info = op.info()
    assert chosen in op.AUTOTUNE_CHUNKS and info["chunk"] == chosen
    assert info["chunk_spread"] in op.AUTOTUNE_CHUNKS
    assert all(t > 0 for t in times.values()) and all(t > 0 for t in op.autotune_spread_times.values())
    assert all(t > 0 for t in op.autotune_residency_times.values())
    assert info["spread_blocks_per_sm"] in (0, 1, 2, 3) and info["spread_tile"] in (0, 1)
    assert all(t > 0 for t in op.autotune_tile_times.values())
    # the spread phase's entry for the joint winner repeats the joint timing
    assert op.autotune_spread_times[chosen] == times[chosen]
    for _ in range(3):
        K1, D1 = op.matvec_all(V)
    assert rel(K1.cpu(), K0.cpu()) < TOL and rel(D1.cpu(), D0.cpu()) < TOL


def test_device_rates_are_plausible(torch_cuda):
    """addker_device_rates: every rate positive; the FP32 rates within the FMA pipe's bound
    (128 lanes per SM, 2 flops per FMA, at the measured clock; twice that for a packed
    FMA issued at full rate) up to timer noise."""
    from paper_2404_17344_gb300.rates import device_rates
    r = device_rates()
    assert r["sms"] > 0 and r["sm_mhz_under_load"] > 100
    bound = r["sms"] * 128 * 2 * r["sm_mhz_under_load"] * 1e6 / 1e12
    for k in ("ffma_tflops", "ffma2_tflops"):
        assert 0.2 * bound < r[k] < 2.2 * bound, (k, r[k], bound)
    assert r["shared_atomic_gops"] > 0 and r["global_atomic_gops"] > 0


@pytest.mark.parametrize("cfg,N", [("c1", 20000), ("c3", 20000)])
def test_every_schedule_matches_the_oracle(torch_cuda, cfg, N):
    """Both 3-D spread register tiles, reduced residency and other item sizes (addker_set_schedule) give the
    oracle's products: the schedule changes only the order of FP32 additions."""
    torch = torch_cuda
    wl = workloads.make(cfg, N=N)
    v = wl.vector()
    op = make_op(torch, wl)
    Kr, dKr = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v.astype(np.float64), wl.bandwidth,
                                 wl.cutoff)
    for chunk, chunk_sp, blocks, tile in [(256, 256, 0, 1), (128, 512, 2, 1), (512, 64, 1, 0), (256, 256, 0, 0)]:
        op.set_schedule(chunk, chunk_sp, blocks, tile)
        info = op.info()
        assert (info["chunk"], info["chunk_spread"], info["spread_blocks_per_sm"], info["spread_tile"]) == \
            (chunk, chunk_sp, blocks, tile)
        Kv, dK = op.matvec_all(torch.from_numpy(v).cuda())
        assert close(Kv.cpu(), Kr) and close(dK.cpu(), dKr), (chunk, chunk_sp, blocks, tile)
    from paper_2404_17344_gb300 import AddkerError
    with pytest.raises(AddkerError):
        op.set_schedule(256, 256, 0, 2)
