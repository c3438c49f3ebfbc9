"""Benchmark: fused additive-kernel products K v + dK/d ell_s v (all s) per second on GB300.

One step = one fused product (addker_matvec_all) on the workload: N = 1e6 points, d = 9, three windows
of 3 consecutive features, ell = (0.3, 0.5, 1.0), sigma_f = 1, bandwidth M = 32, oversampling 2,
cutoff m = 4 (N(0,1) features scaled into the ball of radius 1/4 - eps_B/2; synthetic, seeded).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--N 1000000]
  python bench.py --mode batched [--nrhs 64]        (secondary: 7 mixed windows, 64 right-hand sides)
  python bench.py --mode gp [--nrhs 17 --beta 0.01 --tol 1e-6 --maxit 100]   (secondary: GP gradient, N = 2e6)
  python bench.py --mode grad                       (secondary: vector-Jacobian product, N = 2e5)

--gpus N > 1 runs under torchrun, one rank per GPU: independent replicas (the product needs no
exchange between GPUs at this size), weak scaling; value = all ranks' units / max-over-ranks time.
--impl reference times the FP64 CPU oracle (the plain NFFT fast sum) on the host cores instead.
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "additive K·v + dK/d(ell)·v per sec, N=1M, 3x3 windows, err<=1e-4 vs FP64"
UNIT = "units/s"   # one unit = K v plus dK/d ell_s v for every window s (dK/d sigma_f v = (2/sigma_f) K v is free)
SMS = 152
FP32_LANES_PER_SM = 128


def workload_desc(N):
    return {"workload": f"c1-shaped at N={N}: d=9, windows (0,1,2),(3,4,5),(6,7,8), ell=(0.3,0.5,1.0), "
                        "sigma_f=1, M=32, sigma=2, m=4, eps_B=1/16, separable regularisation (tensor-product "
                        "least-squares Fourier extension per axis), N(0,1) features scaled into the ball",
            "N": N, "d": 9, "P": 3, "bandwidth": 32, "cutoff": 4, "nrhs": 1,
            "l2": "flushed between timed steps (write of a 512 MB buffer)"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.file.flush()
        rows = []
        try:
            with open(self.file.name) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except Exception:
            pass
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def aggregate(total_ms, e2e_sec, steps, world, dist=None, device="cpu"):
    """Replicas: every rank ran `steps` products of its own copy of the workload. The job's time is
    the slowest rank's; value = units of all ranks / that time. Returns (ms_per_step, value, e2e_value)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([float(total_ms), float(e2e_sec)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, e2e_sec = float(t[0]), float(t[1])
    return total_ms / steps, world * steps / (total_ms / 1e3), world / e2e_sec


def cpu_oracle_prepare(wl, v):
    """The oracle's N-independent work, done once before any timed step, as the GPU does it in its
    untimed setup: the Fourier coefficients of every window, the window transforms (cached inside the
    oracle) and loading its C library (one product on 2000 points)."""
    import numpy as np
    import oracle
    X = wl.points.astype(np.float64)
    coefs = [oracle.fastsum.coefficients_for(np.ascontiguousarray(X[:, list(w)]), float(wl.ell[s]),
                                             int(wl.bandwidth[s])) for s, w in enumerate(wl.windows)]
    oracle.fastsum.matvec_all(wl.points[:2000], wl.windows, wl.ell, wl.sigma_f, v[:2000], wl.bandwidth, wl.cutoff,
                              coefs=coefs)
    return coefs


def cpu_oracle_step(wl, v, coefs):
    """One oracle fused product (K v and every dK/d ell_s v) on the whole workload; returns seconds."""
    import oracle
    t0 = time.perf_counter()
    oracle.fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v, wl.bandwidth, wl.cutoff, coefs=coefs)
    return time.perf_counter() - t0


def cpu_threads(n=None):
    """Set (n > 0) and return the oracle's OpenMP thread count."""
    from oracle import _clib
    if n:
        _clib.lib().orc_set_threads(int(n))
    return int(_clib.lib().orc_num_threads())


def cpu_cores():
    return cpu_threads()


CPU_SAMPLE = ("the whole workload: all N points, all 3 windows, one fused product per step; the coefficients and "
              "window transforms are computed once before the timed steps, as the GPU's untimed setup does")


def run_reference(args, rank, world):
    """The FP64 CPU oracle on the host cores: each step is the oracle's fused product on the whole
    workload (every point, every window), after the same untimed setup the GPU plan does."""
    if rank != 0:
        return
    import workloads
    wl = workloads.make("c1", N=args.N)
    v = wl.vector()
    cores = cpu_threads(os.cpu_count())
    coefs = cpu_oracle_prepare(wl, v)
    for _ in range(args.warmup):
        cpu_oracle_step(wl, v, coefs)
    ts = [cpu_oracle_step(wl, v, coefs) for _ in range(args.steps)]
    sec = sum(ts) / len(ts)
    val = 1.0 / sec
    out = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_desc(args.N),
           "impl": "reference",
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": CPU_SAMPLE},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import __graft_entry__
    import workloads
    __graft_entry__.build()
    from paper_2404_17344_gb300 import AddKer

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl", device_id=dev)
        dist = dist_mod

    wl = workloads.make("c1", N=args.N)
    v_np = wl.vector()
    pts = torch.from_numpy(wl.points).to(dev)
    v = torch.from_numpy(v_np).to(dev)
    t0 = time.perf_counter()
    op = AddKer(pts, wl.windows, wl.ell, wl.sigma_f, wl.bandwidth, wl.cutoff)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    N, P = wl.N, wl.P
    Kv = torch.empty(N, device=dev)
    dK = torch.empty(P * N, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, device=dev)

    for _ in range(args.warmup):
        op.matvec_all(v, Kv, dK)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local_rank)
    with ClockSampler(gpu_id) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            op.matvec_all(v, Kv, dK)
            ends[i].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)

    # per-kernel durations: the same K steps again with stage events on the plan's stream (kept out of
    # the timed region above, where the extra events would cost time and break launch overlap)
    op.profile(True)
    for i in range(args.steps):
        flush.zero_()
        op.matvec_all(v, Kv, dK)
    torch.cuda.synchronize()
    stage = op.profile_read()
    op.profile(False)

    # end to end through the host-buffer entry point: pinned host v in, Kv and dK out, copies timed
    vh = torch.from_numpy(v_np).pin_memory()
    Kh = torch.empty(N).pin_memory()
    dKh = torch.empty(N * P).pin_memory()
    for _ in range(2):
        op.matvec_all_host(vh, Kh, dKh)
    e2e_ts = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op.matvec_all_host(vh, Kh, dKh)
        e2e_ts.append(time.perf_counter() - t0)
    e2e_sec = sum(e2e_ts) / len(e2e_ts)
    ms_per_step, value, e2e_value = aggregate(total_ms, e2e_sec, args.steps, world, dist, dev)

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (spread or gather): FP32 FMA pipe, algorithmic flops per launch
    pk, pk_kind = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12          # TFLOP/s
    W3 = (2 * wl.cutoff) ** 3
    flops = {"spread": 2.0 * W3 * N * P, "gather": 2.0 * 2 * W3 * N * P}     # per launch (all windows)
    dom = max(("spread", "gather"), key=lambda k: stage[k][0])
    dom_ms, dom_launches = stage[dom]
    per_launch_s = dom_ms / 1e3 / max(1, dom_launches)
    achieved = flops[dom] / per_launch_s / 1e12
    traffic = None                       # from the last ncu capture, only while the kernel source is unchanged
    tfile = os.path.join(ROOT, "profiles", f"{dom}_traffic.json")
    if os.path.exists(tfile):
        try:
            import hashlib
            rec = json.load(open(tfile))
            srcs = rec.get("sources") or {rec["source"]: rec["source_sha256"]}
            if all(hashlib.sha256(open(os.path.join(ROOT, f), "rb").read()).hexdigest() == h
                   for f, h in srcs.items()):
                traffic = rec["bytes_per_launch"]
        except Exception:
            traffic = None
    # algorithmic HBM bytes per unit: coordinates read twice (36 B each), v (4 B), outputs 4(1+P) B per point
    hbm_bytes = N * (2 * 4 * wl.d + 4 + 4 * (1 + P))
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))

    # measured FP32 and atomic rates of this device (after the timed region)
    from paper_2404_17344_gb300.rates import device_rates
    rates = device_rates()

    # the spread's grid flush against the measured L2 atomic rate: one atomic add per box value (W^3) per
    # work item (every window here is 3-D with m = 4)
    sp_ms, sp_launches = stage["spread"]
    atomics = op.info()["items"] * W3
    sp_s = sp_ms / 1e3 / max(1, sp_launches)
    atomics_line = {"kernel": "spread", "atomic_adds_per_launch": atomics,
                    "achieved_gops": atomics / sp_s / 1e9, "peak_gops": rates["global_atomic_gops"],
                    "frac": atomics / sp_s / 1e9 / rates["global_atomic_gops"],
                    "note": "grid flush: one float atomic add per box value per work item; peak = measured "
                            "rate into an L2-resident grid (device_rates)"}

    # CPU oracle baseline on the whole workload: median of 3 products on all host cores, 1 on one core
    cores = cpu_threads(os.cpu_count())
    coefs = cpu_oracle_prepare(wl, v_np)
    cpu_sec = statistics.median(cpu_oracle_step(wl, v_np, coefs) for _ in range(args.cpu_reps))
    cpu_threads(1)
    cpu_sec_1 = cpu_oracle_step(wl, v_np, coefs)
    cpu_threads(cores)

    # accuracy on sampled rows against the FP64 CPU NFFT (same settings) and the FP64 direct sum
    acc = gate = None
    if not args.no_check:
        import oracle
        rows = np.random.default_rng(0).choice(N, args.check_rows, replace=False)
        Kn, dKn = oracle.fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v_np.astype(np.float64),
                                            wl.bandwidth, wl.cutoff, rows=rows)
        Kd, dKd = oracle.fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v_np.astype(np.float64),
                                        rows=rows)
        Kg = Kv.cpu().numpy()[rows]
        dg = dK.reshape(P, N).cpu().numpy()[:, rows]
        r = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        mr = lambda a, b: float(np.abs(a - b).max() / (np.linalg.norm(b) / np.sqrt(b.size)))
        acc = {"rows": int(args.check_rows),
               "Kv_vs_fp64_nfft": r(Kg, Kn), "dK_vs_fp64_nfft": [r(dg[s], dKn[s]) for s in range(P)],
               "Kv_vs_fp64_direct": r(Kg, Kd), "dK_vs_fp64_direct": [r(dg[s], dKd[s]) for s in range(P)],
               "oracle_nfft_Kv_vs_direct": r(Kn, Kd),
               "oracle_nfft_dK_vs_direct": [r(dKn[s], dKd[s]) for s in range(P)],
               "max_row_vs_fp64_nfft": {"Kv": mr(Kg, Kn), "dK": [mr(dg[s], dKn[s]) for s in range(P)],
                                        "note": "largest row error / RMS of the reference"}}
        nb, db = 1e-5, 1e-4
        gate = {"vs_fp64_nfft": {"bar": nb, "Kv": acc["Kv_vs_fp64_nfft"] <= nb,
                                 "dK": [e <= nb for e in acc["dK_vs_fp64_nfft"]]},
                "vs_fp64_direct": {"bar": db, "Kv": acc["Kv_vs_fp64_direct"] <= db,
                                   "dK": [e <= db for e in acc["dK_vs_fp64_direct"]]},
                "metric": "relative L2 on the sampled rows"}
        gate["pass"] = bool(gate["vs_fp64_nfft"]["Kv"] and all(gate["vs_fp64_nfft"]["dK"]) and
                            gate["vs_fp64_direct"]["Kv"] and all(gate["vs_fp64_direct"]["dK"]))
    else:
        gate = None

    launches = int(sum(c for _, c in stage.values()))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_desc(N),
           "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                        "frac": achieved / fp32_peak, "traffic": traffic,
                        "timing": "CUDA events around the kernel's stage on the plan's stream, over K steps run "
                                  "right after the timed region (same inputs, L2 flushed between steps)",
                        "peak_source": f"FP32 FMA pipe: {SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_max:.0f} MHz "
                                       f"(sm_max_mhz {pk_kind})",
                        "peak_measured": rates["ffma2_tflops"],
                        "frac_of_measured": achieved / rates["ffma2_tflops"] if rates["ffma2_tflops"] > 0 else None,
                        "peak_measured_source": "packed FFMA2 microbenchmark (addker_device_rates) at "
                                                f"{rates['sm_mhz_under_load']:.0f} MHz, after the timed region"},
           "roofline_atomics": atomics_line,
           "roofline_hbm": {"achieved": hbm_bytes / (ms_per_step / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                            "frac": hbm_bytes / (ms_per_step / 1e3) / 1e9 / hbm_peak,
                            "note": f"algorithmic bytes of the whole step, {pk_kind} copy bandwidth"},
           "stage_ms_per_step": {k: t / args.steps for k, (t, _) in stage.items()},
           "cpu_baseline": {"value": 1.0 / cpu_sec, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": CPU_SAMPLE + f"; median of {args.cpu_reps} products",
                            "one_core": {"value": 1.0 / cpu_sec_1, "unit": UNIT, "cores": 1}},
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * N,
                   "d2h_bytes_per_step": 4 * N * (1 + P)},
           "gpu_launches": launches * 1,
           "gpu_launches_per_step": launches / args.steps,
           "device_rates": rates,
           "clocks": clk.summary(), "setup_ms": setup_ms, "wall_s_timed": wall,
           "accuracy": acc, "gate": gate}
    print(json.dumps(out), flush=True)
    op.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def _setup_secondary(args, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local_rank)
    return torch, dev, gpu_id


def run_batched(args, rank, world, local_rank):
    """Secondary workload (multi-RHS batching): the mixed-window configuration (N = 1e6, d = 15, windows of
    3,3,3,2,2,1,1, M = 32 for 3-D and 16 for 1-D/2-D windows) with 64 right-hand sides per step; one unit
    = K v + all dK/d ell_s v for one right-hand side. The work-item size is autotuned first."""
    import numpy as np
    torch, dev, gpu_id = _setup_secondary(args, local_rank)
    import workloads
    from paper_2404_17344_gb300 import AddKer
    N = args.N if args.N != 1_000_000 else 1_000_000
    R = args.nrhs
    wl = workloads.make("c3", N=N)
    op = AddKer(torch.from_numpy(wl.points).to(dev), wl.windows, wl.ell, wl.sigma_f, wl.bandwidth, wl.cutoff)
    Vnp = wl.vector(nrhs=R)
    V = torch.from_numpy(np.ascontiguousarray(Vnp.T)).to(dev).t()          # column-major (N, R) view
    chunk, tune_ms = op.autotune(V[:, :8])
    Kv = torch.empty(N * R, device=dev)
    dK = torch.empty(N * wl.P * R, device=dev)
    for _ in range(args.warmup):
        op.matvec_all(V, out_Kv=Kv, out_dK=dK)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(gpu_id) as clk:
        for a, b in ev:
            a.record()
            op.matvec_all(V, out_Kv=Kv, out_dK=dK)
            b.record()
        torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    # the same product one right-hand side at a time, for the per-solve comparison
    v1 = V[:, 0].contiguous()
    K1 = torch.empty(N, device=dev)
    D1 = torch.empty(N * wl.P, device=dev)
    for _ in range(3):
        op.matvec_all(v1, out_Kv=K1, out_dK=D1)
    torch.cuda.synchronize()
    a1, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a1.record()
    for _ in range(10):
        op.matvec_all(v1, out_Kv=K1, out_dK=D1)
    b1.record()
    torch.cuda.synchronize()
    single_ms = a1.elapsed_time(b1) / 10
    # accuracy: right-hand sides 0 and R-1 on 256 sampled rows against the FP64 CPU NFFT
    import oracle
    rows = np.random.default_rng(0).choice(N, 256, replace=False)
    acc = {}
    Kh = Kv.reshape(R, N).cpu().numpy()
    for j in (0, R - 1):
        Kn, _ = oracle.fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, Vnp[:, j].astype(np.float64),
                                          wl.bandwidth, wl.cutoff, rows=rows)
        acc[f"Kv_rhs{j}_vs_fp64_nfft"] = float(np.linalg.norm(Kh[j][rows] - Kn) / np.linalg.norm(Kn))
    out = {"metric": "batched additive K·V + dK/d(ell)·V, right-hand-side units per sec, N=1M, 7 mixed windows",
           "value": R / (ms / 1e3), "unit": "units/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": f"c3-shaped at N={N}: d=15, windows 3,3,3,2,2,1,1, ell log-U[0.1,2], M=32/16, "
                                  f"m=4, U[-1,1] features scaled into the ball, {R} right-hand sides per step",
                      "N": N, "nrhs": R, "chunk": chunk, "chunk_spread": op.info()["chunk_spread"],
                      "autotune_ms": tune_ms, "autotune_spread_ms": op.autotune_spread_times,
                      "spread_blocks_per_sm": op.info()["spread_blocks_per_sm"],
                      "spread_tile": op.info()["spread_tile"],
                      "autotune_tile_ms": {str(k): v for k, v in op.autotune_tile_times.items()},
                      "autotune_residency_ms": {str(k): v for k, v in op.autotune_residency_times.items()}},
           "per_rhs_ms": ms / R, "single_rhs_ms": single_ms, "speedup_per_solve_vs_single": single_ms / (ms / R),
           "clocks": clk.summary(), "accuracy": acc, "plan": {k: v for k, v in op.info().items() if k != "windows"}}
    print(json.dumps(out), flush=True)
    op.close()


def run_gp(args, rank, world, local_rank):
    """Secondary workload (GP training): the correlated-Gaussian configuration (N = 2e6, d = 24, eight
    windows of 3, ell = 0.5, M = 32) with targets y = a 16-term random-Fourier-feature function per window
    plus N(0, 0.01) noise; one step = one gradient of the GP log marginal likelihood in
    (ell_1..ell_8, sigma_f, beta): CG on (K + beta I) with 1 + 16 right-hand sides
    [y, z_1..z_16] (Rademacher probes, Hutchinson) to relative residual 1e-6, or at most --maxit
    iterations, preconditioned with every window's lowest Fourier modes (--precond band; 0 = plain CG),
    then one fused product on [alpha, z_1..z_16]. At the configuration's beta = 0.01 the FP32 operator's
    error (~1e-7 ||K||, ||K|| ~ 1.6e7) is far above beta, so the solve stalls at a relative residual of a
    few 1e-2 whatever the iteration count; the line reports the residual reached, measured with one more
    product."""
    import numpy as np
    torch, dev, gpu_id = _setup_secondary(args, local_rank)
    import workloads
    from paper_2404_17344_gb300 import AddKer
    N = args.N if args.N != 1_000_000 else 2_000_000
    m = args.nrhs - 1
    wl = workloads.make("c4", N=N)
    op = AddKer(torch.from_numpy(wl.points).to(dev), wl.windows, wl.ell, wl.sigma_f, wl.bandwidth, wl.cutoff)
    op.set_precond(args.precond)
    y = torch.from_numpy(wl.targets()).to(dev)
    Z = torch.from_numpy(wl.probes(m)).to(dev)
    beta, tol = args.beta, args.tol
    for _ in range(max(1, args.warmup // 3)):
        g, fit, alpha, iters = op.gp_grad(y, beta, Z, tol=tol, maxit=args.maxit)
    torch.cuda.synchronize()
    ts, its = [], []
    with ClockSampler(gpu_id) as clk:
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g, fit, alpha, iters = op.gp_grad(y, beta, Z, tol=tol, maxit=args.maxit)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
            its.append(iters)
    ms = statistics.mean(ts)
    # relative residual of alpha, by one more product
    Ka = op.matvec(alpha)
    relres = float(torch.linalg.norm(y - Ka - beta * alpha) / torch.linalg.norm(y))
    out = {"metric": "GP log-marginal-likelihood gradients per sec (Hutchinson, CG), N=2M, 8 windows of 3",
           "value": 1e3 / ms, "unit": "gradients/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": f"c4-shaped at N={N}: d=24, correlated Gaussian features, 8 windows of 3, ell=0.5, "
                                  "M=32, m=4; y = 16-term random Fourier features per window + N(0, 0.01) noise",
                      "N": N, "probes": m, "beta": beta, "cg_tol": tol, "cg_maxit": args.maxit, "cg_iters": its,
                      "precond_band": args.precond, "alpha_relres": relres,
                      "ms_per_cg_iteration": ms / max(1, statistics.mean(its))},
           "grad": list(map(float, g)), "fit": fit, "clocks": clk.summary()}
    print(json.dumps(out), flush=True)
    op.close()


def run_grad(args, rank, world, local_rank):
    """Secondary workload (differentiation): the mixture-of-Gaussians configuration (N = 2e5, d = 12, four
    windows of 3, ell = 0.3, 0.5, 0.7, 1.0, M = 32, m = 4); one step = one vector-Jacobian product of
    f = w^T K v (addker_vjp): the gradients with respect to v, every ell_s, sigma_f and the N x 12 point
    coordinates. Accuracy: the parameter gradients against the oracle's FP64 NFFT gradients."""
    import numpy as np
    torch, dev, gpu_id = _setup_secondary(args, local_rank)
    import workloads
    from paper_2404_17344_gb300 import AddKer
    N = args.N if args.N != 1_000_000 else 200_000
    wl = workloads.make("c2", N=N)
    op = AddKer(torch.from_numpy(wl.points).to(dev), wl.windows, wl.ell, wl.sigma_f, wl.bandwidth, wl.cutoff)
    v_np, w_np = wl.vector(), wl.vector(which=2)
    v, w = torch.from_numpy(v_np).to(dev), torch.from_numpy(w_np).to(dev)
    for _ in range(args.warmup):
        op.vjp(v, w)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(gpu_id) as clk:
        for a, b in ev:
            a.record()
            gv, gt, gx = op.vjp(v, w)
            b.record()
        torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    # one fused product for comparison (K v and every dK/d ell_s v)
    for _ in range(3):
        op.matvec_all(v)
    torch.cuda.synchronize()
    a1, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a1.record()
    for _ in range(10):
        op.matvec_all(v)
    b1.record()
    torch.cuda.synchronize()
    fused_ms = a1.elapsed_time(b1) / 10
    import oracle
    rv, rell, rsf, rx = oracle.gradients.nfft_grad(wl.points, wl.windows, wl.ell, wl.sigma_f, v_np, w_np,
                                                   wl.bandwidth, wl.cutoff)
    gt = gt.cpu().numpy()
    r = lambda a, b: float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))
    out = {"metric": "vector-Jacobian products of w^T K v per sec (grad v, ell, sigma_f, points), N=200k, 4 windows of 3",
           "value": 1e3 / ms, "unit": "gradients/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": f"c2-shaped at N={N}: d=12, mixture of 4 Gaussians, 4 windows of 3, "
                                  "ell=(0.3,0.5,0.7,1.0), M=32, m=4", "N": N},
           "fused_product_ms": fused_ms, "vjp_over_product": ms / fused_ms,
           "accuracy": {"grad_v_vs_fp64_nfft": r(gv.cpu().numpy(), rv), "grad_ell_vs_fp64_nfft": r(gt[:wl.P], rell),
                        "grad_sigma_f_vs_fp64_nfft": abs(gt[wl.P] - rsf) / abs(rsf),
                        "grad_points_vs_fp64_nfft": r(gx.cpu().numpy(), rx)},
           "clocks": clk.summary()}
    print(json.dumps(out), flush=True)
    op.close()


def run_cpu_times(args, rank):
    """CPU context for the headline workload (no GPU): one full-N FP64 oracle product on the host
    cores (the oracle's OpenMP threads; OMP_NUM_THREADS=1 gives the one-core figure) and, with
    --check-rows R, the direct FP64 sums on R random rows. Prints one JSON line."""
    if rank != 0:
        return
    import numpy as np
    import workloads
    import oracle
    wl = workloads.make("c1", N=args.N)
    v = wl.vector().astype(np.float64)
    sample = min(args.N, 20_000)
    oracle.fastsum.matvec_all(wl.points[:sample], wl.windows, wl.ell, wl.sigma_f, v[:sample], wl.bandwidth,
                              wl.cutoff)                                  # builds and warms the oracle library
    t0 = time.perf_counter()
    oracle.fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v, wl.bandwidth, wl.cutoff)
    nfft_s = time.perf_counter() - t0
    rows = np.random.default_rng(0).choice(wl.N, args.check_rows, replace=False)
    t0 = time.perf_counter()
    oracle.fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v, rows=rows)
    direct_s = time.perf_counter() - t0
    print(json.dumps({"mode": "cpu", "threads": cpu_cores(), "N": args.N,
                      "oracle_nfft_units_per_s": 1.0 / nfft_s, "oracle_nfft_s_per_unit": nfft_s,
                      "direct_rows": int(args.check_rows), "direct_s": direct_s}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=1_000_000)
    ap.add_argument("--cpu-reps", type=int, default=3, help="oracle products timed for cpu_baseline")
    ap.add_argument("--check-rows", type=int, default=4096)
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--mode", default="product", choices=["product", "batched", "gp", "grad", "cpu"],
                    help="product: the headline fused product; batched: 7 mixed windows x 64 right-hand sides; "
                         "gp: one GP gradient (CG + Hutchinson) per step; grad: one vector-Jacobian product per "
                         "step (differentiation configuration); cpu: FP64 oracle timings on the host "
                         "cores (no GPU)")
    ap.add_argument("--nrhs", type=int, default=64, help="right-hand sides per step (batched), 1 + probes (gp)")
    ap.add_argument("--beta", type=float, default=0.01,
                    help="gp: regularisation beta (the configuration's noise variance 0.01)")
    ap.add_argument("--precond", type=int, default=1, help="gp: preconditioner band (0 = plain CG)")
    ap.add_argument("--tol", type=float, default=1e-6, help="gp: CG relative residual tolerance")
    ap.add_argument("--maxit", type=int, default=100, help="gp: CG iterations at most")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.mode == "batched":
        run_batched(args, rank, world, local_rank)
    elif args.mode == "cpu":
        run_cpu_times(args, rank)
    elif args.mode == "grad":
        run_grad(args, rank, world, local_rank)
    elif args.mode == "gp":
        if args.nrhs == 64:
            args.nrhs = 17                       # y and 16 probes
        run_gp(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
