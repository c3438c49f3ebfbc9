"""GB300 library for NFFT-based products with additive Gaussian kernels (arXiv 2404.17344).

The compute path is the CUDA library libaddker.so behind the C ABI of include/addker.h; this
package only marshals arguments to it. PyTorch provides device memory and the current stream.

    from paper_2404_17344_gb300 import AddKer
    op = AddKer(points_cuda, windows=[(0, 1, 2), (3, 4, 5)], ell=[0.3, 0.5], sigma_f=1.0,
                bandwidth=32, cutoff=4)
    Kv, dKdell = op.matvec_all(v)        # K v and dK/d ell_s v for every window s
"""
from __future__ import annotations

import ctypes

from . import native
from .native import (ADDKER_ELL, ADDKER_ELL_SHARED, ADDKER_SIGMA_F, AddkerError)  # noqa: F401

__all__ = ["AddKer", "prescale", "ADDKER_ELL", "ADDKER_ELL_SHARED", "ADDKER_SIGMA_F", "AddkerError"]


def _torch():
    import torch
    return torch


def _csr(windows):
    off, feat = [0], []
    for w in windows:
        feat.extend(int(f) for f in w)
        off.append(len(feat))
    return (ctypes.c_int * len(off))(*off), (ctypes.c_int * max(1, len(feat)))(*feat)


def _dev_f32(t, name):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32):
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _stream_ptr():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


class AddKer:
    """A plan for the additive kernel K = sigma_f^2 sum_s K_s over the given windows.

    points: (N, d) float32 CUDA tensor, scaled so that ||x^{W_s}|| <= 1/4 - eps_B/2 for all s.
    windows: list of feature-index tuples (1 to 3 features each).
    ell: per-window length scales; sigma_f: signal standard deviation.
    bandwidth: M (int or per-window list), cutoff: window cutoff m.
    reg: the reading of the regularisation, None (the default: 'separable' for the Gaussian, 'radial'
    for Matern(1/2)), 'separable' or 'radial' (degree p).
    """

    KERNELS = {"gauss": native.ADDKER_KERNEL_GAUSS, "matern": native.ADDKER_KERNEL_MATERN12}
    WINDOWS = {"kb": native.ADDKER_WIN_KB, "es": native.ADDKER_WIN_ES}
    REGS = {None: native.ADDKER_REG_DEFAULT, "separable": native.ADDKER_REG_SEPARABLE,
            "radial": native.ADDKER_REG_RADIAL}

    def __init__(self, points, windows, ell, sigma_f=1.0, bandwidth=32, cutoff=4, eps_B=1.0 / 16.0,
                 p=-1, sigma_os=2.0, kernel="gauss", compensated=False, window="kb", reg=None):
        L = native.lib()
        pts = _dev_f32(points, "points")
        if pts.dim() != 2:
            raise ValueError("points must be (N, d)")
        self.N, self.d = int(pts.shape[0]), int(pts.shape[1])
        self.windows = [tuple(int(f) for f in w) for w in windows]
        self.P = len(self.windows)
        bw = [int(bandwidth)] * self.P if isinstance(bandwidth, int) else [int(b) for b in bandwidth]
        if len(bw) != self.P or len(ell) != self.P:
            raise ValueError("ell and bandwidth need one entry per window")
        off, feat = _csr(self.windows)
        ell_c = (ctypes.c_double * self.P)(*[float(e) for e in ell])
        bw_c = (ctypes.c_int * self.P)(*bw)
        opts = native.addker_opts()
        native.check(L.addker_opts_default(ctypes.byref(opts)), "addker_opts_default")
        opts.sigma_os, opts.eps_B, opts.p = float(sigma_os), float(eps_B), int(p)
        if kernel not in self.KERNELS:
            raise ValueError(f"kernel must be one of {sorted(self.KERNELS)}")
        opts.kernel = self.KERNELS[kernel]
        if window not in self.WINDOWS:
            raise ValueError(f"window must be one of {sorted(self.WINDOWS)}")
        opts.window = self.WINDOWS[window]
        opts.compensated = 1 if compensated else 0
        if reg not in self.REGS:
            raise ValueError("reg must be None, 'separable' or 'radial'")
        opts.reg = self.REGS[reg]
        opts.stream = _stream_ptr()
        plan = ctypes.c_void_p()
        native.check(L.addker_setup(ctypes.byref(plan), ctypes.c_void_p(pts.data_ptr()), self.N, self.d, off, feat,
                                    self.P, ell_c, float(sigma_f), bw_c, int(cutoff), ctypes.byref(opts)),
                     "addker_setup")
        self._plan = plan
        self.ell = [float(e) for e in ell]
        self.sigma_f = float(sigma_f)
        self.bandwidth = bw
        self.cutoff = int(cutoff)
        self.sigma_os = float(sigma_os)
        self.kernel = kernel
        self.window = window

    # -- plumbing ---------------------------------------------------------------------------
    def _ready(self):
        if self._plan is None:
            raise RuntimeError("plan already freed")
        native.check(native.lib().addker_set_stream(self._plan, _stream_ptr()), "addker_set_stream")
        return native.lib()

    def _rhs(self, v):
        torch = _torch()
        if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float32):
            raise TypeError("v must be a float32 CUDA tensor")
        if v.shape[0] != self.N or v.dim() not in (1, 2):
            raise ValueError("v must be (N,) or (N, nrhs) with column j a right-hand side")
        nrhs = 1 if v.dim() == 1 else int(v.shape[1])
        if v.dim() == 2:
            v = v.t()                      # column-major (nrhs, N) storage; a column-major view is not copied
        if not v.is_contiguous():
            v = v.contiguous()
        return v, nrhs

    @staticmethod
    def _shape_out(buf, nrhs, one_shape):
        return buf.reshape(one_shape) if nrhs == 1 else buf.reshape(nrhs, -1).t()

    # -- products ----------------------------------------------------------------------------
    def matvec(self, v):
        """K v; v is (N,) or (N, nrhs)."""
        torch = _torch()
        L = self._ready()
        vv, nrhs = self._rhs(v)
        out = torch.empty(nrhs * self.N, device=vv.device, dtype=torch.float32)
        native.check(L.addker_matvec(self._plan, ctypes.c_void_p(vv.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     nrhs), "addker_matvec")
        return self._shape_out(out, nrhs, (self.N,))

    def dmatvec(self, param, v):
        """dK/d theta v for param = ADDKER_ELL(s), ADDKER_ELL_SHARED or ADDKER_SIGMA_F."""
        torch = _torch()
        L = self._ready()
        vv, nrhs = self._rhs(v)
        out = torch.empty(nrhs * self.N, device=vv.device, dtype=torch.float32)
        native.check(L.addker_dmatvec(self._plan, int(param), ctypes.c_void_p(vv.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), nrhs), "addker_dmatvec")
        return self._shape_out(out, nrhs, (self.N,))

    def matvec_all(self, v, out_Kv=None, out_dK=None):
        """(K v, dK/d ell v): Kv has v's shape; dK is (P, N) for one right-hand side, else (P, N, nrhs)."""
        torch = _torch()
        L = self._ready()
        vv, nrhs = self._rhs(v)
        Kv = out_Kv if out_Kv is not None else torch.empty(nrhs * self.N, device=vv.device, dtype=torch.float32)
        dK = out_dK if out_dK is not None else torch.empty(nrhs * self.P * self.N, device=vv.device,
                                                            dtype=torch.float32)
        native.check(L.addker_matvec_all(self._plan, ctypes.c_void_p(vv.data_ptr()), ctypes.c_void_p(Kv.data_ptr()),
                                         ctypes.c_void_p(dK.data_ptr()), nrhs), "addker_matvec_all")
        if nrhs == 1:
            return Kv.reshape(self.N), dK.reshape(self.P, self.N)
        return Kv.reshape(nrhs, self.N).t(), dK.reshape(nrhs, self.P, self.N).permute(1, 2, 0)

    def matvec_all_host(self, v, Kv, dK, nrhs=1):
        """Fused product on HOST buffers (contiguous float32 CPU torch tensors, pinned for asynchronous
        copies): v and Kv hold N*nrhs values, dK N*P*nrhs (or None), right-hand side j at offset j*N
        (j*N*P for dK). Copies are included; returns when the results are on the host."""
        L = self._ready()
        for t, need in ((v, self.N * nrhs), (Kv, self.N * nrhs)) + (((dK, self.N * self.P * nrhs),) if dK is not None else ()):
            if t.device.type != "cpu" or t.dtype != _torch().float32 or not t.is_contiguous() or t.numel() < need:
                raise ValueError("host buffers must be contiguous float32 CPU tensors of sufficient size")
        native.check(L.addker_matvec_all_host(self._plan, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(Kv.data_ptr()),
                                              ctypes.c_void_p(dK.data_ptr()) if dK is not None else None, int(nrhs)),
                     "addker_matvec_all_host")

    def vjp(self, v, w):
        """Gradients of f = w^T K v: (K w [N], grad_theta [P + 1] float64 = (df/d ell_s..., df/d sigma_f),
        df/dpoints [N, d]). v and w are (N,) float32 CUDA tensors."""
        torch = _torch()
        L = self._ready()
        v = _dev_f32(v, "v")
        w = _dev_f32(w, "w")
        if v.shape != (self.N,) or w.shape != (self.N,):
            raise ValueError("v and w must be (N,)")
        gv = torch.empty(self.N, device=v.device, dtype=torch.float32)
        gt = torch.empty(self.P + 1, device=v.device, dtype=torch.float64)
        gx = torch.empty(self.N, self.d, device=v.device, dtype=torch.float32)
        native.check(L.addker_vjp(self._plan, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                  ctypes.c_void_p(gv.data_ptr()), ctypes.c_void_p(gt.data_ptr()),
                                  ctypes.c_void_p(gx.data_ptr())), "addker_vjp")
        return gv, gt, gx

    # -- plan management ---------------------------------------------------------------------
    def set_params(self, ell=None, sigma_f=None):
        L = self._ready()
        sf = self.sigma_f if sigma_f is None else float(sigma_f)
        ell_c = None
        if ell is not None:
            ell_c = (ctypes.c_double * self.P)(*[float(e) for e in ell])
        native.check(L.addker_set_params(self._plan, ell_c, sf), "addker_set_params")
        if ell is not None:
            self.ell = [float(e) for e in ell]
        self.sigma_f = sf

    def set_graphs(self, enable):
        """Replay repeated identical products as CUDA graphs (default on); False launches every kernel."""
        native.check(self._ready().addker_set_graphs(self._plan, 1 if enable else 0), "addker_set_graphs")

    def set_schedule(self, chunk=256, chunk_spread=256, spread_blocks=0, spread_tile=0):
        """Work-item sizes, persistent-spread blocks per SM (0 = as many as fit) and 3-D spread register tile
        (addker_set_schedule): the choices addker_autotune makes, set directly."""
        native.check(self._ready().addker_set_schedule(self._plan, int(chunk), int(chunk_spread), int(spread_blocks),
                                                        int(spread_tile)), "addker_set_schedule")

    def set_precond(self, band):
        """CG preconditioner with every window's Fourier modes |k|_inf <= band (addker_set_precond; 0 = plain CG,
        default 1)."""
        native.check(self._ready().addker_set_precond(self._plan, int(band)), "addker_set_precond")

    def cg(self, y, beta, tol=1e-3, maxit=1000, x0=None):
        """Solve (K + beta I) x = y by conjugate gradients (addker_cg). y is (N,) or (N, nrhs); returns
        (x shaped like y, iterations per column, relative residual per column)."""
        torch = _torch()
        yy, nrhs = self._rhs(y)
        x = torch.zeros_like(yy) if x0 is None else self._rhs(x0)[0].clone()
        iters = (ctypes.c_int * nrhs)()
        rel = (ctypes.c_double * nrhs)()
        native.check(self._ready().addker_cg(self._plan, float(beta), ctypes.c_void_p(yy.data_ptr()),
                                              ctypes.c_void_p(x.data_ptr()), nrhs, float(tol), int(maxit), iters, rel),
                     "addker_cg")
        return self._shape_out(x.reshape(-1), nrhs, (self.N,)), list(iters), list(rel)

    def gp_grad(self, y, beta, Z=None, tol=1e-3, maxit=1000):
        """Gradient of the GP log marginal likelihood in (ell_1..ell_P, sigma_f, beta) with Hutchinson
        probes Z ((N, m), or None for no trace term) (addker_gp_grad). Returns (grad [P+2] float64 numpy,
        y^T alpha, alpha [N], CG iterations)."""
        import numpy as np
        torch = _torch()
        yv = _dev_f32(y, "y")
        if yv.shape != (self.N,):
            raise ValueError("y must be (N,)")
        m = 0
        zp = None
        if Z is not None:
            zz, m = self._rhs(Z)
            zp = ctypes.c_void_p(zz.data_ptr())
        grad = (ctypes.c_double * (self.P + 2))()
        fit = ctypes.c_double(0.0)
        alpha = torch.empty(self.N, device=yv.device, dtype=torch.float32)
        iters = ctypes.c_int(0)
        native.check(self._ready().addker_gp_grad(self._plan, float(beta), ctypes.c_void_p(yv.data_ptr()), zp, m,
                                                   float(tol), int(maxit), grad, ctypes.byref(fit),
                                                   ctypes.c_void_p(alpha.data_ptr()), ctypes.byref(iters)),
                     "addker_gp_grad")
        return np.array(list(grad)), fit.value, alpha, iters.value

    def gsi(self, v):
        """Global sensitivity indices of the fast-summation polynomial for coefficients v (addker_gsi).
        Returns ({feature subset (tuple): rho}, total variance), subsets by decreasing rho."""
        vv = _dev_f32(v, "v")
        if vv.shape != (self.N,):
            raise ValueError("v must be (N,)")
        L = self._ready()
        cap = sum(2 ** len(w) - 1 for w in self.windows)
        feats = (ctypes.c_int * (3 * cap))()
        rho = (ctypes.c_double * cap)()
        total = ctypes.c_double(0.0)
        n = L.addker_gsi(self._plan, ctypes.c_void_p(vv.data_ptr()), cap, feats, rho, ctypes.byref(total))
        if n < 0:
            native.check(n, "addker_gsi")
        out = {}
        for i in range(min(n, cap)):
            out[tuple(f for f in feats[3 * i:3 * i + 3] if f >= 0)] = rho[i]
        return out, total.value

    AUTOTUNE_CHUNKS = (64, 128, 256, 512, 1024)

    def autotune(self, v):
        """Time the fused product on v ((N,) or (N, nrhs)) for each work-item size in AUTOTUNE_CHUNKS (one
        size for both kernels), then for each spread size with the gather's fixed, then for each persistent-
        spread residency (blocks per SM 1, 2, 3, or as many as fit = 0), then for each 3-D spread register
        tile (0, 1), and keep the fastest. Returns
        (gather chunk, {chunk: ms per product} of the joint phase); the spread's size and residency are
        info()["chunk_spread"], info()["spread_blocks_per_sm"] and info()["spread_tile"], their timings
        autotune_spread_times, autotune_residency_times and autotune_tile_times."""
        vv, nrhs = self._rhs(v)
        chosen = ctypes.c_int(0)
        nc = len(self.AUTOTUNE_CHUNKS)
        times = (ctypes.c_double * (2 * nc + 6))()
        native.check(self._ready().addker_autotune(self._plan, ctypes.c_void_p(vv.data_ptr()), nrhs,
                                                    ctypes.byref(chosen), times, len(times)), "addker_autotune")
        self.autotune_spread_times = dict(zip(self.AUTOTUNE_CHUNKS, list(times)[nc:2 * nc]))
        self.autotune_residency_times = dict(zip((1, 2, 3, 0), list(times)[2 * nc:2 * nc + 4]))
        self.autotune_tile_times = dict(zip((0, 1), list(times)[2 * nc + 4:]))
        return chosen.value, dict(zip(self.AUTOTUNE_CHUNKS, list(times)[:nc]))

    STAGES = ("clear", "spread", "transform", "gather", "window_sum")

    def profile(self, enable=True):
        """Start (clearing) or stop per-stage event timing of later products on this plan."""
        native.check(native.lib().addker_profile(self._plan, 1 if enable else 0), "addker_profile")

    def profile_read(self):
        """{stage: (milliseconds, kernel launches)} summed over the products since profile(True)."""
        ms = (ctypes.c_double * 5)()
        cnt = (ctypes.c_int64 * 5)()
        n = native.lib().addker_profile_read(self._plan, ms, cnt, 5)
        if n < 0:
            native.check(n, "addker_profile_read")
        return {name: (ms[i], cnt[i]) for i, name in enumerate(self.STAGES)}

    def sync(self):
        native.check(native.lib().addker_sync(self._plan), "addker_sync")

    def info(self):
        cap = 11 + 4 * self.P
        buf = (ctypes.c_int64 * cap)()
        n = native.lib().addker_info(self._plan, buf, cap)
        vals = list(buf[:n])
        e = 4 + 4 * self.P
        return {"N": vals[0], "P": vals[1], "items": vals[2], "device_bytes": vals[3],
                "windows": [dict(d=vals[4 + 4 * s], M=vals[5 + 4 * s], n=vals[6 + 4 * s], cells=vals[7 + 4 * s])
                            for s in range(self.P)],
                "slots": vals[e], "graphs": vals[e + 1], "graph_replays": vals[e + 2], "chunk": vals[e + 3],
                "chunk_spread": vals[e + 4], "spread_blocks_per_sm": vals[e + 5], "spread_tile": vals[e + 6]}

    def debug_stage(self, window, stage, v):
        """Stage 0: spread grid (n^d doubles); stage 1: adjoint NFFT S_k (complex M^d). Synchronous."""
        import numpy as np
        L = self._ready()
        v = _dev_f32(v, "v")
        w = self.windows[window]
        M = self.bandwidth[window]
        n = int(round(self.sigma_os * M))
        cap = n ** len(w) if stage == 0 else 2 * M ** len(w)
        out = np.zeros(cap, dtype=np.float64)
        native.check(L.addker_debug_stage(self._plan, int(window), int(stage), ctypes.c_void_p(v.data_ptr()),
                                          ctypes.c_void_p(out.ctypes.data), cap), "addker_debug_stage")
        if stage == 0:
            return out.reshape((n,) * len(w))
        return (out[0::2] + 1j * out[1::2]).reshape((M,) * len(w))

    def close(self):
        if getattr(self, "_plan", None) is not None:
            native.lib().addker_free(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prescale(X, windows, eps_B=1.0 / 16.0, rule="ball"):
    """Sec. 3.2 prescaling on the device: returns (scaled copy of X, factor).
    rule "ball": one global factor into the ball of radius 1/4 - eps_B/2 (addker_prescale);
    rule "cube": the paper's per-feature map onto a cube, then 1/sqrt(d_max) (addker_prescale_cube)."""
    torch = _torch()
    X = _dev_f32(X, "X")
    N, d = int(X.shape[0]), int(X.shape[1])
    off, feat = _csr(windows)
    out = torch.empty_like(X)
    f = ctypes.c_double()
    fn = {"ball": "addker_prescale", "cube": "addker_prescale_cube"}[rule]
    native.check(getattr(native.lib(), fn)(ctypes.c_void_p(X.data_ptr()), N, d, off, feat, len(windows),
                                           float(eps_B), ctypes.c_void_p(out.data_ptr()), ctypes.byref(f),
                                           _stream_ptr()), fn)
    return out, f.value
