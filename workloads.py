"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers and lays them out. It holds none of the
fast-summation arithmetic, so both the CUDA path and the CPU oracle may use it.

Every workload stands in for the paper's UCI/StatLib datasets (Protein,
KEGGundir, Bike Sharing, Housing; Sec. 5), which are not available here. The
draws follow the shapes and distributions of the five benchmark configurations:

  c0  N=2000,  d=3,  U[-1,1]^3, one window {0,1,2}, ell=0.5
  c1  N=1e5 (1e6 for the headline), d=9, N(0,1), windows of 3 consecutive
      features, ell=(0.3, 0.5, 1.0)
  c2  N=2e5, d=12, mixture of 4 isotropic Gaussians (means U[-1,1]^12,
      std 0.3), 4 windows of 3
  c3  N=1e6, d=15, U[-1,1], windows of sizes 3,3,3,2,2,1,1, ell log-U[0.1,2]
  c4  N=2e6, d=24, correlated Gaussian (covariance A A^T, A ~ N(0,1/24)),
      8 windows of 3

Points are then multiplied by one global factor so that every point restricted
to every window lies in the ball of radius rho = 1/4 - eps_B/2 (eps_B = 1/16);
then all pairwise differences inside a window have norm <= 1/2 - eps_B. Length
scales are given in these scaled units. Seeds: numpy PCG64 with
seed = 1000 + config index for the points, +1 for v, +2 for w, +3 for regression
targets (random Fourier features plus noise), +4 for Hutchinson probes.
"""
from __future__ import annotations

import dataclasses
import numpy as np

EPS_B = 1.0 / 16.0
RHO = 0.25 - EPS_B / 2.0          # ball radius that every windowed point must respect


@dataclasses.dataclass
class Workload:
    name: str
    points: np.ndarray            # (N, d) float32, row-major, already scaled into the ball
    windows: list                 # list of tuples of 0-based feature indices
    ell: np.ndarray               # (P,) float64 length scales in scaled units
    sigma_f: float
    bandwidth: list               # per-window bandwidth M_s (even)
    cutoff: int                   # window cutoff m
    seed: int

    @property
    def N(self) -> int:
        return int(self.points.shape[0])

    @property
    def d(self) -> int:
        return int(self.points.shape[1])

    @property
    def P(self) -> int:
        return len(self.windows)

    def vector(self, nrhs: int = 1, which: int = 1) -> np.ndarray:
        """Standard-normal right-hand side(s): shape (N,) for nrhs == 1, else (N, nrhs)
        (column j is right-hand side j). which=1 gives v, which=2 gives w."""
        rng = np.random.Generator(np.random.PCG64(self.seed + which))
        if nrhs == 1:
            return rng.standard_normal(self.N).astype(np.float32)
        return rng.standard_normal((nrhs, self.N)).astype(np.float32).T.copy()

    def targets(self, terms: int = 16, noise_var: float = 0.01) -> np.ndarray:
        """Regression targets for the GP/KRR loop: a sum over the windows of random smooth functions of
        the window's features, each a random-Fourier-feature expansion with `terms` terms,
        f_s(x) = sqrt(2/F) sum_f a_f cos(omega_f . x^W_s + b_f), omega_f ~ N(0, I/ell_s^2),
        a_f ~ N(0, 1), b_f ~ U[0, 2 pi), plus N(0, noise_var) noise. Seed + 3. Shape (N,), float32."""
        rng = np.random.Generator(np.random.PCG64(self.seed + 3))
        y = np.zeros(self.N)
        for s, w in enumerate(self.windows):
            X = self.points[:, list(w)].astype(np.float64)
            omega = rng.standard_normal((terms, len(w))) / float(self.ell[s])
            a = rng.standard_normal(terms)
            b = rng.uniform(0.0, 2.0 * np.pi, size=terms)
            y += np.sqrt(2.0 / terms) * (np.cos(X @ omega.T + b) @ a)
        y += np.sqrt(noise_var) * rng.standard_normal(self.N)
        return y.astype(np.float32)

    def probes(self, m: int) -> np.ndarray:
        """m Rademacher probe vectors for Hutchinson's trace estimator, (N, m) float32. Seed + 4."""
        rng = np.random.Generator(np.random.PCG64(self.seed + 4))
        return rng.choice(np.array([-1.0, 1.0], dtype=np.float32), size=(m, self.N)).T.copy()


def scale_into_ball(X: np.ndarray, windows, rho: float = RHO) -> np.ndarray:
    """One global factor so that max_{j,s} ||x_j^{W_s}|| = rho (up to a hair for float32
    rounding). Returns float32."""
    X = np.asarray(X, dtype=np.float64)
    mx = 0.0
    for w in windows:
        nr = np.sqrt((X[:, list(w)] ** 2).sum(axis=1))
        mx = max(mx, float(nr.max()) if len(nr) else 0.0)
    f = rho * (1.0 - 4e-7) / mx if mx > 0 else 1.0
    return (X * f).astype(np.float32)


def consecutive_windows(sizes):
    out, k = [], 0
    for s in sizes:
        out.append(tuple(range(k, k + s)))
        k += s
    return out


def make(config: str, N: int | None = None) -> Workload:
    """Build a workload by configuration name ('c0' .. 'c4'); N overrides the point count."""
    idx = int(config[1:])
    seed = 1000 + idx
    rng = np.random.Generator(np.random.PCG64(seed))
    if idx == 0:
        N = N or 2000
        X = rng.uniform(-1.0, 1.0, size=(N, 3))
        wins = [(0, 1, 2)]
        ell = [0.5]
        bw = [32]
    elif idx == 1:
        N = N or 100_000
        X = rng.standard_normal((N, 9))
        wins = consecutive_windows([3, 3, 3])
        ell = [0.3, 0.5, 1.0]
        bw = [32, 32, 32]
    elif idx == 2:
        N = N or 200_000
        means = rng.uniform(-1.0, 1.0, size=(4, 12))
        comp = rng.integers(0, 4, size=N)
        X = means[comp] + 0.3 * rng.standard_normal((N, 12))
        wins = consecutive_windows([3, 3, 3, 3])
        ell = [0.3, 0.5, 0.7, 1.0]
        bw = [32] * 4
    elif idx == 3:
        N = N or 1_000_000
        X = rng.uniform(-1.0, 1.0, size=(N, 15))
        wins = consecutive_windows([3, 3, 3, 2, 2, 1, 1])
        ell = list(np.exp(rng.uniform(np.log(0.1), np.log(2.0), size=7)))
        bw = [32 if len(w) == 3 else 16 for w in wins]
    elif idx == 4:
        N = N or 2_000_000
        A = rng.standard_normal((24, 24)) * np.sqrt(1.0 / 24.0)
        X = rng.standard_normal((N, 24)) @ A.T
        wins = consecutive_windows([3] * 8)
        ell = [0.5] * 8
        bw = [32] * 8
    else:
        raise ValueError(f"unknown configuration {config!r}")
    pts = scale_into_ball(X, wins)
    return Workload(name=config, points=pts, windows=wins, ell=np.asarray(ell, dtype=np.float64),
                    sigma_f=1.0, bandwidth=bw, cutoff=4, seed=seed)


def tiny(N: int = 40, d: int = 3, windows=None, seed: int = 7, ell=None) -> Workload:
    """Small uniform case for brute-force checks."""
    windows = windows or [tuple(range(d))]
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.uniform(-1.0, 1.0, size=(N, d))
    pts = scale_into_ball(X, windows)
    ell = np.asarray(ell if ell is not None else [0.4] * len(windows), dtype=np.float64)
    return Workload(name=f"tiny{N}", points=pts, windows=list(windows), ell=ell, sigma_f=1.3,
                    bandwidth=[16] * len(windows), cutoff=3, seed=seed)
