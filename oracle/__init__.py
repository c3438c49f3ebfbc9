"""FP64 CPU oracle for the NFFT-based additive-kernel products.

TEST INFRASTRUCTURE. Only the tests, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg (`bench.py --impl reference` and the
`cpu_baseline` field) may import or run this package. The CUDA library and its
Python binding never do; they share no code with it.

Contents (each function cites the passage of Wagner, Nestler, Stoll, "Fast
Evaluation of Additive Kernels: Feature Arrangement, Fourier Methods, and Kernel
Derivatives" that it follows):

  fastsum.direct        O(N^2) (or row-subset) direct sums of K v and dK/d ell_s v
  fastsum.ndft_fastsum  exact trigonometric fast sum (eq. "approx fast sum")
  fastsum.nfft_fastsum  plain FP64 NFFT fast summation (adjoint NFFT, multiply, NFFT)
  fastsum.matvec_all    additive combination over windows, with the derivative scalings
  kernels.*             kernels, regularisation (radial, and the separable reading: tensor-product
                        coefficients of 1-D least-squares Fourier extensions), discrete Fourier
                        coefficients
  window.*              Kaiser-Bessel window and its Fourier transform
  bounds.*              the error bounds of Sec. 3.4 and the analytic coefficients
  gp.*                  regression system (CG), GP log marginal likelihood and its gradient,
                        Hutchinson's trace estimator (Sec. 3.3)
  gsi.*                 global sensitivity indices (Sec. 4, Algorithm "Computation of GSI")

Parity status: every function is pinned by a CPU test against something other
than itself (closed forms, brute force, the paper's printed constants, bounds,
invariants), except the absolute error level of the regularised periodisation
against the paper's figures, which are not available ("parity unpinned" for that
one number only; the regularisation itself is pinned by its defining conditions).
"""
from . import bounds, fastsum, gp, gradients, gsi, kernels, window  # noqa: F401
from ._clib import build  # noqa: F401
