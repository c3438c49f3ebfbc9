/*
 * addker.h - C ABI of the GB300 library for NFFT-based products with additive
 * Gaussian kernels and their hyperparameter derivatives.
 *
 * Operation (Wagner, Nestler, Stoll, "Fast Evaluation of Additive Kernels",
 * arXiv 2404.17344):
 *
 *   K v              = sigma_f^2 sum_{s=1}^{P} K_s v,
 *   (K_s)_{ij}       = exp(-||x_i^{W_s} - x_j^{W_s}||^2 / (2 ell_s^2))
 *                      (Sec. 1 eq. "wind_gauss_anova_kernel", Sec. 3.3 eq. "add_gauss_kernel"),
 *   dK/d ell_s v     = sigma_f^2 (2/ell_s) K_s^der v,
 *   (K_s^der)_{ij}   = (r^2/(2 ell_s^2)) exp(-r^2/(2 ell_s^2)),  r = ||x_i^{W_s} - x_j^{W_s}||
 *                      (Sec. 3.3 eq. "implement_der_gaussian_kernel" with c = sqrt(2) ell),
 *   dK/d sigma_f v   = (2/sigma_f) K v                          (Sec. 3.3),
 *
 * each K_s v and K_s^der v approximated by the NFFT fast summation of Sec. 3.1
 * (eq. "approx fast sum"): spreading onto an oversampled grid (adjoint NFFT),
 * FFT, multiplication by the Fourier coefficients of the regularised kernel
 * (Lemma "aliasing error": coefficients from M^{d_s} samples), inverse FFT,
 * interpolation (NFFT). Every step of a product runs in CUDA kernels on the
 * device; FP32 arithmetic, FP64 only in the coefficient precomputation and in
 * the inner products of the solvers.
 *
 * Entry points:
 *   plan         addker_opts_default, addker_setup, addker_set_params, addker_set_stream,
 *                addker_set_graphs, addker_set_precond, addker_set_schedule, addker_autotune, addker_free,
 *                addker_info
 *   products     addker_matvec, addker_dmatvec, addker_matvec_all (device buffers),
 *                addker_matvec_all_host (host buffers), addker_fastsum_noalloc (no plan)
 *   gradients    addker_vjp (w^T K v with respect to v, ell, sigma_f and the points)
 *   solvers      addker_cg (regression system, Sec. 3.3), addker_gp_grad (GP training)
 *   analysis     addker_gsi (global sensitivity indices, Sec. 4)
 *   utilities    addker_prescale, addker_prescale_cube, addker_sync, addker_strerror, addker_profile,
 *                addker_profile_read, addker_debug_stage
 * The additive Matern(1/2) kernel of Sec. 5 is selected by addker_opts.kernel.
 *
 * Conventions for every call:
 *   - Return 0 on success or a negative ADDKER_E* code; addker_strerror() names it.
 *     No C++ exception crosses this interface.
 *   - Pointers marked "device" must point to CUDA device memory of the current
 *     device; "host" pointers to ordinary (or pinned) host memory.
 *   - The caller owns every buffer it passes in. A plan owns the device buffers
 *     it allocates (sorted copies of the points, grids, spectra, coefficients)
 *     and frees them in addker_free().
 *   - Products are enqueued on the plan's stream (addker_set_stream) and return
 *     without waiting; the outputs are ready when that stream reaches them.
 *     Kernel launch failures are reported by the call that launched them, or by
 *     addker_sync().
 *   - A plan is not thread-safe: calls on one plan must not overlap in time, and
 *     two products on one plan must not run concurrently on different streams
 *     (they share the plan's grids).
 */
#ifndef ADDKER_H
#define ADDKER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define ADDKER_OK        0
#define ADDKER_EINVAL   -1   /* bad argument (sizes, window layout, bandwidth, cutoff, NULL) */
#define ADDKER_EDOMAIN  -2   /* a point lies outside the ball ||x^{W_s}|| <= 1/4 - eps_B/2, or is not finite */
#define ADDKER_ENOMEM   -3   /* a device allocation failed */
#define ADDKER_ECUDA    -4   /* a CUDA runtime call or kernel launch failed */
#define ADDKER_ETIMEOUT -5   /* a bounded device wait gave up (reserved) */
#define ADDKER_ELIMIT   -6   /* request larger than the fixed memory of addker_fastsum_noalloc */

/* ---- derivative selectors for addker_dmatvec --------------------------- */
#define ADDKER_ELL(s)        (s)   /* dK/d ell_s v for window s, 0 <= s < P */
#define ADDKER_ELL_SHARED   (-1)   /* sum_s dK/d ell_s v: the derivative for one ell shared by all windows */
#define ADDKER_SIGMA_F      (-2)   /* dK/d sigma_f v = (2/sigma_f) K v */

/* NFFT windows (addker_opts.window), support |n x| <= m (2m grid points per axis); the paper leaves the
 * window to the NFFT literature (Sec. 3.1):
 *   ADDKER_WIN_KB  Kaiser-Bessel, phi(x) = sinh(b sqrt(m^2 - (n x)^2)) / (pi sqrt(m^2 - (n x)^2)),
 *                  b = pi (2 - 1/sigma)
 *   ADDKER_WIN_ES  exponential of semicircle (Barnett, Magland, af Klinteberg 2019),
 *                  phi(x) = exp(beta (sqrt(1 - (n x/m)^2) - 1)), beta = 2.30 * 2m * (1 - 1/(2 sigma)) / (3/4)
 *                  (2.30 * 2m at sigma = 2). Products only: addker_vjp returns ADDKER_EINVAL for it (its
 *                  derivative is unbounded at the support edge). */
#define ADDKER_WIN_KB 0
#define ADDKER_WIN_ES 1

/* Kernel families (addker_opts.kernel):
 *   ADDKER_KERNEL_GAUSS     kappa_s(r) = exp(-r^2/(2 ell_s^2)), derivative kernel (r^2/(2 ell_s^2)) kappa_s,
 *                           dK/d ell_s = sigma_f^2 (2/ell_s) K_s^der (Sec. 3.3)
 *   ADDKER_KERNEL_MATERN12  kappa_s(r) = exp(-r/ell_s), derivative kernel (r/ell_s) kappa_s,
 *                           dK/d ell_s = sigma_f^2 (1/ell_s) K_s^der (Sec. 5, "Extension to Other
 *                           Kernels"). Same boundary regularisation; the kink at r = 0 is not corrected
 *                           (the paper describes no near-field correction), so the Fourier error is
 *                           far larger than the Gaussian's at equal M (e.g. 3e-3 at M = 32, 5e-4 at
 *                           M = 64, relative, ell = 0.3). */
#define ADDKER_KERNEL_GAUSS 0
#define ADDKER_KERNEL_MATERN12 1

/* How the non-periodic kernel becomes a trigonometric polynomial (addker_opts.reg). The paper smooths
 * the periodisation near the boundary of the period (Sec. 3.1, after Potts and Steidl) without writing
 * the construction down; two readings are built:
 *   ADDKER_REG_SEPARABLE  (default for the Gaussian) Sec. 3.4's tensor-product form: the Gaussian's
 *                         coefficients c_k = prod_t c_{k_t}(f), the derivative kernel's the d_s-term sum
 *                         sum_t c_{k_t}(g) prod_{u != t} c_{k_u}(f), f(x) = exp(-x^2/(2 ell^2)),
 *                         g(x) = (x^2/(2 ell^2)) f(x); each 1-D factor is the least-squares Fourier
 *                         extension (cosines of degree < M/2, FP64 Householder QR on 4M equispaced nodes)
 *                         of f or g on [0, a_t], a_t = min(1/2 - eps_B, max(max(1/4, 1/2 - 4/M),
 *                         2 max_j |x_{j,t}|)): the interval that holds every coordinate difference of
 *                         axis t. Gaussian family only.
 *   ADDKER_REG_RADIAL     the radial profile kept up to a = 1/2 - eps_B, joined to the constant kappa(1/2)
 *                         by the degree 2p-1 two-point Hermite polynomial (opts.p), sampled on the M^d
 *                         grid and transformed (Lemma "aliasing error"). The only choice for Matern(1/2).
 * At M = 32 on the nine-feature benchmark's windows the derivative products against the direct sums are
 * below 1e-5 with the separable reading and 3.6e-4 .. 2.8e-3 with the radial one. */
#define ADDKER_REG_DEFAULT (-1)
#define ADDKER_REG_SEPARABLE 0
#define ADDKER_REG_RADIAL 1

typedef struct addker_plan addker_plan;

/* Optional settings; pass NULL to addker_setup for the defaults. */
typedef struct {
    double sigma_os;     /* oversampling factor sigma; grid n = sigma * M per dimension (default 2.0) */
    double eps_B;        /* boundary width eps_B of the regularisation (default 1/16); points must satisfy
                            ||x^{W_s}|| <= 1/4 - eps_B/2 */
    int    p;            /* radial reading only: regularisation degree (transition polynomial of degree 2p-1);
                            -1 = default max(1, floor(M eps_B + 1/2)); 0 = no regularisation (plain periodic
                            continuation) */
    int    window;       /* ADDKER_WIN_KB (default) or ADDKER_WIN_ES */
    int    kernel;       /* ADDKER_KERNEL_GAUSS (default) or ADDKER_KERNEL_MATERN12 */
    int    compensated;  /* 1: compensated grid accumulation: the spread's FP32 tile sums are added into an
                            FP64 grid (no rounding error from the order of the atomic adds), which the
                            forward transform rounds once to FP32; 0 (default): plain FP32 adds */
    int    reg;          /* ADDKER_REG_DEFAULT (separable for the Gaussian, radial for Matern(1/2)),
                            ADDKER_REG_SEPARABLE (Gaussian only) or ADDKER_REG_RADIAL */
    void*  stream;       /* cudaStream_t for every product of this plan; NULL = legacy default stream */
} addker_opts;

/* Fill *opts with the defaults above. Returns ADDKER_EINVAL for NULL. */
int addker_opts_default(addker_opts* opts);

/*
 * Build a plan: validate, sort the points of every window by grid cell, and
 * precompute the Fourier multipliers (Sec. 3.1 and Sec. 3.3).
 *
 *   plan       out: the new plan (NULL on failure)
 *   points     device, N x d float32, row-major; already scaled so that every
 *              windowed point satisfies ||x^{W_s}|| <= 1/4 - eps_B/2 (Sec. 3.2);
 *              copied, the caller may free it after the call
 *   N, d       number of points (N >= 1) and features (d >= 1)
 *   win_off    host, P+1 ints, CSR offsets of the windows (win_off[0] = 0)
 *   win_feat   host, win_off[P] ints: 0-based feature indices of window s are
 *              win_feat[win_off[s] .. win_off[s+1]); 1 <= d_s <= 3, distinct, < d
 *   P          number of windows, 1 <= P <= 64
 *   ell        host, P doubles > 0: length scale of each window, in the units of `points`
 *   sigma_f    signal standard deviation (> 0)
 *   bandwidth  host, P ints: M_s, even, 4 <= M_s <= 64 (number of Fourier coefficients per dimension)
 *   cutoff     window cutoff m, 2 <= m <= 8, with m + 1 <= n/4 + n eps_B/2 for n = sigma M_s
 *              (so no support wraps around the grid)
 *   opts       host or NULL
 *
 * Under the separable reading the coefficients also depend on the points' largest |coordinate| per
 * feature (the fit intervals), taken here and kept for addker_set_params.
 *
 * Errors: ADDKER_EINVAL for bad sizes/layout (or the separable reading with Matern(1/2)), ADDKER_EDOMAIN
 * for a point outside the ball (checked on the device), ADDKER_ENOMEM, ADDKER_ECUDA. Synchronises the
 * plan's stream before returning.
 */
int addker_setup(addker_plan** plan, const float* points, int64_t N, int d,
                 const int* win_off, const int* win_feat, int P,
                 const double* ell, double sigma_f, const int* bandwidth, int cutoff,
                 const addker_opts* opts);

/* Replace the hyperparameters (host ell[P], sigma_f) and recompute the multipliers; the
 * sorted points are kept. ell may be NULL to keep the length scales. Synchronous. */
int addker_set_params(addker_plan* plan, const double* ell, double sigma_f);

/*
 * CUDA graphs for repeated products (enable = 1, the default; 0 = every call launches its kernels).
 * When a product entry point (addker_matvec, addker_dmatvec, addker_matvec_all and the host variant)
 * is called twice in a row with the same pointers, nrhs and selector, the second call captures the
 * product on a private stream and every later identical call replays it on the plan's stream. Graphs
 * bake in pointers and sigma_f: addker_set_params, slot growth and this call discard them. No graph
 * is used while stage profiling is on or while the plan's stream is itself being captured (the
 * caller's capture then records the kernels). EINVAL for enable other than 0/1. Synchronises the
 * plan's stream.
 */
int addker_set_graphs(addker_plan* plan, int enable);

/*
 * Autotuning of the spread and gather schedules. The spread and gather kernels take the points of each
 * non-empty grid cell in work items of at most `chunk` points (default 256 for both lists), their
 * scheduling grain, and the persistent spread runs as many blocks per SM as fit. This call times the
 * fused product (addker_matvec_all semantics) on v (device, N x nrhs, column-major), one warm-up and
 * three timed products per candidate, without graphs: first one item size for both kernels, chunk in
 * {64, 128, 256, 512, 1024}; then, with the gather's size fixed at the fastest, the spread's size over the
 * same candidates; then the persistent spread's residency, 1, 2 or 3 blocks per SM or as many as fit
 * (fewer resident warps contend less for the grid's atomic adds, more hide more latency); then the 3-D
 * spread's register tile (each lane accumulating a 4 x 4 x 2 or an 8 x 2 x 2 block of the 8 x 8 x 8 box:
 * the second needs half the packed products per point and one more shared load). The fastest setting is
 * kept for later products; chosen (host, may be NULL) receives the gather's size (the spread's size,
 * residency and tile are addker_info's last three values) and times (host, may be NULL) up to `cap`
 * milliseconds per product: the five joint candidates, the five spread candidates, the four residencies,
 * then the two tiles. Allocates and frees its own output buffers; synchronous on the plan's stream. The paper has
 * no counterpart (its library runs on the CPU): these are scheduling choices of the GPU path.
 */
int addker_autotune(addker_plan* plan, const float* v, int nrhs, int* chosen, double* times, int cap);

/*
 * Set the schedule that addker_autotune chooses, directly (for instance one tuned earlier): work items
 * of at most `chunk` points for the gathers and `chunk_spread` for the spread (16 .. 4096; the items are
 * re-cut when a size changes), the persistent spread's blocks per SM (0 = as many as fit, else 1 .. 8) and
 * the 3-D spread's register tile (0 or 1, see addker_autotune). Results do not depend on the schedule
 * beyond FP32 rounding order. EINVAL for values outside these ranges, ENOMEM if re-cutting fails.
 * Synchronises the plan's stream and drops captured graphs.
 */
int addker_set_schedule(addker_plan* plan, int chunk, int chunk_spread, int spread_blocks, int spread_tile);

/*
 * Conjugate gradients for the regression system (K + beta I) x = y (Sec. 3.3, eq. "regression_system";
 * the paper solves it with unpreconditioned CG to a relative residual tolerance), for nrhs independent
 * columns at once; preconditioned by default (addker_set_precond).
 *   beta    regularisation (>= 0; K + beta I must be positive definite)
 *   y       device, N x nrhs float32, column-major (column j at y + j N)
 *   x       device, N x nrhs float32: the initial guess in, the solution out
 *   tol     stop a column once ||y - (K + beta I) x|| <= tol ||y|| (> 0); the residual is the CG
 *           recurrence's, FP64 norms of FP32 vectors
 *   maxit   iterations at most (>= 0); a column still above tol after maxit keeps its last iterate
 *   iters, relres  host, nrhs each (may be NULL): iterations taken and the final relative residual
 * Each iteration is one batched product (graph-replayed after the first) plus three vector kernels with
 * FP64 dot products; the host reads the nrhs residual norms once per iteration. A column with y = 0
 * returns x = 0. Synchronous. EINVAL for bad sizes or non-device pointers, ENOMEM for workspace.
 */
int addker_cg(addker_plan* plan, double beta, const float* y, float* x, int nrhs, double tol, int maxit,
              int* iters, double* relres);

/*
 * Preconditioner of addker_cg and addker_gp_grad (not in the paper, which uses plain CG). At a small beta
 * the regression system is ill-conditioned (condition number ~ N / beta for a kernel wide against the
 * data): K's large eigenvalues belong to every window's lowest Fourier modes (Sec. 3.1: the even
 * coefficients give each pair +-k the term 2 c_hat_k [cos(2 pi k.x) cos(2 pi k.x') + sin sin]). The
 * preconditioner B = beta I + U W U^T keeps, for every window, the modes |k|_inf <= band whose weight
 * sigma_f^2 2 c_hat_k times N is at least beta (plus the shared constant mode, weight sigma_f^2 sum_s c_hat_0),
 * U = their cosines and sines at the points (N x r, at most 1024 columns; FP32), and applies B^{-1} by the
 * Woodbury identity with U^T U accumulated in FP64 and factored by FP64 Cholesky. It is built on the first
 * solve for a given beta (about 0.1 s and 4 N r bytes of device memory at N = 2e6) and kept until the
 * hyperparameters, beta or this setting change; CG then runs the flexible (Polak-Ribiere) preconditioned
 * iteration. band 0 gives plain CG; 1 (the default) to 3. If no mode qualifies or the factorisation fails,
 * plain CG runs. EINVAL for band outside 0..3. Synchronises the plan's stream.
 */
int addker_set_precond(addker_plan* plan, int band);

/*
 * Gradient of the GP log marginal likelihood L = -1/2 y^T A^{-1} y - 1/2 log det A - N/2 log 2 pi,
 * A = K + beta I, with respect to (ell_1 .. ell_P, sigma_f, beta):
 *   dL/dtheta = 1/2 alpha^T (dA/dtheta) alpha - 1/2 tr(A^{-1} dA/dtheta),   alpha = A^{-1} y,
 * the trace by Hutchinson's estimator (1/m) sum_i (A^{-1} z_i)^T (dA/dtheta) z_i over the m probes
 * given in Z (the caller draws them, e.g. Rademacher). dA/d ell_s are the derivative-kernel products
 * (Sec. 3.3), dA/d sigma_f = (2/sigma_f) K, dA/d beta = I. One CG solve (addker_cg semantics, x0 = 0)
 * with the 1 + m columns [y, Z], then one fused product on [alpha, Z], then FP64 dot products.
 *   y      device, N float32;  Z  device, N x m float32 column-major (NULL if m = 0: no trace term)
 *   grad   host, P + 2 doubles out;  fit  host, 1 double out (y^T alpha; may be NULL)
 *   alpha  device, N float32 out (may be NULL);  iters  host, 1 int out: the most CG iterations of
 *          any column (may be NULL)
 * Synchronous. EINVAL / ENOMEM as addker_cg.
 */
int addker_gp_grad(addker_plan* plan, double beta, const float* y, const float* Z, int m, double tol, int maxit,
                   double* grad, double* fit, float* alpha, int* iters);

/*
 * Global sensitivity indices (Sec. 4, Algorithm "Computation of GSI") of the plan's fast-summation
 * polynomial h~(x) = sum_s sum_k c_hat_k S(k, W_s) e^{2 pi i k.x^W_s} for coefficients v (device, N
 * float32): S(k, W_s) is the adjoint NFFT of v over window s (the plan's own spread and forward
 * transform), and the variance |c_hat_k S(k, W_s)|^2 of each frequency goes to the feature subset on
 * which k is non-zero; subsets shared by several windows add up. Windows of any length (<= 3) and
 * length scale use their own coefficients (the paper's algorithm assumes equal windows; the general
 * case is the one it calls analogous). S uses the exponent sign of eq. "approx fast sum".
 * Outputs, sorted by decreasing index: feats (host, cap x 3 ints: the subset's feature indices,
 * ascending, padded with -1), rho (host, cap doubles: theta_u / total), total (host, may be NULL:
 * the total variance). Returns the number of distinct non-empty subsets (>= 0; only the first cap are
 * written) or a negative status. Synchronous.
 */
int addker_gsi(addker_plan* plan, const float* v, int cap, int* feats, double* rho, double* total);

/* Set the CUDA stream (cudaStream_t, NULL = legacy default) used by later products. */
int addker_set_stream(addker_plan* plan, void* stream);

/*
 * Kv = K v. v and Kv: device, N x nrhs float32, column-major (column j is
 * right-hand side j, leading dimension N). nrhs >= 1.
 *
 * Batches (all product entry points): right-hand sides are processed up to eight
 * at a time, each stage one launch per kernel kind for the whole group, every
 * right-hand side with its own grid slot. The plan allocates slots on demand: the
 * first call with a larger nrhs (up to 8, rounded up to a power of two)
 * synchronises the plan's stream and grows the per-window grid memory by that
 * factor. If that allocation fails the call runs one right-hand side at a
 * time instead (ADDKER_ENOMEM only if even one slot cannot be allocated). The
 * right-hand sides share the sorted points and the
 * Fourier multipliers (Sec. 3.1: the coefficients depend only on the kernel).
 */
int addker_matvec(addker_plan* plan, const float* v, float* Kv, int nrhs);

/*
 * out = (dK/d theta) v for theta selected by `param` (ADDKER_ELL(s), ADDKER_ELL_SHARED,
 * ADDKER_SIGMA_F). v and out: device, N x nrhs float32, column-major.
 */
int addker_dmatvec(addker_plan* plan, int param, const float* v, float* out, int nrhs);

/*
 * The fused product: one spreading per window gives both
 *   Kv     = K v                      (device, N x nrhs, column-major), and
 *   dKdell = dK/d ell_s v, s = 0..P-1 (device, N x P x nrhs: column s + P*j holds
 *            window s of right-hand side j, each column of length N).
 * dK/d sigma_f v is (2/sigma_f) Kv and is not written. dKdell may be NULL.
 */
int addker_matvec_all(addker_plan* plan, const float* v, float* Kv, float* dKdell, int nrhs);

/*
 * addker_matvec_all with HOST buffers (same layouts): copies v to the device,
 * runs the fused product on the plan's stream, copies Kv and dKdell back, and
 * waits for the stream. Pinned host memory makes the copies asynchronous.
 * Uses plan-owned device staging buffers (allocated on first use).
 */
int addker_matvec_all_host(addker_plan* plan, const float* v, float* Kv, float* dKdell, int nrhs);

/*
 * Vector-Jacobian product of the product K v: the gradients of f = w^T K v (K the operator as the
 * fast summation computes it, Sec. 3.1 and 3.3) with respect to v, the hyperparameters and the points.
 *   v, w         device, N floats each
 *   grad_v       device, N floats: K w  (K is symmetric)
 *   grad_theta   device, P + 1 doubles: w^T (dK/d ell_s) v for s = 0..P-1, then w^T (dK/d sigma_f) v
 *   grad_points  device, N x d floats, row-major like `points`: df/dx (a feature used by several
 *                windows gets the sum of their contributions); must not be NULL
 * The coordinate gradient differentiates the interpolation window (the NFFT's last step) at the
 * target point; with f = w^T A B A^T v it is w_k grad(A h(v))_k + v_k grad(A h(w))_k per window.
 * Nothing from earlier products is kept: the grids of v and of w are computed here (two spreads,
 * two sets of transforms). Enqueued on the plan's stream; uses the plan's window-sum scratch.
 */
int addker_vjp(addker_plan* plan, const float* v, const float* w, float* grad_v, double* grad_theta,
               float* grad_points);

/* Wait for the plan's stream; report a failed kernel as ADDKER_ECUDA. */
int addker_sync(addker_plan* plan);

/* Release the plan and every device buffer it owns. NULL is accepted. */
int addker_free(addker_plan* plan);

/* Human-readable name of a status code (static string). */
const char* addker_strerror(int status);

/*
 * Data prescaling of Sec. 3.2 for the given windows: one global factor
 *   f = (1/4 - eps_B/2) / max_{j,s} ||x_j^{W_s}||
 * so that every windowed point lands in the ball that addker_setup requires.
 * X and Xs: device, N x d float32 row-major (Xs may equal X). factor: host, out.
 * Length scales chosen for X must be multiplied by the same factor. Synchronous
 * on the given stream (NULL = legacy default).
 */
int addker_prescale(const float* X, int64_t N, int d, const int* win_off, const int* win_feat, int P,
                    double eps_B, float* Xs, double* factor, void* stream);

/*
 * Data prescaling of Sec. 3.2 in the paper's own two steps: every feature f is first mapped affinely
 * from its range [min_f, max_f] onto [-r, r] (the paper: onto [-1/4, 1/4]), then all features are
 * divided by sqrt(d_max), d_max the longest window; every windowed point then lies in the ball of
 * radius r. Here r = (1/4 - eps_B/2)(1 - 4e-7), which adds the boundary width eps_B the fast summation
 * needs and a margin for FP32 rounding. A constant feature maps to 0.
 * X and Xs: device, N x d float32 row-major (Xs may equal X). factor: host, out, = 4 r / sqrt(d_max): a
 * length scale chosen for data in [-1/4, 1/4]^d is multiplied by it (the paper's ell / sqrt(d_max)).
 * ADDKER_EDOMAIN if X holds a non-finite value. Synchronous on the given stream (NULL = legacy default).
 */
int addker_prescale_cube(const float* X, int64_t N, int d, const int* win_off, const int* win_feat, int P,
                         double eps_B, float* Xs, double* factor, void* stream);

/*
 * Plan inspection for tests and benchmarks. Writes up to `cap` int64 values into info:
 *   [0] N  [1] P  [2] number of work items over all windows  [3] bytes of device memory owned
 *   then per window s: [4+4s] d_s  [5+4s] M_s  [6+4s] n_s  [7+4s] number of non-empty cells,
 *   then [4+4P] right-hand-side slots allocated  [5+4P] captured product graphs held
 *   [6+4P] product graph replays so far  [7+4P] points per gather work item at most
 *   [8+4P] points per spread work item at most (x8 for 2-D windows)
 *   [9+4P] blocks per SM of the persistent spread (0: as many as fit)
 *   [10+4P] register tile of the 3-D spread (0: a 4 x 4 x 2 block of the 8 x 8 x 8 box per lane, 1: 8 x 2 x 2).
 * Returns the number of values available.
 */
int addker_info(const addker_plan* plan, int64_t* info, int cap);

/*
 * Stage timing for tracing and roofline accounting (not in the paper). While enabled, every
 * product records CUDA events on the plan's stream around its stages
 *   0 clearing the grids, 1 spreading, 2 the DFTs with the multiplication, 3 interpolation
 *   (gather), 4 the sum over windows
 * and counts the kernels it launches per stage. addker_profile(plan, 1) clears and starts,
 * addker_profile(plan, 0) stops. addker_profile_read waits for the stream and writes, for
 * up to `cap` stages, the summed milliseconds ms[i] and kernel launches launches[i]; it returns
 * the number of stages (5). Either output may be NULL.
 */
int addker_profile(addker_plan* plan, int enable);
int addker_profile_read(addker_plan* plan, double* ms, int64_t* launches, int cap);

/*
 * Stage-wise check of one window (tests only; synchronous): runs the steps up to `stage`
 * for right-hand side v (device, N floats) and copies a result to host doubles:
 *   stage 0: the spread grid g_l, l in I_n^{d_s} (n^{d_s} values, last axis fastest), in the
 *            normalisation of the window phi(x) = sinh(b sqrt(m^2 - n^2 x^2))/(pi sqrt(m^2 - n^2 x^2));
 *   stage 1: the adjoint NFFT result S_k ~= sum_j v_j exp(-2 pi i k.x_j), k in I_M^{d_s}
 *            (2 M^{d_s} values: real, imaginary interleaved, last axis fastest).
 * `cap` is the capacity of out in doubles. Returns ADDKER_EINVAL if it is too small.
 */
int addker_debug_stage(addker_plan* plan, int window, int stage, const float* v, double* out, int64_t cap);

/*
 * The fused product for ONE window without any device allocation. The paper has no counterpart;
 * this entry point exists for callers that cannot call cudaMalloc: servers and real-time loops that
 * forbid device allocation after start-up so that their memory use stays fixed, and hosts whose own
 * allocator owns the device memory. Every working buffer (grids, transform buffers, multipliers,
 * twiddles, the FP64 coefficient work area, the points' coordinate range) lives in one fixed 9 MiB
 * array in device memory that the library declares; every GPU that loads the library keeps it until the
 * process exits.
 *
 *   points   device, N x d float32 row-major: all d features form the window (1 <= d <= 3), each point
 *            inside the ball ||x|| <= 1/4 - eps_B/2 with eps_B = 1/16
 *   ell, sigma_f, bandwidth (M), cutoff (m): as in addker_setup, with oversampling 2, eps_B = 1/16 and
 *            the Gaussian's default reading (ADDKER_REG_SEPARABLE)
 *   v        device, N floats;  Kv, dKdell: device, N floats each (dKdell may be NULL)
 *            Kv = sigma_f^2 K v,  dKdell = sigma_f^2 (2/ell) K^der v
 *   stream   cudaStream_t (NULL = legacy default); the call waits for it before returning
 *
 * Limit: bandwidth M <= 32 (grid n = 64), d <= 3, any N (points are not sorted, so nothing grows with
 * N). Larger requests return ADDKER_ELIMIT; malformed ones ADDKER_EINVAL; a point outside the ball or
 * not finite gives ADDKER_EDOMAIN (outputs then undefined). The first call on a device looks up the
 * array's device address (once per device, with that device current). All calls share the one array and
 * it keeps the last call's contents (each call clears what must start at zero): calls that overlap on
 * the GPU, on any stream or thread, race. No cudaMalloc, cudaFree or other allocating routine is called.
 */
int addker_fastsum_noalloc(const float* points, int64_t N, int d, double ell, double sigma_f,
                           int bandwidth, int cutoff, const float* v, float* Kv, float* dKdell,
                           void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ADDKER_H */
