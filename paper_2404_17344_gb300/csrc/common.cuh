// Internal declarations shared by the library's translation units.
//
// Data layout in device memory, per window s (dimension D = d_s <= 3):
//   pts      N float4, the points sorted by grid cell: (x, y, z, original index as int bits);
//            unused coordinates are 0.
//   grid     the spread grid restricted to its bounding box (the only part any point touches),
//            box[0] x box[1] x box[2] floats, last axis fastest; box[t] = 1 for t >= D.
//   h        the two interpolation grids (K and K^der) on the same box, float2 per grid point.
//   buf1/2   FFT intermediates (float4 = two complex numbers), spec the two spectra.
//   bK, bD   Fourier multipliers on I_M^D (float), see coefficient precomputation.
//   twf/twi  per-axis DFT twiddles on the box (forward e^{-2 pi i k l/n}, inverse e^{+...}).
// Work items partition every window's sorted points by cell into chunks of at most
// kItemPoints points; an item is int4 {first sorted index, count, packed cell, window}.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/addker.h"

namespace addker {

constexpr int kMaxWindows = 64;
constexpr int kMaxRhsChunk = 8;         // right-hand sides processed together by one launch per stage
// kernel kinds of the item lists: m = 4 fast kernels for D = 3, 1, 2, then the generic ones for D = 1, 2, 3
enum { kKindFast3 = 0, kKindLow1 = 1, kKindLow2 = 2, kKindGen1 = 3, kKindGen2 = 4, kKindGen3 = 5, kKinds = 6 };
inline int kind_of(int D, int m) { return m == 4 ? (D == 3 ? kKindFast3 : D) : 2 + D; }
constexpr int kItemPoints = 256;        // default points per work item (one warp); see build_items
constexpr int kLowdChunkFactor = 8;     // spread items of 2-D windows hold this many times more points
constexpr int kMaxBandwidth = 64;
constexpr int kPcMaxBand = 3;           // largest |k|_inf of the CG preconditioner's Fourier modes

// Piecewise polynomial form of the window used by every spreading/interpolation kernel: for a
// coordinate with fractional grid offset frac = n x - floor(n x) in [0, 1) and u = 2 frac - 1, the
// weight of support index q (grid index floor(n x) - m + 1 + q) is a polynomial P_q(u) of degree
// kPolyDeg. The window is even, so piece W-1-q is piece q mirrored, P_{W-1-q}(u) = P_q(-u); with
// P_q(u) = E_q(u^2) + u O_q(u^2) both come from one even and one odd part:
//   w_q = E_q(u^2) + u O_q(u^2),   w_{W-1-q} = E_q(u^2) - u O_q(u^2),   q < m.
// Fitted at setup (FP64 Chebyshev interpolation of the window normalised to peak 1: Kaiser-Bessel or
// exponential of semicircle): at m = 4 degree 7 is within 4e-8 of the peak (derivative 1.1e-6), below
// the window's own NFFT error (~1e-7); degree 9 (1e-10) measured 1% slower. Passed by value, so the
// coefficients sit in the constant bank.
constexpr int kPolyDeg = 7;
constexpr int kMaxW = 16;
constexpr int kHalfCoef = (kPolyDeg + 2) / 2;    // coefficients of E_q and O_q each
struct WinPoly {
    float e[kMaxW / 2][kHalfCoef];
    float o[kMaxW / 2][kHalfCoef];
};

struct WinDev {                          // copied by value into kernel parameter space
    const float4* pts;
    float* grid;
    double* grid64;                      // compensated mode: the spread grid accumulated in FP64 (same
                                         // layout as grid, which it replaces) or NULL
    float2* h;
    float4* buf1;
    float4* buf2;
    float4* spec;
    const float* bK;
    const float* bD;
    const float* dconv;                  // 1 / (n^D prod_t phi_hat(k_t)): the adjoint NFFT's deconvolution
    const float* chat;                   // c_hat_k, the kernel's Fourier coefficients (FP32 copy; GSI)
    // per right-hand-side slots: slot r of grid and h starts at + r*gsz, of buf1 at + r*b1sz, of
    // buf2 at + r*b2sz (elements of the respective type)
    int64_t gsz, b1sz, b2sz;
    const float2* twf[3];                // [axis]: box[axis] x M
    const float2* twi[3];                // [axis]: M x box[axis]
    // the quadratic split (a window whose derivative kernel's quadratic part ||r||^2/(2 ell^2) is
    // evaluated through moments instead of the transforms): pq = 1/(2 ell^2) when split, else 0; the
    // moments of right-hand side r are mom[r * mstride + c], c = 0 .. 4: sum v, sum x v, sum y v,
    // sum z v, sum ||x||^2 v (over this window's coordinates; zeroed by every spread launch)
    double* mom;
    int64_t mstride;
    float pq;
    int D, M, n, m;
    int feat[3];                         // feature (column of the points array) of each axis
    int lo[3];                           // grid-array index (l + n/2) of the box origin per axis
    int box[3];
    float b;                             // window shape (Kaiser-Bessel b or semicircle beta; host only)
};

struct Plan {
    int64_t N = 0;
    int d = 0, P = 0, m = 4;
    double sigma_f = 1.0, sigma_os = 2.0, eps_B = 1.0 / 16.0;
    int p_opt = -1;
    int reg = ADDKER_REG_SEPARABLE;       // reading of the regularisation (addker_opts.reg, resolved)
    float* range = nullptr;               // 2d floats: per-feature [min, max] of the points (fit intervals)
    int kernel = ADDKER_KERNEL_GAUSS;     // radial profile family (addker_opts.kernel)
    int window = ADDKER_WIN_KB;           // NFFT window (addker_opts.window)
    bool comp = false;                    // compensated grid accumulation (addker_opts.compensated)
    cudaStream_t stream = nullptr;
    std::vector<int> dims, bandwidth, feat_off, feat;
    std::vector<double> ell;
    std::vector<WinDev> win;              // host copies of the per-window descriptors
    WinDev* wins_dev = nullptr;           // device copy of `win`
    std::vector<int> n_cells;             // non-empty cells per window
    // work items of all windows in one device array, grouped by kernel kind and, within a kind, by
    // window: items of window s are [item_begin[k][s], item_begin[k][s+1]) for its kind k = kind[s]
    int4* items = nullptr;
    int64_t items_cap = 0;
    int chunk = kItemPoints;              // points per work item at most (gathers)
    int chunk_sp = kItemPoints;           // points per spread work item at most (x8 for 2-D windows)
    int sp_blocks = 0;                    // blocks per SM of the persistent spreads (0: as many as fit)
    int sp_tile = 0;                      // register tile of the 3-D spread (0: 4x4x2 per lane, 1: 8x2x2)
    std::vector<std::vector<int4>> cells; // per window: non-empty cells (first point, count, packed cell, s)
    std::vector<int> item_begin[kKinds];
    std::vector<int> item_begin_sp[kKinds]; // the spread's list (larger items for 2-D windows), same array
    std::vector<int> kind;
    int slots = 0;                        // right-hand-side slots allocated per window
    std::vector<void*> slot_allocs;       // grid, h, buf1, buf2 of all slots (re-made when slots grow)
    int64_t slot_bytes = 0;
    WinPoly poly;                         // window polynomials for cutoff m and shape b
    float* scale_dev = nullptr;           // 3P floats: [0,P) ones, [P,2P) sigma_f^2, [2P,3P) sigma_f^2 2/ell_s
    float* ks = nullptr;                  // slots x P x N per-window K_s v, scratch for the window sum
    float* stage_v = nullptr;             // host-API staging (N x nrhs), allocated on demand
    float* stage_k = nullptr;
    float* stage_d = nullptr;
    int64_t stage_cap = 0;
    std::vector<void*> allocations;
    int64_t bytes = 0;
    // stage profiling (addker_profile): event pairs per recorded stage, launches per stage
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    int64_t launches[5] = {0, 0, 0, 0, 0};
    double* dots = nullptr;               // 2P doubles: gradient dot products (addker_vjp)
    int* counters = nullptr;              // work counters of the persistent kernels (16 ints), followed by
                                          // the moments of the quadratic split: kMaxRhsChunk x P x 8 doubles
                                          // (mom), then P x 8 saved by addker_vjp (mom_saved)
    double* mom = nullptr;
    double* mom_saved = nullptr;
    bool any_split = false;               // some window's quadratic part is split off
    std::vector<double> pq;               // per window: 1/(2 ell^2) when split, else 0 (FP64 copy of WinDev.pq)
    // the CG preconditioner (solver.cu): every window's lowest Fourier modes |k|_inf <= pc_band
    int pc_band = 1;                      // addker_set_precond; 0 = plain CG
    std::vector<std::vector<double>> lowc;  // per window: c_hat_k (FP64) for |k|_inf <= kPcMaxBand, index
                                            // sum_t (k_t + kPcMaxBand) (2 kPcMaxBand + 1)^(D-1-t)
    float* pc_U = nullptr;                // N x r basis (column-major), built on the first preconditioned solve
    double* pc_G = nullptr;               // U^T U (r x r)
    double* pc_L = nullptr;               // Cholesky factor of beta W^{-1} + U^T U for pc_beta (r x r)
    double* pc_w = nullptr;               // r column weights (device)
    int pc_r = 0;
    double pc_beta = -1.0;
    // CUDA graphs of repeated products (addker_set_graphs): a product whose arguments repeat those of
    // the previous call is captured once and replayed; any change of buffers or scalars clears them
    struct GraphKey {
        const float* v;
        float *Kv, *dK;
        int nrhs, window, mode;
        bool operator==(const GraphKey& o) const
        {
            return v == o.v && Kv == o.Kv && dK == o.dK && nrhs == o.nrhs && window == o.window && mode == o.mode;
        }
    };
    bool graphs = true;
    std::vector<std::pair<GraphKey, cudaGraphExec_t>> graph_cache;   // most recent last
    GraphKey last_key = {nullptr, nullptr, nullptr, 0, 0, -1};
    cudaStream_t cap_stream = nullptr;
    cudaStream_t copy_stream = nullptr;   // device-to-host copies overlapped with later gathers (host entry)
    std::vector<cudaEvent_t> win_events;  // one per window: its gather has finished
    int64_t graph_replays = 0;
};

// Launch a kernel on st. With pdl the launch carries the programmatic-serialisation attribute (the
// kernel orders its own accesses with grid_dep_wait()); only for kernels whose predecessor in the
// stream is a kernel of the same product.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args... args)
{
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = pdl ? &attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---- asynchronous staging and launch overlap (inline PTX, sm_90 and later) --------------------
// cp.async: global -> shared copies that do not hold a register; cp_async_wait_all() then a barrier
// makes them visible to the block. Sizes 4, 8 (both .ca) and 16 bytes (.cg), naturally aligned.
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Programmatic dependent launch. The transform kernels, the window sum and the scalings are launched
// with the programmatic-serialisation attribute, so each launch overlaps the end of its predecessor
// (which triggers implicitly on completion: triggering at block start measured slower, because the
// waiting blocks then occupy the SMs). grid_dep_wait() blocks until every prerequisite grid has
// completed and its writes are visible; such a kernel calls it before it reads or writes anything an
// earlier kernel touches. The spread and gather kernels (thousands of blocks) are launched plainly:
// the wait in every warp cost them more than the overlap saved.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Add x to the grid value: into the FP32 grid g, or with compensated accumulation into the FP64 grid
// g64 (when not NULL), whose sum carries no rounding error of the accumulation order (each term is an
// FP32 value; 10^4 of them add exactly to within 1e-12 relative in FP64).
__device__ __forceinline__ void grid_add(float* g, double* g64, float x)
{
    if (g64) atomicAdd(g64, (double)x);
    else atomicAdd(g, x);
}

// ---- device window weights ------------------------------------------------------------
// The W = 2m weights of one coordinate x on a grid of n points; *cell = floor(n x) + n/2.
__device__ __forceinline__ void window_pair(const WinPoly& P, int q, float u, float u2, float* lo, float* hi)
{
    float E = P.e[q][kHalfCoef - 1], O = P.o[q][kHalfCoef - 1];
#pragma unroll
    for (int i = kHalfCoef - 2; i >= 0; --i) {
        E = fmaf(E, u2, P.e[q][i]);
        O = fmaf(O, u2, P.o[q][i]);
    }
    *lo = fmaf(u, O, E);
    *hi = fmaf(-u, O, E);
}

template <int W>
__device__ __forceinline__ void window_weights(const WinPoly& P, float x, int n, float* w, int* cell)
{
    const float s = x * (float)n;
    const float fl = floorf(s);
    const float u = 2.0f * (s - fl) - 1.0f;
    const float u2 = u * u;
    *cell = (int)fl + n / 2;
#pragma unroll
    for (int q = 0; q < W / 2; ++q) window_pair(P, q, u, u2, &w[q], &w[W - 1 - q]);
}

// The moments of the quadratic split, per lane: m[0] += v, m[1..D] += x_t v, m[4] += ||x||^2 v.
template <int D>
__device__ __forceinline__ void moments_add(float* m, float x, float y, float z, float v)
{
    m[0] += v;
    m[1] = fmaf(x, v, m[1]);
    if (D >= 2) m[2] = fmaf(y, v, m[2]);
    if (D >= 3) m[3] = fmaf(z, v, m[3]);
    float r2 = x * x;
    if (D >= 2) r2 = fmaf(y, y, r2);
    if (D >= 3) r2 = fmaf(z, z, r2);
    m[4] = fmaf(r2, v, m[4]);
}

// Sum the five per-lane moments over the warp (every lane must call) and add them to dst in FP64: the
// partial sums of one work item are short, so FP32 within the item and FP64 across items keep the totals
// at FP32 accuracy relative to their own size.
__device__ __forceinline__ void moments_flush(float* m, double* dst, int lane)
{
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        float x = m[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0 && dst) atomicAdd(dst + c, (double)x);
        m[c] = 0.f;
    }
}

// The quadratic part of the derivative product at a target, pq (||x||^2 m0 - 2 x.m1 + m2), from the
// moments of right-hand side r (zero for a window that is not split).
struct Quad {
    float q0, qx, qy, qz, q2;
};
__device__ __forceinline__ Quad quad_of(const WinDev& W, int r)
{
    Quad q = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (W.pq != 0.f) {
        const double* m = W.mom + r * W.mstride;
        const double a = (double)W.pq;
        q.q0 = (float)(a * m[0]);
        q.qx = (float)(-2.0 * a * m[1]);
        q.qy = (float)(-2.0 * a * m[2]);
        q.qz = (float)(-2.0 * a * m[3]);
        q.q2 = (float)(a * m[4]);
    }
    return q;
}
template <int D>
__device__ __forceinline__ float quad_eval(const Quad& q, float x, float y, float z)
{
    float r2 = x * x;
    if (D >= 2) r2 = fmaf(y, y, r2);
    if (D >= 3) r2 = fmaf(z, z, r2);
    float t = fmaf(q.q0, r2, q.q2);
    t = fmaf(q.qx, x, t);
    if (D >= 2) t = fmaf(q.qy, y, t);
    if (D >= 3) t = fmaf(q.qz, z, t);
    return t;
}

// runtime W (generic kernels)
__device__ __forceinline__ void window_weights_n(const WinPoly& P, float x, int n, int W, float* w, int* cell)
{
    const float s = x * (float)n;
    const float fl = floorf(s);
    const float u = 2.0f * (s - fl) - 1.0f;
    const float u2 = u * u;
    *cell = (int)fl + n / 2;
    for (int q = 0; q < W / 2; ++q) window_pair(P, q, u, u2, &w[q], &w[W - 1 - q]);
}

// Weights and their x-derivatives: dw_q = dP_q/du * du/dx with du/dx = 2n. For the mirrored pair,
// with A = 2u E'(u^2) and B = O(u^2) + 2u^2 O'(u^2): dP_q/du = A + B and dP_{W-1-q}/du = A - B.
__device__ __forceinline__ void window_weights_grad_n(const WinPoly& P, float x, int n, int W, float* w, float* dw,
                                                      int* cell)
{
    const float s = x * (float)n;
    const float fl = floorf(s);
    const float u = 2.0f * (s - fl) - 1.0f;
    const float u2 = u * u;
    const float dudx = 2.0f * (float)n;
    *cell = (int)fl + n / 2;
    for (int q = 0; q < W / 2; ++q) {
        float E = P.e[q][kHalfCoef - 1], O = P.o[q][kHalfCoef - 1];
        float dE = (kHalfCoef - 1) * P.e[q][kHalfCoef - 1], dO = (kHalfCoef - 1) * P.o[q][kHalfCoef - 1];
        for (int i = kHalfCoef - 2; i >= 0; --i) {
            E = fmaf(E, u2, P.e[q][i]);
            O = fmaf(O, u2, P.o[q][i]);
            if (i >= 1) {
                dE = fmaf(dE, u2, (float)i * P.e[q][i]);
                dO = fmaf(dO, u2, (float)i * P.o[q][i]);
            }
        }
        w[q] = fmaf(u, O, E);
        w[W - 1 - q] = fmaf(-u, O, E);
        const float A = 2.0f * u * dE;
        const float B = fmaf(2.0f * u2, dO, O);
        dw[q] = (A + B) * dudx;
        dw[W - 1 - q] = (A - B) * dudx;
    }
}

// ---- launchers implemented in the other translation units -------------------------
// Each launcher returns the number of kernels it launched through *count (may be NULL). All of them
// process nrhs (<= kMaxRhsChunk) right-hand sides: rhs r reads v + r*ldv and uses slot r of the grids.
cudaError_t launch_spread(const Plan& p, int window_or_all, const float* v, int64_t ldv, int nrhs, cudaStream_t st,
                          int* count = nullptr);
// Outputs of window s for rhs r and the point with original index i go to
// outK[i + s*strideK + r*rstrideK] and outD[i + s*strideD + r*rstrideD] (either may be NULL), scaled by
// scaleK[s] and scaleD[s] (device arrays).
cudaError_t launch_gather(const Plan& p, int window_or_all, float* outK, int64_t strideK, int64_t rstrideK,
                          float* outD, int64_t strideD, int64_t rstrideD, int nrhs, const float* scaleK,
                          const float* scaleD, cudaStream_t st, int* count = nullptr);
// Gradient gathers of addker_vjp (gradients.cu). Pass 0 reads the grids of w: writes f^K to
// ks[s N + i], accumulates dots[s] += v_i f^K, dots[P + s] += v_i f^D and
// grad_x[i d + feat] += sigma_f^2 v_i grad f^K. Pass 1 reads the grids of v and accumulates
// grad_x[i d + feat] += sigma_f^2 w_i grad f^K.
cudaError_t launch_gather_grad(const Plan& p, int pass, const float* other, float* ks, float* grad_x,
                               cudaStream_t st, int* count);

// Products of a plan (addker.cu): nrhs columns v + j N, mode 0 fused (Kv and/or dK), 1 one window's
// derivative, 2 the shared-length-scale derivative; chunked, graph-replayed when repeated.
int product_all(Plan& p, const float* v, int nrhs, float* Kv, float* dK, int window, int mode);
// Regression system and GP training (solver.cu).
int cg_solve(Plan& p, double beta, const float* Y, float* X, int nrhs, double tol, int maxit, int* iters,
             double* relres);
int gp_grad(Plan& p, double beta, const float* y, const float* Z, int m, double tol, int maxit, double* grad,
            double* fit, float* alpha_out, int* iters);

// The CG preconditioner's device buffers (solver.cu): released here and rebuilt on the next solve.
void pc_release(Plan& p);

// Global sensitivity indices (gsi.cu): returns the number of feature subsets (or a negative status).
int gsi_run(Plan& p, const float* v, int cap, int* feats, double* rho, double* total);

// Building blocks used without a plan (addker_fastsum_noalloc).
void window_poly_for(int m, double sigma_os, WinPoly* poly);
int multipliers_with_scratch(const WinDev& w, double ell, double eps_B, const float* range, const WinPoly& poly,
                             double* scratch, cudaStream_t st, float* pq);
cudaError_t feature_range_async(const float* X, int64_t N, int d, float* range, int* bad, cudaStream_t st);
cudaError_t twiddles_into(const WinDev& w, float2* const tw[3], cudaStream_t st);
cudaError_t launch_transforms_window(const WinDev& w, const WinDev* w_dev, cudaStream_t st);

// grid -> (multiply) -> h for one window or all (window < 0) and nrhs slots. spec_only: stop after
// the forward transform and write S_k = G_k dconv_k (the adjoint NFFT) to slot 0's spec.
cudaError_t launch_transforms(const Plan& p, int window_or_all, int nrhs, cudaStream_t st, int* count, bool spec_only);

}  // namespace addker
