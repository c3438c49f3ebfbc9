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

#include <vector>

#include "../../include/addker.h"

namespace addker {

constexpr int kMaxWindows = 64;
constexpr int kItemPoints = 256;        // points per work item (one warp)
constexpr int kMaxBandwidth = 64;

struct WinDev {                          // copied by value into kernel parameter space
    const float4* pts;
    float* grid;
    float2* h;
    float4* buf1;
    float4* buf2;
    float4* spec;
    const float* bK;
    const float* bD;
    const float* dconv;                  // 1 / (n^D prod_t phi_hat(k_t)): the adjoint NFFT's deconvolution
    const float2* twf[3];                // [axis]: box[axis] x M
    const float2* twi[3];                // [axis]: M x box[axis]
    int D, M, n, m;
    int lo[3];                           // grid-array index (l + n/2) of the box origin per axis
    int box[3];
    float b;                             // Kaiser-Bessel shape pi (2 - 1/sigma)
    float wnorm;                         // 1 / (1 - exp(-2 b m))
};

struct Plan {
    int64_t N = 0;
    int d = 0, P = 0, m = 4;
    double sigma_f = 1.0, sigma_os = 2.0, eps_B = 1.0 / 16.0;
    int p_opt = -1;
    cudaStream_t stream = nullptr;
    std::vector<int> dims, bandwidth, feat_off, feat;
    std::vector<double> ell;
    std::vector<WinDev> win;              // host copies of the per-window descriptors
    WinDev* wins_dev = nullptr;           // device copy of `win`
    std::vector<int> n_cells;             // non-empty cells per window
    // items: fast 3-D kernels (D = 3, m = 4) and generic kernels, grouped by window; items of
    // window s are [begin[s], begin[s+1]) of the respective list
    int4* items_fast = nullptr;
    int4* items_gen = nullptr;
    std::vector<int> item_begin_fast, item_begin_gen;
    float* scale_dev = nullptr;           // 3P floats: [0,P) ones, [P,2P) sigma_f^2, [2P,3P) sigma_f^2 2/ell_s
    float* ks = nullptr;                  // P x N per-window K_s v, scratch for the window sum
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
};

// ---- device window function --------------------------------------------------------
// Kaiser-Bessel window in grid units t = n x - l, normalised to 1 at t = 0:
//   w(t) = (m / s) sinh(b s) / sinh(b m),   s = sqrt(m^2 - t^2),   |t| <= m.
// Written as (m/s) (e^{b(s-m)} - e^{-b(s+m)}) / (1 - e^{-2bm}) so no term overflows; for tiny s
// the series sinh(bs)/s = b (1 + (bs)^2/6) is used.
__device__ __forceinline__ float kb_weight(float t, float b, float m, float wnorm)
{
    float s2 = fmaxf(m * m - t * t, 0.0f);
    float s = sqrtf(s2);
    if (s > 1e-3f) {
        float e1 = expf(b * (s - m));
        float e2 = expf(-b * (s + m));
        return (m / s) * (e1 - e2) * wnorm;
    }
    return m * b * (1.0f + b * b * s2 * (1.0f / 6.0f)) * 2.0f * expf(-b * m) * wnorm;
}

// ---- launchers implemented in the other translation units -------------------------
// Each launcher returns the number of kernels it launched through *count (may be NULL).
cudaError_t launch_spread(const Plan& p, int window_or_all, const float* v, cudaStream_t st, int* count = nullptr);
// Outputs of window s for the point with original index i go to outK[i + s*strideK] and
// outD[i + s*strideD] (either may be NULL), scaled by scaleK[s] and scaleD[s] (device arrays).
cudaError_t launch_gather(const Plan& p, int window_or_all, float* outK, int64_t strideK, float* outD,
                          int64_t strideD, const float* scaleK, const float* scaleD, cudaStream_t st,
                          int* count = nullptr);
cudaError_t launch_fft_forward(const WinDev& w, cudaStream_t st);   // grid -> spec (two spectra), D launches
cudaError_t launch_fft_inverse(const WinDev& w, cudaStream_t st);   // spec -> h, D launches
cudaError_t launch_adjoint_only(const WinDev& w, const float* dconv, float4* out,
                                cudaStream_t st);                    // grid -> S_k (adjoint NFFT)

}  // namespace addker
