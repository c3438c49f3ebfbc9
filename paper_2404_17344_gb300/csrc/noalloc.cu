// addker_fastsum_noalloc: the fused product for one window without allocating device memory.
//
// Some callers cannot call cudaMalloc: inference servers and real-time loops that forbid device
// allocation after start-up so that their memory use stays fixed, and hosts whose own allocator owns
// all device memory (a caching pool that must not be bypassed). For them this entry point takes every
// working buffer from one fixed array in device memory, declared below at file scope. Every GPU that
// loads the library keeps that array for the life of the process.
//
// The array's limit: one window of d <= 3 features, bandwidth M <= 32 (grid n = 2M <= 64), any N
// (the points are not sorted, so no buffer grows with N); the layout below must fit kScratchBytes.
// The variant kernels here spread point by point with atomics into the fixed grid and interpolate
// point by point; the coefficient precomputation (the separable reading, with the fit intervals taken
// from the points' largest |coordinate| per axis) and the transforms are the plan path's own kernels.
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace addker {

namespace {

constexpr size_t kScratchBytes = 9u << 20;                 // 9 MiB
constexpr int kNoallocMaxBandwidth = 32;
constexpr int kMaxDevices = 64;

// The fixed working memory. In host code this name is only a stand-in: its device address comes
// from cudaGetSymbolAddress (see scratch_for_current_device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of g_noalloc_scratch for the current device, looked up once per device.
int scratch_for_current_device(unsigned char** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ADDKER_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return ADDKER_ECUDA;
        }
        g_scratch_addr[dev] = ptr;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return ADDKER_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Spreading, one thread per (unsorted) point, atomics into the full n^D grid. A point whose support
// would leave the grid (outside the ball, or not finite) is skipped and raises *flag. With mom (not
// NULL) the block also adds the moments of the quadratic split (sum v, sum x v, sum ||x||^2 v) to mom[0..5);
// no thread leaves early, so the block's reductions see every lane.
template <int D>
__global__ void __launch_bounds__(128) k_na_spread(const float* __restrict__ X, int64_t N, const float* __restrict__ v,
                                                   float* grid, int n, int m, float rho2, const WinPoly poly, int* flag,
                                                   double* mom)
{
    __shared__ float part[4][5];
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int W = 2 * m;
    float w[3][kMaxW];
    int cell[3] = {0, 0, 0};
    float xs[3] = {0.f, 0.f, 0.f};
    bool ok = j < N;
    if (ok) {
        float r2 = 0.f;
        for (int t = 0; t < D; ++t) {
            xs[t] = X[j * D + t];
            r2 = fmaf(xs[t], xs[t], r2);
        }
        ok = r2 <= rho2;                                       // same ball as addker_setup checks
        for (int t = 0; t < D && ok; ++t) {
            ok = fabsf(xs[t]) < 0.5f;
            if (!ok) break;
            window_weights_n(poly, xs[t], n, W, w[t], &cell[t]);
            ok = cell[t] - m + 1 >= 0 && cell[t] + m <= n - 1;
        }
        if (!ok) atomicOr(flag, 1);
    }
    const float vj = ok ? v[j] : 0.f;
    if (ok) {
        for (int a = 0; a < W; ++a) {
            const int ia = cell[0] - m + 1 + a;
            if (D == 1) { atomicAdd(grid + ia, vj * w[0][a]); continue; }
            for (int b = 0; b < W; ++b) {
                const int ib = cell[1] - m + 1 + b;
                const float vab = vj * w[0][a] * w[1][b];
                if (D == 2) { atomicAdd(grid + (size_t)ia * n + ib, vab); continue; }
                float* row = grid + ((size_t)ia * n + ib) * n + (cell[2] - m + 1);
                for (int c = 0; c < W; ++c) atomicAdd(row + c, vab * w[2][c]);
            }
        }
    }
    if (mom) {                                                  // block-uniform
        float mm[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        moments_add<D>(mm, xs[0], xs[1], xs[2], vj);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int c = 0; c < 5; ++c) {
            float x = mm[c];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) part[warp][c] = x;
        }
        __syncthreads();
        if (threadIdx.x < 5) {
            const float t = part[0][threadIdx.x] + part[1][threadIdx.x] + part[2][threadIdx.x] + part[3][threadIdx.x];
            atomicAdd(mom + threadIdx.x, (double)t);
        }
    }
}

// Interpolation, one thread per point: Kv = sK f^K, dK = sD f^der.
// A split window (pq != 0) adds pq (||x||^2 m0 - 2 x.m1 + m2) to the derivative product.
template <int D>
__global__ void k_na_gather(const float* __restrict__ X, int64_t N, const float2* __restrict__ h, int n, int m,
                            const WinPoly poly, float sK, float sD, float* __restrict__ Kv, float* __restrict__ dK,
                            const double* __restrict__ mom, float pq)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int W = 2 * m;
    float w[3][kMaxW];
    int cell[3] = {0, 0, 0};
    for (int t = 0; t < D; ++t) {
        const float x = X[j * D + t];
        if (!(fabsf(x) < 0.5f)) return;
        window_weights_n(poly, x, n, W, w[t], &cell[t]);
        if (cell[t] - m + 1 < 0 || cell[t] + m > n - 1) return;
    }
    float fK = 0.f, fD = 0.f;
    for (int a = 0; a < W; ++a) {
        const int ia = cell[0] - m + 1 + a;
        float uK = 0.f, uD = 0.f;
        for (int b = 0; b < (D >= 2 ? W : 1); ++b) {
            const int ib = D >= 2 ? cell[1] - m + 1 + b : 0;
            float tK = 0.f, tD = 0.f;
            for (int c = 0; c < (D >= 3 ? W : 1); ++c) {
                const int ic = D >= 3 ? cell[2] - m + 1 + c : 0;
                size_t g = (size_t)ia;
                if (D >= 2) g = g * n + ib;
                if (D >= 3) g = g * n + ic;
                const float2 hv = h[g];
                const float wc = D >= 3 ? w[2][c] : 1.f;
                tK = fmaf(hv.x, wc, tK);
                tD = fmaf(hv.y, wc, tD);
            }
            const float wb = D >= 2 ? w[1][b] : 1.f;
            uK = fmaf(tK, wb, uK);
            uD = fmaf(tD, wb, uD);
        }
        fK = fmaf(uK, w[0][a], fK);
        fD = fmaf(uD, w[0][a], fD);
    }
    Kv[j] = sK * fK;
    if (dK) {
        float qd = 0.f;
        if (pq != 0.f) {
            const double a = (double)pq;
            const Quad q = {(float)(a * mom[0]), (float)(-2.0 * a * mom[1]), (float)(-2.0 * a * mom[2]),
                            (float)(-2.0 * a * mom[3]), (float)(a * mom[4])};
            qd = quad_eval<D>(q, X[j * D], D >= 2 ? X[j * D + 1] : 0.f, D >= 3 ? X[j * D + 2] : 0.f);
        }
        dK[j] = sD * (fD + qd);
    }
}

}  // namespace
}  // namespace addker

using namespace addker;

extern "C" int addker_fastsum_noalloc(const float* points, int64_t N, int d, double ell, double sigma_f,
                                      int bandwidth, int cutoff, const float* v, float* Kv, float* dKdell,
                                      void* stream)
{
    if (!points || !v || !Kv || N < 1 || d < 1 || d > 3 || !(ell > 0.0) || !(sigma_f > 0.0)) return ADDKER_EINVAL;
    if (bandwidth < 4 || (bandwidth & 1) || cutoff < 2 || cutoff > 8) return ADDKER_EINVAL;
    if (bandwidth > kNoallocMaxBandwidth) return ADDKER_ELIMIT;
    const double eps_B = 1.0 / 16.0, sigma_os = 2.0;
    const int M = bandwidth, n = 2 * M, D = d;
    if (cutoff + 1 > n / 4.0 + n * eps_B / 2.0) return ADDKER_EINVAL;

    // layout of the fixed array for this request
    int64_t nd = 1, md = 1;
    for (int t = 0; t < D; ++t) { nd *= n; md *= M; }
    const int64_t b0 = n, b1 = D >= 2 ? n : 1;
    size_t off = 0;
    const size_t o_grid = off; off = align256(off + sizeof(float) * nd);
    const size_t o_h = off;    off = align256(off + sizeof(float2) * nd);
    const size_t o_b1 = off;   off = align256(off + sizeof(float4) * (D == 3 ? b0 * std::max<int64_t>(b1, M) * M : b0 * M));
    const size_t o_b2 = off;   off = align256(off + sizeof(float4) * (D == 3 ? b0 * M * M : 1));
    const size_t o_spec = off; off = align256(off + sizeof(float4) * md);
    const size_t o_mult = off; off = align256(off + sizeof(float) * 3 * md);
    const size_t o_tw = off;   off = align256(off + sizeof(float2) * 2 * (size_t)n * M * D);
    const size_t o_coef = off; off = align256(off + sizeof(double) * (3 * md + 6 * M));
    const size_t o_mom = off;  off = align256(off + sizeof(double) * 8);
    const size_t o_win = off;  off = align256(off + sizeof(WinDev));
    const size_t o_flag = off; off = align256(off + sizeof(int));
    const size_t o_range = off; off = align256(off + sizeof(float) * 2 * 3 + sizeof(int));
    if (off > kScratchBytes) return ADDKER_ELIMIT;

    unsigned char* base = nullptr;
    const int st_ok = scratch_for_current_device(&base);
    if (st_ok != ADDKER_OK) return st_ok;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    WinDev w;
    std::memset(&w, 0, sizeof(w));
    w.D = D;
    w.M = M;
    w.n = n;
    w.m = cutoff;
    w.b = (float)(M_PI * (2.0 - 1.0 / sigma_os));
    for (int t = 0; t < 3; ++t) {
        w.lo[t] = 0;
        w.box[t] = t < D ? n : 1;
    }
    w.gsz = nd;                                                // one right-hand side: slot 0 only
    w.grid = reinterpret_cast<float*>(base + o_grid);
    w.h = reinterpret_cast<float2*>(base + o_h);
    w.buf1 = reinterpret_cast<float4*>(base + o_b1);
    w.buf2 = reinterpret_cast<float4*>(base + o_b2);
    w.spec = reinterpret_cast<float4*>(base + o_spec);
    float* mult = reinterpret_cast<float*>(base + o_mult);
    w.bK = mult;
    w.bD = mult + md;
    w.dconv = mult + 2 * md;
    float2* tw[3] = {nullptr, nullptr, nullptr};
    for (int t = 0; t < D; ++t) {
        tw[t] = reinterpret_cast<float2*>(base + o_tw) + (size_t)t * 2 * n * M;
        w.twf[t] = tw[t];
        w.twi[t] = tw[t] + (size_t)n * M;
    }
    WinDev* w_dev = reinterpret_cast<WinDev*>(base + o_win);
    int* flag = reinterpret_cast<int*>(base + o_flag);
    float* range = reinterpret_cast<float*>(base + o_range);
    double* mom = reinterpret_cast<double*>(base + o_mom);
    int* bad = reinterpret_cast<int*>(range + 2 * 3);

    WinPoly poly;
    window_poly_for(cutoff, sigma_os, &poly);
    // the array keeps the previous call's contents: clear the grid and the flag
    if (cudaMemsetAsync(w.grid, 0, sizeof(float) * nd, st) != cudaSuccess) return ADDKER_ECUDA;
    if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return ADDKER_ECUDA;
    if (cudaMemsetAsync(mom, 0, sizeof(double) * 8, st) != cudaSuccess) return ADDKER_ECUDA;
    if (cudaMemcpyAsync(w_dev, &w, sizeof(WinDev), cudaMemcpyHostToDevice, st) != cudaSuccess) return ADDKER_ECUDA;
    if (twiddles_into(w, tw, st) != cudaSuccess) return ADDKER_ECUDA;
    // the separable reading's fit intervals come from the points' largest |coordinate| per axis
    if (feature_range_async(points, N, D, range, bad, st) != cudaSuccess) return ADDKER_ECUDA;
    float pq = 0.f;                                            // the quadratic split's weight, or 0
    const int mst = multipliers_with_scratch(w, ell, eps_B, range, poly, reinterpret_cast<double*>(base + o_coef), st,
                                             &pq);
    if (mst != ADDKER_OK) return mst;
    double* mom_used = pq != 0.f ? mom : nullptr;

    const int th = 128, bl = (int)((N + th - 1) / th);
    const double rho = 0.25 - eps_B / 2.0;
    const float rho2 = (float)(rho * rho * (1.0 + 4e-6));
    if (D == 1) k_na_spread<1><<<bl, th, 0, st>>>(points, N, v, w.grid, n, cutoff, rho2, poly, flag, mom_used);
    else if (D == 2) k_na_spread<2><<<bl, th, 0, st>>>(points, N, v, w.grid, n, cutoff, rho2, poly, flag, mom_used);
    else k_na_spread<3><<<bl, th, 0, st>>>(points, N, v, w.grid, n, cutoff, rho2, poly, flag, mom_used);
    if (cudaGetLastError() != cudaSuccess) return ADDKER_ECUDA;
    if (launch_transforms_window(w, w_dev, st) != cudaSuccess) return ADDKER_ECUDA;
    const float sK = (float)(sigma_f * sigma_f), sD = (float)(sigma_f * sigma_f * 2.0 / ell);
    if (D == 1) k_na_gather<1><<<bl, th, 0, st>>>(points, N, w.h, n, cutoff, poly, sK, sD, Kv, dKdell, mom, pq);
    else if (D == 2) k_na_gather<2><<<bl, th, 0, st>>>(points, N, w.h, n, cutoff, poly, sK, sD, Kv, dKdell, mom, pq);
    else k_na_gather<3><<<bl, th, 0, st>>>(points, N, w.h, n, cutoff, poly, sK, sD, Kv, dKdell, mom, pq);
    if (cudaGetLastError() != cudaSuccess) return ADDKER_ECUDA;
    int hflag = 0;
    if (cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return ADDKER_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ADDKER_ECUDA;
    return hflag ? ADDKER_EDOMAIN : ADDKER_OK;
}
