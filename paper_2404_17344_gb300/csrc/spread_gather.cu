// Spreading (adjoint NFFT, first step) and interpolation (NFFT, last step) kernels.
//
//   spread:  g_l   = sum_j v_j prod_t w(n x_{j,t} - l_t),   l in the support of x_j
//   gather:  f_i   = sum_l h_l prod_t w(n x_{i,t} - l_t)     for the two grids h^K and h^der
// (Sec. 3.1, eq. "approx fast sum": the inner sums by an adjoint NFFT, the outer sums by an
// NFFT). w is the normalised Kaiser-Bessel window; the support of x along an axis is the 2m
// grid indices floor(n x) - m + 1 .. floor(n x) + m.
//
// Points are sorted by grid cell, so all points of a work item share one support box of
// (2m)^D grid points. The fast kernels (D = 3, m = 4) exploit that:
//   spread: a warp accumulates the item's 8x8x8 box in registers as a sum of outer products
//           (v_j w_x) (x) (w_y (x) w_z) and adds it to the grid once per item;
//   gather: a warp stages the item's 8x8x8 box of both grids in shared memory and every lane
//           contracts it with its own point's weights (broadcast reads, no atomics).
#include "common.cuh"

namespace addker {

namespace {

constexpr int kWarps = 8;                 // warps per block in the item kernels

__device__ __forceinline__ void point_weights(float x, int n, int m, float b, float wnorm, int W,
                                              float* w, int* cell)
{
    float u = x * (float)n;
    float fl = floorf(u);
    float frac = u - fl;
    *cell = (int)fl + n / 2;
    for (int q = 0; q < W; ++q) w[q] = kb_weight(frac + (float)(m - 1 - q), b, (float)m, wnorm);
}

// ----------------------------------------------------------------------------------
// fast 3-D spread, m = 4 (W = 8)
// lane owns the (b, c) pairs (lane >> 3, lane & 7) and (4 + (lane >> 3), lane & 7) for all a.
__global__ void __launch_bounds__(kWarps * 32) k_spread3_w8(const int4* __restrict__ items, int nitems,
                                                           const WinDev* __restrict__ wins,
                                                           const float* __restrict__ v)
{
    constexpr int W = 8;
    constexpr int STRIDE = 28;            // floats per staged point: wx*v[8] wy[8] wz[8] pad[4]
    __shared__ __align__(16) float sw[kWarps][32 * STRIDE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * kWarps + warp;
    if (item >= nitems) return;
    const int4 it = items[item];
    const WinDev& P = wins[it.w];
    const float4* __restrict__ pts = P.pts + it.x;
    const int count = it.y;
    float* ws = sw[warp];
    const int c = lane & 7, b0 = lane >> 3;

    float acc0[W], acc1[W];
#pragma unroll
    for (int a = 0; a < W; ++a) { acc0[a] = 0.f; acc1[a] = 0.f; }

    for (int base = 0; base < count; base += 32) {
        const int k = base + lane;
        float wx[W], wy[W], wz[W];
        if (k < count) {
            float4 p = pts[k];
            float vv = __ldg(v + __float_as_int(p.w));
            int cx, cy, cz;
            point_weights(p.x, P.n, 4, P.b, P.wnorm, W, wx, &cx);
            point_weights(p.y, P.n, 4, P.b, P.wnorm, W, wy, &cy);
            point_weights(p.z, P.n, 4, P.b, P.wnorm, W, wz, &cz);
#pragma unroll
            for (int q = 0; q < W; ++q) wx[q] *= vv;
        } else {
#pragma unroll
            for (int q = 0; q < W; ++q) { wx[q] = 0.f; wy[q] = 0.f; wz[q] = 0.f; }
        }
        float4* dst = reinterpret_cast<float4*>(ws + lane * STRIDE);
        dst[0] = make_float4(wx[0], wx[1], wx[2], wx[3]);
        dst[1] = make_float4(wx[4], wx[5], wx[6], wx[7]);
        dst[2] = make_float4(wy[0], wy[1], wy[2], wy[3]);
        dst[3] = make_float4(wy[4], wy[5], wy[6], wy[7]);
        dst[4] = make_float4(wz[0], wz[1], wz[2], wz[3]);
        dst[5] = make_float4(wz[4], wz[5], wz[6], wz[7]);
        __syncwarp();
        const int cnt = min(32, count - base);
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            const float* src = ws + j * STRIDE;
            float4 xa = *reinterpret_cast<const float4*>(src);
            float4 xb = *reinterpret_cast<const float4*>(src + 4);
            float B0 = src[8 + b0] * src[16 + c];
            float B1 = src[12 + b0] * src[16 + c];
            float xv[W] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
            for (int a = 0; a < W; ++a) {
                acc0[a] = fmaf(xv[a], B0, acc0[a]);
                acc1[a] = fmaf(xv[a], B1, acc1[a]);
            }
        }
        __syncwarp();
    }
    // flush: grid index of (a, b, c) relative to the box origin
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff, cz = (it.z >> 16) & 0xff;
    const int ox = cx - 3 - P.lo[0], oy = cy - 3 - P.lo[1], oz = cz - 3 - P.lo[2];
    const int sy = P.box[2], sx = P.box[1] * P.box[2];
    float* g0 = P.grid + (size_t)ox * sx + (size_t)(oy + b0) * sy + oz + c;
    float* g1 = g0 + 4 * sy;
#pragma unroll
    for (int a = 0; a < W; ++a) {
        atomicAdd(g0 + (size_t)a * sx, acc0[a]);
        atomicAdd(g1 + (size_t)a * sx, acc1[a]);
    }
}

// ----------------------------------------------------------------------------------
// fast 3-D gather, m = 4 (W = 8): lanes own points; the item's box of both grids is staged in
// shared memory as float2 (h^K, h^der) and read back as float4 pairs (broadcast).
template <bool WK, bool WD>
__global__ void __launch_bounds__(kWarps * 32, 2) k_gather3_w8(const int4* __restrict__ items, int nitems,
                                                           const WinDev* __restrict__ wins,
                                                           float* __restrict__ outK, float* __restrict__ outD,
                                                           const float* __restrict__ scaleK,
                                                           const float* __restrict__ scaleD, int64_t strideK,
                                                           int64_t strideD)
{
    constexpr int W = 8;
    __shared__ __align__(16) float2 tile[kWarps][W * W * W];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * kWarps + warp;
    if (item >= nitems) return;
    const int4 it = items[item];
    const WinDev& P = wins[it.w];
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff, cz = (it.z >> 16) & 0xff;
    const int ox = cx - 3 - P.lo[0], oy = cy - 3 - P.lo[1], oz = cz - 3 - P.lo[2];
    const int sy = P.box[2], sx = P.box[1] * P.box[2];
    const float2* __restrict__ h = P.h + (size_t)ox * sx + (size_t)oy * sy + oz;
    float2* t = tile[warp];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        int idx = lane + 32 * i;
        int a = idx >> 6, bb = (idx >> 3) & 7, cc = idx & 7;
        t[idx] = h[(size_t)a * sx + (size_t)bb * sy + cc];
    }
    __syncwarp();
    const float4* t4 = reinterpret_cast<const float4*>(t);
    const float4* __restrict__ pts = P.pts + it.x;
    const float sK = WK ? scaleK[it.w] : 0.f;
    const float sD = WD ? scaleD[it.w] : 0.f;
    for (int k = lane; k < it.y; k += 32) {
        float4 p = pts[k];
        float wx[W], wy[W], wz[W];
        int c0, c1, c2;
        point_weights(p.x, P.n, 4, P.b, P.wnorm, W, wx, &c0);
        point_weights(p.y, P.n, 4, P.b, P.wnorm, W, wy, &c1);
        point_weights(p.z, P.n, 4, P.b, P.wnorm, W, wz, &c2);
        float fK = 0.f, fD = 0.f;
#pragma unroll 1
        for (int a = 0; a < W; ++a) {
            float uK = 0.f, uD = 0.f;
#pragma unroll
            for (int bb = 0; bb < W; ++bb) {
                float tK = 0.f, tD = 0.f;
#pragma unroll
                for (int cc = 0; cc < W; cc += 2) {
                    float4 hv = t4[(a * 64 + bb * 8 + cc) >> 1];
                    tK = fmaf(hv.x, wz[cc], tK);
                    tD = fmaf(hv.y, wz[cc], tD);
                    tK = fmaf(hv.z, wz[cc + 1], tK);
                    tD = fmaf(hv.w, wz[cc + 1], tD);
                }
                uK = fmaf(tK, wy[bb], uK);
                uD = fmaf(tD, wy[bb], uD);
            }
            fK = fmaf(uK, wx[a], fK);
            fD = fmaf(uD, wx[a], fD);
        }
        const int64_t i = (int64_t)__float_as_int(p.w);
        if (WK) outK[i + (int64_t)it.w * strideK] = sK * fK;
        if (WD) outD[i + (int64_t)it.w * strideD] = sD * fD;
    }
}

// ----------------------------------------------------------------------------------
// generic kernels: any D in {1,2,3}, W = 2m <= 16. One block per item; the spread accumulates
// the item's W^D support box in shared memory, then adds it to the grid.
template <int D>
__global__ void __launch_bounds__(256) k_spread_generic(const int4* __restrict__ items,
                                                        const WinDev* __restrict__ wins,
                                                        const float* __restrict__ v)
{
    __shared__ float box[16 * 16 * 16];
    const int4 it = items[blockIdx.x];
    const WinDev& P = wins[it.w];
    const int W = 2 * P.m;
    int WD = W;
    if (D >= 2) WD *= W;
    if (D >= 3) WD *= W;
    for (int i = threadIdx.x; i < WD; i += blockDim.x) box[i] = 0.f;
    __syncthreads();
    for (int k = threadIdx.x; k < it.y; k += blockDim.x) {
        float4 p = P.pts[it.x + k];
        float vv = __ldg(v + __float_as_int(p.w));
        float w0[16], w1[16], w2[16];
        int c;
        point_weights(p.x, P.n, P.m, P.b, P.wnorm, W, w0, &c);
        if (D >= 2) point_weights(p.y, P.n, P.m, P.b, P.wnorm, W, w1, &c);
        if (D >= 3) point_weights(p.z, P.n, P.m, P.b, P.wnorm, W, w2, &c);
        for (int a = 0; a < W; ++a) {
            float va = vv * w0[a];
            if (D == 1) { atomicAdd(&box[a], va); continue; }
            for (int bb = 0; bb < W; ++bb) {
                float vab = va * w1[bb];
                if (D == 2) { atomicAdd(&box[a * W + bb], vab); continue; }
                for (int cc = 0; cc < W; ++cc) atomicAdd(&box[(a * W + bb) * W + cc], vab * w2[cc]);
            }
        }
    }
    __syncthreads();
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff, cz = (it.z >> 16) & 0xff;
    const int ox = cx - P.m + 1 - P.lo[0], oy = cy - P.m + 1 - P.lo[1], oz = cz - P.m + 1 - P.lo[2];
    for (int i = threadIdx.x; i < WD; i += blockDim.x) {
        int a = i, bb = 0, cc = 0;
        if (D == 2) { a = i / W; bb = i % W; }
        if (D == 3) { a = i / (W * W); bb = (i / W) % W; cc = i % W; }
        size_t g = ((size_t)(ox + a) * P.box[1] + (D >= 2 ? oy + bb : 0)) * P.box[2] + (D >= 3 ? oz + cc : 0);
        if (box[i] != 0.f) atomicAdd(P.grid + g, box[i]);
    }
}

template <int D, bool WK, bool WD>
__global__ void __launch_bounds__(256) k_gather_generic(const int4* __restrict__ items,
                                                        const WinDev* __restrict__ wins,
                                                        float* __restrict__ outK, float* __restrict__ outD,
                                                        const float* __restrict__ scaleK,
                                                        const float* __restrict__ scaleD, int64_t strideK,
                                                        int64_t strideD)
{
    const int4 it = items[blockIdx.x];
    const WinDev& P = wins[it.w];
    const int W = 2 * P.m;
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff, cz = (it.z >> 16) & 0xff;
    const int ox = cx - P.m + 1 - P.lo[0], oy = cy - P.m + 1 - P.lo[1], oz = cz - P.m + 1 - P.lo[2];
    for (int k = threadIdx.x; k < it.y; k += blockDim.x) {
        float4 p = P.pts[it.x + k];
        float w0[16], w1[16], w2[16];
        int c;
        point_weights(p.x, P.n, P.m, P.b, P.wnorm, W, w0, &c);
        if (D >= 2) point_weights(p.y, P.n, P.m, P.b, P.wnorm, W, w1, &c);
        if (D >= 3) point_weights(p.z, P.n, P.m, P.b, P.wnorm, W, w2, &c);
        float fK = 0.f, fD = 0.f;
        for (int a = 0; a < W; ++a) {
            float uK = 0.f, uD = 0.f;
            for (int bb = 0; bb < (D >= 2 ? W : 1); ++bb) {
                float tK = 0.f, tD = 0.f;
                for (int cc = 0; cc < (D >= 3 ? W : 1); ++cc) {
                    size_t g = ((size_t)(ox + a) * P.box[1] + (D >= 2 ? oy + bb : 0)) * P.box[2] +
                               (D >= 3 ? oz + cc : 0);
                    float2 hv = P.h[g];
                    float wc = D >= 3 ? w2[cc] : 1.f;
                    tK = fmaf(hv.x, wc, tK);
                    tD = fmaf(hv.y, wc, tD);
                }
                float wb = D >= 2 ? w1[bb] : 1.f;
                uK = fmaf(tK, wb, uK);
                uD = fmaf(tD, wb, uD);
            }
            fK = fmaf(uK, w0[a], fK);
            fD = fmaf(uD, w0[a], fD);
        }
        const int64_t i = (int64_t)__float_as_int(p.w);
        if (WK) outK[i + (int64_t)it.w * strideK] = scaleK[it.w] * fK;
        if (WD) outD[i + (int64_t)it.w * strideD] = scaleD[it.w] * fD;
    }
}

}  // namespace

// Item ranges: items of window s are [begin[s], begin[s+1]) in each list; window < 0 = all.
static void item_range(const std::vector<int>& begin, int window, int* lo, int* hi)
{
    if (window < 0) { *lo = begin.front(); *hi = begin.back(); }
    else { *lo = begin[window]; *hi = begin[window + 1]; }
}

cudaError_t launch_spread(const Plan& p, int window, const float* v, cudaStream_t st, int* count)
{
    int launched = 0;
    const WinDev* wd = p.wins_dev;
    int lo, hi;
    item_range(p.item_begin_fast, window, &lo, &hi);
    if (hi > lo) {
        int n = hi - lo;
        k_spread3_w8<<<(n + kWarps - 1) / kWarps, kWarps * 32, 0, st>>>(p.items_fast + lo, n, wd, v);
        ++launched;
    }
    const std::vector<int>& gb = p.item_begin_gen;
    for (int s = 0; s < p.P; ++s) {
        if (window >= 0 && s != window) continue;
        int n = gb[s + 1] - gb[s];
        if (n == 0) continue;
        const int4* it = p.items_gen + gb[s];
        switch (p.dims[s]) {
            case 1: k_spread_generic<1><<<n, 128, 0, st>>>(it, wd, v); break;
            case 2: k_spread_generic<2><<<n, 128, 0, st>>>(it, wd, v); break;
            default: k_spread_generic<3><<<n, 128, 0, st>>>(it, wd, v); break;
        }
        ++launched;
    }
    if (count) *count = launched;
    return cudaGetLastError();
}

template <bool WK, bool WD>
static int gather_all(const Plan& p, int window, float* outK, int64_t zK, float* outD, int64_t zD,
                      const float* sK, const float* sD, cudaStream_t st)
{
    int launched = 0;
    const WinDev* wd = p.wins_dev;
    int lo, hi;
    item_range(p.item_begin_fast, window, &lo, &hi);
    if (hi > lo) {
        int n = hi - lo;
        k_gather3_w8<WK, WD><<<(n + kWarps - 1) / kWarps, kWarps * 32, 0, st>>>(p.items_fast + lo, n, wd, outK, outD,
                                                                               sK, sD, zK, zD);
        ++launched;
    }
    const std::vector<int>& gb = p.item_begin_gen;
    for (int s = 0; s < p.P; ++s) {
        if (window >= 0 && s != window) continue;
        int n = gb[s + 1] - gb[s];
        if (n == 0) continue;
        const int4* it = p.items_gen + gb[s];
        switch (p.dims[s]) {
            case 1: k_gather_generic<1, WK, WD><<<n, 128, 0, st>>>(it, wd, outK, outD, sK, sD, zK, zD); break;
            case 2: k_gather_generic<2, WK, WD><<<n, 128, 0, st>>>(it, wd, outK, outD, sK, sD, zK, zD); break;
            default: k_gather_generic<3, WK, WD><<<n, 128, 0, st>>>(it, wd, outK, outD, sK, sD, zK, zD); break;
        }
        ++launched;
    }
    return launched;
}

cudaError_t launch_gather(const Plan& p, int window, float* outK, int64_t zK, float* outD, int64_t zD,
                          const float* sK, const float* sD, cudaStream_t st, int* count)
{
    int launched = 0;
    if (outK && outD) launched = gather_all<true, true>(p, window, outK, zK, outD, zD, sK, sD, st);
    else if (outK) launched = gather_all<true, false>(p, window, outK, zK, nullptr, 0, sK, sD, st);
    else if (outD) launched = gather_all<false, true>(p, window, nullptr, 0, outD, zD, sK, sD, st);
    if (count) *count = launched;
    return cudaGetLastError();
}

}  // namespace addker
