// Spreading (adjoint NFFT, first step) and interpolation (NFFT, last step) kernels.
//
//   spread:  g_l   = sum_j v_j prod_t w(n x_{j,t} - l_t),   l in the support of x_j
//   gather:  f_i   = sum_l h_l prod_t w(n x_{i,t} - l_t)     for the two grids h^K and h^der
// (Sec. 3.1, eq. "approx fast sum": the inner sums by an adjoint NFFT, the outer sums by an
// NFFT). w is the normalised Kaiser-Bessel window (evaluated through its piecewise polynomial
// form, see WinPoly); the support of x along an axis is floor(n x) - m + 1 .. floor(n x) + m.
//
// Points are sorted by grid cell, so all points of a work item share one support box of
// (2m)^D grid points. The fast kernels (D = 3, m = 4) exploit that:
//   spread: a warp accumulates the item's 8x8x8 box in registers as a sum of outer products
//           (v_j w_x) (x) w_y (x) w_z; lane (ah, bh, c) owns the 4x4 block a in 4ah..4ah+3,
//           b in 4bh..4bh+3 at z-offset c, so each point costs a lane 3 shared loads, 4 products
//           and 16 FMAs; the box is added to the grid once per item;
//   gather: a warp stages the item's box of both grids in shared memory (float2 (h^K, h^der)) and
//           every lane contracts it with two points at once, so one 16-byte broadcast load feeds
//           8 FMAs.
#include "common.cuh"

namespace addker {

namespace {

constexpr int kWarps = 8;                 // warps per block in the item kernels

// ----------------------------------------------------------------------------------
// fast 3-D spread, m = 4 (W = 8)
__global__ void __launch_bounds__(kWarps * 32) k_spread3_w8(const int4* __restrict__ items, int nitems,
                                                           const WinDev* __restrict__ wins,
                                                           const float* __restrict__ v, const WinPoly poly)
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
    const int n = P.n;
    float* ws = sw[warp];
    const int ah = lane >> 4, bh = (lane >> 3) & 1, c = lane & 7;

    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;

    for (int base = 0; base < count; base += 32) {
        const int k = base + lane;
        float wx[W], wy[W], wz[W];
        int cx, cy, cz;
        if (k < count) {
            const float4 p = pts[k];
            const float vv = __ldg(v + __float_as_int(p.w));
            window_weights<W>(poly, p.x, n, wx, &cx);
            window_weights<W>(poly, p.y, n, wy, &cy);
            window_weights<W>(poly, p.z, n, wz, &cz);
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
        const float* src = ws;
#pragma unroll 4
        for (int j = 0; j < cnt; ++j, src += STRIDE) {
            const float4 xa = *reinterpret_cast<const float4*>(src + 4 * ah);
            const float4 yb = *reinterpret_cast<const float4*>(src + 8 + 4 * bh);
            const float zc = src[16 + c];
            const float B[4] = {yb.x * zc, yb.y * zc, yb.z * zc, yb.w * zc};
            const float X[4] = {xa.x, xa.y, xa.z, xa.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(X[a], B[b], acc[a][b]);
        }
        __syncwarp();
    }
    // flush: grid index of (a, b, c) relative to the box origin
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff, cz = (it.z >> 16) & 0xff;
    const int ox = cx - 3 - P.lo[0], oy = cy - 3 - P.lo[1], oz = cz - 3 - P.lo[2];
    const int sy = P.box[2], sx = P.box[1] * P.box[2];
    float* g = P.grid + (size_t)(ox + 4 * ah) * sx + (size_t)(oy + 4 * bh) * sy + oz + c;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) atomicAdd(g + (size_t)a * sx + (size_t)b * sy, acc[a][b]);
}

// ----------------------------------------------------------------------------------
// fast 3-D gather, m = 4 (W = 8): lanes own points (two each); the item's box of both grids is
// staged in shared memory and read back as float4 (h^K_c, h^D_c, h^K_c+1, h^D_c+1), broadcast.
template <bool WK, bool WD>
__global__ void __launch_bounds__(kWarps * 32, 2) k_gather3_w8(const int4* __restrict__ items, int nitems,
                                                              const WinDev* __restrict__ wins,
                                                              float* __restrict__ outK, float* __restrict__ outD,
                                                              const float* __restrict__ scaleK,
                                                              const float* __restrict__ scaleD, int64_t strideK,
                                                              int64_t strideD, const WinPoly poly)
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
        const int idx = lane + 32 * i;
        const int a = idx >> 6, bb = (idx >> 3) & 7, cc = idx & 7;
        t[idx] = h[(size_t)a * sx + (size_t)bb * sy + cc];
    }
    __syncwarp();
    const float4* t4 = reinterpret_cast<const float4*>(t);
    const float4* __restrict__ pts = P.pts + it.x;
    const float sK = WK ? scaleK[it.w] : 0.f;
    const float sD = WD ? scaleD[it.w] : 0.f;
    const int n = P.n;
    for (int k0 = lane; k0 < it.y; k0 += 64) {
        const int k1 = k0 + 32;
        const bool has1 = k1 < it.y;
        const float4 p0 = pts[k0];
        const float4 p1 = has1 ? pts[k1] : p0;
        float x0[W], y0[W], z0[W], x1[W], y1[W], z1[W];
        int c;
        window_weights<W>(poly, p0.x, n, x0, &c);
        window_weights<W>(poly, p0.y, n, y0, &c);
        window_weights<W>(poly, p0.z, n, z0, &c);
        window_weights<W>(poly, p1.x, n, x1, &c);
        window_weights<W>(poly, p1.y, n, y1, &c);
        window_weights<W>(poly, p1.z, n, z1, &c);
        float fK0 = 0.f, fD0 = 0.f, fK1 = 0.f, fD1 = 0.f;
#pragma unroll 1
        for (int a = 0; a < W; ++a) {
            float uK0 = 0.f, uD0 = 0.f, uK1 = 0.f, uD1 = 0.f;
            const float4* row = t4 + a * 32;
#pragma unroll
            for (int bb = 0; bb < W; ++bb) {
                float tK0 = 0.f, tD0 = 0.f, tK1 = 0.f, tD1 = 0.f;
#pragma unroll
                for (int cc = 0; cc < W; cc += 2) {
                    const float4 hv = row[(bb * 8 + cc) >> 1];
                    tK0 = fmaf(hv.x, z0[cc], tK0);
                    tD0 = fmaf(hv.y, z0[cc], tD0);
                    tK1 = fmaf(hv.x, z1[cc], tK1);
                    tD1 = fmaf(hv.y, z1[cc], tD1);
                    tK0 = fmaf(hv.z, z0[cc + 1], tK0);
                    tD0 = fmaf(hv.w, z0[cc + 1], tD0);
                    tK1 = fmaf(hv.z, z1[cc + 1], tK1);
                    tD1 = fmaf(hv.w, z1[cc + 1], tD1);
                }
                uK0 = fmaf(tK0, y0[bb], uK0);
                uD0 = fmaf(tD0, y0[bb], uD0);
                uK1 = fmaf(tK1, y1[bb], uK1);
                uD1 = fmaf(tD1, y1[bb], uD1);
            }
            fK0 = fmaf(uK0, x0[0], fK0);
            fD0 = fmaf(uD0, x0[0], fD0);
            fK1 = fmaf(uK1, x1[0], fK1);
            fD1 = fmaf(uD1, x1[0], fD1);
            // rotate so that x0[0], x1[0] hold the weights of the next a (keeps indices static)
#pragma unroll
            for (int q = 0; q < W - 1; ++q) { x0[q] = x0[q + 1]; x1[q] = x1[q + 1]; }
        }
        const int64_t i0 = (int64_t)__float_as_int(p0.w);
        if (WK) outK[i0 + (int64_t)it.w * strideK] = sK * fK0;
        if (WD) outD[i0 + (int64_t)it.w * strideD] = sD * fD0;
        if (has1) {
            const int64_t i1 = (int64_t)__float_as_int(p1.w);
            if (WK) outK[i1 + (int64_t)it.w * strideK] = sK * fK1;
            if (WD) outD[i1 + (int64_t)it.w * strideD] = sD * fD1;
        }
    }
}

// ----------------------------------------------------------------------------------
// generic kernels: any D in {1,2,3}, W = 2m <= 16. One block per item; the spread accumulates
// the item's W^D support box in shared memory, then adds it to the grid.
template <int D>
__global__ void __launch_bounds__(128) k_spread_generic(const int4* __restrict__ items,
                                                        const WinDev* __restrict__ wins,
                                                        const float* __restrict__ v, const WinPoly poly)
{
    __shared__ float box[kMaxW * kMaxW * kMaxW];
    const int4 it = items[blockIdx.x];
    const WinDev& P = wins[it.w];
    const int W = 2 * P.m;
    int WD = W;
    if (D >= 2) WD *= W;
    if (D >= 3) WD *= W;
    for (int i = threadIdx.x; i < WD; i += blockDim.x) box[i] = 0.f;
    __syncthreads();
    for (int k = threadIdx.x; k < it.y; k += blockDim.x) {
        const float4 p = P.pts[it.x + k];
        const float vv = __ldg(v + __float_as_int(p.w));
        float w0[kMaxW], w1[kMaxW], w2[kMaxW];
        int c;
        window_weights_n(poly, p.x, P.n, W, w0, &c);
        if (D >= 2) window_weights_n(poly, p.y, P.n, W, w1, &c);
        if (D >= 3) window_weights_n(poly, p.z, P.n, W, w2, &c);
        for (int a = 0; a < W; ++a) {
            const float va = vv * w0[a];
            if (D == 1) { atomicAdd(&box[a], va); continue; }
            for (int bb = 0; bb < W; ++bb) {
                const float vab = va * w1[bb];
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
        const size_t g = ((size_t)(ox + a) * P.box[1] + (D >= 2 ? oy + bb : 0)) * P.box[2] + (D >= 3 ? oz + cc : 0);
        if (box[i] != 0.f) atomicAdd(P.grid + g, box[i]);
    }
}

template <int D, bool WK, bool WD>
__global__ void __launch_bounds__(128) k_gather_generic(const int4* __restrict__ items,
                                                        const WinDev* __restrict__ wins,
                                                        float* __restrict__ outK, float* __restrict__ outD,
                                                        const float* __restrict__ scaleK,
                                                        const float* __restrict__ scaleD, int64_t strideK,
                                                        int64_t strideD, const WinPoly poly)
{
    const int4 it = items[blockIdx.x];
    const WinDev& P = wins[it.w];
    const int W = 2 * P.m;
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff, cz = (it.z >> 16) & 0xff;
    const int ox = cx - P.m + 1 - P.lo[0], oy = cy - P.m + 1 - P.lo[1], oz = cz - P.m + 1 - P.lo[2];
    for (int k = threadIdx.x; k < it.y; k += blockDim.x) {
        const float4 p = P.pts[it.x + k];
        float w0[kMaxW], w1[kMaxW], w2[kMaxW];
        int c;
        window_weights_n(poly, p.x, P.n, W, w0, &c);
        if (D >= 2) window_weights_n(poly, p.y, P.n, W, w1, &c);
        if (D >= 3) window_weights_n(poly, p.z, P.n, W, w2, &c);
        float fK = 0.f, fD = 0.f;
        for (int a = 0; a < W; ++a) {
            float uK = 0.f, uD = 0.f;
            for (int bb = 0; bb < (D >= 2 ? W : 1); ++bb) {
                float tK = 0.f, tD = 0.f;
                for (int cc = 0; cc < (D >= 3 ? W : 1); ++cc) {
                    const size_t g = ((size_t)(ox + a) * P.box[1] + (D >= 2 ? oy + bb : 0)) * P.box[2] +
                                     (D >= 3 ? oz + cc : 0);
                    const float2 hv = P.h[g];
                    const float wc = D >= 3 ? w2[cc] : 1.f;
                    tK = fmaf(hv.x, wc, tK);
                    tD = fmaf(hv.y, wc, tD);
                }
                const float wb = D >= 2 ? w1[bb] : 1.f;
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
        const int n = hi - lo;
        k_spread3_w8<<<(n + kWarps - 1) / kWarps, kWarps * 32, 0, st>>>(p.items_fast + lo, n, wd, v, p.poly);
        ++launched;
    }
    const std::vector<int>& gb = p.item_begin_gen;
    for (int s = 0; s < p.P; ++s) {
        if (window >= 0 && s != window) continue;
        const int n = gb[s + 1] - gb[s];
        if (n == 0) continue;
        const int4* it = p.items_gen + gb[s];
        switch (p.dims[s]) {
            case 1: k_spread_generic<1><<<n, 128, 0, st>>>(it, wd, v, p.poly); break;
            case 2: k_spread_generic<2><<<n, 128, 0, st>>>(it, wd, v, p.poly); break;
            default: k_spread_generic<3><<<n, 128, 0, st>>>(it, wd, v, p.poly); break;
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
        const int n = hi - lo;
        k_gather3_w8<WK, WD><<<(n + kWarps - 1) / kWarps, kWarps * 32, 0, st>>>(p.items_fast + lo, n, wd, outK, outD,
                                                                               sK, sD, zK, zD, p.poly);
        ++launched;
    }
    const std::vector<int>& gb = p.item_begin_gen;
    for (int s = 0; s < p.P; ++s) {
        if (window >= 0 && s != window) continue;
        const int n = gb[s + 1] - gb[s];
        if (n == 0) continue;
        const int4* it = p.items_gen + gb[s];
        switch (p.dims[s]) {
            case 1: k_gather_generic<1, WK, WD><<<n, 128, 0, st>>>(it, wd, outK, outD, sK, sD, zK, zD, p.poly); break;
            case 2: k_gather_generic<2, WK, WD><<<n, 128, 0, st>>>(it, wd, outK, outD, sK, sD, zK, zD, p.poly); break;
            default: k_gather_generic<3, WK, WD><<<n, 128, 0, st>>>(it, wd, outK, outD, sK, sD, zK, zD, p.poly); break;
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
