// Gradient gathers for the vector-Jacobian product of K v (addker_vjp).
//
// For f = w^T K~ v with K~ = sigma_f^2 sum_s A_s B_s A_s^T (Sec. 3.1 fast summation; A_s interpolates
// from window s's grid, B_s is the symmetric multiply between the transforms):
//   df/dv       = K~ w
//   df/d ell_s  = v^T (dK~/d ell_s) w = sigma_f^2 (2/ell_s) v^T A_s h^D_s(w)
//   df/dsigma_f = (2/sigma_f) v^T K~ w
//   df/dx_k     = sigma_f^2 sum_s [ v_k grad(A_s h^K_s(w))_k + w_k grad(A_s h^K_s(v))_k ]
// where h_s(u) are the interpolation grids of u and grad differentiates the interpolation window in
// the target point. One thread per point of a work item (block per item): weights, window
// derivatives, and the (2m)^D support box read from the grid (L1/L2 cached).
#include "common.cuh"

namespace addker {

namespace {

__device__ __forceinline__ double warp_sum(double x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int D, int PASS>
__global__ void __launch_bounds__(128) k_gather_grad(const int4* __restrict__ items, const WinDev* __restrict__ wins,
                                                     const float* __restrict__ other, float* __restrict__ ks,
                                                     float* __restrict__ grad_x, double* __restrict__ dots, int P,
                                                     int d, int64_t N, float sf2, const WinPoly poly)
{
    const int4 it = items[blockIdx.x];
    const WinDev& W = wins[it.w];
    const int Wd = 2 * W.m;
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff, cz = (it.z >> 16) & 0xff;
    const int ox = cx - W.m + 1 - W.lo[0], oy = cy - W.m + 1 - W.lo[1], oz = cz - W.m + 1 - W.lo[2];
    double dk = 0.0, dd = 0.0;
    for (int k = threadIdx.x; k < it.y; k += blockDim.x) {
        const float4 p = W.pts[it.x + k];
        const int i = __float_as_int(p.w);
        float w0[kMaxW], w1[kMaxW], w2[kMaxW], g0[kMaxW], g1[kMaxW], g2[kMaxW];
        int c;
        window_weights_grad_n(poly, p.x, W.n, Wd, w0, g0, &c);
        if (D >= 2) window_weights_grad_n(poly, p.y, W.n, Wd, w1, g1, &c);
        if (D >= 3) window_weights_grad_n(poly, p.z, W.n, Wd, w2, g2, &c);
        // value (K and der) and gradient (K) of the interpolation at the point
        float fK = 0.f, fD = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        for (int a = 0; a < Wd; ++a) {
            float uK = 0.f, uD = 0.f, uKy = 0.f, uKz = 0.f;
            for (int b = 0; b < (D >= 2 ? Wd : 1); ++b) {
                float tK = 0.f, tD = 0.f, tKz = 0.f;
                for (int cc = 0; cc < (D >= 3 ? Wd : 1); ++cc) {
                    const size_t gi = ((size_t)(ox + a) * W.box[1] + (D >= 2 ? oy + b : 0)) * W.box[2] +
                                      (D >= 3 ? oz + cc : 0);
                    const float2 hv = W.h[gi];
                    const float wc = D >= 3 ? w2[cc] : 1.f;
                    tK = fmaf(hv.x, wc, tK);
                    tD = fmaf(hv.y, wc, tD);
                    if (D >= 3) tKz = fmaf(hv.x, g2[cc], tKz);
                }
                const float wb = D >= 2 ? w1[b] : 1.f;
                uK = fmaf(tK, wb, uK);
                uD = fmaf(tD, wb, uD);
                if (D >= 2) uKy = fmaf(tK, g1[b], uKy);
                if (D >= 3) uKz = fmaf(tKz, wb, uKz);
            }
            fK = fmaf(uK, w0[a], fK);
            fD = fmaf(uD, w0[a], fD);
            gx = fmaf(uK, g0[a], gx);
            if (D >= 2) gy = fmaf(uKy, w0[a], gy);
            if (D >= 3) gz = fmaf(uKz, w0[a], gz);
        }
        const float o = other[i];                                  // v_i (pass 0) or w_i (pass 1)
        const float gs = sf2 * o;
        float* gxi = grad_x + (int64_t)i * d;
        atomicAdd(gxi + W.feat[0], gs * gx);
        if (D >= 2) atomicAdd(gxi + W.feat[1], gs * gy);
        if (D >= 3) atomicAdd(gxi + W.feat[2], gs * gz);
        if (PASS == 0) {
            ks[(int64_t)it.w * N + i] = fK;
            dk += (double)o * (double)fK;
            dd += (double)o * (double)fD;
        }
    }
    if (PASS == 0) {
        dk = warp_sum(dk);
        dd = warp_sum(dd);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(dots + it.w, dk);
            atomicAdd(dots + P + it.w, dd);
        }
    }
}

// The same for 3-D windows with cutoff m = 4 (W = 8), one warp per work item: the item's 8x8x8 box of
// (h^K, h^D) is staged in shared memory once, and each lane takes one point at a time. Per grid row (a, b)
// the c-sums give both grids' values (a packed FMA on the pair) and the z-derivative of h^K; the b-sums add
// the y-derivative and the a-sums the x-derivative, so one pass over the box yields f^K, f^D and grad f^K.
template <int PASS>
__global__ void __launch_bounds__(128) k_gather_grad3_w8(const int4* __restrict__ items, int nitems,
                                                         const WinDev* __restrict__ wins,
                                                         const float* __restrict__ other, float* __restrict__ ks,
                                                         float* __restrict__ grad_x, double* __restrict__ dots, int P,
                                                         int d, int64_t N, float sf2, const WinPoly poly)
{
    constexpr int W = 8;
    __shared__ __align__(16) float2 tile[4][512];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * 4 + warp;
    if (item >= nitems) return;                                // warp-uniform: no block-wide barrier follows
    const int4 it = items[item];
    const WinDev& Wd = wins[it.w];
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff, cz = (it.z >> 16) & 0xff;
    const int ox = cx - 3 - Wd.lo[0], oy = cy - 3 - Wd.lo[1], oz = cz - 3 - Wd.lo[2];
    const int sy = Wd.box[2], sx = Wd.box[1] * Wd.box[2];
    const float2* __restrict__ h = Wd.h + (size_t)ox * sx + (size_t)oy * sy + oz;    // slot 0
    float2* t = tile[warp];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int idx = lane + 32 * i;
        const int a = idx >> 6, bb = (idx >> 3) & 7, cc = idx & 7;
        t[idx] = h[(size_t)a * sx + (size_t)bb * sy + cc];
    }
    __syncwarp();
    const float4* t4 = reinterpret_cast<const float4*>(t);
    double dk = 0.0, dd = 0.0;
    for (int k = lane; k < it.y; k += 32) {
        const float4 q = Wd.pts[it.x + k];
        const int i = __float_as_int(q.w);
        float x[W], dx[W], yv[W], dy[W], zv[W], dz[W];
        int c;
        window_weights_grad_n(poly, q.x, Wd.n, W, x, dx, &c);
        window_weights_grad_n(poly, q.y, Wd.n, W, yv, dy, &c);
        window_weights_grad_n(poly, q.z, Wd.n, W, zv, dz, &c);
        float2 f = make_float2(0.f, 0.f);
        float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll 1
        for (int a = 0; a < W; ++a) {
            float2 u = make_float2(0.f, 0.f);
            float uy = 0.f, uz = 0.f;
            const float4* row = t4 + a * 32;
#pragma unroll
            for (int bb = 0; bb < W; ++bb) {
                float2 sv = make_float2(0.f, 0.f);
                float tz = 0.f;
#pragma unroll
                for (int cc = 0; cc < W; cc += 2) {
                    const float4 hv = row[(bb * 8 + cc) >> 1];
                    sv = __ffma2_rn(make_float2(hv.x, hv.y), make_float2(zv[cc], zv[cc]), sv);
                    sv = __ffma2_rn(make_float2(hv.z, hv.w), make_float2(zv[cc + 1], zv[cc + 1]), sv);
                    tz = fmaf(hv.x, dz[cc], tz);
                    tz = fmaf(hv.z, dz[cc + 1], tz);
                }
                u = __ffma2_rn(sv, make_float2(yv[bb], yv[bb]), u);
                uy = fmaf(sv.x, dy[bb], uy);
                uz = fmaf(tz, yv[bb], uz);
            }
            f = __ffma2_rn(u, make_float2(x[0], x[0]), f);
            gx = fmaf(u.x, dx[0], gx);
            gy = fmaf(uy, x[0], gy);
            gz = fmaf(uz, x[0], gz);
            // rotate so that x[0], dx[0] hold the next a's weights (keeps indices static)
#pragma unroll
            for (int j = 0; j < W - 1; ++j) {
                x[j] = x[j + 1];
                dx[j] = dx[j + 1];
            }
        }
        const float o = other[i];
        const float gs = sf2 * o;
        float* gxi = grad_x + (int64_t)i * d;
        atomicAdd(gxi + Wd.feat[0], gs * gx);
        atomicAdd(gxi + Wd.feat[1], gs * gy);
        atomicAdd(gxi + Wd.feat[2], gs * gz);
        if (PASS == 0) {
            ks[(int64_t)it.w * N + i] = f.x;
            dk += (double)o * (double)f.x;
            dd += (double)o * (double)f.y;
        }
    }
    if (PASS == 0) {
        dk = warp_sum(dk);
        dd = warp_sum(dd);
        if (lane == 0) {
            atomicAdd(dots + it.w, dk);
            atomicAdd(dots + P + it.w, dd);
        }
    }
}

template <int PASS>
int launch_pass(const Plan& p, const int4* items, int n, int D, const float* other, float* ks, float* grad_x,
                cudaStream_t st)
{
    const float sf2 = (float)(p.sigma_f * p.sigma_f);
    if (n == 0) return 0;
    if (D == 3 && p.m == 4) {
        launch_k(false, k_gather_grad3_w8<PASS>, dim3((n + 3) / 4), dim3(128), 0, st, items, n,
                 (const WinDev*)p.wins_dev, other, ks, grad_x, p.dots, p.P, p.d, p.N, sf2, p.poly);
        return 1;
    }
    auto kern = D == 1 ? k_gather_grad<1, PASS> : D == 2 ? k_gather_grad<2, PASS> : k_gather_grad<3, PASS>;
    launch_k(false, kern, dim3(n), dim3(128), 0, st, items, (const WinDev*)p.wins_dev, other, ks, grad_x, p.dots,
             p.P, p.d, p.N, sf2, p.poly);
    return 1;
}

}  // namespace

cudaError_t launch_gather_grad(const Plan& p, int pass, const float* other, float* ks, float* grad_x, cudaStream_t st,
                               int* count)
{
    int launched = 0;
    for (int s = 0; s < p.P; ++s) {
        const std::vector<int>& b = p.item_begin[p.kind[s]];
        const int4* items = p.items + b[s];
        const int n = b[s + 1] - b[s];
        if (pass == 0) launched += launch_pass<0>(p, items, n, p.dims[s], other, ks, grad_x, st);
        else launched += launch_pass<1>(p, items, n, p.dims[s], other, ks, grad_x, st);
    }
    if (count) *count = launched;
    return cudaGetLastError();
}

}  // namespace addker
