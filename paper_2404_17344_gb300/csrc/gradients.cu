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

template <int PASS>
int launch_pass(const Plan& p, const int4* items, int n, int D, const float* other, float* ks, float* grad_x,
                cudaStream_t st)
{
    const float sf2 = (float)(p.sigma_f * p.sigma_f);
    if (n == 0) return 0;
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
