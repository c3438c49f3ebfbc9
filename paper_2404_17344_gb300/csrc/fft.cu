// The transforms between the spread grid and the interpolation grids (Sec. 3.1: the FFT inside the
// adjoint NFFT, the multiplication by the kernel's Fourier coefficients, the FFT inside the NFFT).
//
//   forward:  G_k   = sum_l g_l exp(-2 pi i k.l/n),  k in I_M^D, l over the grid's bounding box
//   multiply: S^K_k = bK_k G_k,   S^D_k = bD_k G_k  (bK, bD: coefficients over window transforms)
//   inverse:  h_l   = Re sum_k S_k exp(+2 pi i k.l/n), l over the bounding box, for both spectra
//
// Only the M^D retained frequencies and the box of grid points that points can touch are computed:
// a pruned transform, axis by axis, as small dense DFTs (box <= 64 samples <-> M <= 64 frequencies).
//
// D = 3 (the hot case) uses three fused kernels, each launched once for all windows:
//   k_fwd_yz   per x-slab:   g[x][y][z] -> t[x][ky][kz]         (z then y, in shared memory)
//   k_xround   per column:   t[x][c] -> S[kx][c] -> B[x][c]      (x forward, multiply, x inverse)
//   k_inv_yz   per x-slab:   B[x][ky][kz] -> h[x][y][z]          (y then z inverse, real part)
// The x round trip fuses forward DFT, multiplication and inverse DFT because all three act on the
// same column (ky, kz). D = 1, 2 use the generic one-axis pass k_dft_pass per window.
#include "common.cuh"

namespace addker {

namespace {

enum { IN_REAL = 0, IN_CPLX = 1, IN_PAIR = 2 };
enum { OUT_CPLX = 1, OUT_PAIR = 2, OUT_MUL = 3, OUT_REAL_PAIR = 4 };

__device__ __forceinline__ float2 cmad(float2 a, float2 b, float2 c)      // c + a*b
{
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cmadc(float2 a, float2 w, float2 c)     // c + a*conj(w)
{
    return make_float2(fmaf(a.x, w.x, fmaf(a.y, w.y, c.x)), fmaf(a.y, w.x, fmaf(-a.x, w.y, c.y)));
}

// ------------------------------------------------------------------------ D = 3 fused ----
// Each phase is a small dense complex matrix product done from shared memory, one 2x2 block of
// outputs per thread, so each pair of 16-byte shared loads feeds 16 to 32 FMAs. Twiddles are the
// forward tables twf[axis][l][k] = e^{-2 pi i k l/n}; the inverse uses their conjugates.
constexpr int kT = 256;

// block = (x, window). smem: gs[b1][b2] float, tz[b2][M], ty[b1][M], t1[b1][M] float2.
//   t1[y][kz] = sum_z g[x][y][z] tz[z][kz];   out[x][ky][kz] = sum_y ty[y][ky] t1[y][kz]
// The grid slab is zeroed once read, so d = 3 grids need no separate clearing before a spread.
__global__ void __launch_bounds__(kT) k_fwd_yz(const WinDev* __restrict__ wins, int w0)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const WinDev& W = wins[w0 + blockIdx.y];
    if (W.D != 3) return;
    const int x = blockIdx.x;
    const int b0 = W.box[0], b1 = W.box[1], b2 = W.box[2], M = W.M;
    if (x >= b0) return;
    float2* tz = reinterpret_cast<float2*>(smem);
    float2* ty = tz + b2 * M;
    float2* t1 = ty + b1 * M;
    float* gs = reinterpret_cast<float*>(t1 + b1 * M);
    float* g = W.grid + (size_t)x * b1 * b2;
    for (int i = threadIdx.x; i < b1 * b2; i += kT) {
        gs[i] = g[i];
        g[i] = 0.f;                      // the slab is consumed: leave the grid zeroed for the next spread
    }
    for (int i = threadIdx.x; i < b2 * M; i += kT) tz[i] = W.twf[2][i];
    for (int i = threadIdx.x; i < b1 * M; i += kT) ty[i] = W.twf[1][i];
    __syncthreads();
    const int Mh = M / 2;
    // phase 1: rows y (2 per block, clamped), columns kz (2 per block)
    const int nb1 = (b1 + 1) / 2;
    for (int o = threadIdx.x; o < nb1 * Mh; o += kT) {
        const int y0 = 2 * (o / Mh), y1 = min(y0 + 1, b1 - 1), k0 = 2 * (o % Mh);
        float2 a00 = make_float2(0.f, 0.f), a01 = a00, a10 = a00, a11 = a00;
        const float* r0 = gs + y0 * b2;
        const float* r1 = gs + y1 * b2;
#pragma unroll 4
        for (int z = 0; z < b2; ++z) {
            const float4 w = *reinterpret_cast<const float4*>(tz + z * M + k0);
            const float g0 = r0[z], g1 = r1[z];
            a00.x = fmaf(g0, w.x, a00.x); a00.y = fmaf(g0, w.y, a00.y);
            a01.x = fmaf(g0, w.z, a01.x); a01.y = fmaf(g0, w.w, a01.y);
            a10.x = fmaf(g1, w.x, a10.x); a10.y = fmaf(g1, w.y, a10.y);
            a11.x = fmaf(g1, w.z, a11.x); a11.y = fmaf(g1, w.w, a11.y);
        }
        *reinterpret_cast<float4*>(t1 + y0 * M + k0) = make_float4(a00.x, a00.y, a01.x, a01.y);
        if (y0 + 1 < b1) *reinterpret_cast<float4*>(t1 + y1 * M + k0) = make_float4(a10.x, a10.y, a11.x, a11.y);
    }
    __syncthreads();
    // phase 2: rows ky, columns kz (2x2 blocks)
    float2* out = reinterpret_cast<float2*>(W.buf1) + (size_t)x * M * M;
    for (int o = threadIdx.x; o < Mh * Mh; o += kT) {
        const int ky = 2 * (o / Mh), kz = 2 * (o % Mh);
        float2 a00 = make_float2(0.f, 0.f), a01 = a00, a10 = a00, a11 = a00;
#pragma unroll 4
        for (int y = 0; y < b1; ++y) {
            const float4 w = *reinterpret_cast<const float4*>(ty + y * M + ky);   // ty[y][ky], ty[y][ky+1]
            const float4 t = *reinterpret_cast<const float4*>(t1 + y * M + kz);   // t1[y][kz], t1[y][kz+1]
            const float2 w0 = make_float2(w.x, w.y), w1 = make_float2(w.z, w.w);
            const float2 s0 = make_float2(t.x, t.y), s1 = make_float2(t.z, t.w);
            a00 = cmad(s0, w0, a00);
            a01 = cmad(s1, w0, a01);
            a10 = cmad(s0, w1, a10);
            a11 = cmad(s1, w1, a11);
        }
        *reinterpret_cast<float4*>(out + ky * M + kz) = make_float4(a00.x, a00.y, a01.x, a01.y);
        *reinterpret_cast<float4*>(out + (ky + 1) * M + kz) = make_float4(a10.x, a10.y, a11.x, a11.y);
    }
}

// block = (column tile of 32 columns c = (ky, kz), window). smem: tx[b0][M] float2, ts[b0][32]
// float2, ss[M][32] float4.
//   S[kx][c] = m_k sum_x tx[x][kx] t[x][c];   B[x][c] = sum_kx conj(tx[x][kx]) S[kx][c]
// spec_only: write S (multiplied by dconv) to W.spec and stop.
__global__ void __launch_bounds__(kT) k_xround(const WinDev* __restrict__ wins, int w0, int spec_only)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const WinDev& W = wins[w0 + blockIdx.y];
    if (W.D != 3) return;
    const int M = W.M, b0 = W.box[0];
    const int MM = M * M;
    const int c0 = blockIdx.x * 32;
    if (c0 >= MM) return;
    float2* tx = reinterpret_cast<float2*>(smem);
    float2* ts = tx + b0 * M;
    float4* ss = reinterpret_cast<float4*>(ts + b0 * 32);
    const int cols = min(32, MM - c0);                          // M^2 need not be a multiple of 32
    const float2* t = reinterpret_cast<const float2*>(W.buf1);
    for (int i = threadIdx.x; i < b0 * 32; i += kT)
        ts[i] = (i & 31) < cols ? t[(size_t)(i >> 5) * MM + c0 + (i & 31)] : make_float2(0.f, 0.f);
    for (int i = threadIdx.x; i < b0 * M; i += kT) tx[i] = W.twf[0][i];
    __syncthreads();
    const float* mK = spec_only ? W.dconv : W.bK;
    const float* mD = spec_only ? W.dconv : W.bD;
    const int Mh = M / 2;
    for (int o = threadIdx.x; o < Mh * 16; o += kT) {            // 2x2 blocks (kx, j)
        const int kx = 2 * (o / 16), j = 2 * (o % 16);
        float2 a00 = make_float2(0.f, 0.f), a01 = a00, a10 = a00, a11 = a00;
#pragma unroll 4
        for (int x = 0; x < b0; ++x) {
            const float4 w = *reinterpret_cast<const float4*>(tx + x * M + kx);
            const float4 v = *reinterpret_cast<const float4*>(ts + x * 32 + j);
            const float2 w0 = make_float2(w.x, w.y), w1 = make_float2(w.z, w.w);
            const float2 s0 = make_float2(v.x, v.y), s1 = make_float2(v.z, v.w);
            a00 = cmad(s0, w0, a00);
            a01 = cmad(s1, w0, a01);
            a10 = cmad(s0, w1, a10);
            a11 = cmad(s1, w1, a11);
        }
        const float2 acc[2][2] = {{a00, a01}, {a10, a11}};
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (j + q >= cols) {
                    if (!spec_only) ss[(kx + r) * 32 + j + q] = make_float4(0.f, 0.f, 0.f, 0.f);
                    continue;
                }
                const size_t k = (size_t)(kx + r) * MM + c0 + j + q;
                const float a = __ldg(mK + k), d = __ldg(mD + k);
                const float4 v = make_float4(a * acc[r][q].x, a * acc[r][q].y, d * acc[r][q].x, d * acc[r][q].y);
                if (spec_only) W.spec[k] = v;
                else ss[(kx + r) * 32 + j + q] = v;
            }
    }
    if (spec_only) return;
    __syncthreads();
    const int nbx = (b0 + 1) / 2;
    for (int o = threadIdx.x; o < nbx * 16; o += kT) {           // 2x2 blocks (x, j)
        const int x0 = 2 * (o / 16), x1 = min(x0 + 1, b0 - 1), j = 2 * (o % 16);
        float2 k00 = make_float2(0.f, 0.f), k01 = k00, k10 = k00, k11 = k00;
        float2 d00 = k00, d01 = k00, d10 = k00, d11 = k00;
#pragma unroll 4
        for (int kx = 0; kx < M; ++kx) {
            const float2 w0 = tx[x0 * M + kx], w1 = tx[x1 * M + kx];
            const float4 s0 = ss[kx * 32 + j], s1 = ss[kx * 32 + j + 1];
            k00 = cmadc(make_float2(s0.x, s0.y), w0, k00);
            d00 = cmadc(make_float2(s0.z, s0.w), w0, d00);
            k01 = cmadc(make_float2(s1.x, s1.y), w0, k01);
            d01 = cmadc(make_float2(s1.z, s1.w), w0, d01);
            k10 = cmadc(make_float2(s0.x, s0.y), w1, k10);
            d10 = cmadc(make_float2(s0.z, s0.w), w1, d10);
            k11 = cmadc(make_float2(s1.x, s1.y), w1, k11);
            d11 = cmadc(make_float2(s1.z, s1.w), w1, d11);
        }
        if (j >= cols) continue;
        float4* B = W.buf2 + c0 + j;
        const bool q1 = j + 1 < cols;
        B[(size_t)x0 * MM] = make_float4(k00.x, k00.y, d00.x, d00.y);
        if (q1) B[(size_t)x0 * MM + 1] = make_float4(k01.x, k01.y, d01.x, d01.y);
        if (x0 + 1 < b0) {
            B[(size_t)x1 * MM] = make_float4(k10.x, k10.y, d10.x, d10.y);
            if (q1) B[(size_t)x1 * MM + 1] = make_float4(k11.x, k11.y, d11.x, d11.y);
        }
    }
}

// block = (x, window). smem: ty[b1][M], tz[b2][M] float2, bs[M][M] float4, b1s[b1][M] float4.
//   B1[y][kz] = sum_ky conj(ty[y][ky]) B[x][ky][kz];   h[x][y][z] = Re sum_kz conj(tz[z][kz]) B1[y][kz]
__global__ void __launch_bounds__(kT) k_inv_yz(const WinDev* __restrict__ wins, int w0)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const WinDev& W = wins[w0 + blockIdx.y];
    if (W.D != 3) return;
    const int x = blockIdx.x;
    const int b0 = W.box[0], b1 = W.box[1], b2 = W.box[2], M = W.M;
    if (x >= b0) return;
    const int MM = M * M;
    float4* bs = reinterpret_cast<float4*>(smem);
    float4* b1s = bs + MM;
    float2* ty = reinterpret_cast<float2*>(b1s + b1 * M);
    float2* tz = ty + b1 * M;
    const float4* B = W.buf2 + (size_t)x * MM;
    for (int i = threadIdx.x; i < MM; i += kT) bs[i] = B[i];
    for (int i = threadIdx.x; i < b1 * M; i += kT) ty[i] = W.twf[1][i];
    for (int i = threadIdx.x; i < b2 * M; i += kT) tz[i] = W.twf[2][i];
    __syncthreads();
    const int Mh = M / 2;
    const int nb1 = (b1 + 1) / 2;
    for (int o = threadIdx.x; o < nb1 * Mh; o += kT) {           // 2x2 blocks (y, kz)
        const int y0 = 2 * (o / Mh), y1 = min(y0 + 1, b1 - 1), kz = 2 * (o % Mh);
        float2 k00 = make_float2(0.f, 0.f), k01 = k00, k10 = k00, k11 = k00;
        float2 d00 = k00, d01 = k00, d10 = k00, d11 = k00;
#pragma unroll 4
        for (int ky = 0; ky < M; ++ky) {
            const float2 w0 = ty[y0 * M + ky], w1 = ty[y1 * M + ky];
            const float4 s0 = bs[ky * M + kz], s1 = bs[ky * M + kz + 1];
            k00 = cmadc(make_float2(s0.x, s0.y), w0, k00);
            d00 = cmadc(make_float2(s0.z, s0.w), w0, d00);
            k01 = cmadc(make_float2(s1.x, s1.y), w0, k01);
            d01 = cmadc(make_float2(s1.z, s1.w), w0, d01);
            k10 = cmadc(make_float2(s0.x, s0.y), w1, k10);
            d10 = cmadc(make_float2(s0.z, s0.w), w1, d10);
            k11 = cmadc(make_float2(s1.x, s1.y), w1, k11);
            d11 = cmadc(make_float2(s1.z, s1.w), w1, d11);
        }
        b1s[y0 * M + kz] = make_float4(k00.x, k00.y, d00.x, d00.y);
        b1s[y0 * M + kz + 1] = make_float4(k01.x, k01.y, d01.x, d01.y);
        if (y0 + 1 < b1) {
            b1s[y1 * M + kz] = make_float4(k10.x, k10.y, d10.x, d10.y);
            b1s[y1 * M + kz + 1] = make_float4(k11.x, k11.y, d11.x, d11.y);
        }
    }
    __syncthreads();
    float2* h = W.h + (size_t)x * b1 * b2;
    const int nb2 = (b2 + 1) / 2;
    for (int o = threadIdx.x; o < nb1 * nb2; o += kT) {          // 2x2 blocks (y, z)
        const int y0 = 2 * (o / nb2), y1 = min(y0 + 1, b1 - 1);
        const int z0 = 2 * (o % nb2), z1 = min(z0 + 1, b2 - 1);
        float k00 = 0.f, k01 = 0.f, k10 = 0.f, k11 = 0.f, d00 = 0.f, d01 = 0.f, d10 = 0.f, d11 = 0.f;
#pragma unroll 4
        for (int kz = 0; kz < M; ++kz) {
            const float2 w0 = tz[z0 * M + kz], w1 = tz[z1 * M + kz];
            const float4 s0 = b1s[y0 * M + kz], s1 = b1s[y1 * M + kz];
            // Re(s conj(w)) = s.re w.re + s.im w.im
            k00 = fmaf(s0.x, w0.x, fmaf(s0.y, w0.y, k00));
            d00 = fmaf(s0.z, w0.x, fmaf(s0.w, w0.y, d00));
            k01 = fmaf(s0.x, w1.x, fmaf(s0.y, w1.y, k01));
            d01 = fmaf(s0.z, w1.x, fmaf(s0.w, w1.y, d01));
            k10 = fmaf(s1.x, w0.x, fmaf(s1.y, w0.y, k10));
            d10 = fmaf(s1.z, w0.x, fmaf(s1.w, w0.y, d10));
            k11 = fmaf(s1.x, w1.x, fmaf(s1.y, w1.y, k11));
            d11 = fmaf(s1.z, w1.x, fmaf(s1.w, w1.y, d11));
        }
        h[y0 * b2 + z0] = make_float2(k00, d00);
        if (z0 + 1 < b2) h[y0 * b2 + z1] = make_float2(k01, d01);
        if (y0 + 1 < b1) {
            h[y1 * b2 + z0] = make_float2(k10, d10);
            if (z0 + 1 < b2) h[y1 * b2 + z1] = make_float2(k11, d11);
        }
    }
}

// ------------------------------------------------------------------ generic one-axis pass ----
// out[a][k][b] = sum_l in[a][l][b] tw[l][k]; one thread per output.
template <int IN, int OUT>
__global__ void __launch_bounds__(256) k_dft_pass(const void* __restrict__ in_, void* __restrict__ out_,
                                                  const float2* __restrict__ tw, int A, int L, int K, int B,
                                                  const float* __restrict__ bK, const float* __restrict__ bD)
{
    const int64_t total = (int64_t)A * K * B;
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(o % B);
        const int k = (int)((o / B) % K);
        const int a = (int)(o / ((int64_t)B * K));
        const int64_t ibase = (int64_t)a * L * B + b;
        float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
        for (int l = 0; l < L; ++l) {
            const float2 w = tw[l * K + k];
            const int64_t ii = ibase + (int64_t)l * B;
            if (IN == IN_REAL) {
                const float g = reinterpret_cast<const float*>(in_)[ii];
                s0.x = fmaf(g, w.x, s0.x);
                s0.y = fmaf(g, w.y, s0.y);
            } else if (IN == IN_CPLX) {
                s0 = cmad(reinterpret_cast<const float2*>(in_)[ii], w, s0);
            } else {
                const float4 z = reinterpret_cast<const float4*>(in_)[ii];
                s0 = cmad(make_float2(z.x, z.y), w, s0);
                s1 = cmad(make_float2(z.z, z.w), w, s1);
            }
        }
        if (OUT == OUT_CPLX) {
            reinterpret_cast<float2*>(out_)[o] = s0;
        } else if (OUT == OUT_PAIR) {
            reinterpret_cast<float4*>(out_)[o] = make_float4(s0.x, s0.y, s1.x, s1.y);
        } else if (OUT == OUT_MUL) {
            const float mk = bK[o], md = bD[o];
            reinterpret_cast<float4*>(out_)[o] = make_float4(mk * s0.x, mk * s0.y, md * s0.x, md * s0.y);
        } else {
            reinterpret_cast<float2*>(out_)[o] = make_float2(s0.x, s1.x);
        }
    }
}

template <int IN, int OUT>
void pass(const void* in, void* out, const float2* tw, int A, int L, int K, int B, const float* bK,
          const float* bD, cudaStream_t st)
{
    int64_t total = (int64_t)A * K * B;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_dft_pass<IN, OUT><<<blocks, 256, 0, st>>>(in, out, tw, A, L, K, B, bK, bD);
}

// D = 1, 2: forward (multiply fused into the last pass) then inverse, one window
int generic_window(const WinDev& w, cudaStream_t st, bool spec_only)
{
    const int M = w.M;
    const int b0 = w.box[0], b1 = w.box[1];
    const float* mK = spec_only ? w.dconv : w.bK;
    const float* mD = spec_only ? w.dconv : w.bD;
    int n = 0;
    if (w.D == 1) {
        pass<IN_REAL, OUT_MUL>(w.grid, w.spec, w.twf[0], 1, b0, M, 1, mK, mD, st);
        ++n;
        if (spec_only) return n;
        pass<IN_PAIR, OUT_REAL_PAIR>(w.spec, w.h, w.twi[0], 1, M, b0, 1, nullptr, nullptr, st);
        ++n;
    } else {
        float2* t1 = reinterpret_cast<float2*>(w.buf1);
        pass<IN_REAL, OUT_CPLX>(w.grid, t1, w.twf[1], b0, b1, M, 1, nullptr, nullptr, st);       // [x][k1]
        pass<IN_CPLX, OUT_MUL>(t1, w.spec, w.twf[0], 1, b0, M, M, mK, mD, st);                  // [k0][k1]
        n += 2;
        if (spec_only) return n;
        pass<IN_PAIR, OUT_PAIR>(w.spec, w.buf1, w.twi[0], 1, M, b0, M, nullptr, nullptr, st);         // [x][k1]
        pass<IN_PAIR, OUT_REAL_PAIR>(w.buf1, w.h, w.twi[1], b0, M, b1, 1, nullptr, nullptr, st);     // [x][y]
        n += 2;
    }
    return n;
}

}  // namespace

// Shared memory of the fused D = 3 kernels for the largest box of the windows in range.
static void fused_smem(const Plan& p, int lo, int hi, size_t* s1, size_t* s2, size_t* s3, int* maxb0, int* maxMM)
{
    *s1 = *s2 = *s3 = 0;
    *maxb0 = 0;
    *maxMM = 0;
    for (int s = lo; s < hi; ++s) {
        const WinDev& w = p.win[s];
        if (w.D != 3) continue;
        const int b0 = w.box[0], b1 = w.box[1], b2 = w.box[2], M = w.M;
        *s1 = std::max(*s1, sizeof(float2) * (b2 * M + 2 * b1 * M) + sizeof(float) * b1 * b2);
        *s2 = std::max(*s2, sizeof(float2) * (b0 * M + b0 * 32) + sizeof(float4) * M * 32);
        *s3 = std::max(*s3, sizeof(float4) * (M * M + b1 * M) + sizeof(float2) * (b1 + b2) * M);
        *maxb0 = std::max(*maxb0, b0);
        *maxMM = std::max(*maxMM, M * M);
    }
}

static bool fused_attrs_set = false;

static void ensure_attrs()
{
    if (fused_attrs_set) return;
    const int big = 200 * 1024;
    cudaFuncSetAttribute(k_fwd_yz, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_xround, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_inv_yz, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    fused_attrs_set = true;
}

cudaError_t launch_transforms(const Plan& p, int window, cudaStream_t st, int* count, bool spec_only)
{
    const int lo = window < 0 ? 0 : window, hi = window < 0 ? p.P : window + 1;
    int n = 0;
    size_t s1, s2, s3;
    int maxb0, maxMM;
    fused_smem(p, lo, hi, &s1, &s2, &s3, &maxb0, &maxMM);
    if (maxb0 > 0) {
        ensure_attrs();
        dim3 g1(maxb0, hi - lo), g2((maxMM + 31) / 32, hi - lo);
        k_fwd_yz<<<g1, kT, s1, st>>>(p.wins_dev, lo);
        k_xround<<<g2, kT, s2, st>>>(p.wins_dev, lo, spec_only ? 1 : 0);
        n += 2;
        if (!spec_only) {
            k_inv_yz<<<g1, kT, s3, st>>>(p.wins_dev, lo);
            ++n;
        }
    }
    for (int s = lo; s < hi; ++s)
        if (p.win[s].D != 3) n += generic_window(p.win[s], st, spec_only);
    if (count) *count = n;
    return cudaGetLastError();
}

// One window whose descriptor is already in device memory (w_dev) and on the host (w): the same
// kernels as launch_transforms, without a plan.
cudaError_t launch_transforms_window(const WinDev& w, const WinDev* w_dev, cudaStream_t st)
{
    if (w.D == 3) {
        ensure_attrs();
        const int b0 = w.box[0], b1 = w.box[1], b2 = w.box[2], M = w.M;
        const size_t s1 = sizeof(float2) * (b2 * M + 2 * b1 * M) + sizeof(float) * b1 * b2;
        const size_t s2 = sizeof(float2) * (b0 * M + b0 * 32) + sizeof(float4) * M * 32;
        const size_t s3 = sizeof(float4) * (M * M + b1 * M) + sizeof(float2) * (b1 + b2) * M;
        dim3 g1(b0, 1), g2((M * M + 31) / 32, 1);
        k_fwd_yz<<<g1, kT, s1, st>>>(w_dev, 0);
        k_xround<<<g2, kT, s2, st>>>(w_dev, 0, 0);
        k_inv_yz<<<g1, kT, s3, st>>>(w_dev, 0);
    } else {
        generic_window(w, st, false);
    }
    return cudaGetLastError();
}

}  // namespace addker
