// The transforms between the spread grid and the interpolation grids (Sec. 3.1: the FFT inside the
// adjoint NFFT, the multiplication by the kernel's Fourier coefficients, the FFT inside the NFFT).
//
//   forward:  G_k   = sum_l g_l exp(-2 pi i k.l/n),  k in I_M^D, l over the grid's bounding box
//   multiply: S^K_k = bK_k G_k,   S^D_k = bD_k G_k  (bK, bD: coefficients over window transforms)
//   inverse:  h_l   = Re sum_k S_k exp(+2 pi i k.l/n), l over the bounding box, for both spectra
//
// Only the M^D retained frequencies and the box of grid points that points can touch are ever
// computed: a pruned transform done axis by axis as batched small DFTs (box <= 64 samples to
// M <= 64 frequencies). Each pass is out[a][k][b] = sum_l in[a][l][b] tw[l][k], one thread per
// output; b is the fastest index, so reads are coalesced across a warp.
#include "common.cuh"

namespace addker {

namespace {

enum { IN_REAL = 0, IN_CPLX = 1, IN_PAIR = 2 };
enum { OUT_CPLX = 1, OUT_PAIR = 2, OUT_MUL = 3, OUT_REAL_PAIR = 4 };

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

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
                const float2 z = reinterpret_cast<const float2*>(in_)[ii];
                s0.x = fmaf(z.x, w.x, fmaf(-z.y, w.y, s0.x));
                s0.y = fmaf(z.x, w.y, fmaf(z.y, w.x, s0.y));
            } else {
                const float4 z = reinterpret_cast<const float4*>(in_)[ii];
                s0.x = fmaf(z.x, w.x, fmaf(-z.y, w.y, s0.x));
                s0.y = fmaf(z.x, w.y, fmaf(z.y, w.x, s0.y));
                s1.x = fmaf(z.z, w.x, fmaf(-z.w, w.y, s1.x));
                s1.y = fmaf(z.z, w.y, fmaf(z.w, w.x, s1.y));
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

}  // namespace

// grid (box, real) -> spec = (bK G, bD G) on I_M^D, layout [k0][k1][k2] (last fastest)
static cudaError_t forward_with(const WinDev& w, const float* mK, const float* mD, float4* out, cudaStream_t st)
{
    const int M = w.M;
    const int b0 = w.box[0], b1 = w.box[1], b2 = w.box[2];
    if (w.D == 1) {
        pass<IN_REAL, OUT_MUL>(w.grid, out, w.twf[0], 1, b0, M, 1, mK, mD, st);
    } else if (w.D == 2) {
        float2* t1 = reinterpret_cast<float2*>(w.buf1);
        pass<IN_REAL, OUT_CPLX>(w.grid, t1, w.twf[1], b0, b1, M, 1, nullptr, nullptr, st);     // [x][k1]
        pass<IN_CPLX, OUT_MUL>(t1, out, w.twf[0], 1, b0, M, M, mK, mD, st);                   // [k0][k1]
    } else {
        float2* t1 = reinterpret_cast<float2*>(w.buf1);
        float2* t2 = reinterpret_cast<float2*>(w.buf2);
        pass<IN_REAL, OUT_CPLX>(w.grid, t1, w.twf[2], b0 * b1, b2, M, 1, nullptr, nullptr, st);   // [x][y][k2]
        pass<IN_CPLX, OUT_CPLX>(t1, t2, w.twf[1], b0, b1, M, M, nullptr, nullptr, st);            // [x][k1][k2]
        pass<IN_CPLX, OUT_MUL>(t2, out, w.twf[0], 1, b0, M, M * M, mK, mD, st);                   // [k0][k1][k2]
    }
    return cudaGetLastError();
}

cudaError_t launch_fft_forward(const WinDev& w, cudaStream_t st)
{
    return forward_with(w, w.bK, w.bD, w.spec, st);
}

cudaError_t launch_adjoint_only(const WinDev& w, const float* dconv, float4* out, cudaStream_t st)
{
    return forward_with(w, dconv, dconv, out, st);
}

// spec (two spectra on I_M^D) -> h (box, float2 = (h^K, h^der))
cudaError_t launch_fft_inverse(const WinDev& w, cudaStream_t st)
{
    const int M = w.M;
    const int b0 = w.box[0], b1 = w.box[1], b2 = w.box[2];
    if (w.D == 1) {
        pass<IN_PAIR, OUT_REAL_PAIR>(w.spec, w.h, w.twi[0], 1, M, b0, 1, nullptr, nullptr, st);
    } else if (w.D == 2) {
        pass<IN_PAIR, OUT_PAIR>(w.spec, w.buf1, w.twi[0], 1, M, b0, M, nullptr, nullptr, st);         // [x][k1]
        pass<IN_PAIR, OUT_REAL_PAIR>(w.buf1, w.h, w.twi[1], b0, M, b1, 1, nullptr, nullptr, st);     // [x][y]
    } else {
        pass<IN_PAIR, OUT_PAIR>(w.spec, w.buf2, w.twi[0], 1, M, b0, M * M, nullptr, nullptr, st);     // [x][k1][k2]
        pass<IN_PAIR, OUT_PAIR>(w.buf2, w.buf1, w.twi[1], b0, M, b1, M, nullptr, nullptr, st);        // [x][y][k2]
        pass<IN_PAIR, OUT_REAL_PAIR>(w.buf1, w.h, w.twi[2], b0 * b1, M, b2, 1, nullptr, nullptr, st); // [x][y][z]
    }
    return cudaGetLastError();
}

}  // namespace addker
