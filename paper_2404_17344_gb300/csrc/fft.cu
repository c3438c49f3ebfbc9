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
// same column (ky, kz); k_inv_yz also clears the consumed spread grid. D = 1, 2 use k_small_transform: one block per window does every pass.
// Each right-hand side has its own slot in every buffer (blockIdx.z, or blockIdx.y for the small
// kernel), so one launch transforms up to kMaxRhsChunk right-hand sides of all windows.
#include "common.cuh"

namespace addker {

namespace {

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
// The work is tiny (about 1e8 FMAs per product) and latency-bound, so it is spread over many small
// blocks: each x-slab is split over kSplit blocks (k_fwd_yz by kz columns, k_inv_yz by y rows, with
// no repeated arithmetic), and k_xround takes kTile columns per block.
constexpr int kT = 256;                   // threads of the single-block d < 3 transform
constexpr int kT3 = 128;                  // threads of the d = 3 blocks
constexpr int kSplit = 4;                 // blocks per x-slab
constexpr int kTile = 8;                  // columns (ky, kz) per k_xround block (16: 2 us slower)

// Pair range [lo, hi) of part `part` when `pairs` pairs are dealt out to kSplit parts.
__host__ __device__ inline void part_range(int pairs, int part, int* lo, int* hi)
{
    const int per = (pairs + kSplit - 1) / kSplit;
    *lo = min(pairs, part * per);
    *hi = min(pairs, *lo + per);
}

// Row strides that keep the second passes free of shared-memory bank conflicts: twiddle rows are read
// by lanes that differ in the row index, so a row of M float2 (a multiple of 128 bytes) is padded by one
// element; k_xround's tx region is rounded up to an even element count so the float4 arrays behind it
// stay 16-byte aligned, and k_inv_yz keeps its z twiddles transposed, tzT[kz][z] with an even row length,
// so that one float4 load gives the pair (z0, z0 + 1).
__host__ __device__ inline int even_up(int n) { return n + (n & 1); }
__host__ __device__ inline int xround_tx(int b0, int M) { return even_up(b0 * (M + 1)); }

// Shared memory of the three kernels for one box (b0, b1, b2) and bandwidth M.
__host__ __device__ inline void fused3_smem(int b0, int b1, int b2, int M, size_t* s)
{
    const int kw = 2 * ((M / 2 + kSplit - 1) / kSplit);                 // kz columns per k_fwd_yz block
    const int ny = 2 * (((b1 + 1) / 2 + kSplit - 1) / kSplit);           // y rows per k_inv_yz block
    s[0] = sizeof(float2) * (b2 * kw + b1 * M + b1 * kw) + sizeof(float) * b1 * b2;
    s[1] = sizeof(float2) * (xround_tx(b0, M) + b0 * kTile) + sizeof(float4) * M * kTile + 2 * sizeof(float) * M * kTile;
    s[2] = sizeof(float4) * (M * M + ny * M) + sizeof(float2) * (ny * (M + 1) + M * even_up(b2));
}

// block = (x-slab and kz part, window, rhs). smem: tz[b2][kw], ty[b1][M], t1[b1][kw] float2, gs[b1][b2].
//   t1[y][k] = sum_z g[x][y][z] tz[z][k];   out[x][ky][k] = sum_y ty[y][ky] t1[y][k]
// for the block's kz columns k.
__global__ void __launch_bounds__(kT3) k_fwd_yz(const WinDev* __restrict__ wins, int w0)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const WinDev& W = wins[w0 + blockIdx.y];
    if (W.D != 3) return;
    const int x = blockIdx.x / kSplit, part = blockIdx.x % kSplit;
    const int b0 = W.box[0], b1 = W.box[1], b2 = W.box[2], M = W.M;
    if (x >= b0) return;
    const int Mh = M / 2;
    int p0, p1;
    part_range(Mh, part, &p0, &p1);
    const int np = p1 - p0;
    if (np <= 0) return;
    const int kw = 2 * np, kb = 2 * p0;                         // columns kz in [kb, kb + kw)
    float2* tz = reinterpret_cast<float2*>(smem);
    float2* ty = tz + b2 * kw;
    float2* t1 = ty + b1 * M;
    float* gs = reinterpret_cast<float*>(t1 + b1 * kw);
    const int r = blockIdx.z;                                  // right-hand-side slot
    for (int i = threadIdx.x; i < b2 * kw; i += kT3) cp_async8(tz + i, W.twf[2] + (i / kw) * M + kb + i % kw);
    for (int i = threadIdx.x; i < b1 * M; i += kT3) cp_async8(ty + i, W.twf[1] + i);
    grid_dep_wait();                                           // the spread grid is complete from here on
    if (W.grid64) {                                            // compensated: the FP64 grid, rounded once
        const double* g = W.grid64 + r * W.gsz + (size_t)x * b1 * b2;
        for (int i = threadIdx.x; i < b1 * b2; i += kT3) gs[i] = (float)g[i];
    } else {
        const float* g = W.grid + r * W.gsz + (size_t)x * b1 * b2;
        for (int i = threadIdx.x; i < b1 * b2; i += kT3) cp_async4(gs + i, g + i);
    }
    cp_async_wait_all();
    __syncthreads();
    // phase 1: rows y (2 per thread, clamped), columns k (2 per thread)
    const int nb1 = (b1 + 1) / 2;
    for (int o = threadIdx.x; o < nb1 * np; o += kT3) {
        const int y0 = 2 * (o / np), y1 = min(y0 + 1, b1 - 1), k0 = 2 * (o % np);
        float2 a00 = make_float2(0.f, 0.f), a01 = a00, a10 = a00, a11 = a00;
        const float* r0 = gs + y0 * b2;
        const float* r1 = gs + y1 * b2;
#pragma unroll 4
        for (int z = 0; z < b2; ++z) {
            const float4 w = *reinterpret_cast<const float4*>(tz + z * kw + k0);
            const float g0 = r0[z], g1 = r1[z];
            a00.x = fmaf(g0, w.x, a00.x); a00.y = fmaf(g0, w.y, a00.y);
            a01.x = fmaf(g0, w.z, a01.x); a01.y = fmaf(g0, w.w, a01.y);
            a10.x = fmaf(g1, w.x, a10.x); a10.y = fmaf(g1, w.y, a10.y);
            a11.x = fmaf(g1, w.z, a11.x); a11.y = fmaf(g1, w.w, a11.y);
        }
        *reinterpret_cast<float4*>(t1 + y0 * kw + k0) = make_float4(a00.x, a00.y, a01.x, a01.y);
        if (y0 + 1 < b1) *reinterpret_cast<float4*>(t1 + y1 * kw + k0) = make_float4(a10.x, a10.y, a11.x, a11.y);
    }
    __syncthreads();
    // phase 2: rows ky, columns k (2x2 blocks)
    float2* out = reinterpret_cast<float2*>(W.buf1 + r * W.b1sz) + (size_t)x * M * M + kb;
    for (int o = threadIdx.x; o < Mh * np; o += kT3) {
        const int ky = 2 * (o / np), k = 2 * (o % np);
        float2 a00 = make_float2(0.f, 0.f), a01 = a00, a10 = a00, a11 = a00;
#pragma unroll 4
        for (int y = 0; y < b1; ++y) {
            const float4 w = *reinterpret_cast<const float4*>(ty + y * M + ky);   // ty[y][ky], ty[y][ky+1]
            const float4 t = *reinterpret_cast<const float4*>(t1 + y * kw + k);   // t1[y][k], t1[y][k+1]
            const float2 w0 = make_float2(w.x, w.y), w1 = make_float2(w.z, w.w);
            const float2 s0 = make_float2(t.x, t.y), s1 = make_float2(t.z, t.w);
            a00 = cmad(s0, w0, a00);
            a01 = cmad(s1, w0, a01);
            a10 = cmad(s0, w1, a10);
            a11 = cmad(s1, w1, a11);
        }
        *reinterpret_cast<float4*>(out + ky * M + k) = make_float4(a00.x, a00.y, a01.x, a01.y);
        *reinterpret_cast<float4*>(out + (ky + 1) * M + k) = make_float4(a10.x, a10.y, a11.x, a11.y);
    }
}

// block = (tile of kTile columns c = (ky, kz), window, rhs). smem: tx[b0][M + 1] float2, ts[b0][kTile]
// float2, ss[M][kTile] float4, then the tile's multipliers mK[M][kTile], mD[M][kTile] (staged with
// cp.async beside the tile rather than read from global memory inside the product loop).
//   S[kx][c] = m_k sum_x tx[x][kx] t[x][c];   B[x][c] = sum_kx conj(tx[x][kx]) S[kx][c]
// spec_only: write S (multiplied by dconv) to W.spec and stop.
__global__ void __launch_bounds__(kT3) k_xround(const WinDev* __restrict__ wins, int w0, int spec_only)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const WinDev& W = wins[w0 + blockIdx.y];
    if (W.D != 3) return;
    const int M = W.M, b0 = W.box[0];
    const int MM = M * M;
    const int c0 = blockIdx.x * kTile;
    if (c0 >= MM) return;
    constexpr int JP = kTile / 2;                               // column pairs per tile
    const int TXS = M + 1;                                      // padded row of tx
    float2* tx = reinterpret_cast<float2*>(smem);
    float2* ts = tx + xround_tx(b0, M);
    float4* ss = reinterpret_cast<float4*>(ts + b0 * kTile);
    const int cols = min(kTile, MM - c0);                       // M^2 need not be a multiple of kTile
    const int r = blockIdx.z;                                  // right-hand-side slot
    const float2* t = reinterpret_cast<const float2*>(W.buf1 + r * W.b1sz);
    for (int i = threadIdx.x; i < b0 * M; i += kT3) cp_async8(tx + (i / M) * TXS + i % M, W.twf[0] + i);
    grid_dep_wait();
    for (int i = threadIdx.x; i < b0 * kTile; i += kT3) {
        const int x = i / kTile, j = i % kTile;
        if (j < cols) cp_async8(ts + i, t + (size_t)x * MM + c0 + j);
        else ts[i] = make_float2(0.f, 0.f);
    }
    // the tile's multipliers, staged beside it
    float* mks = reinterpret_cast<float*>(ss + M * kTile);
    float* mds = mks + M * kTile;
    {
        const float* mK = spec_only ? W.dconv : W.bK;
        const float* mD = spec_only ? W.dconv : W.bD;
        for (int i = threadIdx.x; i < M * kTile; i += kT3) {
            const int kx = i / kTile, j = i % kTile;
            if (j < cols) {
                cp_async4(mks + i, mK + (size_t)kx * MM + c0 + j);
                cp_async4(mds + i, mD + (size_t)kx * MM + c0 + j);
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const int Mh = M / 2;
    for (int o = threadIdx.x; o < Mh * JP; o += kT3) {            // 2x2 blocks (kx, j)
        const int kx = 2 * (o / JP), j = 2 * (o % JP);
        float2 a00 = make_float2(0.f, 0.f), a01 = a00, a10 = a00, a11 = a00;
#pragma unroll 4
        for (int x = 0; x < b0; ++x) {
            const float2 w0 = tx[x * TXS + kx], w1 = tx[x * TXS + kx + 1];
            const float4 v = *reinterpret_cast<const float4*>(ts + x * kTile + j);
            const float2 s0 = make_float2(v.x, v.y), s1 = make_float2(v.z, v.w);
            a00 = cmad(s0, w0, a00);
            a01 = cmad(s1, w0, a01);
            a10 = cmad(s0, w1, a10);
            a11 = cmad(s1, w1, a11);
        }
        const float2 acc[2][2] = {{a00, a01}, {a10, a11}};
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (j + q >= cols) {
                    if (!spec_only) ss[(kx + rr) * kTile + j + q] = make_float4(0.f, 0.f, 0.f, 0.f);
                    continue;
                }
                const size_t k = (size_t)(kx + rr) * MM + c0 + j + q;
                const float a = mks[(kx + rr) * kTile + j + q], d = mds[(kx + rr) * kTile + j + q];
                const float4 v = make_float4(a * acc[rr][q].x, a * acc[rr][q].y, d * acc[rr][q].x, d * acc[rr][q].y);
                if (spec_only) W.spec[k] = v;
                else ss[(kx + rr) * kTile + j + q] = v;
            }
    }
    if (spec_only) return;
    __syncthreads();
    const int nbx = (b0 + 1) / 2;
    for (int o = threadIdx.x; o < nbx * JP; o += kT3) {           // 2x2 blocks (x, j)
        const int x0 = 2 * (o / JP), x1 = min(x0 + 1, b0 - 1), j = 2 * (o % JP);
        float2 k00 = make_float2(0.f, 0.f), k01 = k00, k10 = k00, k11 = k00;
        float2 d00 = k00, d01 = k00, d10 = k00, d11 = k00;
#pragma unroll 4
        for (int kx = 0; kx < M; ++kx) {
            const float2 w0 = tx[x0 * TXS + kx], w1 = tx[x1 * TXS + kx];
            const float4 s0 = ss[kx * kTile + j], s1 = ss[kx * kTile + j + 1];
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
        float4* B = W.buf2 + r * W.b2sz + c0 + j;
        const bool q1 = j + 1 < cols;
        B[(size_t)x0 * MM] = make_float4(k00.x, k00.y, d00.x, d00.y);
        if (q1) B[(size_t)x0 * MM + 1] = make_float4(k01.x, k01.y, d01.x, d01.y);
        if (x0 + 1 < b0) {
            B[(size_t)x1 * MM] = make_float4(k10.x, k10.y, d10.x, d10.y);
            if (q1) B[(size_t)x1 * MM + 1] = make_float4(k11.x, k11.y, d11.x, d11.y);
        }
    }
}

// block = (x-slab and y part, window, rhs). smem: bs[M][M] float4, b1s[ny][M] float4, ty[ny][M + 1],
// tzT[M][even_up(b2)] float2, for the block's rows y = yb .. yb + ny - 1 (the last row repeated when b1 is odd):
//   B1[y][kz] = sum_ky conj(ty[y][ky]) B[x][ky][kz];   h[x][y][z] = Re sum_kz conj(tz[z][kz]) B1[y][kz]
// The block also zeroes its rows of the spread grid, which k_fwd_yz has consumed, so d = 3 grids
// need no separate clearing before the next spread.
__global__ void __launch_bounds__(kT3) k_inv_yz(const WinDev* __restrict__ wins, int w0)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const WinDev& W = wins[w0 + blockIdx.y];
    if (W.D != 3) return;
    const int x = blockIdx.x / kSplit, part = blockIdx.x % kSplit;
    const int b0 = W.box[0], b1 = W.box[1], b2 = W.box[2], M = W.M;
    if (x >= b0) return;
    const int nb1 = (b1 + 1) / 2;
    int q0, q1;
    part_range(nb1, part, &q0, &q1);
    const int nq = q1 - q0;
    if (nq <= 0) return;
    const int yb = 2 * q0, ny = 2 * nq;                         // local rows; global y = yb + local
    const int MM = M * M;
    float4* bs = reinterpret_cast<float4*>(smem);
    float4* b1s = bs + MM;
    const int TYS = M + 1, TZS = even_up(b2);                   // padded ty row; transposed tz row
    float2* ty = reinterpret_cast<float2*>(b1s + ny * M);
    float2* tzT = ty + ny * TYS;
    const int r = blockIdx.z;                                  // right-hand-side slot
    const float4* B = W.buf2 + r * W.b2sz + (size_t)x * MM;
    for (int i = threadIdx.x; i < ny * M; i += kT3)
        cp_async8(ty + (i / M) * TYS + i % M, W.twf[1] + min(yb + i / M, b1 - 1) * M + i % M);
    for (int i = threadIdx.x; i < b2 * M; i += kT3) cp_async8(tzT + (i % M) * TZS + i / M, W.twf[2] + i);
    if (b2 & 1)
        for (int kz = threadIdx.x; kz < M; kz += kT3) tzT[kz * TZS + b2] = make_float2(0.f, 0.f);
    grid_dep_wait();
    for (int i = threadIdx.x; i < MM; i += kT3) cp_async16(bs + i, B + i);
    const int zrows = min(ny, b1 - yb);
    if (W.grid64) {
        double* g = W.grid64 + r * W.gsz + (size_t)x * b1 * b2 + (size_t)yb * b2;
        for (int i = threadIdx.x; i < zrows * b2; i += kT3) g[i] = 0.0;
    } else {
        float* g = W.grid + r * W.gsz + (size_t)x * b1 * b2 + (size_t)yb * b2;
        for (int i = threadIdx.x; i < zrows * b2; i += kT3) g[i] = 0.f;
    }
    cp_async_wait_all();
    __syncthreads();
    const int Mh = M / 2;
    for (int o = threadIdx.x; o < nq * Mh; o += kT3) {            // 2x2 blocks (y, kz), local rows
        // columns kz and kz + M/2, so the lanes of a row read one contiguous run of bs
        const int y0 = 2 * (o / Mh), kz = o % Mh, kz1 = kz + Mh;
        float2 k00 = make_float2(0.f, 0.f), k01 = k00, k10 = k00, k11 = k00;
        float2 d00 = k00, d01 = k00, d10 = k00, d11 = k00;
#pragma unroll 4
        for (int ky = 0; ky < M; ++ky) {
            const float2 w0 = ty[y0 * TYS + ky], w1 = ty[(y0 + 1) * TYS + ky];
            const float4 s0 = bs[ky * M + kz], s1 = bs[ky * M + kz1];
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
        b1s[y0 * M + kz1] = make_float4(k01.x, k01.y, d01.x, d01.y);
        b1s[(y0 + 1) * M + kz] = make_float4(k10.x, k10.y, d10.x, d10.y);
        b1s[(y0 + 1) * M + kz1] = make_float4(k11.x, k11.y, d11.x, d11.y);
    }
    __syncthreads();
    float2* h = W.h + r * W.gsz + (size_t)x * b1 * b2;
    const int nb2 = (b2 + 1) / 2;
    for (int o = threadIdx.x; o < nq * nb2; o += kT3) {          // 2x2 blocks (y, z), local rows
        const int l0 = 2 * (o / nb2);
        const int z0 = 2 * (o % nb2), z1 = z0 + 1;                // z1 = b2 reads the zero padding of tzT
        float k00 = 0.f, k01 = 0.f, k10 = 0.f, k11 = 0.f, d00 = 0.f, d01 = 0.f, d10 = 0.f, d11 = 0.f;
#pragma unroll 4
        for (int kz = 0; kz < M; ++kz) {
            const float4 w = *reinterpret_cast<const float4*>(tzT + kz * TZS + z0);
            const float2 w0 = make_float2(w.x, w.y), w1 = make_float2(w.z, w.w);
            const float4 s0 = b1s[l0 * M + kz], s1 = b1s[(l0 + 1) * M + kz];
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
        const int y0 = yb + l0, y1 = y0 + 1;
        h[y0 * b2 + z0] = make_float2(k00, d00);
        if (z0 + 1 < b2) h[y0 * b2 + z1] = make_float2(k01, d01);
        if (y1 < b1) {
            h[y1 * b2 + z0] = make_float2(k10, d10);
            if (z0 + 1 < b2) h[y1 * b2 + z1] = make_float2(k11, d11);
        }
    }
}

// ------------------------------------------------------------ D = 1, 2: one block per window ----
// The whole transform of a small grid in one block (box <= 64^2 samples, M <= 64), every pass from
// shared memory, one thread per output:
//   D = 1:  G[k] = sum_x g[x] tf[x][k];  S = (bK, bD) G;  h[x] = Re sum_k S[k] conj(tf[x][k])
//   D = 2:  t[x][ky] = sum_y g[x][y] tf1[y][ky];  G[kx][ky] = sum_x t[x][ky] tf0[x][kx];  S = (bK, bD) G;
//           B[x][ky] = sum_kx S[kx][ky] conj(tf0[x][kx]);  h[x][y] = Re sum_ky B[x][ky] conj(tf1[y][ky])
// The grid is zeroed once read. spec_only: write G dconv to spec and stop.
// Bytes in front of S: the grid, t and G of the forward passes, or B of the inverse, whichever is larger
// (16-byte multiple).
__host__ __device__ inline size_t small_front(int b0, int b1, int M, int D)
{
    const int MD = D == 2 ? M * M : M;
    const size_t fwd = sizeof(float) * ((b0 * b1 + 3) & ~3) + sizeof(float2) * ((D == 2 ? b0 * M : 0) + MD + (MD & 1));
    const size_t inv = D == 2 ? sizeof(float4) * b0 * M : 0;
    return fwd > inv ? fwd : inv;
}

template <int D>
__global__ void __launch_bounds__(kT) k_small_transform(const WinDev* __restrict__ wins, int w0, int spec_only,
                                                        int smem_bytes)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const WinDev& W = wins[w0 + blockIdx.x];
    if (W.D != D) return;
    const int r = blockIdx.y;
    const int b0 = W.box[0], b1 = D == 2 ? W.box[1] : 1, M = W.M;
    const int MD = D == 2 ? M * M : M;
    float* grid = W.grid + r * W.gsz;
    float2* h = W.h + r * W.gsz;
    // gs, t and G are dead once S is written, so B reuses their space (see small_smem)
    float* gs = reinterpret_cast<float*>(smem);                                   // b0 * b1
    float2* t = reinterpret_cast<float2*>(smem + sizeof(float) * ((b0 * b1 + 3) & ~3));   // b0 * M (D = 2)
    float2* G = t + (D == 2 ? b0 * M : 0);                                       // MD
    float4* B = reinterpret_cast<float4*>(smem);                                 // b0 * M (D = 2)
    float4* S = reinterpret_cast<float4*>(smem + small_front(b0, b1, M, D));     // MD
    // the twiddles go to shared memory too when the launch provided room (every pass reads them
    // b0 or M times; from global memory each pass would wait on L2 per term)
    float2* tws = reinterpret_cast<float2*>(S + MD);
    const bool stw = small_front(b0, b1, M, D) + sizeof(float4) * MD + sizeof(float2) * (b0 + (D == 2 ? b1 : 0)) * M <=
                     (size_t)smem_bytes;
    if (stw) {
        for (int i = threadIdx.x; i < b0 * M; i += kT) cp_async8(tws + i, W.twf[0] + i);
        if (D == 2)
            for (int i = threadIdx.x; i < b1 * M; i += kT) cp_async8(tws + b0 * M + i, W.twf[1] + i);
    }
    const float2* tf0 = stw ? tws : W.twf[0];
    const float2* tf1 = stw ? tws + b0 * M : W.twf[1];
    grid_dep_wait();
    if (W.grid64) {                                            // compensated: the FP64 grid, rounded once
        double* g64 = W.grid64 + r * W.gsz;
        for (int i = threadIdx.x; i < b0 * b1; i += kT) {
            gs[i] = (float)g64[i];
            g64[i] = 0.0;                                      // each thread clears what it read
        }
    } else {
        for (int i = threadIdx.x; i < b0 * b1; i += kT) cp_async4(gs + i, grid + i);
        cp_async_wait_all();
        for (int i = threadIdx.x; i < b0 * b1; i += kT) grid[i] = 0.f;     // each thread clears what it copied
    }
    __syncthreads();
    if (D == 1) {
        for (int k = threadIdx.x; k < M; k += kT) {
            float2 acc = make_float2(0.f, 0.f);
            for (int x = 0; x < b0; ++x) {
                const float2 w = tf0[x * M + k];
                acc.x = fmaf(gs[x], w.x, acc.x);
                acc.y = fmaf(gs[x], w.y, acc.y);
            }
            G[k] = acc;
        }
    } else {
        for (int o = threadIdx.x; o < b0 * M; o += kT) {
            const int x = o / M, ky = o % M;
            float2 acc = make_float2(0.f, 0.f);
            for (int y = 0; y < b1; ++y) {
                const float2 w = tf1[y * M + ky];
                acc.x = fmaf(gs[x * b1 + y], w.x, acc.x);
                acc.y = fmaf(gs[x * b1 + y], w.y, acc.y);
            }
            t[o] = acc;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < MD; o += kT) {
            const int kx = o / M, ky = o % M;
            float2 acc = make_float2(0.f, 0.f);
            for (int x = 0; x < b0; ++x) acc = cmad(t[x * M + ky], tf0[x * M + kx], acc);
            G[o] = acc;
        }
    }
    __syncthreads();
    const float* mK = spec_only ? W.dconv : W.bK;
    const float* mD = spec_only ? W.dconv : W.bD;
    for (int o = threadIdx.x; o < MD; o += kT) {
        const float a = mK[o], d = mD[o];
        const float4 v = make_float4(a * G[o].x, a * G[o].y, d * G[o].x, d * G[o].y);
        if (spec_only) W.spec[o] = v;
        else S[o] = v;
    }
    if (spec_only) return;
    __syncthreads();
    if (D == 1) {
        for (int x = threadIdx.x; x < b0; x += kT) {
            float hK = 0.f, hD = 0.f;
            for (int k = 0; k < M; ++k) {
                const float4 v = S[k];
                const float2 w = tf0[x * M + k];
                hK = fmaf(v.x, w.x, fmaf(v.y, w.y, hK));      // Re(s conj(w))
                hD = fmaf(v.z, w.x, fmaf(v.w, w.y, hD));
            }
            h[x] = make_float2(hK, hD);
        }
    } else {
        for (int o = threadIdx.x; o < b0 * M; o += kT) {
            const int x = o / M, ky = o % M;
            float2 aK = make_float2(0.f, 0.f), aD = make_float2(0.f, 0.f);
            for (int kx = 0; kx < M; ++kx) {
                const float4 v = S[kx * M + ky];
                const float2 w = tf0[x * M + kx];
                aK = cmadc(make_float2(v.x, v.y), w, aK);
                aD = cmadc(make_float2(v.z, v.w), w, aD);
            }
            B[o] = make_float4(aK.x, aK.y, aD.x, aD.y);
        }
        __syncthreads();
        for (int o = threadIdx.x; o < b0 * b1; o += kT) {
            const int x = o / b1, y = o % b1;
            float hK = 0.f, hD = 0.f;
            for (int ky = 0; ky < M; ++ky) {
                const float4 v = B[x * M + ky];
                const float2 w = tf1[y * M + ky];
                hK = fmaf(v.x, w.x, fmaf(v.y, w.y, hK));
                hD = fmaf(v.z, w.x, fmaf(v.w, w.y, hD));
            }
            h[o] = make_float2(hK, hD);
        }
    }
}

// Shared memory of k_small_transform for window w: the passes' buffers, plus the twiddles when that
// stays within 160 KB (the kernel checks the launch size itself).
size_t small_smem(const WinDev& w)
{
    const int b0 = w.box[0], b1 = w.D == 2 ? w.box[1] : 1, M = w.M;
    const int MD = w.D == 2 ? M * M : M;
    const size_t base = small_front(b0, b1, M, w.D) + sizeof(float4) * MD;
    const size_t with_tw = base + sizeof(float2) * (b0 + (w.D == 2 ? b1 : 0)) * M;
    return with_tw <= 160 * 1024 ? with_tw : base;
}

}  // namespace

// Shared memory of the fused D = 3 kernels for the largest box of the windows in range.
static void fused_smem(const Plan& p, int lo, int hi, size_t* sm, int* maxb0, int* maxMM)
{
    sm[0] = sm[1] = sm[2] = 0;
    *maxb0 = 0;
    *maxMM = 0;
    for (int s = lo; s < hi; ++s) {
        const WinDev& w = p.win[s];
        if (w.D != 3) continue;
        size_t t[3];
        fused3_smem(w.box[0], w.box[1], w.box[2], w.M, t);
        for (int q = 0; q < 3; ++q) sm[q] = std::max(sm[q], t[q]);
        *maxb0 = std::max(*maxb0, w.box[0]);
        *maxMM = std::max(*maxMM, w.M * w.M);
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
    cudaFuncSetAttribute(k_small_transform<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_small_transform<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    fused_attrs_set = true;
}

cudaError_t launch_transforms(const Plan& p, int window, int nrhs, cudaStream_t st, int* count, bool spec_only)
{
    const int lo = window < 0 ? 0 : window, hi = window < 0 ? p.P : window + 1;
    if (spec_only) nrhs = 1;
    int n = 0;
    size_t f3[3];
    int maxb0, maxMM;
    fused_smem(p, lo, hi, f3, &maxb0, &maxMM);
    ensure_attrs();
    if (maxb0 > 0) {
        dim3 g1(maxb0 * kSplit, hi - lo, nrhs), g2((maxMM + kTile - 1) / kTile, hi - lo, nrhs);
        launch_k(true, k_fwd_yz, g1, dim3(kT3), f3[0], st, (const WinDev*)p.wins_dev, lo);
        launch_k(true, k_xround, g2, dim3(kT3), f3[1], st, (const WinDev*)p.wins_dev, lo, spec_only ? 1 : 0);
        n += 2;
        if (!spec_only) {
            launch_k(true, k_inv_yz, g1, dim3(kT3), f3[2], st, (const WinDev*)p.wins_dev, lo);
            ++n;
        }
    }
    size_t sm[3] = {0, 0, 0};
    for (int s = lo; s < hi; ++s)
        if (p.win[s].D < 3) sm[p.win[s].D] = std::max(sm[p.win[s].D], small_smem(p.win[s]));
    for (int D = 1; D <= 2; ++D) {
        if (sm[D] == 0) continue;
        launch_k(true, D == 1 ? k_small_transform<1> : k_small_transform<2>, dim3(hi - lo, nrhs), dim3(kT), sm[D],
                 st, (const WinDev*)p.wins_dev, lo, spec_only ? 1 : 0, (int)sm[D]);
        ++n;
    }
    if (count) *count = n;
    return cudaGetLastError();
}

// One window whose descriptor is already in device memory (w_dev) and on the host (w): the same
// kernels as launch_transforms, without a plan, one right-hand side.
cudaError_t launch_transforms_window(const WinDev& w, const WinDev* w_dev, cudaStream_t st)
{
    ensure_attrs();
    if (w.D == 3) {
        size_t f3[3];
        fused3_smem(w.box[0], w.box[1], w.box[2], w.M, f3);
        dim3 g1(w.box[0] * kSplit, 1, 1), g2((w.M * w.M + kTile - 1) / kTile, 1, 1);
        k_fwd_yz<<<g1, kT3, f3[0], st>>>(w_dev, 0);
        k_xround<<<g2, kT3, f3[1], st>>>(w_dev, 0, 0);
        k_inv_yz<<<g1, kT3, f3[2], st>>>(w_dev, 0);
    } else if (w.D == 2) {
        k_small_transform<2><<<dim3(1, 1), kT, small_smem(w), st>>>(w_dev, 0, 0, (int)small_smem(w));
    } else {
        k_small_transform<1><<<dim3(1, 1), kT, small_smem(w), st>>>(w_dev, 0, 0, (int)small_smem(w));
    }
    return cudaGetLastError();
}

}  // namespace addker
