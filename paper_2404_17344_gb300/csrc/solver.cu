// The regression system and GP training on top of the fast products (include/addker.h:
// addker_cg, addker_gp_grad).
//
// Sec. 3.3: (K + beta I) x = y (eq. "regression_system"), solved as in the paper with unpreconditioned
// conjugate gradients, here for several right-hand sides at once: every CG iteration is one batched
// product K P (the fast summation, up to eight right-hand sides per launch) plus three small kernels
// on the N x nrhs vectors. Vectors are FP32 like the products; every inner product is accumulated in
// FP64 (per-block sums in FP64 registers, one double atomic add per block). The host reads the nrhs
// residual norms after each iteration to decide convergence (one small copy per iteration).
//
// GP training: with A = K + beta I, alpha = A^{-1} y and probes z_i (Hutchinson's trace estimator),
//   dL/dtheta = 1/2 alpha^T (dA/dtheta) alpha - 1/2 (1/m) sum_i (A^{-1} z_i)^T (dA/dtheta) z_i,
// dA/d ell_s = dK/d ell_s (the derivative-kernel products), dA/d sigma_f = (2/sigma_f) K,
// dA/d beta = I: one CG solve with 1 + m right-hand sides and one fused product on [alpha, z_1..z_m].
#include <cmath>
#include <vector>

#include "common.cuh"

namespace addker {

namespace {

// return the ABI status of a failed CUDA call / of a failed step
#define CK(call)                                                                   \
    do {                                                                           \
        const cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? ADDKER_ENOMEM : ADDKER_ECUDA; \
    } while (0)
#define CS(status)                        \
    do {                                  \
        const int s_ = (status);          \
        if (s_ != ADDKER_OK) return s_;   \
    } while (0)

constexpr int kT = 256;

__device__ __forceinline__ double block_sum(double x)
{
    __shared__ double ws[kT / 32];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) ws[warp] = x;
    __syncthreads();
    x = 0.0;
    if (warp == 0) {
        x = lane < kT / 32 ? ws[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    }
    return x;                              // valid in thread 0
}

// out[j] += sum_i A[j sa + i] (B[j sb + i] + c A[j sa + i]), column j = blockIdx.y
__global__ void __launch_bounds__(kT) k_dot_cols(const float* __restrict__ A, int64_t sa, const float* __restrict__ B,
                                                int64_t sb, float c, int64_t N, double* __restrict__ out)
{
    const int j = blockIdx.y;
    const float* a = A + j * sa;
    const float* b = B + j * sb;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < N; i += (int64_t)gridDim.x * kT)
        acc += (double)a[i] * ((double)b[i] + (double)c * (double)a[i]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) atomicAdd(out + j, acc);
}

// R = Y - (KX + beta X), P = R; column j = blockIdx.y (all N x nrhs, leading dimension N)
__global__ void __launch_bounds__(kT) k_cg_init(const float* __restrict__ Y, const float* __restrict__ X,
                                               const float* __restrict__ KX, float beta, int64_t N,
                                               float* __restrict__ R, float* __restrict__ P)
{
    const int64_t o = blockIdx.y * N;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < N; i += (int64_t)gridDim.x * kT) {
        const float r = Y[o + i] - (KX[o + i] + beta * X[o + i]);
        R[o + i] = r;
        P[o + i] = r;
    }
}

// alpha_j = rr_j / pAp_j (0 for a finished column); X += alpha P; R -= alpha (KP + beta P); rr_new_j += R.R
__global__ void __launch_bounds__(kT) k_cg_step(float* __restrict__ X, float* __restrict__ R,
                                               const float* __restrict__ P, const float* __restrict__ KP, float beta,
                                               const double* __restrict__ rr, const double* __restrict__ pAp,
                                               const int* __restrict__ active, int64_t N, double* __restrict__ rr_new)
{
    const int j = blockIdx.y;
    const int64_t o = j * N;
    const float a = active[j] ? (float)(rr[j] / pAp[j]) : 0.f;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < N; i += (int64_t)gridDim.x * kT) {
        const float pi = P[o + i];
        X[o + i] = fmaf(a, pi, X[o + i]);
        const float r = fmaf(-a, KP[o + i] + beta * pi, R[o + i]);
        R[o + i] = r;
        acc += (double)r * (double)r;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) atomicAdd(rr_new + j, acc);
}

// P = R + (rr_new_j / rr_j) P for the columns still iterating
__global__ void __launch_bounds__(kT) k_cg_dir(const float* __restrict__ R, float* __restrict__ P,
                                              const double* __restrict__ rr, const double* __restrict__ rr_new,
                                              const int* __restrict__ active, int64_t N)
{
    const int j = blockIdx.y;
    if (!active[j]) return;
    const int64_t o = j * N;
    const float b = (float)(rr_new[j] / rr[j]);
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < N; i += (int64_t)gridDim.x * kT)
        P[o + i] = fmaf(b, P[o + i], R[o + i]);
}

// ------------------------------------------------------------------ the preconditioner ----
// Not in the paper, which solves with plain CG to tolerance 1e-3. At a small noise variance beta the
// system is ill-conditioned (kappa ~ N / beta for a kernel wide against the data): K's large eigenvalues
// belong to every window's lowest Fourier modes, since K_s = sum_k c_hat_k e^{2 pi i k.(x - x')} with even
// coefficients gives each pair +-k the term 2 c_hat_k [cos cos + sin sin]. The preconditioner
//     B = beta I + U W U^T,   U = [1, cos(2 pi k.x^{W_s}), sin(2 pi k.x^{W_s}), ...],
//     W = diag(sigma_f^2 sum_s c_hat_0^s, sigma_f^2 2 c_hat_k^s, ...)
// keeps the modes |k|_inf <= band of every window with N sigma_f^2 2 c_hat_k >= beta (they lift an
// eigenvalue above the noise level) and is applied by the Woodbury identity
//     B^{-1} r = (r - U (beta W^{-1} + U^T U)^{-1} U^T r) / beta,
// with U^T U accumulated in FP64 (the cosines of nearby frequencies on a small data ball are nearly
// dependent: condition numbers of 1e13 are typical) and factored by Cholesky in FP64.

// out[idx] = the window's point with original index idx (scatter of the cell-sorted copy)
__global__ void k_unsort(const float4* __restrict__ pts, int64_t N, float4* __restrict__ out)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    const float4 q = pts[j];
    out[__float_as_int(q.w)] = q;
}

// Columns col0 + 2m (cosine) and col0 + 2m + 1 (sine) of U for the nm modes kv[3m .. 3m+3) of one window,
// from its points in original order.
__global__ void k_fourier_cols(const float4* __restrict__ x, int64_t N, const int* __restrict__ kv, int nm,
                               float* __restrict__ U, int col0)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 q = x[i];
    for (int m = 0; m < nm; ++m) {
        const float ph = (float)kv[3 * m] * q.x + (float)kv[3 * m + 1] * q.y + (float)kv[3 * m + 2] * q.z;
        float sn, cs;
        sincospif(2.0f * ph, &sn, &cs);
        U[(int64_t)(col0 + 2 * m) * N + i] = cs;
        U[(int64_t)(col0 + 2 * m + 1) * N + i] = sn;
    }
}

__global__ void k_fill(float* __restrict__ a, int64_t n, float v)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// G[a r + b] += sum_i U[a][i] U[b][i] (FP64) for the 16 x 16 tile pair (ta <= tb) of blockIdx.x, over the row
// chunks blockIdx.y, blockIdx.y + gridDim.y, ...; the lower triangle is mirrored afterwards.
constexpr int kGT = 16, kGR = 256;
__global__ void __launch_bounds__(kGT * kGT) k_gram(const float* __restrict__ U, int64_t N, int r,
                                                    const int2* __restrict__ tiles, double* __restrict__ G)
{
    __shared__ float sa[kGR][kGT + 1];
    __shared__ float sb[kGR][kGT + 1];
    const int2 tp = tiles[blockIdx.x];
    const int ti = threadIdx.x / kGT, tj = threadIdx.x % kGT;
    const int a = tp.x * kGT + ti, b = tp.y * kGT + tj;
    double acc = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.y * kGR; i0 < N; i0 += (int64_t)gridDim.y * kGR) {
        for (int e = threadIdx.x; e < kGR * kGT; e += blockDim.x) {
            const int c = e / kGR, row = e % kGR;
            const int64_t i = i0 + row;
            const int ca = tp.x * kGT + c, cb = tp.y * kGT + c;
            sa[row][c] = (i < N && ca < r) ? U[(int64_t)ca * N + i] : 0.f;
            sb[row][c] = (i < N && cb < r) ? U[(int64_t)cb * N + i] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int row = 0; row < kGR; ++row) acc = fma((double)sa[row][ti], (double)sb[row][tj], acc);
        __syncthreads();
    }
    if (a < r && b < r && (tp.x != tp.y || ti <= tj)) atomicAdd(G + (int64_t)a * r + b, acc);
}

// L = Cholesky factor (lower, row-major r x r) of beta diag(1/w) + G, G given in its upper triangle.
// One block. *fail = 1 when a pivot is not positive (the preconditioner is then not used).
__global__ void k_cholesky(const double* __restrict__ G, const double* __restrict__ w, double beta, int r,
                           double* __restrict__ L, int* __restrict__ fail)
{
    __shared__ double piv;
    for (int64_t e = threadIdx.x; e < (int64_t)r * r; e += blockDim.x) {
        const int i = (int)(e / r), j = (int)(e % r);
        L[e] = i >= j ? G[(int64_t)j * r + i] + (i == j ? beta / w[i] : 0.0) : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        if (threadIdx.x == 0) {
            const double d = L[(int64_t)k * r + k];
            piv = d > 0.0 ? sqrt(d) : 0.0;
            if (!(d > 0.0)) *fail = 1;
            L[(int64_t)k * r + k] = piv;
        }
        __syncthreads();
        if (piv == 0.0) return;
        for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) L[(int64_t)i * r + k] /= piv;
        __syncthreads();
        const int m = r - k - 1;
        for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
            const int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
            if (j <= i) L[(int64_t)i * r + j] -= L[(int64_t)i * r + k] * L[(int64_t)j * r + k];
        }
        __syncthreads();
    }
}

// T[c ng + j] += sum_i U[c][i] R[j][i] for the rows of chunk blockIdx.x and ng <= 8 columns of R (leading
// dimension N): the chunk of R in shared memory, one warp per column c of U at a time.
constexpr int kCH = 1024;
__global__ void __launch_bounds__(256) k_utr(const float* __restrict__ U, int64_t N, int r, const float* __restrict__ R,
                                             int ng, double* __restrict__ T)
{
    __shared__ float rs[kCH][9];
    const int64_t i0 = (int64_t)blockIdx.x * kCH;
    for (int e = threadIdx.x; e < kCH * ng; e += blockDim.x) {
        const int j = e / kCH, row = e % kCH;
        rs[row][j] = i0 + row < N ? R[(int64_t)j * N + i0 + row] : 0.f;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = warp; c < r; c += blockDim.x >> 5) {
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const float* u = U + (int64_t)c * N + i0;
        for (int row = lane; row < kCH; row += 32) {
            const float uv = i0 + row < N ? u[row] : 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < ng) acc[j] = fmaf(uv, rs[row][j], acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j >= ng) break;
            float x = acc[j];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) atomicAdd(T + (int64_t)c * ng + j, (double)x);
        }
    }
}

// T[:, j] <- (L L^T)^{-1} T[:, j] in place, warp j (ng warps, one block); L lower, row-major r x r.
__global__ void k_pc_solve(const double* __restrict__ L, int r, int ng, double* __restrict__ T)
{
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (j >= ng) return;
    for (int k = 0; k < r; ++k) {                              // L y = t
        double acc = 0.0;
        for (int i = lane; i < k; i += 32) acc += L[(int64_t)k * r + i] * T[(int64_t)i * ng + j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) T[(int64_t)k * ng + j] = (T[(int64_t)k * ng + j] - acc) / L[(int64_t)k * r + k];
        __syncwarp();
    }
    for (int k = r - 1; k >= 0; --k) {                         // L^T z = y
        double acc = 0.0;
        for (int i = k + 1 + lane; i < r; i += 32) acc += L[(int64_t)i * r + k] * T[(int64_t)i * ng + j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) T[(int64_t)k * ng + j] = (T[(int64_t)k * ng + j] - acc) / L[(int64_t)k * r + k];
        __syncwarp();
    }
}

// Z[j][i] = (R[j][i] - sum_c U[c][i] T[c ng + j]) / beta for ng <= 8 columns, one thread per row.
constexpr int kMaxPcCols = 1024;
__global__ void __launch_bounds__(256) k_pc_combine(const float* __restrict__ U, int64_t N, int r,
                                                    const float* __restrict__ R, const double* __restrict__ T, int ng,
                                                    float inv_beta, float* __restrict__ Z)
{
    __shared__ float ts[kMaxPcCols * 8];
    for (int e = threadIdx.x; e < r * ng; e += blockDim.x) ts[e] = (float)T[e];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = j < ng ? R[(int64_t)j * N + i] : 0.f;
    for (int c = 0; c < r; ++c) {
        const float uv = U[(int64_t)c * N + i];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < ng) acc[j] = fmaf(-uv, ts[c * ng + j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if (j < ng) Z[(int64_t)j * N + i] = acc[j] * inv_beta;
}

// P = Zn + b_j P with the flexible (Polak-Ribiere) b_j = (Zn.R - Zo.R) / (R_old.Zo) for the active columns
__global__ void __launch_bounds__(256) k_pcg_dir(const float* __restrict__ Zn, float* __restrict__ P,
                                                 const double* __restrict__ rzn, const double* __restrict__ rzo,
                                                 const double* __restrict__ rz, const int* __restrict__ active,
                                                 int64_t N)
{
    const int j = blockIdx.y;
    if (!active[j]) return;
    const int64_t o = j * N;
    const float b = (float)((rzn[j] - rzo[j]) / rz[j]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        P[o + i] = fmaf(b, P[o + i], Zn[o + i]);
}

int vec_blocks(int64_t N)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (N + kT - 1) / kT;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, 4 * (int64_t)std::max(sms, 1)));
}

// Device buffers released on scope exit.
struct Scratch {
    std::vector<void*> ptrs;
    template <typename T>
    T* get(size_t count)
    {
        void* q = nullptr;
        if (cudaMalloc(&q, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(q);
        return static_cast<T*>(q);
    }
    ~Scratch()
    {
        for (void* q : ptrs) cudaFree(q);
    }
};

}  // namespace

static void pc_free(Plan& p)
{
    for (void* q : {(void*)p.pc_U, (void*)p.pc_G, (void*)p.pc_L, (void*)p.pc_w})
        if (q) cudaFree(q);
    p.pc_U = nullptr;
    p.pc_G = p.pc_L = p.pc_w = nullptr;
    p.pc_r = 0;
    p.pc_beta = -1.0;
}

struct PcMode {
    int s;                                 // window, -1 for the shared constant
    int k[3];
};

// The retained modes and their column weights (host): the constant first, then per window the modes
// |k|_inf <= band, one of each +-k pair (the first non-zero component positive), with
// N sigma_f^2 2 c_hat_k >= beta.
static void pc_modes(const Plan& p, int band, double beta, std::vector<PcMode>* modes, std::vector<double>* wcol)
{
    const int B = 2 * kPcMaxBand + 1;
    const double sf2 = p.sigma_f * p.sigma_f;
    double c0 = 0.0;
    for (int s = 0; s < p.P; ++s) {
        int64_t centre = 0;
        for (int t = 0; t < p.dims[s]; ++t) centre = centre * B + kPcMaxBand;
        c0 += p.lowc[s][centre];
    }
    modes->assign(1, PcMode{-1, {0, 0, 0}});
    wcol->assign(1, sf2 * c0);
    for (int s = 0; s < p.P; ++s) {
        const int D = p.dims[s];
        const int b = std::min(band, p.bandwidth[s] / 2 - 1);
        int k[3] = {0, 0, 0};
        int64_t count = 1;
        for (int t = 0; t < D; ++t) count *= 2 * b + 1;
        for (int64_t o = 0; o < count; ++o) {
            int64_t rem = o, idx = 0;
            for (int t = D - 1; t >= 0; --t) {
                k[t] = (int)(rem % (2 * b + 1)) - b;
                rem /= 2 * b + 1;
            }
            int first = 0;
            for (int t = 0; t < D && first == 0; ++t) first = k[t];
            if (first <= 0) continue;                          // the zero mode, or the negative of a kept one
            for (int t = 0; t < D; ++t) idx = idx * B + (k[t] + kPcMaxBand);
            const double val = 2.0 * sf2 * p.lowc[s][idx];
            if (!(val > 0.0) || (double)p.N * val < beta) continue;
            modes->push_back(PcMode{s, {k[0], D > 1 ? k[1] : 0, D > 2 ? k[2] : 0}});
            wcol->push_back(val);
            wcol->push_back(val);
        }
    }
}

// Build the preconditioner for beta (basis, Gram matrix, Cholesky factor). Returns ADDKER_OK, or
// ADDKER_EINVAL when there is nothing to precondition with (then plain CG runs).
static int pc_build(Plan& p, double beta, cudaStream_t st)
{
    if (p.pc_U && p.pc_beta == beta) return ADDKER_OK;
    pc_free(p);
    std::vector<PcMode> modes;
    std::vector<double> w;
    int band = p.pc_band;
    for (;; --band) {
        pc_modes(p, band, beta, &modes, &w);
        if ((int)w.size() <= kMaxPcCols || band <= 1) break;
    }
    const int r = (int)w.size();
    if (r < 2 || r > kMaxPcCols) return ADDKER_EINVAL;
    const int64_t N = p.N;
    Scratch tmp;
    float4* xo = tmp.get<float4>(N);
    int* kv = tmp.get<int>(3 * modes.size());
    int* fail = tmp.get<int>(1);
    const int nt = (r + kGT - 1) / kGT;
    std::vector<int2> tl;
    for (int a = 0; a < nt; ++a)
        for (int b = a; b < nt; ++b) tl.push_back(make_int2(a, b));
    int2* tiles = tmp.get<int2>(tl.size());
    if (!xo || !kv || !fail || !tiles) return ADDKER_ENOMEM;
    CK(cudaMalloc(&p.pc_U, sizeof(float) * (size_t)N * r));
    CK(cudaMalloc(&p.pc_G, sizeof(double) * (size_t)r * r));
    CK(cudaMalloc(&p.pc_L, sizeof(double) * (size_t)r * r));
    CK(cudaMalloc(&p.pc_w, sizeof(double) * (size_t)r));
    p.pc_r = r;
    std::vector<int> hk(3 * modes.size());
    for (size_t m = 0; m < modes.size(); ++m)
        for (int t = 0; t < 3; ++t) hk[3 * m + t] = modes[m].k[t];
    CK(cudaMemcpyAsync(kv, hk.data(), sizeof(int) * hk.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(p.pc_w, w.data(), sizeof(double) * r, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(tiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice, st));
    const int th = 256;
    const int nb = (int)((N + th - 1) / th);
    k_fill<<<nb, th, 0, st>>>(p.pc_U, N, 1.0f);                 // the constant column
    int col = 1;
    for (int s = 0; s < p.P; ++s) {
        size_t m0 = 0, nm = 0;
        for (size_t m = 1; m < modes.size(); ++m)
            if (modes[m].s == s) { if (!nm) m0 = m; ++nm; }
        if (!nm) continue;
        k_unsort<<<nb, th, 0, st>>>(p.win[s].pts, N, xo);
        k_fourier_cols<<<nb, th, 0, st>>>(xo, N, kv + 3 * m0, (int)nm, p.pc_U, col);
        col += 2 * (int)nm;
    }
    CK(cudaMemsetAsync(p.pc_G, 0, sizeof(double) * (size_t)r * r, st));
    CK(cudaMemsetAsync(fail, 0, sizeof(int), st));
    const int gy = (int)std::min<int64_t>(64, (N + kGR - 1) / kGR);
    k_gram<<<dim3((unsigned)tl.size(), gy), kGT * kGT, 0, st>>>(p.pc_U, N, r, tiles, p.pc_G);
    k_cholesky<<<1, 512, 0, st>>>(p.pc_G, p.pc_w, beta, r, p.pc_L, fail);
    CK(cudaGetLastError());
    int hf = 0;
    CK(cudaMemcpyAsync(&hf, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hf) {
        pc_free(p);
        return ADDKER_EINVAL;
    }
    p.pc_beta = beta;
    return ADDKER_OK;
}

// Z = B^{-1} R for nrhs columns (leading dimension N); T: scratch of r x 8 doubles.
static int pc_apply(const Plan& p, const float* R, float* Z, int nrhs, double beta, double* T, cudaStream_t st)
{
    const int64_t N = p.N;
    const int r = p.pc_r;
    for (int j0 = 0; j0 < nrhs; j0 += 8) {
        const int ng = std::min(8, nrhs - j0);
        CK(cudaMemsetAsync(T, 0, sizeof(double) * (size_t)r * ng, st));
        k_utr<<<(unsigned)((N + kCH - 1) / kCH), 256, 0, st>>>(p.pc_U, N, r, R + (size_t)j0 * N, ng, T);
        k_pc_solve<<<1, 32 * ng, 0, st>>>(p.pc_L, r, ng, T);
        k_pc_combine<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(p.pc_U, N, r, R + (size_t)j0 * N, T, ng,
                                                                (float)(1.0 / beta), Z + (size_t)j0 * N);
    }
    CK(cudaGetLastError());
    return ADDKER_OK;
}

void pc_release(Plan& p) { pc_free(p); }

// CG on (K + beta I) X = Y for nrhs columns (device, N x nrhs); X holds the initial guess and receives
// the solution. iters[j] and relres[j] (host) report each column.
int cg_solve(Plan& p, double beta, const float* Y, float* X, int nrhs, double tol, int maxit, int* iters,
             double* relres)
{
    const int64_t N = p.N;
    const size_t NV = (size_t)N * nrhs;
    cudaStream_t st = p.stream;
    Scratch s;
    float* R = s.get<float>(NV);
    float* Pd = s.get<float>(NV);
    float* KP = s.get<float>(NV);
    double* sc = s.get<double>(4 * (size_t)nrhs);              // rr, |y|^2, rr_new, pAp
    int* act = s.get<int>(nrhs);
    if (!R || !Pd || !KP || !sc || !act) return ADDKER_ENOMEM;
    double *rr = sc, *yy = sc + nrhs, *rr_new = sc + 2 * nrhs, *pAp = sc + 3 * nrhs;
    const dim3 grid(vec_blocks(N), nrhs);
    const float fb = (float)beta;
    // R = Y - A X, P = R
    CS(product_all(p, X, nrhs, KP, nullptr, -1, 0));
    k_cg_init<<<grid, kT, 0, st>>>(Y, X, KP, fb, N, R, Pd);
    CK(cudaMemsetAsync(sc, 0, sizeof(double) * 4 * nrhs, st));
    k_dot_cols<<<grid, kT, 0, st>>>(R, N, R, N, 0.f, N, rr);
    k_dot_cols<<<grid, kT, 0, st>>>(Y, N, Y, N, 0.f, N, yy);
    CK(cudaGetLastError());
    std::vector<double> h(2 * nrhs);
    CK(cudaMemcpyAsync(h.data(), rr, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h.data() + nrhs, yy, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<int> active(nrhs), it(nrhs, 0);
    std::vector<double> rel(nrhs);
    int n_active = 0;
    for (int j = 0; j < nrhs; ++j) {
        if (h[nrhs + j] == 0.0) {                  // y_j = 0: the solution is 0
            CK(cudaMemsetAsync(X + (size_t)j * N, 0, sizeof(float) * N, st));
            rel[j] = 0.0;
            active[j] = 0;
            continue;
        }
        rel[j] = std::sqrt(h[j] / h[nrhs + j]);
        active[j] = rel[j] > tol;
        n_active += active[j];
    }
    CK(cudaMemcpyAsync(act, active.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
    // preconditioned: flexible PCG with B = beta I + U W U^T (built once per beta; plain CG if none can be)
    const bool pcg = n_active > 0 && beta > 0.0 && p.pc_band > 0 && pc_build(p, beta, st) == ADDKER_OK;
    if (pcg) {
        float* Z = s.get<float>(NV);
        float* Zn = s.get<float>(NV);
        double* pd = s.get<double>(3 * (size_t)nrhs);             // rz, rzn, rzo
        double* T = s.get<double>((size_t)p.pc_r * 8);
        if (!Z || !Zn || !pd || !T) return ADDKER_ENOMEM;
        double *rz = pd, *rzn = pd + nrhs, *rzo = pd + 2 * nrhs;
        CS(pc_apply(p, R, Z, nrhs, beta, T, st));
        CK(cudaMemcpyAsync(Pd, Z, sizeof(float) * NV, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemsetAsync(rz, 0, sizeof(double) * nrhs, st));
        k_dot_cols<<<grid, kT, 0, st>>>(R, N, Z, N, 0.f, N, rz);
        for (int k = 0; k < maxit && n_active > 0; ++k) {
            CS(product_all(p, Pd, nrhs, KP, nullptr, -1, 0));
            CK(cudaMemsetAsync(rr_new, 0, sizeof(double) * 2 * nrhs, st));    // rr_new and pAp
            k_dot_cols<<<grid, kT, 0, st>>>(Pd, N, KP, N, fb, N, pAp);
            k_cg_step<<<grid, kT, 0, st>>>(X, R, Pd, KP, fb, rz, pAp, act, N, rr_new);   // alpha = r.z / p.Ap
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(h.data(), rr_new, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
            CS(pc_apply(p, R, Zn, nrhs, beta, T, st));
            CK(cudaMemsetAsync(rzn, 0, sizeof(double) * 2 * nrhs, st));        // rzn and rzo
            k_dot_cols<<<grid, kT, 0, st>>>(R, N, Zn, N, 0.f, N, rzn);
            k_dot_cols<<<grid, kT, 0, st>>>(R, N, Z, N, 0.f, N, rzo);
            k_pcg_dir<<<grid, kT, 0, st>>>(Zn, Pd, rzn, rzo, rz, act, N);
            CK(cudaMemcpyAsync(rz, rzn, sizeof(double) * nrhs, cudaMemcpyDeviceToDevice, st));
            CK(cudaGetLastError());
            std::swap(Z, Zn);
            CK(cudaStreamSynchronize(st));
            bool changed = false;
            for (int j = 0; j < nrhs; ++j) {
                if (!active[j]) continue;
                ++it[j];
                rel[j] = std::sqrt(h[j] / h[nrhs + j]);
                if (!(rel[j] > tol)) {
                    active[j] = 0;
                    --n_active;
                    changed = true;
                }
            }
            if (changed) CK(cudaMemcpyAsync(act, active.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
        }
    }
    for (int k = 0; !pcg && k < maxit && n_active > 0; ++k) {
        CS(product_all(p, Pd, nrhs, KP, nullptr, -1, 0));
        CK(cudaMemsetAsync(rr_new, 0, sizeof(double) * 2 * nrhs, st));       // rr_new and pAp
        k_dot_cols<<<grid, kT, 0, st>>>(Pd, N, KP, N, fb, N, pAp);
        k_cg_step<<<grid, kT, 0, st>>>(X, R, Pd, KP, fb, rr, pAp, act, N, rr_new);
        k_cg_dir<<<grid, kT, 0, st>>>(R, Pd, rr, rr_new, act, N);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h.data(), rr_new, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        bool changed = false;
        for (int j = 0; j < nrhs; ++j) {
            if (!active[j]) continue;
            ++it[j];
            rel[j] = std::sqrt(h[j] / h[nrhs + j]);
            if (!(rel[j] > tol)) {
                active[j] = 0;
                --n_active;
                changed = true;
            }
        }
        // rr <- rr_new (device), then the next iteration accumulates a fresh rr_new
        CK(cudaMemcpyAsync(rr, rr_new, sizeof(double) * nrhs, cudaMemcpyDeviceToDevice, st));
        if (changed) CK(cudaMemcpyAsync(act, active.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
    }
    CK(cudaStreamSynchronize(st));
    for (int j = 0; j < nrhs; ++j) {
        if (iters) iters[j] = it[j];
        if (relres) relres[j] = rel[j];
    }
    return ADDKER_OK;
}

int gp_grad(Plan& p, double beta, const float* y, const float* Z, int m, double tol, int maxit, double* grad,
            double* fit, float* alpha_out, int* iters)
{
    const int64_t N = p.N;
    const int P = p.P, nc = 1 + m;
    cudaStream_t st = p.stream;
    Scratch s;
    float* B = s.get<float>((size_t)N * nc);                  // [y, z_1 .. z_m], then [alpha, z_1 .. z_m]
    float* S = s.get<float>((size_t)N * nc);                  // [alpha, w_1 .. w_m]
    float* KC = s.get<float>((size_t)N * nc);
    float* dKC = s.get<float>((size_t)N * P * nc);
    double* d = s.get<double>((size_t)(P + 2) * 2 * nc + 1);
    if (!B || !S || !KC || !dKC || !d) return ADDKER_ENOMEM;
    CK(cudaMemcpyAsync(B, y, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    if (m > 0) CK(cudaMemcpyAsync(B + N, Z, sizeof(float) * N * m, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(S, 0, sizeof(float) * N * nc, st));
    std::vector<int> it(nc);
    std::vector<double> rel(nc);
    CS(cg_solve(p, beta, B, S, nc, tol, maxit, it.data(), rel.data()));
    // C = [alpha, z_1 .. z_m]: products K C and dK/d ell_s C
    CK(cudaMemcpyAsync(B, S, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    CS(product_all(p, B, nc, KC, dKC, -1, 0));
    // FP64 dots, per column j: [s][j] = S_j . dK_s C_j  (s < P), [P][j] = S_j . K C_j, [P+1][j] = S_j . C_j
    CK(cudaMemsetAsync(d, 0, sizeof(double) * ((size_t)(P + 2) * 2 * nc + 1), st));
    const dim3 grid(vec_blocks(N), nc);
    for (int q = 0; q < P; ++q)
        k_dot_cols<<<grid, kT, 0, st>>>(S, N, dKC + (size_t)q * N, (int64_t)P * N, 0.f, N, d + (size_t)q * nc);
    k_dot_cols<<<grid, kT, 0, st>>>(S, N, KC, N, 0.f, N, d + (size_t)P * nc);
    k_dot_cols<<<grid, kT, 0, st>>>(S, N, B, N, 0.f, N, d + (size_t)(P + 1) * nc);
    k_dot_cols<<<dim3(vec_blocks(N), 1), kT, 0, st>>>(S, N, y, N, 0.f, N, d + (size_t)(P + 2) * 2 * nc);   // y^T alpha
    CK(cudaGetLastError());
    std::vector<double> h((size_t)(P + 2) * 2 * nc + 1);
    CK(cudaMemcpyAsync(h.data(), d, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
    if (alpha_out) CK(cudaMemcpyAsync(alpha_out, S, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    for (int q = 0; q < P + 2; ++q) {
        const double* dq = h.data() + (size_t)q * nc;
        double tr = 0.0;
        for (int j = 1; j < nc; ++j) tr += dq[j];
        const double f = q == P ? 2.0 / p.sigma_f : 1.0;                      // dA/d sigma_f = (2/sigma_f) K
        grad[q] = f * (0.5 * dq[0] - (m > 0 ? 0.5 * tr / m : 0.0));
    }
    if (fit) *fit = h[(size_t)(P + 2) * 2 * nc];
    if (iters) {
        int mx = 0;
        for (int j = 0; j < nc; ++j) mx = std::max(mx, it[j]);
        *iters = mx;
    }
    return ADDKER_OK;
}

}  // namespace addker
