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
    for (int k = 0; k < maxit && n_active > 0; ++k) {
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
