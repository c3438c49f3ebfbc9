// C ABI (include/addker.h): plan setup, coefficient precomputation and the product entry points.
//
// Setup (not timed with the products):
//   1. per window, every point's grid cell floor(n x_t) + n/2 and the ball check ||x^W|| <= rho;
//   2. a counting sort of the points by cell (histogram on the device, offsets and work items on
//      the host, scatter on the device);
//   3. the Fourier multipliers, FP64 on the device: samples of the regularised kernel on the
//      M^D grid j/M, a cosine DFT (Lemma "aliasing error"), division by the window transform;
//   4. the per-axis twiddles of the pruned DFTs.
// A product then runs, per right-hand side: clear grids, spread, forward DFT + multiply,
// inverse DFT, gather (+ window sum), all on the plan's stream.
#include <algorithm>
#include <limits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <type_traits>

#include "common.cuh"

using namespace addker;

struct addker_plan {
    Plan p;
};

namespace {

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) {                                  \
            return e_ == cudaErrorMemoryAllocation ? ADDKER_ENOMEM : ADDKER_ECUDA; \
        }                                                         \
    } while (0)

#define CS(status)                        \
    do {                                  \
        int s_ = (status);                \
        if (s_ != ADDKER_OK) return s_;   \
    } while (0)

template <class T>
int dalloc(Plan& p, T** ptr, int64_t count)
{
    *ptr = nullptr;
    if (count <= 0) count = 1;
    void* raw = nullptr;
    cudaError_t e = cudaMalloc(&raw, sizeof(T) * (size_t)count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ADDKER_ENOMEM;
    }
    p.allocations.push_back(raw);
    p.bytes += (int64_t)(sizeof(T) * (size_t)count);
    *ptr = static_cast<T*>(raw);
    return ADDKER_OK;
}

// Forget every captured product (buffers, slots or scalars they bake in have changed).
void clear_graphs(Plan& p)
{
    for (auto& e : p.graph_cache) cudaGraphExecDestroy(e.second);
    p.graph_cache.clear();
    p.last_key = {nullptr, nullptr, nullptr, 0, 0, -1};
}

void release(Plan& p)
{
    clear_graphs(p);
    pc_release(p);
    if (p.cap_stream) cudaStreamDestroy(p.cap_stream);
    p.cap_stream = nullptr;
    if (p.copy_stream) cudaStreamDestroy(p.copy_stream);
    p.copy_stream = nullptr;
    for (cudaEvent_t e : p.win_events) cudaEventDestroy(e);
    p.win_events.clear();
    if (p.items) cudaFree(p.items);
    p.items = nullptr;
    p.items_cap = 0;
    for (void* a : p.allocations) cudaFree(a);
    p.allocations.clear();
    for (void* a : p.slot_allocs) cudaFree(a);
    p.slot_allocs.clear();
    p.slots = 0;
    p.slot_bytes = 0;
    p.bytes = 0;
}

// ------------------------------------------------------------------ setup kernels ----

template <int D>
__global__ void k_cell_keys(const float* __restrict__ X, int64_t N, int d, int f0, int f1, int f2, int n,
                            float rho2, int* __restrict__ keys, int* __restrict__ hist, int* __restrict__ bounds,
                            int* __restrict__ flag)
{
    __shared__ int smin[3], smax[3];
    if (threadIdx.x < 3) { smin[threadIdx.x] = 1 << 30; smax[threadIdx.x] = -(1 << 30); }
    __syncthreads();
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < N) {
        const int f[3] = {f0, f1, f2};
        float x[3] = {0.f, 0.f, 0.f};
        float r2 = 0.f;
        for (int t = 0; t < D; ++t) {
            x[t] = X[j * d + f[t]];
            r2 = fmaf(x[t], x[t], r2);
        }
        if (!(r2 <= rho2)) {            // also catches NaN
            atomicOr(flag, 1);
            keys[j] = -1;
        } else {
            int key = 0;
            for (int t = 0; t < D; ++t) {
                int c = (int)floorf(x[t] * (float)n) + n / 2;
                key = key * n + c;
                atomicMin(&smin[t], c);
                atomicMax(&smax[t], c);
            }
            keys[j] = key;
            atomicAdd(&hist[key], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x < D) {
        atomicMin(&bounds[threadIdx.x], smin[threadIdx.x]);
        atomicMax(&bounds[3 + threadIdx.x], smax[threadIdx.x]);
    }
}

template <int D>
__global__ void k_scatter(const float* __restrict__ X, int64_t N, int d, int f0, int f1, int f2,
                          const int* __restrict__ keys, int* __restrict__ cursor, float4* __restrict__ pts)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int f[3] = {f0, f1, f2};
    float x[3] = {0.f, 0.f, 0.f};
    for (int t = 0; t < D; ++t) x[t] = X[j * d + f[t]];
    int pos = atomicAdd(&cursor[keys[j]], 1);
    pts[pos] = make_float4(x[0], x[1], x[2], __int_as_float((int)j));
}

// ---------------------------------------------------------- coefficients (FP64) ----

struct Transition {                      // T(r) = sum_i s[i] ((r - a)/h)^i on a < r <= 1/2
    int np;                              // 2p coefficients (0: no regularisation)
    int family;                          // ADDKER_KERNEL_GAUSS or ADDKER_KERNEL_MATERN12
    double s[2][32];                     // [kind][i], kind 0 the kernel, 1 its derivative kernel
    double a, h, vb[2];
};

// Radial profiles (Sec. 3.3, eqs. "implement_gaussian_kernel", "implement_der_gaussian_kernel"; Sec. 5
// for Matern(1/2)): Gaussian exp(-q), q = r^2/(2 ell^2), and q exp(-q); Matern exp(-t), t = r/ell, and
// t exp(-t).
__host__ __device__ inline double kernel_value(double r, double ell, int kind, int family)
{
    if (family == ADDKER_KERNEL_MATERN12) {
        const double t = r / ell, e = exp(-t);
        return kind == 0 ? e : t * e;
    }
    const double q = r * r / (2.0 * ell * ell), e = exp(-q);
    return kind == 0 ? e : q * e;
}

template <int D>
__global__ void k_coef_sample(int M, double ell, Transition tr, double* __restrict__ outK, double* __restrict__ outD)
{
    int64_t total = 1;
    for (int t = 0; t < D; ++t) total *= M;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    double r2 = 0.0;
    int64_t rem = idx;
    for (int t = 0; t < D; ++t) {
        int j = (int)(rem % M) - M / 2;
        rem /= M;
        double x = (double)j / (double)M;
        r2 += x * x;
    }
    double r = sqrt(r2);
    for (int kind = 0; kind < 2; ++kind) {
        double val;
        if (tr.np == 0 || r <= tr.a) {
            val = kernel_value(r, ell, kind, tr.family);
        } else if (r <= 0.5) {
            double sg = (r - tr.a) / tr.h, acc = 0.0;
            for (int i = tr.np - 1; i >= 0; --i) acc = acc * sg + tr.s[kind][i];
            val = acc;
        } else {
            val = tr.vb[kind];
        }
        (kind == 0 ? outK : outD)[idx] = val;
    }
}

// ------------------------------------------- separable coefficients (FP64), Sec. 3.4 ----
// The Gaussian's coefficients are a tensor product over the window's axes, c_k = prod_t c_{k_t}(f), and
// the derivative kernel's the D-term sum sum_t c_{k_t}(g) prod_{u != t} c_{k_u}(f), f(x) = exp(-x^2/(2 ell^2)),
// g(x) = (x^2/(2 ell^2)) f(x). Each 1-D factor is the least-squares Fourier extension of f (or g) on the
// interval [0, a_t] that holds every coordinate difference of axis t:
//   a_t = min(1/2 - eps_B, max(max(1/4, 1/2 - 4/M), 2 max_j |x_{j,t}|)),
// fitted on J = 4M equispaced nodes a_t i/(J-1) by cos(2 pi k x), k < K = M/2. The floor keeps the
// basis well conditioned (condition number below ~1e5); the fit is already within 1e-8 there.

// One block per axis t: Householder QR of the J x K cosine matrix with the three right-hand sides f, g and
// p(x) = x^2/(2 ell^2) appended (J x (K+3), column-major in dynamic shared memory), then back substitution.
// range: per-feature [min, max] of the points (2 floats per feature); feat[t]: the axis's feature.
// out[(3t + q) K + k] = b_k of f (q = 0), g (q = 1) or p (q = 2).
__global__ void k_fit_extension(int M, double ell, double eps_B, const float* __restrict__ range, int f0, int f1,
                                int f2, double* __restrict__ out)
{
    extern __shared__ double A[];
    __shared__ double red[32];
    __shared__ double s_beta, s_alpha;
    const int t = blockIdx.x;
    const int f = t == 0 ? f0 : (t == 1 ? f1 : f2);
    const int J = 4 * M, K = M / 2, C = K + 3;
    const double maxabs = fmax(-(double)range[2 * f], (double)range[2 * f + 1]);
    const double a = fmin(0.5 - eps_B, fmax(fmax(0.25, 0.5 - 4.0 / M), 2.0 * maxabs));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int i = tid; i < J; i += blockDim.x) {
        const double x = a * i / (J - 1);
        for (int k = 0; k < K; ++k) A[k * J + i] = cospi(2.0 * k * x);
        const double q = x * x / (2.0 * ell * ell), e = exp(-q);
        A[K * J + i] = e;
        A[(K + 1) * J + i] = q * e;
        A[(K + 2) * J + i] = q;
    }
    __syncthreads();
    for (int c = 0; c < K; ++c) {
        double ss = 0.0;
        for (int i = c + tid; i < J; i += blockDim.x) ss += A[c * J + i] * A[c * J + i];
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) red[warp] = ss;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < nwarps; ++w) tot += red[w];
            const double x0 = A[c * J + c];
            const double alpha = x0 >= 0.0 ? -sqrt(tot) : sqrt(tot);
            const double v0 = x0 - alpha;                  // no cancellation: alpha has x0's opposite sign
            const double vv = tot - x0 * x0 + v0 * v0;
            s_beta = vv > 0.0 ? 2.0 / vv : 0.0;
            s_alpha = alpha;
            A[c * J + c] = v0;                             // the reflector v = (v0, A[c+1.., c])
        }
        __syncthreads();
        for (int j = c + 1 + warp; j < C; j += nwarps) {   // apply I - beta v v^T to the later columns
            double dt = 0.0;
            for (int i = c + lane; i < J; i += 32) dt += A[c * J + i] * A[j * J + i];
            for (int o = 16; o > 0; o >>= 1) dt += __shfl_xor_sync(0xffffffffu, dt, o);
            const double sc = s_beta * dt;
            for (int i = c + lane; i < J; i += 32) A[j * J + i] -= sc * A[c * J + i];
        }
        __syncthreads();
        if (tid == 0) A[c * J + c] = s_alpha;              // R's diagonal
        __syncthreads();
    }
    if (tid < 3) {                                         // R b = (Q^T rhs)[0..K), R[k][j] = A[j J + k]
        double x[kMaxBandwidth / 2];
        for (int k = K - 1; k >= 0; --k) {
            double acc = A[(K + tid) * J + k];
            for (int j = k + 1; j < K; ++j) acc -= A[j * J + k] * x[j];
            x[k] = acc / A[k * J + k];
        }
        for (int k = 0; k < K; ++k) out[(3 * t + tid) * K + k] = x[k];
    }
}

// c_hat, c_hat^der and the quadratic's c_hat^P on I_M^D (layout [k_0]..[k_{D-1}], last fastest) from the
// fitted factors: c_{k}(.) = b_0 at k = 0, b_|k| / 2 for 0 < |k| < M/2, 0 at k = -M/2;
// c^P_k = sum_t c_{k_t}(p) prod_{u != t} [k_u = 0] (P(r) = sum_t p(r_t)).
template <int D>
__global__ void k_coef_tensor(int M, const double* __restrict__ fit, double* __restrict__ outK,
                              double* __restrict__ outD, double* __restrict__ outP)
{
    int64_t total = 1;
    for (int t = 0; t < D; ++t) total *= M;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int K = M / 2;
    double fv[3], gv[3], pv[3];
    int zero[3];
    int64_t rem = idx;
    for (int t = D - 1; t >= 0; --t) {
        const int k = (int)(rem % M) - K;
        rem /= M;
        const int ak = k < 0 ? -k : k;
        const double* bf = fit + (3 * t) * K;
        const double* bg = fit + (3 * t + 1) * K;
        const double* bp = fit + (3 * t + 2) * K;
        zero[t] = k == 0;
        if (ak >= K) { fv[t] = 0.0; gv[t] = 0.0; pv[t] = 0.0; }
        else if (ak == 0) { fv[t] = bf[0]; gv[t] = bg[0]; pv[t] = bp[0]; }
        else { fv[t] = 0.5 * bf[ak]; gv[t] = 0.5 * bg[ak]; pv[t] = 0.5 * bp[ak]; }
    }
    double cK = 1.0, cD = 0.0, cP = 0.0;
    for (int t = 0; t < D; ++t) {
        double term = gv[t];
        bool others_zero = true;
        for (int u = 0; u < D; ++u)
            if (u != t) {
                term *= fv[u];
                others_zero = others_zero && zero[u];
            }
        cD += term;
        if (others_zero) cP += pv[t];
        cK *= fv[t];
    }
    outK[idx] = cK;
    outD[idx] = cD;
    outP[idx] = cP;
}

// Enqueue the separable coefficients of one window (D axes, features feat[0..D)) into cK, cD, cP (M^D
// doubles each), using fit (3 D K doubles) for the 1-D factors.
cudaError_t separable_coefficients(int D, int M, double ell, double eps_B, const float* range, const int* feat,
                                   double* fit, double* cK, double* cD, double* cP, cudaStream_t st)
{
    const int J = 4 * M, K = M / 2;
    const size_t shm = sizeof(double) * (size_t)J * (K + 3);
    cudaError_t e = cudaFuncSetAttribute(k_fit_extension, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    k_fit_extension<<<D, 128, shm, st>>>(M, ell, eps_B, range, feat[0], D > 1 ? feat[1] : 0, D > 2 ? feat[2] : 0,
                                         fit);
    int64_t total = 1;
    for (int t = 0; t < D; ++t) total *= M;
    const int th = 256, bl = (int)((total + th - 1) / th);
    if (D == 1) k_coef_tensor<1><<<bl, th, 0, st>>>(M, fit, cK, cD, cP);
    else if (D == 2) k_coef_tensor<2><<<bl, th, 0, st>>>(M, fit, cK, cD, cP);
    else k_coef_tensor<3><<<bl, th, 0, st>>>(M, fit, cK, cD, cP);
    return cudaGetLastError();
}

// The quadratic split. For a kernel wide against the data the derivative kernel q e^{-q},
// q = ||r||^2/(2 ell^2), is nearly its quadratic part P = q; as a trigonometric polynomial P needs a
// constant term many times the product (about 24 times at ell = 1 on the nine-feature benchmark) that
// cancels against the low frequencies, and every FP32 rounding in the transforms is multiplied by that
// factor. P is a rank-5 kernel (sum_j ||x_i - x_j||^2 v_j = ||x_i||^2 m0 - 2 x_i.m1 + m2 with the
// moments m0 = sum v, m1 = sum x v, m2 = sum ||x||^2 v), so a split window sends only the remainder
// c_hat^der - c_hat^P through the transforms and adds P v from moments the spread accumulates. Rule:
// split when that shrinks the constant coefficient, |c_0^der - c_0^P| < 0.9 |c_0^der| (for a narrow
// kernel the remainder would be the larger one). Reads the two constant terms.
int decide_split(int D, int M, const double* cD, const double* cP, cudaStream_t st, bool* split)
{
    int64_t c = 0;
    for (int t = 0; t < D; ++t) c = c * M + M / 2;
    double h[2];
    if (cudaMemcpyAsync(&h[0], cD + c, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&h[1], cP + c, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ADDKER_ECUDA;
    *split = std::fabs(h[0] - h[1]) < 0.9 * std::fabs(h[0]);
    return ADDKER_OK;
}

// out[a][k][b] = (1/M) sum_j in[a][j][b] cos(2 pi (j - M/2)(k - M/2) / M); the sine part of the DFT
// vanishes for even, real samples.
__global__ void k_coef_dft(const double* __restrict__ in, double* __restrict__ out, int A, int M, int B)
{
    int64_t total = (int64_t)A * M * B;
    int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (o >= total) return;
    int b = (int)(o % B);
    int k = (int)((o / B) % M) - M / 2;
    int a = (int)(o / ((int64_t)B * M));
    double acc = 0.0;
    for (int jj = 0; jj < M; ++jj) {
        int j = jj - M / 2;
        int ph = ((j * k) % M + M) % M;
        acc += in[((int64_t)a * M + jj) * B + b] * cospi(2.0 * ph / M);
    }
    out[o] = acc / M;
}

// bK = c_hat / (n^D prod_t phi_hat(k_t))^2, bD likewise, dconv = 1 / (n^D prod_t phi_hat(k_t)),
// with phat[k + M/2] the Fourier transform of the window the kernels spread with.
// With cP (not NULL) the derivative multiplier is that of the remainder c_hat^der - c_hat^P (quadratic split).
template <int D>
__global__ void k_multipliers(const double* __restrict__ cK, const double* __restrict__ cD, int M, int n,
                              const double* __restrict__ phat, float* __restrict__ bK, float* __restrict__ bD,
                              float* __restrict__ dconv, float* __restrict__ chat, const double* __restrict__ cP)
{
    int64_t total = 1;
    for (int t = 0; t < D; ++t) total *= M;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    double ph = 1.0, nd = 1.0;
    int64_t rem = idx;
    for (int t = 0; t < D; ++t) {
        ph *= phat[rem % M];
        rem /= M;
        nd *= n;
    }
    double den = nd * ph;
    bK[idx] = (float)(cK[idx] / (den * den));
    bD[idx] = (float)((cP ? cD[idx] - cP[idx] : cD[idx]) / (den * den));
    dconv[idx] = (float)(1.0 / den);
    if (chat) chat[idx] = (float)cK[idx];
}

// forward twiddles tf[i][kk] = e^{-2 pi i k l / n}, inverse ti[kk][i] = e^{+2 pi i k l / n},
// k = kk - M/2, l = lo + i - n/2 (centred index of grid position lo + i)
__global__ void k_twiddles(float2* __restrict__ tf, float2* __restrict__ ti, int lo, int box, int M, int n)
{
    int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= box * M) return;
    int i = o / M, kk = o % M;
    int k = kk - M / 2, l = lo + i - n / 2;
    int ph = (int)((((int64_t)k * l) % n + n) % n);
    double s, c;
    sincospi(2.0 * ph / n, &s, &c);
    tf[i * M + kk] = make_float2((float)c, (float)-s);
    ti[kk * box + i] = make_float2((float)c, (float)s);
}

// ---------------------------------------------------------------- products ----

// out[i] = scale sum_s ks[s N + i]; four consecutive i per thread (16-byte accesses when vec: N % 4 == 0
// and out 16-byte aligned)
__global__ void k_window_sum(const float* __restrict__ ks, int P, int64_t N, float scale, float* __restrict__ out,
                             int64_t ld, int vec)
{
    grid_dep_wait();
    const int64_t i0 = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
    if (i0 >= N) return;
    ks += blockIdx.y * (int64_t)P * N;                         // right-hand side blockIdx.y
    out += blockIdx.y * ld;
    if (vec) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int s = 0; s < P; ++s) {
            const float4 k = *reinterpret_cast<const float4*>(ks + (int64_t)s * N + i0);
            acc.x += k.x; acc.y += k.y; acc.z += k.z; acc.w += k.w;
        }
        *reinterpret_cast<float4*>(out + i0) = make_float4(scale * acc.x, scale * acc.y, scale * acc.z, scale * acc.w);
        return;
    }
    for (int64_t i = i0; i < i0 + 4 && i < N; ++i) {
        float acc = 0.f;
        for (int s = 0; s < P; ++s) acc += ks[(int64_t)s * N + i];
        out[i] = scale * acc;
    }
}

struct ThetaScale {
    double s[2 * kMaxWindows + 1];       // [0,P): sigma_f^2 2/ell_s ; P: 2 sigma_f
    double q[kMaxWindows];               // the quadratic split's weight 1/(2 ell_s^2), or 0
};

// grad_theta[s] = sigma_f^2 (2/ell_s) (dots[P + s] + v^T P_s w)  (s < P);  grad_theta[P] = 2 sigma_f sum_s dots[s].
// For a split window the remainder's part is in dots and the quadratic part comes from the moments of
// v (mv) and of w (mw): v^T P w = q (m0(v) m2(w) - 2 m1(v).m1(w) + m2(v) m0(w)).
__global__ void k_theta_grad(const double* __restrict__ dots, int P, ThetaScale sc, const double* __restrict__ mv,
                             const double* __restrict__ mw, double* __restrict__ out)
{
    grid_dep_wait();
    const int s = threadIdx.x;
    if (s < P) {
        double d = dots[P + s];
        if (sc.q[s] != 0.0) {
            const double* a = mv + 8 * s;
            const double* b = mw + 8 * s;
            d += sc.q[s] * (a[0] * b[4] - 2.0 * (a[1] * b[1] + a[2] * b[2] + a[3] * b[3]) + a[4] * b[0]);
        }
        out[s] = sc.s[s] * d;
    }
    if (s == 0) {
        double acc = 0.0;
        for (int q = 0; q < P; ++q) acc += dots[q];
        out[P] = sc.s[P] * acc;
    }
}

__global__ void k_max_norm(const float* __restrict__ X, int64_t N, int d, const int* __restrict__ off,
                           const int* __restrict__ feat, int P, unsigned* __restrict__ result)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float best = 0.f;
    if (j < N) {
        for (int s = 0; s < P; ++s) {
            float r2 = 0.f;
            for (int q = off[s]; q < off[s + 1]; ++q) {
                float x = X[j * d + feat[q]];
                r2 = fmaf(x, x, r2);
            }
            best = fmaxf(best, r2);
        }
        if (!(best == best)) best = __int_as_float(0x7f800000);
    }
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(result, __float_as_uint(best));
}

// Order-preserving atomic min / max of floats through their bit patterns (non-negative floats order
// like ints, negative ones reversed like unsigned); mm[2f] starts at +inf, mm[2f + 1] at -inf.
__device__ __forceinline__ void atomic_min_float(float* a, float v)
{
    if (v >= 0.f) atomicMin(reinterpret_cast<int*>(a), __float_as_int(v));
    else atomicMax(reinterpret_cast<unsigned*>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_float(float* a, float v)
{
    if (v >= 0.f) atomicMax(reinterpret_cast<int*>(a), __float_as_int(v));
    else atomicMin(reinterpret_cast<unsigned*>(a), __float_as_uint(v));
}

// Per-feature range of X (N x d row-major): mm[2f] = min_j X[j][f], mm[2f + 1] = max_j X[j][f];
// *bad = 1 if any value is not finite. Block (feature column chunk): threads stride over rows.
__global__ void k_feature_range(const float* __restrict__ X, int64_t N, int d, float* __restrict__ mm,
                                int* __restrict__ bad)
{
    const int f = blockIdx.y;
    float lo = __int_as_float(0x7f800000), hi = -lo;
    int nonfinite = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const float x = X[j * d + f];
        if (!isfinite(x)) nonfinite = 1;
        lo = fminf(lo, x);
        hi = fmaxf(hi, x);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        nonfinite |= __shfl_xor_sync(0xffffffffu, nonfinite, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_min_float(mm + 2 * f, lo);
        atomic_max_float(mm + 2 * f + 1, hi);
        if (nonfinite) atomicOr(bad, 1);
    }
}

// range[2f] = +inf, range[2f + 1] = -inf for f < d, *bad = 0: the start of k_feature_range.
__global__ void k_range_init(float* __restrict__ range, int d, int* __restrict__ bad)
{
    for (int f = threadIdx.x; f < d; f += blockDim.x) {
        range[2 * f] = __int_as_float(0x7f800000);
        range[2 * f + 1] = -__int_as_float(0x7f800000);
    }
    if (threadIdx.x == 0) *bad = 0;
}

// Y[j][f] = X[j][f] * scale[f] + shift[f]
__global__ void k_affine_features(const float* __restrict__ X, int64_t N, int d, const float* __restrict__ scale,
                                  const float* __restrict__ shift, float* __restrict__ Y)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N * d) return;
    const int f = (int)(i % d);
    Y[i] = fmaf(X[i], scale[f], shift[f]);
}

// dst[i] = src[i], i < n, where one side may be page-locked host memory reached over the CPU-GPU
// link: every SM streams 16-byte words, which moves more than one copy engine does.
__global__ void k_copy(const float* __restrict__ src, float* __restrict__ dst, int64_t n, int vec)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t done = 0;
    if (vec) {
        const int64_t n4 = n / 4;
        const float4* s4 = reinterpret_cast<const float4*>(src);
        float4* d4 = reinterpret_cast<float4*>(dst);
        for (int64_t k = i; k < n4; k += stride) d4[k] = s4[k];
        done = 4 * n4;
    }
    for (int64_t k = done + i; k < n; k += stride) dst[k] = src[k];
}

__global__ void k_scale(const float* __restrict__ X, int64_t n, float f, float* __restrict__ Y)
{
    grid_dep_wait();
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) Y[i] = X[i] * f;
}

// ------------------------------------------------------------------ host helpers ----

// Taylor coefficients at r = a of the Gaussian (kind 0) or the derivative kernel (kind 1), orders
// 0..p-1, by power-series arithmetic: exp(-(a+t)^2/c^2) = exp(-a^2/c^2) exp(q(t)),
// q(t) = -(2 a t + t^2)/c^2, and E = exp(q) satisfies E' = q' E.
void taylor_at(double a, double ell, int p, int kind, int family, double* out)
{
    if (family == ADDKER_KERNEL_MATERN12) {
        // k-th Taylor coefficient at a: (-1/ell)^k e^{-a/ell} / k!, times (a/ell - k) for t e^{-t}
        double f = std::exp(-a / ell);
        for (int k = 0; k < p; ++k) {
            out[k] = kind == 0 ? f : f * (a / ell - k);
            f *= -1.0 / (ell * (k + 1));
        }
        return;
    }
    double c2 = 2.0 * ell * ell;
    double q1 = -2.0 * a / c2, q2 = -1.0 / c2;
    std::vector<double> e(p + 2, 0.0);
    e[0] = 1.0;
    for (int k = 1; k < p + 2; ++k) e[k] = (q1 * e[k - 1] + (k >= 2 ? 2.0 * q2 * e[k - 2] : 0.0)) / k;
    double base = std::exp(-a * a / c2);
    for (int k = 0; k < p + 2; ++k) e[k] *= base;
    for (int k = 0; k < p; ++k) {
        if (kind == 0) {
            out[k] = e[k];
        } else {                       // ((a + t)^2 / c^2) * series
            double v = a * a / c2 * e[k];
            if (k >= 1) v += 2.0 * a / c2 * e[k - 1];
            if (k >= 2) v += 1.0 / c2 * e[k - 2];
            out[k] = v;
        }
    }
}

// Transition polynomial of degree 2p-1 on [a, 1/2] (in sigma = (r - a)/h): matches the kernel's
// first p Taylor coefficients at a, the value kernel(1/2) at 1/2 and p-1 vanishing derivatives there.
int make_transition(double ell, int p, double eps_B, int family, Transition* tr)
{
    std::memset(tr, 0, sizeof(*tr));
    tr->a = 0.5 - eps_B;
    tr->h = eps_B;
    tr->family = family;
    for (int kind = 0; kind < 2; ++kind) tr->vb[kind] = kernel_value(0.5, ell, kind, family);
    if (p == 0) return ADDKER_OK;
    if (p > 12) return ADDKER_EINVAL;
    tr->np = 2 * p;
    for (int kind = 0; kind < 2; ++kind) {
        double t[16];
        taylor_at(tr->a, ell, p, kind, family, t);
        double* s = tr->s[kind];
        for (int i = 0; i < p; ++i) s[i] = t[i] * std::pow(tr->h, i);
        // equations j = 0..p-1 at sigma = 1: sum_i ff(i, j) s_i = (j == 0 ? vb : 0), ff = falling factorial
        double A[12][13];
        for (int j = 0; j < p; ++j) {
            double rhs = j == 0 ? tr->vb[kind] : 0.0;
            for (int i = 0; i < 2 * p; ++i) {
                double ff = 1.0;
                if (i < j) ff = 0.0;
                else for (int r = 0; r < j; ++r) ff *= (double)(i - r);
                if (i < p) rhs -= ff * s[i];
                else A[j][i - p] = ff;
            }
            A[j][p] = rhs;
        }
        for (int col = 0; col < p; ++col) {            // Gaussian elimination, partial pivoting
            int piv = col;
            for (int r = col + 1; r < p; ++r) if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
            if (A[piv][col] == 0.0) return ADDKER_EINVAL;
            for (int c = 0; c <= p; ++c) std::swap(A[col][c], A[piv][c]);
            for (int r = 0; r < p; ++r) {
                if (r == col) continue;
                double f = A[r][col] / A[col][col];
                for (int c = col; c <= p; ++c) A[r][c] -= f * A[col][c];
            }
        }
        for (int j = 0; j < p; ++j) s[p + j] = A[j][p] / A[j][j];
    }
    return ADDKER_OK;
}

int grid_blocks(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

// Normalised Kaiser-Bessel window in grid units: w(t) = (m/s) sinh(b s)/sinh(b m), s = sqrt(m^2 - t^2).
double kb_window(double t, int m, double b)
{
    double s2 = (double)m * m - t * t;
    if (s2 < 0.0) return 0.0;
    double s = std::sqrt(s2);
    double bm = b * m;
    if (s < 1e-7) return m * b * (2.0 * std::exp(-bm)) / (1.0 - std::exp(-2.0 * bm));
    return (m / s) * (std::exp(b * (s - m)) - std::exp(-b * (s + m))) / (1.0 - std::exp(-2.0 * bm));
}

// Exponential-of-semicircle window in grid units, peak 1: w(t) = exp(beta (sqrt(1 - (t/m)^2) - 1)).
double es_window(double t, int m, double beta)
{
    const double z = t / m;
    const double s2 = 1.0 - z * z;
    if (s2 < 0.0) return 0.0;
    return std::exp(beta * (std::sqrt(s2) - 1.0));
}

// Shape of the window of the given kind: b = pi (2 - 1/sigma) (Kaiser-Bessel) or
// beta = 2.30 * 2m * (1 - 1/(2 sigma)) / (3/4) (exponential of semicircle).
double window_shape(int kind, int m, double sigma_os)
{
    if (kind == ADDKER_WIN_ES) return 2.30 * 2.0 * m * (1.0 - 1.0 / (2.0 * sigma_os)) / 0.75;
    return M_PI * (2.0 - 1.0 / sigma_os);
}

// Piece q of the window as a polynomial in u = 2 frac - 1 (t = frac + m - 1 - q): Chebyshev
// interpolation at kPolyDeg + 1 nodes, converted to monomial coefficients, stored as its even part
// (coefficients of u^0, u^2, ...) and odd part (u^1, u^3, ...); pieces q >= m are the mirror images.
void fit_window_poly(int m, double b, WinPoly* out, int kind = ADDKER_WIN_KB)
{
    std::memset(out, 0, sizeof(*out));
    const int N = kPolyDeg + 1;
    for (int q = 0; q < m; ++q) {
        double f[kPolyDeg + 1], a[kPolyDeg + 1];
        for (int j = 0; j < N; ++j) {
            double x = std::cos(M_PI * (j + 0.5) / N);
            const double t = (x + 1.0) / 2.0 + m - 1 - q;
            f[j] = kind == ADDKER_WIN_ES ? es_window(t, m, b) : kb_window(t, m, b);
        }
        for (int k = 0; k < N; ++k) {
            double acc = 0.0;
            for (int j = 0; j < N; ++j) acc += f[j] * std::cos(M_PI * k * (j + 0.5) / N);
            a[k] = 2.0 * acc / N;
        }
        a[0] *= 0.5;
        double Tm[kPolyDeg + 1] = {0}, Tk[kPolyDeg + 1] = {0}, mono[kPolyDeg + 1] = {0};
        Tm[0] = 1.0;                       // T_0
        Tk[1] = 1.0;                       // T_1
        mono[0] += a[0];
        for (int i = 0; i <= kPolyDeg; ++i) mono[i] += a[1] * Tk[i];
        for (int k = 2; k < N; ++k) {      // T_k = 2 u T_{k-1} - T_{k-2}
            double Tn[kPolyDeg + 1] = {0};
            for (int i = 0; i < kPolyDeg; ++i) Tn[i + 1] += 2.0 * Tk[i];
            for (int i = 0; i <= kPolyDeg; ++i) Tn[i] -= Tm[i];
            for (int i = 0; i <= kPolyDeg; ++i) mono[i] += a[k] * Tn[i];
            std::memcpy(Tm, Tk, sizeof(Tm));
            std::memcpy(Tk, Tn, sizeof(Tk));
        }
        for (int i = 0; i <= kPolyDeg; ++i) {
            if (i % 2 == 0) out->e[q][i / 2] = (float)mono[i];
            else out->o[q][i / 2] = (float)mono[i];
        }
    }
}

// Value of window piece q at u, from the stored even/odd parts (the device evaluates the same form).
double window_piece(const WinPoly& poly, int m, int q, double u)
{
    const bool mirror = q >= m;
    const int qq = mirror ? 2 * m - 1 - q : q;
    double E = 0.0, O = 0.0, u2 = u * u;
    for (int i = kHalfCoef - 1; i >= 0; --i) {
        E = E * u2 + (double)poly.e[qq][i];
        O = O * u2 + (double)poly.o[qq][i];
    }
    return mirror ? E - u * O : E + u * O;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n from the three-term recurrence).
void gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Fourier transform of the window the kernels use (the polynomial pieces, in FP64):
//   phi_hat(k) = (1/n) int w(t) cos(2 pi k t / n) dt,  piece q covering t in [m-1-q, m-q).
void window_transform(const WinPoly& poly, int m, int n, int M, double* out)
{
    const int nq = 24;
    double gx[nq], gw[nq];
    gauss_legendre(nq, gx, gw);
    for (int kk = 0; kk < M; ++kk) {
        const int k = kk - M / 2;
        double acc = 0.0;
        for (int q = 0; q < 2 * m; ++q) {
            for (int i = 0; i < nq; ++i) {
                double u = gx[i];                            // u in [-1, 1], frac = (u + 1)/2
                double t = (u + 1.0) / 2.0 + m - 1 - q;
                acc += 0.5 * gw[i] * window_piece(poly, m, q, u) * std::cos(2.0 * M_PI * k * t / n);
            }
        }
        out[kk] = acc / n;
    }
}

int compute_multipliers(Plan& p, int s)
{
    WinDev& w = p.win[s];
    int64_t total = 1;
    for (int t = 0; t < w.D; ++t) total *= w.M;
    double *a = nullptr, *b = nullptr, *c = nullptr, *d = nullptr, *ph = nullptr, *fit = nullptr, *cp = nullptr;
    CK(cudaMalloc(&a, sizeof(double) * (total * 5 + 6 * w.M)));
    b = a + total;
    c = b + total;
    d = c + total;
    cp = d + total;
    ph = cp + total;
    fit = ph + w.M;                                   // 3 D (M/2) <= 4.5 M doubles
    bool split = false;
    std::vector<double> phat(w.M);
    window_transform(p.poly, w.m, w.n, w.M, phat.data());
    cudaStream_t st = p.stream;
    int th = 256, bl = grid_blocks(total, th);
    double* src[2] = {a, b};
    if (cudaMemcpy(ph, phat.data(), sizeof(double) * w.M, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(a);
        return ADDKER_ECUDA;
    }
    if (p.reg == ADDKER_REG_SEPARABLE) {
        if (separable_coefficients(w.D, w.M, p.ell[s], p.eps_B, p.range, w.feat, fit, a, b, cp, st) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(a);
            return ADDKER_ECUDA;
        }
        const int ds = decide_split(w.D, w.M, b, cp, st, &split);
        if (ds != ADDKER_OK) {
            cudaFree(a);
            return ds;
        }
    } else {
        // radial reading: default degree M eps_B rounded half up, at least 1
        int ps = p.p_opt >= 0 ? p.p_opt : std::max(1, (int)std::floor(w.M * p.eps_B + 0.5));
        Transition tr;
        int ts = make_transition(p.ell[s], ps, p.eps_B, p.kernel, &tr);
        if (ts != ADDKER_OK) {
            cudaFree(a);
            return ts;
        }
        if (w.D == 1) k_coef_sample<1><<<bl, th, 0, st>>>(w.M, p.ell[s], tr, a, b);
        else if (w.D == 2) k_coef_sample<2><<<bl, th, 0, st>>>(w.M, p.ell[s], tr, a, b);
        else k_coef_sample<3><<<bl, th, 0, st>>>(w.M, p.ell[s], tr, a, b);
        // separable DFT along each axis (in place via ping-pong): layout [k0]..[k_{D-1}], last fastest
        double* dst[2] = {c, d};
        for (int t = 0; t < w.D; ++t) {
            int64_t B = 1, A = 1;
            for (int u = t + 1; u < w.D; ++u) B *= w.M;
            for (int u = 0; u < t; ++u) A *= w.M;
            for (int q = 0; q < 2; ++q) {
                k_coef_dft<<<bl, th, 0, st>>>(src[q], dst[q], (int)A, w.M, (int)B);
                std::swap(src[q], dst[q]);
            }
        }
    }
    float* mk[4] = {(float*)w.bK, (float*)w.bD, (float*)w.dconv, (float*)w.chat};
    const double* sub = split ? cp : nullptr;
    if (w.D == 1) k_multipliers<1><<<bl, th, 0, st>>>(src[0], src[1], w.M, w.n, ph, mk[0], mk[1], mk[2], mk[3], sub);
    else if (w.D == 2)
        k_multipliers<2><<<bl, th, 0, st>>>(src[0], src[1], w.M, w.n, ph, mk[0], mk[1], mk[2], mk[3], sub);
    else k_multipliers<3><<<bl, th, 0, st>>>(src[0], src[1], w.M, w.n, ph, mk[0], mk[1], mk[2], mk[3], sub);
    cudaError_t e = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(st);
    // the lowest modes' coefficients (FP64) for the CG preconditioner
    std::vector<double> all(total);
    cudaError_t e3 = e == cudaSuccess && e2 == cudaSuccess
                         ? cudaMemcpy(all.data(), src[0], sizeof(double) * total, cudaMemcpyDeviceToHost)
                         : cudaSuccess;
    cudaFree(a);
    if (e != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return ADDKER_ECUDA;
    {
        const int B = 2 * kPcMaxBand + 1;
        int64_t nb = 1;
        for (int t = 0; t < w.D; ++t) nb *= B;
        std::vector<double>& lc = p.lowc[s];
        lc.assign(nb, 0.0);
        for (int64_t o = 0; o < nb; ++o) {
            int64_t rem = o, src_idx = 0, mult = 1;
            bool inside = true;
            for (int t = w.D - 1; t >= 0; --t) {
                const int k = (int)(rem % B) - kPcMaxBand;
                rem /= B;
                if (k <= -w.M / 2 || k >= w.M / 2) inside = false;
                src_idx += (int64_t)(k + w.M / 2) * mult;
                mult *= w.M;
            }
            if (inside) lc[o] = all[src_idx];
        }
    }
    p.pq[s] = split ? 1.0 / (2.0 * p.ell[s] * p.ell[s]) : 0.0;
    w.pq = (float)p.pq[s];
    p.any_split = false;
    for (double q : p.pq) p.any_split = p.any_split || q != 0.0;
    return ADDKER_OK;
}

// dK/d ell_s = sigma_f^2 (f / ell_s) K_s^der: f = 2 for the Gaussian (Sec. 3.3), 1 for Matern(1/2) (Sec. 5)
double der_factor(const Plan& p) { return p.kernel == ADDKER_KERNEL_MATERN12 ? 1.0 : 2.0; }

int upload_scales(Plan& p)
{
    std::vector<float> sc(3 * p.P);
    for (int s = 0; s < p.P; ++s) {
        sc[s] = 1.0f;
        sc[p.P + s] = (float)(p.sigma_f * p.sigma_f);
        sc[2 * p.P + s] = (float)(p.sigma_f * p.sigma_f * der_factor(p) / p.ell[s]);
    }
    CK(cudaMemcpy(p.scale_dev, sc.data(), sizeof(float) * sc.size(), cudaMemcpyHostToDevice));
    return ADDKER_OK;
}

int setup_window(Plan& p, int s, const float* X, int* keys, int* flag)
{
    WinDev& w = p.win[s];
    const int D = w.D, n = w.n;
    int f[3] = {0, 0, 0};
    for (int t = 0; t < D; ++t) f[t] = p.feat[p.feat_off[s] + t];
    for (int t = 0; t < 3; ++t) w.feat[t] = f[t];
    int64_t cells = 1;
    for (int t = 0; t < D; ++t) cells *= n;
    int* hist = nullptr;
    int* bounds = nullptr;
    CK(cudaMalloc(&hist, sizeof(int) * (cells + 6)));
    bounds = hist + cells;
    CK(cudaMemset(hist, 0, sizeof(int) * cells));
    int binit[6] = {1 << 30, 1 << 30, 1 << 30, -(1 << 30), -(1 << 30), -(1 << 30)};
    CK(cudaMemcpy(bounds, binit, sizeof(binit), cudaMemcpyHostToDevice));
    double rho = 0.25 - p.eps_B / 2.0;
    float rho2 = (float)(rho * rho * (1.0 + 4e-6));
    int th = 256, bl = grid_blocks(p.N, th);
    if (D == 1) k_cell_keys<1><<<bl, th>>>(X, p.N, p.d, f[0], f[1], f[2], n, rho2, keys, hist, bounds, flag);
    else if (D == 2) k_cell_keys<2><<<bl, th>>>(X, p.N, p.d, f[0], f[1], f[2], n, rho2, keys, hist, bounds, flag);
    else k_cell_keys<3><<<bl, th>>>(X, p.N, p.d, f[0], f[1], f[2], n, rho2, keys, hist, bounds, flag);
    CK(cudaGetLastError());
    std::vector<int> h(cells);
    int bh[6], fl = 0;
    CK(cudaMemcpy(h.data(), hist, sizeof(int) * cells, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(bh, bounds, sizeof(bh), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&fl, flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (fl) { cudaFree(hist); return ADDKER_EDOMAIN; }
    // offsets and the non-empty cells (first point, count, packed cell, window); work items are cut
    // from the cells by build_items
    std::vector<int> off(cells);
    int64_t acc = 0;
    std::vector<int4>& cl = p.cells[s];
    cl.clear();
    for (int64_t k = 0; k < cells; ++k) {
        off[k] = (int)acc;
        int cnt = h[k];
        if (cnt > 0) {
            int c[3] = {0, 0, 0};
            int64_t rem = k;
            for (int t = D - 1; t >= 0; --t) { c[t] = (int)(rem % n); rem /= n; }
            int packed = c[0] | (c[1] << 8) | (c[2] << 16);
            cl.push_back(make_int4((int)acc, cnt, packed, s));
        }
        acc += cnt;
    }
    p.n_cells[s] = (int)cl.size();
    // scatter
    CK(cudaMemcpy(hist, off.data(), sizeof(int) * cells, cudaMemcpyHostToDevice));
    float4* pts;
    CS(dalloc(p, &pts, p.N));
    w.pts = pts;
    if (D == 1) k_scatter<1><<<bl, th>>>(X, p.N, p.d, f[0], f[1], f[2], keys, hist, pts);
    else if (D == 2) k_scatter<2><<<bl, th>>>(X, p.N, p.d, f[0], f[1], f[2], keys, hist, pts);
    else k_scatter<3><<<bl, th>>>(X, p.N, p.d, f[0], f[1], f[2], keys, hist, pts);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    cudaFree(hist);
    // bounding box of every support: [cmin - m + 1, cmax + m] per axis
    for (int t = 0; t < 3; ++t) {
        if (t < D) {
            w.lo[t] = bh[t] - w.m + 1;
            w.box[t] = bh[3 + t] + w.m - w.lo[t] + 1;
            if (w.lo[t] < 0 || w.lo[t] + w.box[t] > n) return ADDKER_EDOMAIN;
        } else {
            w.lo[t] = 0;
            w.box[t] = 1;
        }
    }
    // buffers that do not depend on the right-hand side (grids: ensure_slots)
    const int M = w.M;
    int64_t md = 1;
    for (int t = 0; t < D; ++t) md *= M;
    float4* spec;
    float* mult;
    w.gsz = (int64_t)w.box[0] * w.box[1] * w.box[2];
    w.b1sz = D == 3 ? (int64_t)w.box[0] * std::max(w.box[1], M) * M : 0;
    w.b2sz = D == 3 ? (int64_t)w.box[0] * M * M : 0;
    w.grid = nullptr;
    w.h = nullptr;
    w.buf1 = w.buf2 = nullptr;
    CS(dalloc(p, &spec, md));
    CS(dalloc(p, &mult, 4 * md));
    w.spec = spec;
    w.bK = mult;
    w.bD = mult + md;
    w.dconv = mult + 2 * md;
    w.chat = mult + 3 * md;
    for (int t = 0; t < 3; ++t) { w.twf[t] = nullptr; w.twi[t] = nullptr; }
    for (int t = 0; t < D; ++t) {
        float2* tw;
        CS(dalloc(p, &tw, 2 * (int64_t)w.box[t] * M));
        k_twiddles<<<grid_blocks((int64_t)w.box[t] * M, 128), 128>>>(tw, tw + (int64_t)w.box[t] * M, w.lo[t],
                                                                     w.box[t], M, n);
        CK(cudaGetLastError());
        w.twf[t] = tw;
        w.twi[t] = tw + (int64_t)w.box[t] * M;
    }
    return ADDKER_OK;
}

// Per-feature [min, max] of the points into the plan-owned p.range (the separable reading's fit
// intervals); the points were checked for finiteness and the ball by the cell keys already.
int feature_range(Plan& p, const float* X)
{
    if (p.d > 65535) return ADDKER_EINVAL;
    CS(dalloc(p, &p.range, 2 * (int64_t)p.d + 1));
    int* bad = reinterpret_cast<int*>(p.range + 2 * (int64_t)p.d);
    CK(feature_range_async(X, p.N, p.d, p.range, bad, nullptr));
    int hbad = 0;
    CK(cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost));
    return hbad ? ADDKER_EDOMAIN : ADDKER_OK;
}

bool valid_stream_ptrs(const void* ptr)
{
    if (!ptr) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ---- stage profiling --------------------------------------------------------------
cudaEvent_t take_event(Plan& p)
{
    if (!p.ev_pool.empty()) {
        cudaEvent_t e = p.ev_pool.back();
        p.ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct Stage {                            // brackets one stage of a product with events when profiling
    Plan& p;
    int id;
    cudaEvent_t a = nullptr;
    Stage(Plan& plan, int stage) : p(plan), id(stage)
    {
        if (p.prof) {
            a = take_event(p);
            cudaEventRecord(a, p.stream);
        }
    }
    void done(int launched)
    {
        if (!p.prof) return;
        p.launches[id] += launched;
        cudaEvent_t b = take_event(p);
        cudaEventRecord(b, p.stream);
        p.ev_used.push_back({id, {a, b}});
    }
};

int vec_ok(const Plan& p, const float* out, int64_t ld)
{
    return (p.N % 4 == 0) && (ld % 4 == 0) && (reinterpret_cast<uintptr_t>(out) % 16 == 0);
}

// Work items: every non-empty cell's points in chunks of at most `chunk`, heaviest first within a
// window; one device array holding the kernel kinds one after another (item_begin[k][s] absolute).
// The chunk is the scheduling grain of the spread and gather kernels (addker_autotune chooses it).
int build_items(Plan& p, int chunk, int chunk_sp)
{
    if (chunk_sp <= 0) chunk_sp = chunk;
    // two lists: the one every kernel uses, and the spread's, which differs for 2-D windows only
    std::vector<int4> lists[2][kKinds];
    for (int k = 0; k < kKinds; ++k) {
        p.item_begin[k].assign(1, 0);
        p.item_begin_sp[k].assign(1, 0);
    }
    for (int s = 0; s < p.P; ++s) {
        for (int l = 0; l < 2; ++l) {
            // spreading a 2-D window: few crowded cells whose 8x8 boxes overlap, so every item ends with
            // atomic adds to the same few hundred grid values; those items are kLowdChunkFactor times
            // larger (1-D windows, and the gathers, need the parallelism of small items more)
            const int ch = l == 0 ? chunk : (p.dims[s] == 2 ? chunk_sp * kLowdChunkFactor : chunk_sp);
            std::vector<int4> items;
            for (const int4& c : p.cells[s])
                for (int st = 0; st < c.y; st += ch)
                    items.push_back(make_int4(c.x + st, std::min(ch, c.y - st), c.z, s));
            std::stable_sort(items.begin(), items.end(), [](const int4& a, const int4& b) { return a.y > b.y; });
            std::vector<int4>& dst = lists[l][p.kind[s]];
            dst.insert(dst.end(), items.begin(), items.end());
        }
        for (int k = 0; k < kKinds; ++k) {
            p.item_begin[k].push_back((int)lists[0][k].size());
            p.item_begin_sp[k].push_back((int)lists[1][k].size());
        }
    }
    std::vector<int4> all;
    for (int l = 0; l < 2; ++l)
        for (int k = 0; k < kKinds; ++k) {
            const int base = (int)all.size();
            for (int& b : (l == 0 ? p.item_begin[k] : p.item_begin_sp[k])) b += base;
            all.insert(all.end(), lists[l][k].begin(), lists[l][k].end());
        }
    if ((int64_t)all.size() > p.items_cap) {
        if (p.items) cudaFree(p.items);
        p.items = nullptr;
        p.items_cap = 0;
        if (cudaMalloc(&p.items, sizeof(int4) * all.size()) != cudaSuccess) {
            cudaGetLastError();
            return ADDKER_ENOMEM;
        }
        p.items_cap = (int64_t)all.size();
    }
    if (!all.empty()) CK(cudaMemcpy(p.items, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice));
    p.chunk = chunk;
    p.chunk_sp = chunk_sp;
    return ADDKER_OK;
}

// Per-window grids for `want` right-hand sides at once (grid, h and the D = 3 transform buffers, one
// slot per right-hand side) and the window-sum scratch ks (slots x P x N). Grown on demand: the old
// buffers are freed after the stream has drained, the grids of the new ones are zeroed, and the
// device descriptors are re-uploaded.
int ensure_slots(Plan& p, int want)
{
    want = std::min(std::max(want, 1), kMaxRhsChunk);
    if (want <= p.slots) return ADDKER_OK;
    int r = 1;
    while (r < want) r *= 2;
    r = std::min(r, kMaxRhsChunk);
    CK(cudaStreamSynchronize(p.stream));
    clear_graphs(p);                               // captured products point at the old slots
    for (void* a : p.slot_allocs) cudaFree(a);
    p.slot_allocs.clear();
    p.bytes -= p.slot_bytes;
    p.slot_bytes = 0;
    p.slots = 0;
    auto take = [&](auto** ptr, int64_t count) -> int {
        using T = std::remove_pointer_t<std::remove_reference_t<decltype(*ptr)>>;
        void* raw = nullptr;
        if (count == 0) { *ptr = nullptr; return ADDKER_OK; }
        if (cudaMalloc(&raw, sizeof(T) * (size_t)count) != cudaSuccess) { cudaGetLastError(); return ADDKER_ENOMEM; }
        p.slot_allocs.push_back(raw);
        p.slot_bytes += (int64_t)(sizeof(T) * (size_t)count);
        p.bytes += (int64_t)(sizeof(T) * (size_t)count);
        *ptr = static_cast<T*>(raw);
        return ADDKER_OK;
    };
    for (int s = 0; s < p.P; ++s) {
        WinDev& w = p.win[s];
        float* grid;
        double* grid64 = nullptr;
        float2* hh;
        float4 *b1, *b2;
        CS(take(&grid, r * w.gsz));
        if (p.comp) {
            CS(take(&grid64, r * w.gsz));
            CK(cudaMemsetAsync(grid64, 0, sizeof(double) * (size_t)(r * w.gsz), p.stream));
        }
        CS(take(&hh, r * w.gsz));
        CS(take(&b1, r * w.b1sz));
        CS(take(&b2, r * w.b2sz));
        CK(cudaMemsetAsync(grid, 0, sizeof(float) * (size_t)(r * w.gsz), p.stream));
        w.grid = grid;
        w.grid64 = grid64;
        w.h = hh;
        w.buf1 = b1;
        w.buf2 = b2;
    }
    float* ks = nullptr;
    if (p.P > 1) CS(take(&ks, (int64_t)r * p.P * p.N));
    p.ks = ks;
    CK(cudaMemcpyAsync(p.wins_dev, p.win.data(), sizeof(WinDev) * p.P, cudaMemcpyHostToDevice, p.stream));
    CK(cudaStreamSynchronize(p.stream));
    p.slots = r;
    return ADDKER_OK;
}

// Sum of the per-window outputs ks (R x P x N, right-hand side r at r P N) into out + r ld, scaled.
void window_sum(Plan& p, int R, float scale, float* out, int64_t ld, cudaStream_t st)
{
    const dim3 grid(grid_blocks((p.N + 3) / 4, 256), R);
    launch_k(true, k_window_sum, grid, dim3(256), 0, st, (const float*)p.ks, p.P, p.N, scale, out, ld,
             vec_ok(p, out, ld));
}

// One product for R <= slots right-hand sides v + r ldv (r < R), every stage one launch per kernel kind.
//   mode 0: Kv + r ldk = K v_r (if Kv) and dK + r ldd + s N = dK/d ell_s v_r for all s (if dK)
//   mode 1: dK + r ldd = dK/d ell_s v_r for the single window `window`
//   mode 2: Kv + r ldk = sum_s dK/d ell_s v_r (shared length scale)
int product(Plan& p, const float* v, int64_t ldv, int R, float* Kv, int64_t ldk, float* dK, int64_t ldd, int window,
            int mode)
{
    cudaStream_t st = p.stream;
    const int only = mode == 1 ? window : -1;
    {
        // d = 3 grids are zeroed by the forward transform that consumes them, d < 3 grids by the small
        // transform, and every grid at allocation, so nothing is cleared here
        Stage sg(p, 1);
        int n = 0;
        CK(launch_spread(p, only, v, ldv, R, st, &n));
        sg.done(n);
    }
    {
        Stage sg(p, 2);
        int n = 0;
        CK(launch_transforms(p, only, R, st, &n, false));
        sg.done(n);
    }
    const float* ones = p.scale_dev;
    const float* sf2 = p.scale_dev + p.P;
    const float* sder = p.scale_dev + 2 * p.P;
    const int64_t PN = (int64_t)p.P * p.N;
    int n = 0;
    Stage sg(p, 3);
    if (mode == 1) {                               // window s only, written at offset 0
        CK(launch_gather(p, only, nullptr, 0, 0, dK, 0, ldd, R, ones, sder, st, &n));
        sg.done(n);
        return ADDKER_OK;
    }
    if (mode == 2) {
        if (p.P == 1) {
            CK(launch_gather(p, -1, nullptr, 0, 0, Kv, 0, ldk, R, ones, sder, st, &n));
            sg.done(n);
            return ADDKER_OK;
        }
        CK(launch_gather(p, -1, nullptr, 0, 0, p.ks, p.N, PN, R, ones, sder, st, &n));
        sg.done(n);
        Stage sum(p, 4);
        window_sum(p, R, 1.0f, Kv, ldk, st);
        CK(cudaGetLastError());
        sum.done(1);
        return ADDKER_OK;
    }
    if (p.P == 1) {
        CK(launch_gather(p, -1, Kv, 0, ldk, dK, p.N, ldd, R, sf2, sder, st, &n));
        sg.done(n);
        return ADDKER_OK;
    }
    CK(launch_gather(p, -1, p.ks, p.N, PN, dK, p.N, ldd, R, ones, sder, st, &n));
    sg.done(n);
    Stage sum(p, 4);
    window_sum(p, R, (float)(p.sigma_f * p.sigma_f), Kv, ldk, st);
    CK(cudaGetLastError());
    sum.done(1);
    return ADDKER_OK;
}

// nrhs right-hand sides (columns of length N, v + j N) in chunks of at most kMaxRhsChunk.
int product_chunks(Plan& p, const float* v, int nrhs, float* Kv, float* dK, int window, int mode)
{
    const int64_t N = p.N;
    const int64_t ldd = mode == 0 ? N * p.P : N;
    for (int j = 0; j < nrhs; j += p.slots) {
        const int R = std::min(p.slots, nrhs - j);
        CS(product(p, v + j * N, N, R, Kv ? Kv + j * N : nullptr, N, dK ? dK + j * ldd : nullptr, ldd, window, mode));
    }
    return ADDKER_OK;
}

}  // namespace

// All products go through here. With graphs on (and no stage profiling, and a stream that is not itself
// being captured), the second consecutive call with the same arguments is captured on a private stream
// and every later one replays the graph on the plan's stream: one launch instead of one per kernel.
int addker::product_all(Plan& p, const float* v, int nrhs, float* Kv, float* dK, int window, int mode)
{
    // a batch that cannot get more slots runs in single-right-hand-side chunks
    if (ensure_slots(p, nrhs) != ADDKER_OK) CS(ensure_slots(p, 1));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!p.graphs || p.prof || cudaStreamIsCapturing(p.stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return product_chunks(p, v, nrhs, Kv, dK, window, mode);
    }
    const Plan::GraphKey key = {v, Kv, dK, nrhs, window, mode};
    for (size_t i = 0; i < p.graph_cache.size(); ++i)
        if (p.graph_cache[i].first == key) {
            auto e = p.graph_cache[i];
            p.graph_cache.erase(p.graph_cache.begin() + i);
            p.graph_cache.push_back(e);
            CK(cudaGraphLaunch(e.second, p.stream));
            ++p.graph_replays;
            return ADDKER_OK;
        }
    if (!(p.last_key == key)) {                    // first sighting: run eagerly, capture if it repeats
        p.last_key = key;
        return product_chunks(p, v, nrhs, Kv, dK, window, mode);
    }
    if (!p.cap_stream) CK(cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(p.cap_stream, cudaStreamCaptureModeThreadLocal));
    const cudaStream_t user = p.stream;
    p.stream = p.cap_stream;
    const int status = product_chunks(p, v, nrhs, Kv, dK, window, mode);
    p.stream = user;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p.cap_stream, &graph);
    if (status != ADDKER_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return status != ADDKER_OK ? status : ADDKER_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ei);
    constexpr size_t kMaxGraphs = 8;
    if (p.graph_cache.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(p.graph_cache.front().second);
        p.graph_cache.erase(p.graph_cache.begin());
    }
    p.graph_cache.push_back({key, exec});
    CK(cudaGraphLaunch(exec, p.stream));
    return ADDKER_OK;
}

namespace {

}  // namespace

// ---- building blocks for callers that bring their own device memory ---------------------
namespace addker {

// Window polynomials for cutoff m and oversampling sigma_os.
void window_poly_for(int m, double sigma_os, WinPoly* poly)
{
    fit_window_poly(m, M_PI * (2.0 - 1.0 / sigma_os), poly);
}

// Fourier multipliers bK, bD, dconv of window w (pointers already set) for length scale ell under the
// separable reading (axis t is feature t of range: device, per-feature [min, max] of the window's
// points), with the quadratic split decided as for a plan (*pq receives 1/(2 ell^2) or 0), computed in
// the caller's FP64 scratch of at least 3 M^D + 6 M doubles. Enqueued on st and waited for.
int multipliers_with_scratch(const WinDev& w, double ell, double eps_B, const float* range, const WinPoly& poly,
                             double* scratch, cudaStream_t st, float* pq)
{
    int64_t total = 1;
    for (int t = 0; t < w.D; ++t) total *= w.M;
    double* a = scratch;
    double* b = a + total;
    double* cp = b + total;
    double* ph = cp + total;
    double* fit = ph + w.M;
    double phat[kMaxBandwidth];
    window_transform(poly, w.m, w.n, w.M, phat);
    CK(cudaMemcpyAsync(ph, phat, sizeof(double) * w.M, cudaMemcpyHostToDevice, st));
    const int feat[3] = {0, 1, 2};
    CK(separable_coefficients(w.D, w.M, ell, eps_B, range, feat, fit, a, b, cp, st));
    bool split = false;
    CS(decide_split(w.D, w.M, b, cp, st, &split));
    const double* sub = split ? cp : nullptr;
    const int th = 256, bl = grid_blocks(total, th);
    float* bK = const_cast<float*>(w.bK);
    float* bD = const_cast<float*>(w.bD);
    float* dc = const_cast<float*>(w.dconv);
    if (w.D == 1) k_multipliers<1><<<bl, th, 0, st>>>(a, b, w.M, w.n, ph, bK, bD, dc, nullptr, sub);
    else if (w.D == 2) k_multipliers<2><<<bl, th, 0, st>>>(a, b, w.M, w.n, ph, bK, bD, dc, nullptr, sub);
    else k_multipliers<3><<<bl, th, 0, st>>>(a, b, w.M, w.n, ph, bK, bD, dc, nullptr, sub);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    *pq = split ? (float)(1.0 / (2.0 * ell * ell)) : 0.f;
    return ADDKER_OK;
}

// Per-feature [min, max] of X (N x d row-major) into range (2d floats) and *bad = 1 for a value that is
// not finite; range and *bad are initialised on the device first.
cudaError_t feature_range_async(const float* X, int64_t N, int d, float* range, int* bad, cudaStream_t st)
{
    k_range_init<<<1, 64, 0, st>>>(range, d, bad);
    const int bx = (int)std::min<int64_t>(64, (N + 255) / 256);
    k_feature_range<<<dim3(bx, d), 256, 0, st>>>(X, N, d, range, bad);
    return cudaGetLastError();
}

// Per-axis twiddles of window w (box and lo set) into tw[t] (forward) and tw[t] + box*M (inverse).
cudaError_t twiddles_into(const WinDev& w, float2* const tw[3], cudaStream_t st)
{
    for (int t = 0; t < w.D; ++t)
        k_twiddles<<<grid_blocks((int64_t)w.box[t] * w.M, 128), 128, 0, st>>>(tw[t], tw[t] + (int64_t)w.box[t] * w.M,
                                                                             w.lo[t], w.box[t], w.M, w.n);
    return cudaGetLastError();
}

}  // namespace addker

// =================================================================== C ABI ====

extern "C" {

const char* addker_strerror(int status)
{
    switch (status) {
        case ADDKER_OK: return "ok";
        case ADDKER_EINVAL: return "invalid argument";
        case ADDKER_EDOMAIN: return "point outside the ball ||x^W|| <= 1/4 - eps_B/2 (or not finite)";
        case ADDKER_ENOMEM: return "device allocation failed";
        case ADDKER_ECUDA: return "CUDA error";
        case ADDKER_ETIMEOUT: return "device wait timed out";
        case ADDKER_ELIMIT: return "request exceeds the fixed memory limit of addker_fastsum_noalloc "
                                   "(bandwidth <= 32, at most 3 features)";
        default: return "unknown status";
    }
}

int addker_opts_default(addker_opts* o)
{
    if (!o) return ADDKER_EINVAL;
    o->sigma_os = 2.0;
    o->eps_B = 1.0 / 16.0;
    o->p = -1;
    o->window = ADDKER_WIN_KB;
    o->kernel = ADDKER_KERNEL_GAUSS;
    o->compensated = 0;
    o->reg = ADDKER_REG_DEFAULT;
    o->stream = nullptr;
    return ADDKER_OK;
}

int addker_setup(addker_plan** out, const float* points, int64_t N, int d, const int* win_off, const int* win_feat,
                 int P, const double* ell, double sigma_f, const int* bandwidth, int cutoff, const addker_opts* opts)
{
    if (!out) return ADDKER_EINVAL;
    *out = nullptr;
    addker_opts o;
    addker_opts_default(&o);
    if (opts) o = *opts;
    if (N < 1 || N > 0x7fffffffLL || d < 1 || P < 1 || P > kMaxWindows || !win_off || !win_feat || !ell || !bandwidth)
        return ADDKER_EINVAL;
    if (!(sigma_f > 0.0) || cutoff < 2 || cutoff > 8 || (o.window != ADDKER_WIN_KB && o.window != ADDKER_WIN_ES) ||
        (o.kernel != ADDKER_KERNEL_GAUSS && o.kernel != ADDKER_KERNEL_MATERN12) ||
        (o.compensated != 0 && o.compensated != 1) ||
        (o.reg != ADDKER_REG_DEFAULT && o.reg != ADDKER_REG_SEPARABLE && o.reg != ADDKER_REG_RADIAL) ||
        (o.reg == ADDKER_REG_SEPARABLE && o.kernel != ADDKER_KERNEL_GAUSS))
        return ADDKER_EINVAL;
    if (!(o.eps_B > 0.0 && o.eps_B < 0.5) || !(o.sigma_os >= 1.25 && o.sigma_os <= 4.0) || o.p < -1 || o.p > 12)
        return ADDKER_EINVAL;
    if (win_off[0] != 0) return ADDKER_EINVAL;
    for (int s = 0; s < P; ++s) {
        int ds = win_off[s + 1] - win_off[s];
        if (ds < 1 || ds > 3 || !(ell[s] > 0.0)) return ADDKER_EINVAL;
        for (int q = win_off[s]; q < win_off[s + 1]; ++q) {
            if (win_feat[q] < 0 || win_feat[q] >= d) return ADDKER_EINVAL;
            for (int r = win_off[s]; r < q; ++r) if (win_feat[r] == win_feat[q]) return ADDKER_EINVAL;
        }
        int M = bandwidth[s];
        if (M < 4 || M > kMaxBandwidth || (M & 1)) return ADDKER_EINVAL;
        double nd = o.sigma_os * M;
        int n = (int)std::lround(nd);
        if (std::fabs(nd - n) > 1e-9 || (n & 1) || n > 128) return ADDKER_EINVAL;
        if (cutoff + 1 > n / 4.0 + n * o.eps_B / 2.0) return ADDKER_EINVAL;
    }
    if (!valid_stream_ptrs(points)) return ADDKER_EINVAL;

    addker_plan* plan = new (std::nothrow) addker_plan;
    if (!plan) return ADDKER_ENOMEM;
    Plan& p = plan->p;
    p.N = N;
    p.d = d;
    p.P = P;
    p.m = cutoff;
    p.sigma_f = sigma_f;
    p.sigma_os = o.sigma_os;
    p.eps_B = o.eps_B;
    p.p_opt = o.p;
    p.reg = o.reg != ADDKER_REG_DEFAULT ? o.reg
                                        : (o.kernel == ADDKER_KERNEL_GAUSS ? ADDKER_REG_SEPARABLE : ADDKER_REG_RADIAL);
    p.kernel = o.kernel;
    p.window = o.window;
    p.comp = o.compensated == 1;
    p.stream = static_cast<cudaStream_t>(o.stream);
    p.feat_off.assign(win_off, win_off + P + 1);
    p.feat.assign(win_feat, win_feat + win_off[P]);
    p.ell.assign(ell, ell + P);
    p.bandwidth.assign(bandwidth, bandwidth + P);
    p.win.resize(P);
    p.dims.resize(P);
    p.kind.resize(P);
    p.n_cells.assign(P, 0);
    const double b_shape = window_shape(o.window, cutoff, o.sigma_os);
    for (int s = 0; s < P; ++s) {
        WinDev& w = p.win[s];
        std::memset(&w, 0, sizeof(w));
        w.D = win_off[s + 1] - win_off[s];
        p.dims[s] = w.D;
        p.kind[s] = kind_of(w.D, cutoff);
        w.M = bandwidth[s];
        w.n = (int)std::lround(o.sigma_os * w.M);
        w.m = cutoff;
        w.b = (float)b_shape;
    }
    fit_window_poly(cutoff, b_shape, &p.poly, o.window);
    int* keys = nullptr;
    int* flag = nullptr;
    int status = ADDKER_OK;
    p.cells.assign(P, {});
    if (cudaMalloc(&keys, sizeof(int) * (size_t)(N + 1)) != cudaSuccess) status = ADDKER_ENOMEM;
    if (status == ADDKER_OK) {
        flag = keys + N;
        if (cudaMemset(flag, 0, sizeof(int)) != cudaSuccess) status = ADDKER_ECUDA;
    }
    for (int s = 0; s < P && status == ADDKER_OK; ++s) status = setup_window(p, s, points, keys, flag);
    if (keys) cudaFree(keys);
    if (status == ADDKER_OK) status = feature_range(p, points);
    if (status == ADDKER_OK) status = build_items(p, kItemPoints, kItemPoints);
    if (status == ADDKER_OK) status = dalloc(p, &p.wins_dev, P);
    if (status == ADDKER_OK) status = dalloc(p, &p.scale_dev, 3 * P);
    if (status == ADDKER_OK) status = dalloc(p, &p.dots, 2 * P);
    if (status == ADDKER_OK) {
        // the persistent kernels' counter (16 ints), then the moments: kMaxRhsChunk slots x P windows x 8,
        // then P x 8 kept by addker_vjp
        double* buf = nullptr;
        status = dalloc(p, &buf, 8 + 8 * (int64_t)P * (kMaxRhsChunk + 1));
        if (status == ADDKER_OK) {
            p.counters = reinterpret_cast<int*>(buf);
            p.mom = buf + 8;
            p.mom_saved = p.mom + 8 * (int64_t)P * kMaxRhsChunk;
            for (int s = 0; s < P; ++s) {
                p.win[s].mom = p.mom + 8 * s;
                p.win[s].mstride = 8 * (int64_t)P;
            }
        }
    }
    p.pq.assign(P, 0.0);
    p.lowc.assign(P, {});
    for (int s = 0; s < P && status == ADDKER_OK; ++s) status = compute_multipliers(p, s);
    if (status == ADDKER_OK && cudaMemcpy(p.wins_dev, p.win.data(), sizeof(WinDev) * P, cudaMemcpyHostToDevice) != cudaSuccess)
        status = ADDKER_ECUDA;
    if (status == ADDKER_OK) status = upload_scales(p);
    if (status == ADDKER_OK) status = ensure_slots(p, 1);
    if (status == ADDKER_OK && cudaDeviceSynchronize() != cudaSuccess) status = ADDKER_ECUDA;
    if (status != ADDKER_OK) {
        cudaGetLastError();
        release(p);
        delete plan;
        return status;
    }
    *out = plan;
    return ADDKER_OK;
}

int addker_set_params(addker_plan* plan, const double* ell, double sigma_f)
{
    if (!plan || !(sigma_f > 0.0)) return ADDKER_EINVAL;
    Plan& p = plan->p;
    if (ell) {
        for (int s = 0; s < p.P; ++s) if (!(ell[s] > 0.0)) return ADDKER_EINVAL;
        p.ell.assign(ell, ell + p.P);
    }
    p.sigma_f = sigma_f;
    CK(cudaStreamSynchronize(p.stream));
    clear_graphs(p);                               // sigma_f is baked into captured window sums
    pc_release(p);                                 // the preconditioner's modes and weights change
    for (int s = 0; s < p.P; ++s) CS(compute_multipliers(p, s));
    CK(cudaMemcpy(p.wins_dev, p.win.data(), sizeof(WinDev) * p.P, cudaMemcpyHostToDevice));   // the split may change
    return upload_scales(p);
}

int addker_set_schedule(addker_plan* plan, int chunk, int chunk_spread, int spread_blocks, int spread_tile)
{
    if (!plan || chunk < 16 || chunk > 4096 || chunk_spread < 16 || chunk_spread > 4096 || spread_blocks < 0 ||
        spread_blocks > 8 || (spread_tile != 0 && spread_tile != 1))
        return ADDKER_EINVAL;
    Plan& p = plan->p;
    CK(cudaStreamSynchronize(p.stream));
    clear_graphs(p);
    if (chunk != p.chunk || chunk_spread != p.chunk_sp) CS(build_items(p, chunk, chunk_spread));
    p.sp_blocks = spread_blocks;
    p.sp_tile = spread_tile;
    return ADDKER_OK;
}

int addker_set_precond(addker_plan* plan, int band)
{
    if (!plan || band < 0 || band > kPcMaxBand) return ADDKER_EINVAL;
    Plan& p = plan->p;
    CK(cudaStreamSynchronize(p.stream));
    pc_release(p);
    p.pc_band = band;
    return ADDKER_OK;
}

int addker_set_graphs(addker_plan* plan, int enable)
{
    if (!plan || (enable != 0 && enable != 1)) return ADDKER_EINVAL;
    Plan& p = plan->p;
    CK(cudaStreamSynchronize(p.stream));
    clear_graphs(p);
    p.graphs = enable == 1;
    return ADDKER_OK;
}

int addker_autotune(addker_plan* plan, const float* v, int nrhs, int* chosen, double* times, int cap)
{
    if (!plan || !v || nrhs < 1) return ADDKER_EINVAL;
    Plan& p = plan->p;
    if (!valid_stream_ptrs(v)) return ADDKER_EINVAL;
    static const int cand[] = {64, 128, 256, 512, 1024};
    constexpr int nc = sizeof(cand) / sizeof(cand[0]);
    CS(ensure_slots(p, nrhs));
    float *Kv = nullptr, *dK = nullptr;
    if (cudaMalloc(&Kv, sizeof(float) * (size_t)p.N * nrhs) != cudaSuccess ||
        cudaMalloc(&dK, sizeof(float) * (size_t)p.N * p.P * nrhs) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(Kv);
        return ADDKER_ENOMEM;
    }
    const bool graphs = p.graphs, prof = p.prof;
    p.graphs = false;
    p.prof = false;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int status = ADDKER_OK, best = p.chunk, best_sp = p.chunk_sp;
    double best_ms = 1e300;
    // ms per product for the items cut by (chunk, chunk_sp); 0 on failure (status set)
    auto time_items = [&](int chunk, int chunk_sp) -> double {
        if (cudaStreamSynchronize(p.stream) != cudaSuccess) { status = ADDKER_ECUDA; return 0.0; }
        status = build_items(p, chunk, chunk_sp);
        if (status == ADDKER_OK) status = product_all(p, v, nrhs, Kv, dK, -1, 0);       // warm-up
        cudaEventRecord(a, p.stream);
        for (int rep = 0; rep < 3 && status == ADDKER_OK; ++rep) status = product_all(p, v, nrhs, Kv, dK, -1, 0);
        cudaEventRecord(b, p.stream);
        float ms = 0.f;
        if (status == ADDKER_OK && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
            return ms / 3.0;
        if (status == ADDKER_OK) status = ADDKER_ECUDA;
        return 0.0;
    };
    // phase 1: one size for both lists; phase 2: the spread's size alone, the gather's kept
    for (int c = 0; c < nc && status == ADDKER_OK; ++c) {
        const double ms = time_items(cand[c], cand[c]);
        if (status != ADDKER_OK) break;
        if (times && c < cap) times[c] = ms;
        if (ms < best_ms) { best_ms = ms; best = best_sp = cand[c]; }
    }
    const double joint_ms = best_ms;
    for (int c = 0; c < nc && status == ADDKER_OK; ++c) {
        const double ms = cand[c] == best ? joint_ms : time_items(best, cand[c]);
        if (status != ADDKER_OK) break;
        if (times && nc + c < cap) times[nc + c] = ms;
        if (ms < best_ms) { best_ms = ms; best_sp = cand[c]; }
    }
    // phase 3: the persistent spread's residency, blocks per SM 1, 2, 3 and as many as fit (0)
    static const int res[] = {1, 2, 3, 0};
    const int sp_blocks0 = p.sp_blocks;
    int best_res = sp_blocks0;
    for (int c = 0; c < 4 && status == ADDKER_OK; ++c) {
        p.sp_blocks = res[c];
        const double ms = time_items(best, best_sp);
        if (status != ADDKER_OK) break;
        if (times && 2 * nc + c < cap) times[2 * nc + c] = ms;
        if (ms < best_ms) { best_ms = ms; best_res = res[c]; }
    }
    p.sp_blocks = status == ADDKER_OK ? best_res : sp_blocks0;
    // phase 4: the 3-D spread's register tile (4 a x 4 b x 2 c or 8 a x 2 b x 2 c per lane)
    const int sp_tile0 = p.sp_tile;
    int best_tile = sp_tile0;
    for (int c = 0; c < 2 && status == ADDKER_OK; ++c) {
        p.sp_tile = c;
        const double ms = time_items(best, best_sp);
        if (status != ADDKER_OK) break;
        if (times && 2 * nc + 4 + c < cap) times[2 * nc + 4 + c] = ms;
        if (ms < best_ms) { best_ms = ms; best_tile = c; }
    }
    p.sp_tile = status == ADDKER_OK ? best_tile : sp_tile0;
    cudaStreamSynchronize(p.stream);
    if (status == ADDKER_OK) status = build_items(p, best, best_sp);
    clear_graphs(p);
    p.graphs = graphs;
    p.prof = prof;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(Kv);
    cudaFree(dK);
    if (status == ADDKER_OK && chosen) *chosen = best;
    return status;
}

int addker_cg(addker_plan* plan, double beta, const float* y, float* x, int nrhs, double tol, int maxit, int* iters,
              double* relres)
{
    if (!plan || !y || !x || nrhs < 1 || !(beta >= 0.0) || !(tol > 0.0) || maxit < 0) return ADDKER_EINVAL;
    if (!valid_stream_ptrs(y) || !valid_stream_ptrs(x)) return ADDKER_EINVAL;
    return cg_solve(plan->p, beta, y, x, nrhs, tol, maxit, iters, relres);
}

int addker_gp_grad(addker_plan* plan, double beta, const float* y, const float* Z, int m, double tol, int maxit,
                   double* grad, double* fit, float* alpha, int* iters)
{
    if (!plan || !y || !grad || m < 0 || (m > 0 && !Z) || !(beta >= 0.0) || !(tol > 0.0) || maxit < 0)
        return ADDKER_EINVAL;
    if (!valid_stream_ptrs(y) || (m > 0 && !valid_stream_ptrs(Z)) || (alpha && !valid_stream_ptrs(alpha)))
        return ADDKER_EINVAL;
    return gp_grad(plan->p, beta, y, Z, m, tol, maxit, grad, fit, alpha, iters);
}

int addker_gsi(addker_plan* plan, const float* v, int cap, int* feats, double* rho, double* total)
{
    if (!plan || !v || cap < 0 || (cap > 0 && (!feats || !rho))) return ADDKER_EINVAL;
    if (!valid_stream_ptrs(v)) return ADDKER_EINVAL;
    Plan& p = plan->p;
    CS(ensure_slots(p, 1));
    return gsi_run(p, v, cap, feats, rho, total);
}

int addker_set_stream(addker_plan* plan, void* stream)
{
    if (!plan) return ADDKER_EINVAL;
    plan->p.stream = static_cast<cudaStream_t>(stream);
    return ADDKER_OK;
}

int addker_matvec_all(addker_plan* plan, const float* v, float* Kv, float* dKdell, int nrhs)
{
    if (!plan || !v || !Kv || nrhs < 1) return ADDKER_EINVAL;
    return product_all(plan->p, v, nrhs, Kv, dKdell, -1, 0);
}

int addker_matvec(addker_plan* plan, const float* v, float* Kv, int nrhs)
{
    return addker_matvec_all(plan, v, Kv, nullptr, nrhs);
}

int addker_dmatvec(addker_plan* plan, int param, const float* v, float* out, int nrhs)
{
    if (!plan || !v || !out || nrhs < 1) return ADDKER_EINVAL;
    Plan& p = plan->p;
    if (param >= p.P || param < ADDKER_SIGMA_F) return ADDKER_EINVAL;
    if (param >= 0) return product_all(p, v, nrhs, nullptr, out, param, 1);
    if (param == ADDKER_ELL_SHARED) return product_all(p, v, nrhs, out, nullptr, -1, 2);
    CS(product_all(p, v, nrhs, out, nullptr, -1, 0));
    const int64_t len = p.N * (int64_t)nrhs;
    launch_k(true, k_scale, dim3(grid_blocks(len, 256)), dim3(256), 0, p.stream, (const float*)out, len,
             (float)(2.0 / p.sigma_f), out);
    CK(cudaGetLastError());
    return ADDKER_OK;
}

int addker_vjp(addker_plan* plan, const float* v, const float* w, float* grad_v, double* grad_theta,
               float* grad_points)
{
    if (!plan || !v || !w || !grad_v || !grad_theta || !grad_points) return ADDKER_EINVAL;
    Plan& p = plan->p;
    if (p.window != ADDKER_WIN_KB) return ADDKER_EINVAL;         // needs a window with a bounded derivative
    CS(ensure_slots(p, 1));
    cudaStream_t st = p.stream;
    float* gx = grad_points;
    CK(cudaMemsetAsync(gx, 0, sizeof(float) * (size_t)p.N * p.d, st));
    CK(cudaMemsetAsync(p.dots, 0, sizeof(double) * 2 * p.P, st));
    // scratch for the per-window f^K of w: the plan's window-sum buffer (N for P = 1 is grad_v itself)
    float* ks = p.P > 1 ? p.ks : grad_v;
    for (int pass = 0; pass < 2; ++pass) {
        const float* u = pass == 0 ? w : v;
        CK(launch_spread(p, -1, u, p.N, 1, st, nullptr));         // slot 0; the transforms re-zero the grids
        if (pass == 0 && p.any_split)                              // w's moments, before v's replace them
            CK(cudaMemcpyAsync(p.mom_saved, p.mom, sizeof(double) * 8 * p.P, cudaMemcpyDeviceToDevice, st));
        CK(launch_transforms(p, -1, 1, st, nullptr, false));
        CK(launch_gather_grad(p, pass, pass == 0 ? v : w, ks, gx, st, nullptr));
        if (pass == 0) {
            if (p.P > 1)
                window_sum(p, 1, (float)(p.sigma_f * p.sigma_f), grad_v, p.N, st);
            else
                launch_k(true, k_scale, dim3(grid_blocks(p.N, 256)), dim3(256), 0, st, (const float*)grad_v,
                         p.N, (float)(p.sigma_f * p.sigma_f), grad_v);
            CK(cudaGetLastError());
        }
    }
    ThetaScale sc;
    for (int s = 0; s < p.P; ++s) {
        sc.s[s] = p.sigma_f * p.sigma_f * der_factor(p) / p.ell[s];
        sc.q[s] = p.pq[s];
    }
    sc.s[p.P] = 2.0 * p.sigma_f;
    launch_k(true, k_theta_grad, dim3(1), dim3(64), 0, st, (const double*)p.dots, p.P, sc, (const double*)p.mom,
             (const double*)p.mom_saved, grad_theta);
    CK(cudaGetLastError());
    return ADDKER_OK;
}

int addker_matvec_all_host(addker_plan* plan, const float* v, float* Kv, float* dKdell, int nrhs)
{
    if (!plan || !v || !Kv || nrhs < 1) return ADDKER_EINVAL;
    Plan& p = plan->p;
    int64_t need = p.N * (int64_t)nrhs;
    if (need > p.stage_cap) {
        CS(dalloc(p, &p.stage_v, need));
        CS(dalloc(p, &p.stage_k, need));
        CS(dalloc(p, &p.stage_d, need * p.P));
        p.stage_cap = need;
    }
    cudaStream_t st = p.stream;
    // page-locked host buffers are read and written by copy kernels over the CPU-GPU link (more
    // bandwidth than one copy engine); pageable ones go through cudaMemcpyAsync
    auto mapped = [](const void* q) -> void* {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
    };
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int cb = 4 * std::max(sms, 1);
    auto copy = [&](const float* src, float* dst, int64_t n) {
        const int vec = (reinterpret_cast<uintptr_t>(src) % 16 == 0) && (reinterpret_cast<uintptr_t>(dst) % 16 == 0);
        k_copy<<<cb, 256, 0, st>>>(src, dst, n, vec);
        return cudaGetLastError();
    };
    if (nrhs == 1 && dKdell && p.P > 1) {
        // one right-hand side: the windows are gathered one launch each, and each window's derivative
        // product is copied to the host on a second stream while the next window is gathered; only K v
        // (after the window sum) and the last window's copy remain after the last gather
        if (!p.copy_stream) CK(cudaStreamCreateWithFlags(&p.copy_stream, cudaStreamNonBlocking));
        while ((int)p.win_events.size() < p.P) {
            cudaEvent_t e;
            CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            p.win_events.push_back(e);
        }
        CS(ensure_slots(p, 1));
        const int64_t N = p.N;
        CK(cudaMemcpyAsync(p.stage_v, v, sizeof(float) * N, cudaMemcpyHostToDevice, st));
        CK(launch_spread(p, -1, p.stage_v, N, 1, st));
        CK(launch_transforms(p, -1, 1, st, nullptr, false));
        const float* ones = p.scale_dev;
        const float* sder = p.scale_dev + 2 * p.P;
        for (int s = 0; s < p.P; ++s) {
            CK(launch_gather(p, s, p.ks, N, 0, p.stage_d, N, 0, 1, ones, sder, st));
            CK(cudaEventRecord(p.win_events[s], st));
            CK(cudaStreamWaitEvent(p.copy_stream, p.win_events[s], 0));
            CK(cudaMemcpyAsync(dKdell + s * N, p.stage_d + s * N, sizeof(float) * N, cudaMemcpyDeviceToHost,
                               p.copy_stream));
        }
        window_sum(p, 1, (float)(p.sigma_f * p.sigma_f), p.stage_k, N, st);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(Kv, p.stage_k, sizeof(float) * N, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(p.copy_stream));
        CK(cudaStreamSynchronize(st));
        return ADDKER_OK;
    }
    const float* vm = static_cast<const float*>(mapped(v));
    float* Km = static_cast<float*>(mapped(Kv));
    float* Dm = dKdell ? static_cast<float*>(mapped(dKdell)) : nullptr;
    if (vm) CK(copy(vm, p.stage_v, need));
    else CK(cudaMemcpyAsync(p.stage_v, v, sizeof(float) * need, cudaMemcpyHostToDevice, st));
    CS(addker_matvec_all(plan, p.stage_v, p.stage_k, dKdell ? p.stage_d : nullptr, nrhs));
    if (Km) CK(copy(p.stage_k, Km, need));
    else CK(cudaMemcpyAsync(Kv, p.stage_k, sizeof(float) * need, cudaMemcpyDeviceToHost, st));
    if (dKdell) {
        if (Dm) CK(copy(p.stage_d, Dm, need * p.P));
        else CK(cudaMemcpyAsync(dKdell, p.stage_d, sizeof(float) * need * p.P, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    return ADDKER_OK;
}

int addker_sync(addker_plan* plan)
{
    if (!plan) return ADDKER_EINVAL;
    CK(cudaStreamSynchronize(plan->p.stream));
    CK(cudaGetLastError());
    return ADDKER_OK;
}

int addker_profile(addker_plan* plan, int enable)
{
    if (!plan) return ADDKER_EINVAL;
    Plan& p = plan->p;
    CK(cudaStreamSynchronize(p.stream));
    for (auto& u : p.ev_used) {
        p.ev_pool.push_back(u.second.first);
        p.ev_pool.push_back(u.second.second);
    }
    p.ev_used.clear();
    if (enable) for (int i = 0; i < 5; ++i) p.launches[i] = 0;
    p.prof = enable != 0;
    return ADDKER_OK;
}

int addker_profile_read(addker_plan* plan, double* ms, int64_t* launches, int cap)
{
    if (!plan || cap < 0) return ADDKER_EINVAL;
    Plan& p = plan->p;
    CK(cudaStreamSynchronize(p.stream));
    double acc[5] = {0, 0, 0, 0, 0};
    for (auto& u : p.ev_used) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, u.second.first, u.second.second));
        acc[u.first] += t;
    }
    for (int i = 0; i < cap && i < 5; ++i) {
        if (ms) ms[i] = acc[i];
        if (launches) launches[i] = p.launches[i];
    }
    return 5;
}

int addker_free(addker_plan* plan)
{
    if (!plan) return ADDKER_OK;
    cudaStreamSynchronize(plan->p.stream);
    for (auto& u : plan->p.ev_used) {
        cudaEventDestroy(u.second.first);
        cudaEventDestroy(u.second.second);
    }
    for (cudaEvent_t e : plan->p.ev_pool) cudaEventDestroy(e);
    release(plan->p);
    delete plan;
    return ADDKER_OK;
}

int addker_prescale(const float* X, int64_t N, int d, const int* win_off, const int* win_feat, int P, double eps_B,
                    float* Xs, double* factor, void* stream)
{
    if (!X || !Xs || !factor || N < 1 || d < 1 || P < 1 || !win_off || !win_feat || !(eps_B > 0.0 && eps_B < 0.5))
        return ADDKER_EINVAL;
    for (int s = 0; s < P; ++s) {
        if (win_off[s + 1] <= win_off[s]) return ADDKER_EINVAL;
        for (int q = win_off[s]; q < win_off[s + 1]; ++q) if (win_feat[q] < 0 || win_feat[q] >= d) return ADDKER_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* buf = nullptr;
    int nf = win_off[P];
    CK(cudaMalloc(&buf, sizeof(int) * (P + 1 + nf + 1)));
    unsigned* res = reinterpret_cast<unsigned*>(buf + P + 1 + nf);
    cudaMemcpyAsync(buf, win_off, sizeof(int) * (P + 1), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(buf + P + 1, win_feat, sizeof(int) * nf, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(res, 0, sizeof(unsigned), st);
    k_max_norm<<<grid_blocks(N, 256), 256, 0, st>>>(X, N, d, buf, buf + P + 1, P, res);
    unsigned bits = 0;
    cudaMemcpyAsync(&bits, res, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaFree(buf); return ADDKER_ECUDA; }
    float mx2;
    std::memcpy(&mx2, &bits, sizeof(float));
    if (!std::isfinite(mx2)) { cudaFree(buf); return ADDKER_EDOMAIN; }
    double f = mx2 > 0.f ? (0.25 - eps_B / 2.0) * (1.0 - 4e-7) / std::sqrt((double)mx2) : 1.0;
    k_scale<<<grid_blocks(N * d, 256), 256, 0, st>>>(X, N * d, (float)f, Xs);
    e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) return ADDKER_ECUDA;
    *factor = f;
    return ADDKER_OK;
}

int addker_prescale_cube(const float* X, int64_t N, int d, const int* win_off, const int* win_feat, int P,
                         double eps_B, float* Xs, double* factor, void* stream)
{
    if (!X || !Xs || !factor || N < 1 || d < 1 || d > 65535 || P < 1 || !win_off || !win_feat ||
        !(eps_B > 0.0 && eps_B < 0.5) || win_off[0] != 0)
        return ADDKER_EINVAL;
    int dmax = 0;
    for (int s = 0; s < P; ++s) {
        if (win_off[s + 1] <= win_off[s]) return ADDKER_EINVAL;
        for (int q = win_off[s]; q < win_off[s + 1]; ++q) if (win_feat[q] < 0 || win_feat[q] >= d) return ADDKER_EINVAL;
        dmax = std::max(dmax, win_off[s + 1] - win_off[s]);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* mm = nullptr;                                     // 2d range values, 2d affine coefficients, flag
    CK(cudaMalloc(&mm, sizeof(float) * (4 * (size_t)d + 1)));
    int* bad = reinterpret_cast<int*>(mm + 4 * (size_t)d);
    std::vector<float> h(2 * (size_t)d);
    for (int f = 0; f < d; ++f) {
        h[2 * f] = std::numeric_limits<float>::infinity();
        h[2 * f + 1] = -std::numeric_limits<float>::infinity();
    }
    int hbad = 0;
    cudaError_t e = cudaMemcpyAsync(mm, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        const int bx = (int)std::min<int64_t>(64, (N + 255) / 256);
        k_feature_range<<<dim3(bx, d), 256, 0, st>>>(X, N, d, mm, bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), mm, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(mm);
        return ADDKER_ECUDA;
    }
    if (hbad) {
        cudaFree(mm);
        return ADDKER_EDOMAIN;
    }
    // [min_f, max_f] -> [-r, r] per feature, then / sqrt(d_max); r = (1/4 - eps_B/2) shrunk by 4e-7 so that
    // FP32 rounding of the map cannot leave the ball
    const double r = (0.25 - eps_B / 2.0) * (1.0 - 4e-7);
    const double inv = 1.0 / std::sqrt((double)dmax);
    std::vector<float> coef(2 * (size_t)d);
    for (int f = 0; f < d; ++f) {
        const double lo = h[2 * f], hi = h[2 * f + 1];
        const double a = hi > lo ? 2.0 * r / (hi - lo) * inv : 0.0;
        coef[f] = (float)a;
        coef[d + f] = (float)(hi > lo ? -(lo + hi) / 2.0 * a : 0.0);
    }
    e = cudaMemcpyAsync(mm + 2 * (size_t)d, coef.data(), sizeof(float) * coef.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_affine_features<<<grid_blocks(N * d, 256), 256, 0, st>>>(X, N, d, mm + 2 * (size_t)d, mm + 3 * (size_t)d, Xs);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(mm);
    if (e != cudaSuccess) return ADDKER_ECUDA;
    *factor = 4.0 * r * inv;
    return ADDKER_OK;
}

int addker_info(const addker_plan* plan, int64_t* info, int cap)
{
    if (!plan) return ADDKER_EINVAL;
    const Plan& p = plan->p;
    std::vector<int64_t> v = {p.N, p.P, (int64_t)p.item_begin[kKinds - 1].back(), p.bytes};
    for (int s = 0; s < p.P; ++s) {
        v.push_back(p.win[s].D);
        v.push_back(p.win[s].M);
        v.push_back(p.win[s].n);
        v.push_back(p.n_cells[s]);
    }
    v.push_back(p.slots);
    v.push_back((int64_t)p.graph_cache.size());
    v.push_back(p.graph_replays);
    v.push_back(p.chunk);
    v.push_back(p.chunk_sp);
    v.push_back(p.sp_blocks);
    v.push_back(p.sp_tile);
    for (int i = 0; i < cap && i < (int)v.size(); ++i) info[i] = v[i];
    return (int)v.size();
}

int addker_debug_stage(addker_plan* plan, int window, int stage, const float* v, double* out, int64_t cap)
{
    if (!plan || !v || !out) return ADDKER_EINVAL;
    Plan& p = plan->p;
    if (window < 0 || window >= p.P || stage < 0 || stage > 1) return ADDKER_EINVAL;
    WinDev& w = p.win[window];
    int64_t full = 1, md = 1;
    for (int t = 0; t < w.D; ++t) { full *= w.n; md *= w.M; }
    if ((stage == 0 && cap < full) || (stage == 1 && cap < 2 * md)) return ADDKER_EINVAL;
    CS(ensure_slots(p, 1));
    cudaStream_t st = p.stream;
    int64_t gsz = (int64_t)w.box[0] * w.box[1] * w.box[2];
    CK(cudaMemsetAsync(w.grid, 0, sizeof(float) * gsz, st));
    CK(launch_spread(p, window, v, p.N, 1, st));                     // slot 0
    if (stage == 0) {
        std::vector<float> g(gsz);
        std::vector<double> g64(w.grid64 ? gsz : 0);
        if (w.grid64) {
            CK(cudaMemcpyAsync(g64.data(), w.grid64, sizeof(double) * gsz, cudaMemcpyDeviceToHost, st));
            CK(cudaMemsetAsync(w.grid64, 0, sizeof(double) * gsz, st));    // products expect a zeroed grid
        } else {
            CK(cudaMemcpyAsync(g.data(), w.grid, sizeof(float) * gsz, cudaMemcpyDeviceToHost, st));
            CK(cudaMemsetAsync(w.grid, 0, sizeof(float) * gsz, st));
        }
        CK(cudaStreamSynchronize(st));
        // the device window is w = phi * C with C = pi m / sinh(b m) (Kaiser-Bessel; 1 for the
        // exponential of semicircle, whose peak is 1); report in phi's normalisation
        double b = M_PI * (2.0 - 1.0 / p.sigma_os);
        double C = p.window == ADDKER_WIN_ES ? 1.0 : M_PI * w.m / std::sinh(b * w.m);
        double scale = std::pow(C, -w.D);
        std::fill(out, out + full, 0.0);
        for (int64_t i = 0; i < gsz; ++i) {
            int64_t i0 = i / ((int64_t)w.box[1] * w.box[2]), i1 = (i / w.box[2]) % w.box[1], i2 = i % w.box[2];
            int64_t a0 = w.lo[0] + i0, a1 = w.lo[1] + i1, a2 = w.lo[2] + i2;
            int64_t idx = a0;
            if (w.D >= 2) idx = idx * w.n + a1;
            if (w.D >= 3) idx = idx * w.n + a2;
            out[idx] = (w.grid64 ? g64[i] : (double)g[i]) * scale;
        }
        return ADDKER_OK;
    }
    CK(launch_transforms(p, window, 1, st, nullptr, true));
    CK(cudaMemsetAsync(w.grid, 0, sizeof(float) * gsz, st));        // d = 3: the inverse pass that clears it did not run
    if (w.grid64) CK(cudaMemsetAsync(w.grid64, 0, sizeof(double) * gsz, st));
    std::vector<float4> s(md);
    CK(cudaMemcpyAsync(s.data(), w.spec, sizeof(float4) * md, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < md; ++i) {
        out[2 * i] = s[i].x;
        out[2 * i + 1] = s[i].y;
    }
    return ADDKER_OK;
}

}  // extern "C"
