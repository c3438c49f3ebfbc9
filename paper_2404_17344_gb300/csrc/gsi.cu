// Global sensitivity indices of the fast-summation polynomial (include/addker.h: addker_gsi).
//
// Sec. 4, Algorithm "Computation of GSI": per window s, the adjoint NFFT S(k, W_s) of v (step 2(a)) —
// here the plan's own spread and forward transform, S_k = G_k dconv_k, all windows in one launch per
// stage — then for every non-empty subset of the window's features the sum of |c_hat_k S_k|^2 over the
// frequencies whose non-zero coordinates are exactly that subset (step 2(b)); the host adds the
// windows' contributions per feature subset, the total variance (step 3) and the ratios (step 4).
// Windows of length 1..3 with their own length scales use their own coefficients.
#include <algorithm>
#include <map>
#include <vector>

#include "common.cuh"

namespace addker {

namespace {

constexpr int kT = 256;

// theta[b] += sum over k with non-zero pattern b of c_hat_k^2 |S_k|^2 (b = bit t set iff k_t != 0)
template <int D>
__global__ void __launch_bounds__(kT) k_gsi_reduce(const WinDev* __restrict__ wins, int s, double* __restrict__ theta)
{
    constexpr int NB = 1 << D;
    const WinDev& W = wins[s];
    const int M = W.M;
    int64_t total = M;
    if (D >= 2) total *= M;
    if (D >= 3) total *= M;
    double acc[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[b] = 0.0;
    for (int64_t o = blockIdx.x * (int64_t)kT + threadIdx.x; o < total; o += (int64_t)gridDim.x * kT) {
        int64_t rem = o;
        int pat = 0;
#pragma unroll
        for (int t = D - 1; t >= 0; --t) {
            const int kk = (int)(rem % M) - M / 2;
            rem /= M;
            pat |= (kk != 0) << t;
        }
        const float4 S = W.spec[o];
        const double c = (double)W.chat[o];
        const double e = c * c * ((double)S.x * S.x + (double)S.y * S.y);
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[b] += b == pat ? e : 0.0;
    }
#pragma unroll
    for (int b = 1; b < NB; ++b) {
        double x = acc[b];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(theta + (size_t)s * 8 + b, x);
    }
}

}  // namespace

int gsi_run(Plan& p, const float* v, int cap, int* feats, double* rho, double* total_out)
{
    cudaStream_t st = p.stream;
    double* theta = nullptr;
    if (cudaMalloc(&theta, sizeof(double) * 8 * p.P) != cudaSuccess) {
        cudaGetLastError();
        return ADDKER_ENOMEM;
    }
    std::vector<double> h(8 * (size_t)p.P);
    cudaError_t e = cudaMemsetAsync(theta, 0, sizeof(double) * 8 * p.P, st);
    if (e == cudaSuccess) e = launch_spread(p, -1, v, p.N, 1, st);                 // slot 0
    if (e == cudaSuccess) e = launch_transforms(p, -1, 1, st, nullptr, true);       // spec = S_k per window
    for (int s = 0; s < p.P && e == cudaSuccess; ++s) {
        const WinDev& w = p.win[s];
        // the spectrum-only pass skips the inverse that clears d = 3 grids
        if (w.D == 3 && w.grid64) e = cudaMemsetAsync(w.grid64, 0, sizeof(double) * (size_t)w.gsz, st);
        else if (w.D == 3) e = cudaMemsetAsync(w.grid, 0, sizeof(float) * (size_t)w.gsz, st);
        int64_t tot = 1;
        for (int t = 0; t < w.D; ++t) tot *= w.M;
        const int nb = (int)std::min<int64_t>(1024, (tot + kT - 1) / kT);
        if (w.D == 1) k_gsi_reduce<1><<<nb, kT, 0, st>>>(p.wins_dev, s, theta);
        else if (w.D == 2) k_gsi_reduce<2><<<nb, kT, 0, st>>>(p.wins_dev, s, theta);
        else k_gsi_reduce<3><<<nb, kT, 0, st>>>(p.wins_dev, s, theta);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), theta, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(theta);
    if (e != cudaSuccess) return ADDKER_ECUDA;
    // per feature subset (sorted feature indices), summed over the windows that contain it
    std::map<std::vector<int>, double> by_subset;
    for (int s = 0; s < p.P; ++s) {
        const WinDev& w = p.win[s];
        for (int b = 1; b < (1 << w.D); ++b) {
            std::vector<int> u;
            for (int t = 0; t < w.D; ++t)
                if (b >> t & 1) u.push_back(w.feat[t]);
            std::sort(u.begin(), u.end());
            by_subset[u] += h[(size_t)s * 8 + b];
        }
    }
    double total = 0.0;
    for (const auto& kv : by_subset) total += kv.second;
    std::vector<std::pair<double, std::vector<int>>> out;
    for (const auto& kv : by_subset) out.push_back({kv.second, kv.first});
    std::stable_sort(out.begin(), out.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    for (int i = 0; i < cap && i < (int)out.size(); ++i) {
        if (rho) rho[i] = total > 0.0 ? out[i].first / total : 0.0;
        if (feats)
            for (int t = 0; t < 3; ++t) feats[3 * i + t] = t < (int)out[i].second.size() ? out[i].second[t] : -1;
    }
    if (total_out) *total_out = total;
    return (int)out.size();
}

}  // namespace addker
