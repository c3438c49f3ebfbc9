// Device rates that bound the product's kernels (include/addker_rates.h: addker_device_rates), built into
// its own library, libaddker_rates.so, apart from the product's.
//
// The spread and the gather of 3-D windows are bound by the FP32 FMA pipe and by how fast the
// register tiles reach the grid (global atomic adds into an L2-resident grid); shared-memory atomics
// are the alternative accumulation a shared-memory spread would use. Each rate is measured with
// a kernel that does nothing else, long enough (tens of milliseconds) for the clock to settle:
//   FFMA   8 independent FMA chains per thread, 2048 threads per SM;
//   FFMA2  the same with packed two-wide FMAs (the form the product's inner loops use);
//   shared atomics: every thread adds into its own shared word (distinct banks within a warp);
//   global atomic adds: warps add rows of 32 consecutive floats (or doubles) into a 1 MiB (2 MiB)
//          grid (L2-resident), the access shape of a tile flush.
// The SM clock under load comes from clock64() against the global timer inside the FFMA kernel.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "../../include/addker_rates.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kRateThreads = 512;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// clk[2 * block] = SM cycles, clk[2 * block + 1] = nanoseconds between the block's first and last
// instruction (thread 0)
__global__ void __launch_bounds__(kRateThreads) k_rate_ffma(float* out, long long* clk, int iters, float a, float b)
{
    long long c0 = 0;
    unsigned long long t0 = 0;
    if (threadIdx.x == 0) {
        c0 = clock64();
        t0 = global_ns();
    }
    float acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = 1e-3f * (float)threadIdx.x + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) acc[i] = fmaf(acc[i], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += acc[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) {
        clk[2 * blockIdx.x] = clock64() - c0;
        clk[2 * blockIdx.x + 1] = (long long)(global_ns() - t0);
    }
}

__global__ void __launch_bounds__(kRateThreads) k_rate_ffma2(float* out, int iters, float a, float b)
{
    float2 acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = make_float2(1e-3f * (float)threadIdx.x + (float)i, (float)i);
    const float2 A = make_float2(a, a), B = make_float2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) acc[i] = __ffma2_rn(acc[i], A, B);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += acc[i].x + acc[i].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kRateThreads) k_rate_shared_atomic(float* out, int iters)
{
    __shared__ float s[kRateThreads];
    s[threadIdx.x] = 0.f;
    __syncthreads();
    float* p = s + threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) atomicAdd(p, 1.0f);
    }
    __syncthreads();
    out[blockIdx.x * blockDim.x + threadIdx.x] = s[threadIdx.x];
}

// grid of 2^18 floats; warp w of the launch adds 1 to row (w * 97 + it * 31) mod 2^13 (32 floats each)
__global__ void __launch_bounds__(kRateThreads) k_rate_global_atomic(float* grid, int iters)
{
    const int lane = threadIdx.x & 31;
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const unsigned row = (warp * 97u + (unsigned)(it * kUnroll + u) * 31u) & ((1u << 13) - 1u);
            atomicAdd(grid + row * 32u + lane, 1.0f);
        }
    }
}

// the same access shape with double atomic adds (an FP64 grid accumulates without rounding error in
// practice); grid of 2^18 doubles
__global__ void __launch_bounds__(kRateThreads) k_rate_global_atomic64(double* grid, int iters)
{
    const int lane = threadIdx.x & 31;
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const unsigned row = (warp * 97u + (unsigned)(it * kUnroll + u) * 31u) & ((1u << 13) - 1u);
            atomicAdd(grid + row * 32u + lane, 1.0);
        }
    }
}

struct Buf {
    void* p = nullptr;
    ~Buf() { cudaFree(p); }
};

}  // namespace

extern "C" int addker_device_rates(double* out, int cap)
{
    if (!out || cap < 0) return ADDKER_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return ADDKER_ECUDA;
    }
    const int blocks = nsm * 4;                      // 2048 threads per SM
    const int64_t threads = (int64_t)blocks * kRateThreads;
    Buf o, c, g;
    if (cudaMalloc(&o.p, sizeof(float) * threads) != cudaSuccess || cudaMalloc(&c.p, sizeof(long long) * 2 * blocks) != cudaSuccess ||
        cudaMalloc(&g.p, sizeof(double) << 18) != cudaSuccess) {
        cudaGetLastError();
        return ADDKER_ENOMEM;
    }
    float* of = static_cast<float*>(o.p);
    long long* ck = static_cast<long long*>(c.p);
    float* gf = static_cast<float*>(g.p);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (st) cudaStreamDestroy(st);
        if (e0) cudaEventDestroy(e0);
        return ADDKER_ECUDA;
    }
    cudaError_t err = cudaMemsetAsync(gf, 0, sizeof(double) << 18, st);
    // the median of 3 timed launches after one warm-up launch, in ms
    auto timed = [&](auto launch) -> double {
        std::vector<double> ms;
        for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
            err = cudaEventRecord(e0, st);
            launch();
            if (err == cudaSuccess) err = cudaGetLastError();
            if (err == cudaSuccess) err = cudaEventRecord(e1, st);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float t = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms.push_back(t);
        }
        if (err != cudaSuccess) return 0.0;
        std::sort(ms.begin(), ms.end());
        return ms[ms.size() / 2];
    };
    const int it_fma = 16384, it_atom = 8192, it_red = 256;
    const float a = 0.9999999f, b = 1e-7f;
    const double t_fma = timed([&] { k_rate_ffma<<<blocks, kRateThreads, 0, st>>>(of, ck, it_fma, a, b); });
    std::vector<long long> hc(2 * (size_t)blocks);
    if (err == cudaSuccess) err = cudaMemcpy(hc.data(), ck, sizeof(long long) * hc.size(), cudaMemcpyDeviceToHost);
    const double t_fma2 = timed([&] { k_rate_ffma2<<<blocks, kRateThreads, 0, st>>>(of, it_fma, a, b); });
    const double t_sat = timed([&] { k_rate_shared_atomic<<<blocks, kRateThreads, 0, st>>>(of, it_atom); });
    const double t_red = timed([&] { k_rate_global_atomic<<<blocks, kRateThreads, 0, st>>>(gf, it_red); });
    if (err == cudaSuccess) err = cudaMemsetAsync(gf, 0, sizeof(double) << 18, st);
    const double t_red64 =
        timed([&] { k_rate_global_atomic64<<<blocks, kRateThreads, 0, st>>>(reinterpret_cast<double*>(gf), it_red); });
    cudaStreamDestroy(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return ADDKER_ECUDA;
    }
    std::vector<double> mhz;
    for (int i = 0; i < blocks; ++i)
        if (hc[2 * i + 1] > 0) mhz.push_back(1e3 * (double)hc[2 * i] / (double)hc[2 * i + 1]);
    std::sort(mhz.begin(), mhz.end());
    const double fmas = (double)threads * it_fma * kUnroll * kChains;
    const double vals[8] = {
        (double)nsm,
        mhz.empty() ? 0.0 : mhz[mhz.size() / 2],
        2.0 * fmas / (t_fma * 1e-3) / 1e12,               // FFMA TFLOP/s
        4.0 * fmas / (t_fma2 * 1e-3) / 1e12,              // FFMA2 TFLOP/s (two FMAs per instruction)
        (double)threads * it_atom * kUnroll / (t_sat * 1e-3) / 1e9,   // shared atomics, G/s
        (double)threads * it_red * kUnroll / (t_red * 1e-3) / 1e9,    // global atomic adds, G/s
        t_fma,
        (double)threads * it_red * kUnroll / (t_red64 * 1e-3) / 1e9,  // global double atomic adds, G/s
    };
    for (int i = 0; i < cap && i < 8; ++i) out[i] = vals[i];
    return 8;
}
