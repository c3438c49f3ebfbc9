// Spreading (adjoint NFFT, first step) and interpolation (NFFT, last step) kernels.
//
//   spread:  g_l   = sum_j v_j prod_t w(n x_{j,t} - l_t),   l in the support of x_j
//   gather:  f_i   = sum_l h_l prod_t w(n x_{i,t} - l_t)     for the two grids h^K and h^der
// (Sec. 3.1, eq. "approx fast sum": the inner sums by an adjoint NFFT, the outer sums by an
// NFFT). w is the plan's window normalised to peak 1 (Kaiser-Bessel or exponential of semicircle),
// evaluated through its piecewise polynomial form (WinPoly); the support of x along an axis is
// floor(n x) - m + 1 .. floor(n x) + m.
//
// Points are sorted by grid cell, so all points of a work item share one support box of
// (2m)^D grid points. The fast kernels (D = 3, m = 4) exploit that:
//   spread: a warp accumulates the item's 8x8x8 box in registers as a sum of outer products
//           (v_j w_x) (x) w_y (x) w_z; lane (ah, bh, c) owns the 4x4 block a in 4ah..4ah+3,
//           b in 4bh..4bh+3 at z-offset c, so each point costs a lane 4 shared loads, 2 packed
//           products and 8 packed FMAs; the box is added to the grid once per item;
//   gather: a warp stages the item's box of both grids in shared memory (float2 (h^K, h^der)) and
//           every lane contracts it with two points at once, the grid pair in one packed FMA, so
//           one 16-byte broadcast load feeds 8 FMAs in 4 instructions.
#include <map>
#include <mutex>

#include "common.cuh"

namespace addker {

namespace {

constexpr int kWarps = 4;                 // warps per block in the item kernels (8: 2% slower)

// ----------------------------------------------------------------------------------
// Packed FP32 pairs (one instruction, two FMAs): the fast kernels keep their accumulators in
// float2 pairs and use __ffma2_rn.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Running totals of the quadratic split's moments in the persistent spreads: a warp's consecutive units
// mostly share (window, right-hand side), so their warp-summed FP32 moments are added into lane c's FP64
// register (c < 5) and reach global memory only when that pair changes and when the warp finishes. One
// flush per unit put five FP64 atomics per unit on the same few addresses, whose queue slowed the grid's
// own atomic adds in the same L2 slices.
struct MomAcc {
    double a;
    int key;                              // window * kMaxRhsChunk + rhs of the running total, or -1
};
__device__ __forceinline__ void mom_flush(const MomAcc& acc, const WinDev* __restrict__ wins, int lane)
{
    if (acc.key >= 0 && lane < 5) {
        const WinDev& W = wins[acc.key / kMaxRhsChunk];
        atomicAdd(W.mom + (acc.key % kMaxRhsChunk) * W.mstride + lane, acc.a);
    }
}
// End of a unit of split window w, right-hand side r: fold the lanes' moments mm into the running total.
__device__ __forceinline__ void mom_unit_end(MomAcc& acc, float* mm, const WinDev* __restrict__ wins, int w, int r,
                                             int lane)
{
    float t = 0.f;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        float x = mm[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == c) t = x;
        mm[c] = 0.f;
    }
    const int key = w * kMaxRhsChunk + r;
    if (key != acc.key) {
        mom_flush(acc, wins, lane);
        acc.key = key;
        acc.a = 0.0;
    }
    acc.a += (double)t;
}

// The 3-D spread's register tile (m = 4, W = 8): each lane of half-warp hw holds 32 values of the item's
// 8x8x8 box, acc[16] float2, summed over the staged points its half takes (alternate points). Two shapes:
//   TILE 0: a in 4ah..4ah+3, b in 4bh..4bh+3, c in {2cq, 2cq+1}: acc[(2a' + p) 2 + i] =
//           (g[4ah+a'][4bh+2p][2cq+i], g[4ah+a'][4bh+2p+1][2cq+i]); per point 3 shared loads (40 B),
//           4 packed products y (x) z and 16 packed FMAs;
//   TILE 1: a in 0..7, b in {2bp, 2bp+1}, c in {2cq, 2cq+1}: acc[2a + i] = (g[a][2bp][2cq+i], g[a][2bp+1][2cq+i]);
//           per point 4 shared loads (48 B), 2 packed products and 16 packed FMAs.
// The duplicated operands the packed FMAs need are formed in registers. Staged rows: x v [8] | y [8] | z [8].
template <int TILE>
__device__ __forceinline__ void spread3_points(float2 (&acc)[16], const float* ws, int stride, int cnt, int lane)
{
    const int hw = lane >> 4, cq = lane & 3;
    const float* src = ws + hw * stride;
    if (TILE == 0) {
        const int ah = (lane >> 3) & 1, bh = (lane >> 2) & 1;
#pragma unroll 2
        for (int j = 0; j < cnt; j += 2, src += 2 * stride) {
            const float4 xa = *reinterpret_cast<const float4*>(src + 4 * ah);         // a = 4ah .. 4ah+3
            const float4 yb = *reinterpret_cast<const float4*>(src + 8 + 4 * bh);     // b = 4bh .. 4bh+3
            const float2 zc = *reinterpret_cast<const float2*>(src + 16 + 2 * cq);    // c = 2cq, 2cq+1
            const float2 Y[2] = {f2(yb.x, yb.y), f2(yb.z, yb.w)};
            const float2 Z[2] = {f2(zc.x, zc.x), f2(zc.y, zc.y)};
            const float2 X[4] = {f2(xa.x, xa.x), f2(xa.y, xa.y), f2(xa.z, xa.z), f2(xa.w, xa.w)};
            float2 B[2][2];
#pragma unroll
            for (int q = 0; q < 4; ++q) B[q >> 1][q & 1] = __fmul2_rn(Y[q >> 1], Z[q & 1]);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[a * 4 + q] = __ffma2_rn(X[a], B[q >> 1][q & 1], acc[a * 4 + q]);
        }
    } else {
        const int bp = (lane >> 2) & 3;
#pragma unroll 2
        for (int j = 0; j < cnt; j += 2, src += 2 * stride) {
            const float4 x0 = *reinterpret_cast<const float4*>(src);                  // a = 0 .. 3
            const float4 x1 = *reinterpret_cast<const float4*>(src + 4);              // a = 4 .. 7
            const float2 yb = *reinterpret_cast<const float2*>(src + 8 + 2 * bp);     // b = 2bp, 2bp+1
            const float2 zc = *reinterpret_cast<const float2*>(src + 16 + 2 * cq);    // c = 2cq, 2cq+1
            const float2 B[2] = {__fmul2_rn(yb, f2(zc.x, zc.x)), __fmul2_rn(yb, f2(zc.y, zc.y))};
            const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const float2 X = f2(xs[a], xs[a]);
                acc[2 * a] = __ffma2_rn(X, B[0], acc[2 * a]);
                acc[2 * a + 1] = __ffma2_rn(X, B[1], acc[2 * a + 1]);
            }
        }
    }
}

// Sum the two halves' tiles (half hw keeps the values with c = 2cq + hw and receives its partner's) and add
// the 16 kept values per lane to the grid of window P, right-hand side r, for the item's cell.
template <int TILE>
__device__ __forceinline__ void spread3_flush(float2 (&acc)[16], const WinDev* P, const int4 it, int r, int lane)
{
    const int hw = lane >> 4, cq = lane & 3;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float2 send = hw ? acc[2 * k] : acc[2 * k + 1];
        float2 keep = hw ? acc[2 * k + 1] : acc[2 * k];
        keep.x += __shfl_xor_sync(0xffffffffu, send.x, 16);
        keep.y += __shfl_xor_sync(0xffffffffu, send.y, 16);
        acc[2 * k] = keep;
    }
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff, cz = (it.z >> 16) & 0xff;
    const int ox = cx - 3 - P->lo[0], oy = cy - 3 - P->lo[1], oz = cz - 3 - P->lo[2];
    const int sy = P->box[2], sx = P->box[1] * P->box[2];
    const int a0 = TILE == 0 ? 4 * ((lane >> 3) & 1) : 0;
    const int b0 = TILE == 0 ? 4 * ((lane >> 2) & 1) : 2 * ((lane >> 2) & 3);
    const size_t o0 = r * P->gsz + (size_t)(ox + a0) * sx + (size_t)(oy + b0) * sy + oz + 2 * cq + hw;
    float* g = P->grid + o0;
    double* ge = P->grid64 ? P->grid64 + o0 : nullptr;
    // k-th kept pair: TILE 0 (a = k / 2, b = 2 (k % 2) + {0, 1}); TILE 1 (a = k, b = {0, 1})
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const size_t o = TILE == 0 ? (size_t)(k >> 1) * sx + (size_t)(2 * (k & 1)) * sy : (size_t)k * sx;
        grid_add(g + o, ge ? ge + o : nullptr, acc[2 * k].x);
        grid_add(g + o + sy, ge ? ge + o + sy : nullptr, acc[2 * k].y);
    }
}

// fast 3-D spread, m = 4 (W = 8)
// Staged per point (STRIDE floats): x_a v [8] | y [8] | z [8]. The two half-warps take alternate
// staged points (hw = lane >> 4). Within a half-warp, lane (ah, bh, cq) accumulates
// acc[a][p][i] = (g[4ah+a][4bh+2p][2cq+i], g[4ah+a][4bh+2p+1][2cq+i]): the whole box per half-warp,
// 32 values per lane, so each point costs a lane 3 shared loads (16 + 16 + 8 bytes), 4 packed
// products and 16 packed FMAs; the duplicated operands (x_a, x_a) and (z_c, z_c) the packed FMAs need
// are formed in registers, which keeps the shared-memory traffic (the loop's tighter limit) at 40
// bytes per lane and point. The two halves are summed once per item, before the atomic adds.
//
// Persistent: each warp takes work units (item, right-hand side) from a global counter, one unit
// ahead, and loads the first batch of the next unit while it finishes the current one, so neither
// the chain item -> points -> v at the start of an item nor the drain of the atomic adds at its end
// stalls the warp. Unit u is item u % nitems of right-hand side u / nitems.
template <int TILE>
__global__ void __launch_bounds__(kWarps * 32, 4) k_spread3_w8(const int4* __restrict__ items, int nitems,
                                                              int nunits, int* __restrict__ counter,
                                                              const WinDev* __restrict__ wins,
                                                              const float* __restrict__ v, int64_t ldv,
                                                              const WinPoly poly)
{
    constexpr int W = 8;
    constexpr int STRIDE = 28;            // 8 + 8 + 8 floats, padded so staging stores avoid conflicts
    __shared__ __align__(16) float sw[kWarps][32 * STRIDE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* ws = sw[warp];

    int u = 0;
    if (lane == 0) u = atomicAdd(counter, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= nunits) return;
    int un = 0;
    if (lane == 0) un = atomicAdd(counter, 1);
    un = __shfl_sync(0xffffffffu, un, 0);
    int4 it = items[u % nitems];
    int r = u / nitems;
    int4 itn = un < nunits ? items[un % nitems] : make_int4(0, 0, 0, 0);
    const WinDev* P = wins + it.w;
    const float4* __restrict__ pts = P->pts + it.x;
    const float* __restrict__ vr = v + r * ldv;
    // software pipeline: the next batch's point (and then its v) is in flight during this batch
    float4 pn = make_float4(0.f, 0.f, 0.f, 0.f);
    float vn = 0.f;
    if (lane < it.y) {
        pn = pts[lane];
        vn = __ldg(vr + __float_as_int(pn.w));
    }
    float mm[5] = {0.f, 0.f, 0.f, 0.f, 0.f};      // moments of the quadratic split over this unit
    MomAcc macc = {0.0, -1};
    while (true) {
        float2 acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = f2(0.f, 0.f);
        const int count = it.y;
        const int n = P->n;
        const bool more = un < nunits;
        const bool split = P->pq != 0.f;
        for (int base = 0; base < count; base += 32) {
            const float4 p = pn;
            const float vv = vn;
            const bool valid = base + lane < count;
            const bool last = base + 32 >= count;
            // prefetch: the next batch of this item, or the first batch of the next unit
            const float4* __restrict__ npts = last ? wins[itn.w].pts + itn.x : pts + base + 32;
            const int ncount = last ? (more ? itn.y : 0) : count - base - 32;
            if (lane < ncount) pn = npts[lane];
            float wx[W], wy[W], wz[W];
            int cx, cy, cz;
            if (valid) {
                window_weights<W>(poly, p.x, n, wx, &cx);
                window_weights<W>(poly, p.y, n, wy, &cy);
                window_weights<W>(poly, p.z, n, wz, &cz);
#pragma unroll
                for (int q = 0; q < W; ++q) wx[q] *= vv;
                if (split) moments_add<3>(mm, p.x, p.y, p.z, vv);
            } else {
#pragma unroll
                for (int q = 0; q < W; ++q) { wx[q] = 0.f; wy[q] = 0.f; wz[q] = 0.f; }
            }
            if (lane < ncount) vn = __ldg((last ? v + (un / nitems) * ldv : vr) + __float_as_int(pn.w));
            float4* dst = reinterpret_cast<float4*>(ws + lane * STRIDE);
            dst[0] = make_float4(wx[0], wx[1], wx[2], wx[3]);
            dst[1] = make_float4(wx[4], wx[5], wx[6], wx[7]);
            dst[2] = make_float4(wy[0], wy[1], wy[2], wy[3]);
            dst[3] = make_float4(wy[4], wy[5], wy[6], wy[7]);
            dst[4] = make_float4(wz[0], wz[1], wz[2], wz[3]);
            dst[5] = make_float4(wz[4], wz[5], wz[6], wz[7]);
            __syncwarp();
            // rows cnt .. 31 hold zeros (lanes without a point stage zero weights), so an odd count is safe
            const int cnt = min(32, count - base);
            spread3_points<TILE>(acc, ws, STRIDE, cnt, lane);
            __syncwarp();
        }
        spread3_flush<TILE>(acc, P, it, r, lane);
        if (split) mom_unit_end(macc, mm, wins, it.w, r, lane);
        if (!more) break;
        // advance: the prefetched unit becomes current; take the one after it
        it = itn;
        r = un / nitems;
        P = wins + it.w;
        pts = P->pts + it.x;
        vr = v + r * ldv;
        if (lane == 0) un = atomicAdd(counter, 1);
        un = __shfl_sync(0xffffffffu, un, 0);
        itn = un < nunits ? items[un % nitems] : make_int4(0, 0, 0, 0);
    }
    mom_flush(macc, wins, lane);
}

// Contraction of the staged box t4 with NP points per lane, p[i] written out where has[i]. The pair
// (h^K, h^D) of a grid point is multiplied by duplicated weights in one packed FMA.
template <int NP, bool WK, bool WD>
__device__ __forceinline__ void gather_points(const float4* t4, const float4 (&p)[2], const bool (&has)[2], int n,
                                              const WinPoly& poly, float* __restrict__ outK,
                                              float* __restrict__ outD, float sK, float sD, int64_t offK,
                                              int64_t offD, const Quad& Q)
{
    constexpr int W = 8;
    float x[NP][W];
    float2 y[NP][W], z[NP][W];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        float a[W], b[W];
        int c;
        window_weights<W>(poly, p[i].x, n, x[i], &c);
        window_weights<W>(poly, p[i].y, n, a, &c);
        window_weights<W>(poly, p[i].z, n, b, &c);
#pragma unroll
        for (int q = 0; q < W; ++q) { y[i][q] = f2(a[q], a[q]); z[i][q] = f2(b[q], b[q]); }
    }
    // (K, der) per point; the derivative's quadratic part (quadratic split, zero otherwise) starts its sum, so
    // the moments' coefficients are not live through the contraction
    float2 f[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) f[i] = f2(0.f, WD ? quad_eval<3>(Q, p[i].x, p[i].y, p[i].z) : 0.f);
#pragma unroll 1
    for (int a = 0; a < W; ++a) {
        float2 u[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) u[i] = f2(0.f, 0.f);
        const float4* row = t4 + a * 32;
#pragma unroll
        for (int bb = 0; bb < W; ++bb) {
            float2 s[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) s[i] = f2(0.f, 0.f);
#pragma unroll
            for (int cc = 0; cc < W; cc += 2) {
                const float4 hv = row[(bb * 8 + cc) >> 1];
                const float2 hc = f2(hv.x, hv.y), hd = f2(hv.z, hv.w);
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    s[i] = __ffma2_rn(hc, z[i][cc], s[i]);
                    s[i] = __ffma2_rn(hd, z[i][cc + 1], s[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < NP; ++i) u[i] = __ffma2_rn(s[i], y[i][bb], u[i]);
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            f[i] = __ffma2_rn(u[i], f2(x[i][0], x[i][0]), f[i]);
            // rotate so that x[i][0] holds the weight of the next a (keeps indices static)
#pragma unroll
            for (int q = 0; q < W - 1; ++q) x[i][q] = x[i][q + 1];
        }
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        if (!has[i]) continue;
        const int64_t idx = (int64_t)__float_as_int(p[i].w);
        if (WK) outK[idx + offK] = sK * f[i].x;
        if (WD) outD[idx + offD] = sD * f[i].y;
    }
}

// ----------------------------------------------------------------------------------
// fast 3-D gather, m = 4 (W = 8): lanes own points (two each); the item's box of both grids is
// staged in shared memory as float2 (h^K, h^D) and read back as float4 (two such pairs). The pair
// (h^K, h^D) is contracted with duplicated weights in one packed FMA, so each 16-byte broadcast load
// feeds 4 packed FMAs (8 FMAs) for the lane's two points.
// The gather arguments every item routine takes: outputs (window s and right-hand side r of point i
// at out[i + s*stride + r*rstride]), per-window scales, and the window polynomials.
struct GatherArgs {
    float* outK;
    float* outD;
    const float* scaleK;
    const float* scaleD;
    int64_t strideK, strideD, rstrideK, rstrideD;
};

// One 3-D item (m = 4) by one warp; t is the warp's 512-entry tile.
template <bool WK, bool WD>
__device__ __forceinline__ void gather3_item(const int4 it, const WinDev& P, float2* t, int lane, int r,
                                             const GatherArgs& g, const WinPoly& poly)
{
    float* __restrict__ outK = g.outK;
    float* __restrict__ outD = g.outD;
    const int64_t strideK = g.strideK, strideD = g.strideD, rstrideK = g.rstrideK, rstrideD = g.rstrideD;
    const float* __restrict__ scaleK = g.scaleK;
    const float* __restrict__ scaleD = g.scaleD;
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff, cz = (it.z >> 16) & 0xff;
    const int ox = cx - 3 - P.lo[0], oy = cy - 3 - P.lo[1], oz = cz - 3 - P.lo[2];
    const int sy = P.box[2], sx = P.box[1] * P.box[2];
    const float2* __restrict__ h = P.h + r * P.gsz + (size_t)ox * sx + (size_t)oy * sy + oz;
    const float4* __restrict__ pts = P.pts + it.x;
    const int count = it.y;
    // the first round's points load while the box is staged; each round loads the next round's
    float4 pa[2];
    pa[0] = pts[min(lane, count - 1)];
    pa[1] = pts[min(lane + 32, count - 1)];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int idx = lane + 32 * i;
        const int a = idx >> 6, bb = (idx >> 3) & 7, cc = idx & 7;
        t[idx] = h[(size_t)a * sx + (size_t)bb * sy + cc];
    }
    __syncwarp();
    const float4* t4 = reinterpret_cast<const float4*>(t);
    const float sK = WK ? scaleK[it.w] : 0.f;
    const float sD = WD ? scaleD[it.w] : 0.f;
    const Quad Q = WD ? quad_of(P, r) : Quad{0.f, 0.f, 0.f, 0.f, 0.f};
    const int n = P.n;
    // two points per lane while more than 32 remain, then one, so tail lanes do no dead work
    const int64_t offK = it.w * strideK + r * rstrideK, offD = it.w * strideD + r * rstrideD;
    for (int base = 0; base < count;) {
        const int np = count - base > 32 ? 2 : 1;
        const float4 pc[2] = {pa[0], pa[1]};
        const bool has[2] = {base + lane < count, np == 2 && base + 32 + lane < count};
        const int nb = base + 32 * np;
        if (nb < count) {
            pa[0] = pts[min(nb + lane, count - 1)];
            pa[1] = pts[min(nb + 32 + lane, count - 1)];
        }
        if (np == 2) gather_points<2, WK, WD>(t4, pc, has, n, poly, outK, outD, sK, sD, offK, offD, Q);
        else if (has[0]) gather_points<1, WK, WD>(t4, pc, has, n, poly, outK, outD, sK, sD, offK, offD, Q);
        base = nb;
    }
}

template <bool WK, bool WD>
__global__ void __launch_bounds__(kWarps * 32, 4) k_gather3_w8(const int4* __restrict__ items, int nitems,
                                                              const WinDev* __restrict__ wins, GatherArgs g,
                                                              const WinPoly poly)
{
    __shared__ __align__(16) float2 tile[kWarps][512];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * kWarps + warp;
    if (item >= nitems) return;
    const int4 it = items[item];
    gather3_item<WK, WD>(it, wins[it.w], tile[warp], lane, blockIdx.y, g, poly);
}

// ----------------------------------------------------------------------------------
// fast 1-D and 2-D kernels, m = 4 (W = 8): one warp per work item, lanes own points. The spread
// accumulates the item's whole support box (8 or 8x8 values) in each lane's registers and reduces it
// across the warp once per item (a transpose-reduction: each halving step trades half of a lane's
// values with its partner), so no atomics touch a grid value more than once per item.

// Sum each of the NV entries v[0..NV) over the 32 lanes of the warp (NV a power of two <= 64) by
// recursive halving: at offset off a lane swaps half of its current entries with lane ^ off, keeping the
// lower half if bit off is clear and the upper half otherwise. Afterwards v[0..held) are complete totals of
// entries base .. base + held - 1, with held = max(1, NV / 32); for NV < 32 each entry is held by
// 32 / NV lanes (those equal in the bits used for halving).
template <int NV>
__device__ __forceinline__ void warp_transpose_reduce(float* v, int lane, int* base_out, int* held_out)
{
    int held = NV;
    int base = 0;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        if (held == 1) {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
            continue;
        }
        const int half = held / 2;
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < NV / 2; ++i) {
            if (i < half) {
                const float send = upper ? v[i] : v[i + half];
                const float keep = upper ? v[i + half] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
            }
        }
        if (upper) base += half;
        held = half;
    }
    *base_out = base;
    *held_out = held;
}

// One 1-D or 2-D spread item (m = 4) by one warp: rhs r reads v (already offset to that rhs).
template <int D>
__device__ __forceinline__ void spread_lowd_item(const int4 it, const WinDev& P, const float* __restrict__ v, int r,
                                                 int lane, const WinPoly& poly)
{
    constexpr int W = 8;
    constexpr int NV = D == 1 ? W : W * W;
    const float4* __restrict__ pts = P.pts + it.x;
    float acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.f;
    float mm[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    // U points per lane per round, their loads issued together (the work per point is small, so one
    // point at a time would leave the loop waiting on memory); points past the item weigh 0
    constexpr int U = 4;
    for (int k0 = lane; k0 < it.y; k0 += 32 * U) {
        float4 p[U];
        float vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) p[u] = pts[min(k0 + 32 * u, it.y - 1)];
#pragma unroll
        for (int u = 0; u < U; ++u) vv[u] = k0 + 32 * u < it.y ? __ldg(v + __float_as_int(p[u].w)) : 0.f;
        // one point at a time (the arrays rotate so that indices stay static and in registers)
#pragma unroll 1
        for (int u = 0; u < U; ++u) {
            const float4 pu = p[0];
            const float vu = vv[0];
#pragma unroll
            for (int z = 0; z < U - 1; ++z) { p[z] = p[z + 1]; vv[z] = vv[z + 1]; }
            float wx[W];
            int c;
            window_weights<W>(poly, pu.x, P.n, wx, &c);
            moments_add<D>(mm, pu.x, pu.y, 0.f, vu);          // vu = 0 past the item's end
            if (D == 1) {
#pragma unroll
                for (int a = 0; a < W; ++a) acc[a] = fmaf(vu, wx[a], acc[a]);
            } else {
                float wy[W];
                window_weights<W>(poly, pu.y, P.n, wy, &c);
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    const float xa = vu * wx[a];
#pragma unroll
                    for (int b = 0; b < W; b += 2) {
                        float2 t = make_float2(acc[a * W + b], acc[a * W + b + 1]);
                        t = __ffma2_rn(make_float2(xa, xa), make_float2(wy[b], wy[b + 1]), t);
                        acc[a * W + b] = t.x;
                        acc[a * W + b + 1] = t.y;
                    }
                }
            }
        }
    }
    if (P.pq != 0.f) moments_flush(mm, P.mom + r * P.mstride, lane);
    int base, held;
    warp_transpose_reduce<NV>(acc, lane, &base, &held);
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff;
    const int ox = cx - 3 - P.lo[0], oy = cy - 3 - P.lo[1];
    // for NV < 32 several lanes hold the same total: the lowest of them adds it
    const bool first = NV >= 32 || (lane & (32 / NV - 1)) == 0;
    if (first) {
#pragma unroll
        for (int e = 0; e < (NV >= 32 ? NV / 32 : 1); ++e) {
            const int idx = base + e;
            const int a = D == 1 ? idx : idx / W, b = D == 1 ? 0 : idx % W;
            const size_t o = r * P.gsz + (size_t)(ox + a) * P.box[1] + (D >= 2 ? oy + b : 0);
            grid_add(P.grid + o, P.grid64 ? P.grid64 + o : nullptr, acc[e]);
        }
    }
}

template <int D>
__global__ void __launch_bounds__(kWarps * 32) k_spread_lowd_w8(const int4* __restrict__ items, int nitems,
                                                               const WinDev* __restrict__ wins,
                                                               const float* __restrict__ v, int64_t ldv,
                                                               const WinPoly poly)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * kWarps + warp;
    if (item >= nitems) return;
    const int4 it = items[item];
    const int r = blockIdx.y;                                  // right-hand side
    spread_lowd_item<D>(it, wins[it.w], v + r * ldv, r, lane, poly);
}

// Every m = 4 spread item of every window (3-D, 2-D and 1-D, any mix) in one persistent launch: the
// 3-D units run the pipelined register-tile loop above, the others the one-warp low-d routine; a
// 3-D unit's first batch is prefetched by the unit before it only when that one is 3-D as well.
// Unit u takes item (u % nitems + rot) % nitems: with rot = the number of 3-D items the low-d items
// (latency-bound, few) go first and overlap the 3-D work, whose light items then form the tail.
template <int TILE>
__global__ void __launch_bounds__(kWarps * 32, 4) k_spread_w8_all(const int4* __restrict__ items, int nitems,
                                                              int nunits, int rot, int* __restrict__ counter,
                                                              const WinDev* __restrict__ wins,
                                                              const float* __restrict__ v, int64_t ldv,
                                                              const WinPoly poly)
{
    constexpr int W = 8;
    constexpr int STRIDE = 28;            // 8 + 8 + 8 floats, padded so staging stores avoid conflicts
    __shared__ __align__(16) float sw[kWarps][32 * STRIDE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* ws = sw[warp];

    int u = 0;
    if (lane == 0) u = atomicAdd(counter, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= nunits) return;
    int un = 0;
    if (lane == 0) un = atomicAdd(counter, 1);
    un = __shfl_sync(0xffffffffu, un, 0);
    int4 it = items[(u % nitems + rot) % nitems];
    int r = u / nitems;
    int4 itn = un < nunits ? items[(un % nitems + rot) % nitems] : make_int4(0, 0, 0, 0);
    const WinDev* P = wins + it.w;
    const float4* __restrict__ pts = P->pts + it.x;
    const float* __restrict__ vr = v + r * ldv;
    // software pipeline: the next batch's point (and then its v) is in flight during this batch;
    // `primed`: the current 3-D unit's first batch is already loaded
    float4 pn = make_float4(0.f, 0.f, 0.f, 0.f);
    float vn = 0.f;
    bool primed = false;
    float mm[5] = {0.f, 0.f, 0.f, 0.f, 0.f};      // moments of the quadratic split over this unit
    MomAcc macc = {0.0, -1};
    while (true) {
        const bool more = un < nunits;
        if (P->D != 3) {
            if (P->D == 2) spread_lowd_item<2>(it, *P, vr, r, lane, poly);
            else spread_lowd_item<1>(it, *P, vr, r, lane, poly);
            primed = false;
            if (!more) break;
            it = itn;
            r = un / nitems;
            P = wins + it.w;
            pts = P->pts + it.x;
            vr = v + r * ldv;
            if (lane == 0) un = atomicAdd(counter, 1);
            un = __shfl_sync(0xffffffffu, un, 0);
            itn = un < nunits ? items[(un % nitems + rot) % nitems] : make_int4(0, 0, 0, 0);
            continue;
        }
        if (!primed && lane < it.y) {
            pn = pts[lane];
            vn = __ldg(vr + __float_as_int(pn.w));
        }
        float2 acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = f2(0.f, 0.f);
        const int count = it.y;
        const int n = P->n;
        const bool split = P->pq != 0.f;
        // the next unit is prefetched only if it is 3-D as well
        const bool n3 = more && wins[itn.w].D == 3;
        for (int base = 0; base < count; base += 32) {
            const float4 p = pn;
            const float vv = vn;
            const bool valid = base + lane < count;
            const bool last = base + 32 >= count;
            // prefetch: the next batch of this item, or the first batch of the next unit
            const float4* __restrict__ npts = last ? wins[itn.w].pts + itn.x : pts + base + 32;
            const int ncount = last ? (n3 ? itn.y : 0) : count - base - 32;
            if (lane < ncount) pn = npts[lane];
            float wx[W], wy[W], wz[W];
            int cx, cy, cz;
            if (valid) {
                window_weights<W>(poly, p.x, n, wx, &cx);
                window_weights<W>(poly, p.y, n, wy, &cy);
                window_weights<W>(poly, p.z, n, wz, &cz);
#pragma unroll
                for (int q = 0; q < W; ++q) wx[q] *= vv;
                if (split) moments_add<3>(mm, p.x, p.y, p.z, vv);
            } else {
#pragma unroll
                for (int q = 0; q < W; ++q) { wx[q] = 0.f; wy[q] = 0.f; wz[q] = 0.f; }
            }
            if (lane < ncount) vn = __ldg((last ? v + (un / nitems) * ldv : vr) + __float_as_int(pn.w));
            float4* dst = reinterpret_cast<float4*>(ws + lane * STRIDE);
            dst[0] = make_float4(wx[0], wx[1], wx[2], wx[3]);
            dst[1] = make_float4(wx[4], wx[5], wx[6], wx[7]);
            dst[2] = make_float4(wy[0], wy[1], wy[2], wy[3]);
            dst[3] = make_float4(wy[4], wy[5], wy[6], wy[7]);
            dst[4] = make_float4(wz[0], wz[1], wz[2], wz[3]);
            dst[5] = make_float4(wz[4], wz[5], wz[6], wz[7]);
            __syncwarp();
            // rows cnt .. 31 hold zeros (lanes without a point stage zero weights), so an odd count is safe
            const int cnt = min(32, count - base);
            spread3_points<TILE>(acc, ws, STRIDE, cnt, lane);
            __syncwarp();
        }
        spread3_flush<TILE>(acc, P, it, r, lane);
        if (split) mom_unit_end(macc, mm, wins, it.w, r, lane);
        primed = n3;
        if (!more) break;
        // advance: the prefetched unit becomes current; take the one after it
        it = itn;
        r = un / nitems;
        P = wins + it.w;
        pts = P->pts + it.x;
        vr = v + r * ldv;
        if (lane == 0) un = atomicAdd(counter, 1);
        un = __shfl_sync(0xffffffffu, un, 0);
        itn = un < nunits ? items[(un % nitems + rot) % nitems] : make_int4(0, 0, 0, 0);
    }
    mom_flush(macc, wins, lane);
}

// One 1-D or 2-D item (m = 4) by one warp; t holds at least (2m)^D entries.
template <int D, bool WK, bool WD>
__device__ __forceinline__ void gather_lowd_item(const int4 it, const WinDev& P, float2* t, int lane, int r,
                                                 const GatherArgs& g, const WinPoly& poly)
{
    constexpr int W = 8;
    constexpr int NV = D == 1 ? W : W * W;
    float* __restrict__ outK = g.outK;
    float* __restrict__ outD = g.outD;
    const int64_t strideK = g.strideK, strideD = g.strideD, rstrideK = g.rstrideK, rstrideD = g.rstrideD;
    const float* __restrict__ scaleK = g.scaleK;
    const float* __restrict__ scaleD = g.scaleD;
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff;
    const int ox = cx - 3 - P.lo[0], oy = cy - 3 - P.lo[1];
    const float2* __restrict__ h = P.h + r * P.gsz;
    for (int i = lane; i < NV; i += 32) {
        const int a = D == 1 ? i : i / W, b = D == 1 ? 0 : i % W;
        t[i] = h[(size_t)(ox + a) * P.box[1] + (D >= 2 ? oy + b : 0)];
    }
    __syncwarp();
    const float4* __restrict__ pts = P.pts + it.x;
    const float sK = WK ? scaleK[it.w] : 0.f;
    const float sD = WD ? scaleD[it.w] : 0.f;
    const Quad Q = WD ? quad_of(P, r) : Quad{0.f, 0.f, 0.f, 0.f, 0.f};
    constexpr int U = 4;                                       // points per lane per round, loads together
    for (int k0 = lane; k0 < it.y; k0 += 32 * U) {
        float4 pp[U];
#pragma unroll
        for (int q = 0; q < U; ++q) pp[q] = pts[min(k0 + 32 * q, it.y - 1)];
        // one point at a time (the array rotates so that indices stay static and in registers)
#pragma unroll 1
        for (int q = 0; q < U; ++q) {
            if (k0 + 32 * q >= it.y) break;
            const float4 p = pp[0];
#pragma unroll
            for (int z = 0; z < U - 1; ++z) pp[z] = pp[z + 1];
            float wx[W];
            int c;
            window_weights<W>(poly, p.x, P.n, wx, &c);
            float2 f = make_float2(0.f, WD ? quad_eval<D>(Q, p.x, p.y, 0.f) : 0.f);
            if (D == 1) {
#pragma unroll
                for (int a = 0; a < W; ++a) f = __ffma2_rn(t[a], make_float2(wx[a], wx[a]), f);
            } else {
                float wy[W];
                window_weights<W>(poly, p.y, P.n, wy, &c);
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    float2 u = make_float2(0.f, 0.f);
                    const float4* row = reinterpret_cast<const float4*>(t + a * W);
#pragma unroll
                    for (int b = 0; b < W; b += 2) {
                        const float4 hv = row[b / 2];
                        u = __ffma2_rn(make_float2(hv.x, hv.y), make_float2(wy[b], wy[b]), u);
                        u = __ffma2_rn(make_float2(hv.z, hv.w), make_float2(wy[b + 1], wy[b + 1]), u);
                    }
                    f = __ffma2_rn(u, make_float2(wx[a], wx[a]), f);
                }
            }
            const int64_t i = (int64_t)__float_as_int(p.w);
            if (WK) outK[i + it.w * strideK + r * rstrideK] = sK * f.x;
            if (WD) outD[i + it.w * strideD + r * rstrideD] = sD * f.y;
        }
    }
}

template <int D, bool WK, bool WD>
__global__ void __launch_bounds__(kWarps * 32) k_gather_lowd_w8(const int4* __restrict__ items, int nitems,
                                                               const WinDev* __restrict__ wins, GatherArgs g,
                                                               const WinPoly poly)
{
    __shared__ __align__(16) float2 tile[kWarps][D == 1 ? 8 : 64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * kWarps + warp;
    if (item >= nitems) return;
    const int4 it = items[item];
    gather_lowd_item<D, WK, WD>(it, wins[it.w], tile[warp], lane, blockIdx.y, g, poly);
}

// Every m = 4 item of every window in one launch (items of the 3-D, 1-D and 2-D kinds are contiguous):
// each warp takes the routine of its item's dimension, so mixed windows share one grid and one tail.
template <bool WK, bool WD>
__global__ void __launch_bounds__(kWarps * 32, 4) k_gather_w8_all(const int4* __restrict__ items, int nitems,
                                                                 const WinDev* __restrict__ wins, GatherArgs g,
                                                                 const WinPoly poly)
{
    __shared__ __align__(16) float2 tile[kWarps][512];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * kWarps + warp;
    if (item >= nitems) return;
    const int4 it = items[item];
    const WinDev& P = wins[it.w];
    if (P.D == 3) gather3_item<WK, WD>(it, P, tile[warp], lane, blockIdx.y, g, poly);
    else if (P.D == 2) gather_lowd_item<2, WK, WD>(it, P, tile[warp], lane, blockIdx.y, g, poly);
    else gather_lowd_item<1, WK, WD>(it, P, tile[warp], lane, blockIdx.y, g, poly);
}

// ----------------------------------------------------------------------------------
// generic kernels: any D in {1,2,3}, W = 2m <= 16. One block per item; the spread accumulates
// the item's W^D support box in shared memory, then adds it to the grid.
template <int D>
__global__ void __launch_bounds__(128) k_spread_generic(const int4* __restrict__ items,
                                                        const WinDev* __restrict__ wins,
                                                        const float* __restrict__ v, int64_t ldv,
                                                        const WinPoly poly)
{
    __shared__ float box[kMaxW * kMaxW * kMaxW];
    const int4 it = items[blockIdx.x];
    const WinDev& P = wins[it.w];
    const int r = blockIdx.y;                                  // right-hand side
    v += r * ldv;
    const int W = 2 * P.m;
    int WD = W;
    if (D >= 2) WD *= W;
    if (D >= 3) WD *= W;
    for (int i = threadIdx.x; i < WD; i += blockDim.x) box[i] = 0.f;
    __syncthreads();
    float mm[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = threadIdx.x; k < it.y; k += blockDim.x) {
        const float4 p = P.pts[it.x + k];
        const float vv = __ldg(v + __float_as_int(p.w));
        moments_add<D>(mm, p.x, p.y, p.z, vv);
        float w0[kMaxW], w1[kMaxW], w2[kMaxW];
        int c;
        window_weights_n(poly, p.x, P.n, W, w0, &c);
        if (D >= 2) window_weights_n(poly, p.y, P.n, W, w1, &c);
        if (D >= 3) window_weights_n(poly, p.z, P.n, W, w2, &c);
        for (int a = 0; a < W; ++a) {
            const float va = vv * w0[a];
            if (D == 1) { atomicAdd(&box[a], va); continue; }
            for (int bb = 0; bb < W; ++bb) {
                const float vab = va * w1[bb];
                if (D == 2) { atomicAdd(&box[a * W + bb], vab); continue; }
                for (int cc = 0; cc < W; ++cc) atomicAdd(&box[(a * W + bb) * W + cc], vab * w2[cc]);
            }
        }
    }
    if (P.pq != 0.f) moments_flush(mm, P.mom + r * P.mstride, threadIdx.x & 31);
    __syncthreads();
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff, cz = (it.z >> 16) & 0xff;
    const int ox = cx - P.m + 1 - P.lo[0], oy = cy - P.m + 1 - P.lo[1], oz = cz - P.m + 1 - P.lo[2];
    for (int i = threadIdx.x; i < WD; i += blockDim.x) {
        int a = i, bb = 0, cc = 0;
        if (D == 2) { a = i / W; bb = i % W; }
        if (D == 3) { a = i / (W * W); bb = (i / W) % W; cc = i % W; }
        const size_t g = ((size_t)(ox + a) * P.box[1] + (D >= 2 ? oy + bb : 0)) * P.box[2] + (D >= 3 ? oz + cc : 0);
        if (box[i] != 0.f) grid_add(P.grid + r * P.gsz + g, P.grid64 ? P.grid64 + r * P.gsz + g : nullptr, box[i]);
    }
}

template <int D, bool WK, bool WD>
__global__ void __launch_bounds__(128) k_gather_generic(const int4* __restrict__ items,
                                                        const WinDev* __restrict__ wins,
                                                        float* __restrict__ outK, float* __restrict__ outD,
                                                        const float* __restrict__ scaleK,
                                                        const float* __restrict__ scaleD, int64_t strideK,
                                                        int64_t strideD, int64_t rstrideK, int64_t rstrideD,
                                                        const WinPoly poly)
{
    const int4 it = items[blockIdx.x];
    const WinDev& P = wins[it.w];
    const int W = 2 * P.m;
    const int r = blockIdx.y;                                  // right-hand side
    const float2* __restrict__ h = P.h + r * P.gsz;
    const int cx = it.z & 0xff, cy = (it.z >> 8) & 0xff, cz = (it.z >> 16) & 0xff;
    const int ox = cx - P.m + 1 - P.lo[0], oy = cy - P.m + 1 - P.lo[1], oz = cz - P.m + 1 - P.lo[2];
    const Quad Q = WD ? quad_of(P, r) : Quad{0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = threadIdx.x; k < it.y; k += blockDim.x) {
        const float4 p = P.pts[it.x + k];
        float w0[kMaxW], w1[kMaxW], w2[kMaxW];
        int c;
        window_weights_n(poly, p.x, P.n, W, w0, &c);
        if (D >= 2) window_weights_n(poly, p.y, P.n, W, w1, &c);
        if (D >= 3) window_weights_n(poly, p.z, P.n, W, w2, &c);
        float fK = 0.f, fD = 0.f;
        for (int a = 0; a < W; ++a) {
            float uK = 0.f, uD = 0.f;
            for (int bb = 0; bb < (D >= 2 ? W : 1); ++bb) {
                float tK = 0.f, tD = 0.f;
                for (int cc = 0; cc < (D >= 3 ? W : 1); ++cc) {
                    const size_t g = ((size_t)(ox + a) * P.box[1] + (D >= 2 ? oy + bb : 0)) * P.box[2] +
                                     (D >= 3 ? oz + cc : 0);
                    const float2 hv = h[g];
                    const float wc = D >= 3 ? w2[cc] : 1.f;
                    tK = fmaf(hv.x, wc, tK);
                    tD = fmaf(hv.y, wc, tD);
                }
                const float wb = D >= 2 ? w1[bb] : 1.f;
                uK = fmaf(tK, wb, uK);
                uD = fmaf(tD, wb, uD);
            }
            fK = fmaf(uK, w0[a], fK);
            fD = fmaf(uD, w0[a], fD);
        }
        const int64_t i = (int64_t)__float_as_int(p.w);
        if (WK) outK[i + it.w * strideK + r * rstrideK] = scaleK[it.w] * fK;
        if (WD) outD[i + it.w * strideD + r * rstrideD] = scaleD[it.w] * (fD + quad_eval<D>(Q, p.x, p.y, p.z));
    }
}

}  // namespace

// Blocks of `kernel` (block threads, no dynamic shared memory) resident on the whole device at once,
// cached per device and kernel.
template <typename K>
static int resident_blocks(K kernel, int threads)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_pair(dev, reinterpret_cast<const void*>(kernel));
    std::lock_guard<std::mutex> lock(mu);
    auto f = cache.find(key);
    if (f != cache.end()) return f->second;
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
    const int nb = std::max(1, sms * std::max(1, per));
    cache[key] = nb;
    return nb;
}

// Blocks of a persistent spread: as many as fit (sp_blocks = 0) or sp_blocks per SM (autotuned), never more
// than the units need.
template <typename K>
static int spread_blocks(const Plan& p, K kernel, int units)
{
    int nb = resident_blocks(kernel, kWarps * 32);
    if (p.sp_blocks > 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        nb = std::min(nb, p.sp_blocks * std::max(sms, 1));
    }
    return std::max(1, std::min(nb, (units + kWarps - 1) / kWarps));
}

// Items of one kind for one window, or for all windows (window < 0).
static void item_range(const Plan& p, int kind, int window, int* lo, int* hi, bool spread = false)
{
    const std::vector<int>& b = spread ? p.item_begin_sp[kind] : p.item_begin[kind];
    if (window < 0) { *lo = b.front(); *hi = b.back(); }
    else { *lo = b[window]; *hi = b[window + 1]; }
}

// One launch per kernel kind that has items: all windows of a kind together, all right-hand sides
// along gridDim.y.
cudaError_t launch_spread(const Plan& p, int window, const float* v, int64_t ldv, int nrhs, cudaStream_t st, int* count)
{
    int launched = 0;
    const WinDev* wd = p.wins_dev;
    int k0 = 0;
    // the persistent kernels' work counter and, when a window is split, the moments of these right-hand
    // sides (they lie right after the counter: one memset)
    const size_t zero = 16 * sizeof(int) + (p.any_split ? sizeof(double) * 8 * p.P * (size_t)nrhs : 0);
    if (cudaMemsetAsync(p.counters, 0, zero, st) != cudaSuccess) return cudaGetLastError();
    if (window < 0) {
        // the m = 4 kinds (3-D, 1-D, 2-D fast) lie next to each other in the spread list: one persistent
        // launch for all of them, units taken from a zeroed counter
        const int lo = p.item_begin_sp[kKindFast3].front(), hi = p.item_begin_sp[kKindLow2].back();
        const int n3 = p.item_begin_sp[kKindFast3].back() - lo;
        if (hi > lo) {
            const int n = hi - lo, units = n * nrhs;
            if (n3 == n) {                    // 3-D items only: the kernel without the per-unit branch
                auto kern = p.sp_tile == 1 ? k_spread3_w8<1> : k_spread3_w8<0>;
                const int nb = spread_blocks(p, kern, units);
                launch_k(false, kern, dim3(nb), dim3(kWarps * 32), 0, st, p.items + lo, n, units, p.counters, wd, v,
                         ldv, p.poly);
            } else {
                auto kern = p.sp_tile == 1 ? k_spread_w8_all<1> : k_spread_w8_all<0>;
                const int nb = spread_blocks(p, kern, units);
                launch_k(false, kern, dim3(nb), dim3(kWarps * 32), 0, st, p.items + lo, n, units, n3, p.counters, wd,
                         v, ldv, p.poly);
            }
            ++launched;
        }
        k0 = kKindGen1;
    }
    for (int k = k0; k < kKinds; ++k) {
        int lo, hi;
        item_range(p, k, window, &lo, &hi, true);
        if (hi <= lo) continue;
        const int n = hi - lo;
        const int4* it = p.items + lo;
        const dim3 warps((n + kWarps - 1) / kWarps, nrhs), blocks(n, nrhs);
        const bool pdl = false;                // the first kernel of a product follows arbitrary stream work
        const dim3 T(kWarps * 32), T2(128);
        switch (k) {
            case kKindFast3: {
                // persistent: as many blocks as fit at once, units taken from a zeroed counter
                const int units = n * nrhs;
                auto kern = p.sp_tile == 1 ? k_spread3_w8<1> : k_spread3_w8<0>;
                const int nb = spread_blocks(p, kern, units);
                launch_k(pdl, kern, dim3(nb), T, 0, st, it, n, units, p.counters, wd, v, ldv, p.poly);
                break;
            }
            case kKindLow1: launch_k(pdl, k_spread_lowd_w8<1>, warps, T, 0, st, it, n, wd, v, ldv, p.poly); break;
            case kKindLow2: launch_k(pdl, k_spread_lowd_w8<2>, warps, T, 0, st, it, n, wd, v, ldv, p.poly); break;
            case kKindGen1: launch_k(pdl, k_spread_generic<1>, blocks, T2, 0, st, it, wd, v, ldv, p.poly); break;
            case kKindGen2: launch_k(pdl, k_spread_generic<2>, blocks, T2, 0, st, it, wd, v, ldv, p.poly); break;
            default: launch_k(pdl, k_spread_generic<3>, blocks, T2, 0, st, it, wd, v, ldv, p.poly); break;
        }
        ++launched;
    }
    if (count) *count = launched;
    return cudaGetLastError();
}

template <bool WK, bool WD>
static int gather_all(const Plan& p, int window, float* oK, int64_t zK, int64_t rK, float* oD, int64_t zD,
                      int64_t rD, int nrhs, const float* sK, const float* sD, cudaStream_t st)
{
    int launched = 0;
    const WinDev* wd = p.wins_dev;
    const GatherArgs g = {oK, oD, sK, sD, zK, zD, rK, rD};
    const dim3 T(kWarps * 32), T2(128);
    int k0 = 0;
    if (window < 0) {
        // the m = 4 kinds (3-D, 1-D, 2-D fast) lie next to each other: one launch for all of them
        const int lo = p.item_begin[kKindFast3].front(), hi = p.item_begin[kKindLow2].back();
        if (hi > lo) {
            const int n = hi - lo;
            launch_k(false, k_gather_w8_all<WK, WD>, dim3((n + kWarps - 1) / kWarps, nrhs), T, 0, st, p.items + lo, n,
                     wd, g, p.poly);
            ++launched;
        }
        k0 = kKindGen1;
    }
    for (int k = k0; k < kKinds; ++k) {
        int lo, hi;
        item_range(p, k, window, &lo, &hi);
        if (hi <= lo) continue;
        const int n = hi - lo;
        const int4* it = p.items + lo;
        const dim3 warps((n + kWarps - 1) / kWarps, nrhs), blocks(n, nrhs);
        switch (k) {
            case kKindFast3: launch_k(false, k_gather3_w8<WK, WD>, warps, T, 0, st, it, n, wd, g, p.poly); break;
            case kKindLow1: launch_k(false, k_gather_lowd_w8<1, WK, WD>, warps, T, 0, st, it, n, wd, g, p.poly); break;
            case kKindLow2: launch_k(false, k_gather_lowd_w8<2, WK, WD>, warps, T, 0, st, it, n, wd, g, p.poly); break;
            case kKindGen1:
                launch_k(false, k_gather_generic<1, WK, WD>, blocks, T2, 0, st, it, wd, oK, oD, sK, sD, zK, zD, rK, rD,
                         p.poly);
                break;
            case kKindGen2:
                launch_k(false, k_gather_generic<2, WK, WD>, blocks, T2, 0, st, it, wd, oK, oD, sK, sD, zK, zD, rK, rD,
                         p.poly);
                break;
            default:
                launch_k(false, k_gather_generic<3, WK, WD>, blocks, T2, 0, st, it, wd, oK, oD, sK, sD, zK, zD, rK, rD,
                         p.poly);
                break;
        }
        ++launched;
    }
    return launched;
}

cudaError_t launch_gather(const Plan& p, int window, float* outK, int64_t zK, int64_t rK, float* outD, int64_t zD,
                          int64_t rD, int nrhs, const float* sK, const float* sD, cudaStream_t st, int* count)
{
    int launched = 0;
    if (outK && outD) launched = gather_all<true, true>(p, window, outK, zK, rK, outD, zD, rD, nrhs, sK, sD, st);
    else if (outK) launched = gather_all<true, false>(p, window, outK, zK, rK, nullptr, 0, 0, nrhs, sK, sD, st);
    else if (outD) launched = gather_all<false, true>(p, window, nullptr, 0, 0, outD, zD, rD, nrhs, sK, sD, st);
    if (count) *count = launched;
    return cudaGetLastError();
}

}  // namespace addker
