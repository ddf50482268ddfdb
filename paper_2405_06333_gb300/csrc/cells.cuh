// Shared machinery of the real-space kernels: the screened-Coulomb pair factors, the
// enumeration of a charge's sources (the charge and its images near the slab, Eq. 3.2 -
// Eq. 3.3 with the coefficients of reading A4), and the kernels that build the sorted
// cell list of those sources (count, scan, scatter, per-cell key order).  Included by
// the cell-scan pair kernel (real_kernels.cu) and the pair-list kernels
// (pairlist_kernels.cu); everything here has internal linkage.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rbe2d_internal.h"

namespace rbe2d {
namespace {

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    typedef float4 type;
};
template <>
struct Vec4<double> {
    typedef double4_32a type;
};

// Screened-Coulomb pair factors for a pair at distance r (r2 = r^2, ax = alpha r):
//   ec = erfc(alpha r),  g = exp(-alpha^2 r^2),  ir = 1/r.
// float32: erfc by Abramowitz and Stegun's rational approximation 7.1.26
// (|error| <= 1.5e-7 for x >= 0), which shares its exponential with the Gaussian term;
// float64: the library erfc and exp.
constexpr float kAsP = 0.3275911f;  // 7.1.26: erfc x ~ t (a1 + t (a2 + ...)) e^{-x^2}, t = 1 / (1 + p x)
__device__ constexpr float kAsA[5] = {0.254829592f, -0.284496736f, 1.421413741f, -1.453152027f, 1.061405429f};

__device__ __forceinline__ void screened(float r2, float a, float& ec, float& g, float& ir) {
    ir = rsqrtf(r2);
    const float x = a * r2 * ir;
    g = __expf(-x * x);
    const float t = __fdividef(1.0f, fmaf(kAsP, x, 1.0f));
    const float p = fmaf(fmaf(fmaf(fmaf(kAsA[4], t, kAsA[3]), t, kAsA[2]), t, kAsA[1]), t, kAsA[0]);
    ec = t * p * g;
}
// The same for two distances at once (x and y halves) on paired float32 instructions; the
// reciprocal square root, exponential and reciprocal stay one MUFU operation each.
__device__ __forceinline__ void screened2(float2 r2, float a, float2& ec, float2& g, float2& ir) {
    ir = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 x = __fmul2_rn(__fmul2_rn(make_float2(a, a), r2), ir);
    const float2 xx = __fmul2_rn(x, x);
    g = make_float2(__expf(-xx.x), __expf(-xx.y));
    const float2 den = __ffma2_rn(make_float2(kAsP, kAsP), x, make_float2(1.f, 1.f));
    const float2 t = make_float2(__fdividef(1.0f, den.x), __fdividef(1.0f, den.y));
    float2 p = make_float2(kAsA[4], kAsA[4]);
#pragma unroll
    for (int i = 3; i >= 0; i--) p = __ffma2_rn(p, t, make_float2(kAsA[i], kAsA[i]));
    ec = __fmul2_rn(__fmul2_rn(t, p), g);
}
__device__ __forceinline__ void screened(double r2, double a, double& ec, double& g, double& ir) {
    const double r = sqrt(r2);
    ir = 1.0 / r;
    ec = erfc(a * r);
    g = exp(-a * a * r2);
}

// Fixed-order sum of n doubles by all threads of one CTA (strided partial sums, then
// warps in order); thread 0 gets the total.
__device__ double cta_sum_ordered(const double* __restrict__ v, unsigned n, double* red) {
    double t = 0.0;
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) t += __ldcg(&v[i]);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
    return s;
}

__device__ __forceinline__ int wrap_cell(int c, int n) {
    c %= n;
    return c < 0 ? c + n : c;
}

// Cell of a source at (x, y, z) (x, y already in [0, L)) and its corner-relative coords.
__device__ __forceinline__ int cell_of(const CellGrid& g, double x, double y, double z, double* xl, double* yl,
                                       double* zl) {
    int cx = (int)floor(x * g.inv_hx), cy = (int)floor(y * g.inv_hy), cz = (int)floor((z - g.z0) * g.inv_hz);
    cx = min(max(cx, 0), g.ncx - 1);
    cy = min(max(cy, 0), g.ncy - 1);
    cz = min(max(cz, 0), g.ncz - 1);
    *xl = x - cx * g.hx;
    *yl = y - cy * g.hy;
    *zl = z - (g.z0 + cz * g.hz);
    return (cz * g.ncy + cy) * g.ncx + cx;
}

// The sources of particle j: slot 0 the charge itself, slots 2l-1 / 2l its images of
// level l above / below the slab (Eq. 3.3, coefficients of reading A4), kept if their
// height is within r_c of the slab.  f(slot, x, y, z, qg) is called for each.
template <typename TIn, typename F>
__device__ __forceinline__ void for_each_source(const DevParams& dp, const CellGrid& g, const TIn* pos, const TIn* q,
                                                int64_t j, F f) {
    double x = (double)pos[3 * j], y = (double)pos[3 * j + 1], z = (double)pos[3 * j + 2];
    const double qj = (double)q[j];
    x -= floor(x * dp.inv_Lx) * dp.Lx;
    y -= floor(y * dp.inv_Ly) * dp.Ly;
    // keep every source inside the grid even for non-finite or far-away input
    x = isfinite(x) ? fmin(fmax(x, 0.0), dp.Lx) : 0.0;
    y = isfinite(y) ? fmin(fmax(y, 0.0), dp.Ly) : 0.0;
    z = isfinite(z) ? z : 0.0;
    if (x >= dp.Lx) x -= dp.Lx;
    if (y >= dp.Ly) y -= dp.Ly;
    f(0, x, y, z, qj);
    const double lo = -dp.r_c, hi = dp.H + dp.r_c;
    double gp_up = 1.0, gp_dn = 1.0;  // running gt^ceil(l/2) gb^floor(l/2) and its mirror
    for (int l = 1; l <= g.lmax; l++) {
        // gamma_+^(l) = gt^ceil(l/2) gb^floor(l/2): multiply by gt on odd l, by gb on even l
        if (l & 1) { gp_up *= dp.gt; gp_dn *= dp.gb; }
        else { gp_up *= dp.gb; gp_dn *= dp.gt; }
        const double sg = (l & 1) ? -1.0 : 1.0;
        const double zp = sg * z + 2.0 * ((l + 1) / 2) * dp.H;
        const double zm = sg * z - 2.0 * (l / 2) * dp.H;
        if (gp_up != 0.0 && zp > lo && zp < hi) f(2 * l - 1, x, y, zp, qj * gp_up);
        if (gp_dn != 0.0 && zm > lo && zm < hi) f(2 * l, x, y, zm, qj * gp_dn);
    }
}

// The same enumeration for float32 storage, in fixed point: x and y as 32-bit turn
// fractions of the cell (the periodic wrap is exact and the cell index is
// (u n_cells) >> 32), z over the extended range [-r_c, H + r_c) as a 32-bit fraction
// with the images reached by integer steps of 2H.  Three float64 conversions per charge
// (float64 is 1/64 of the float32 rate on GB300); corner-relative coordinates keep
// 2^-24 of a cell.  f(slot, cell, xl, yl, zl, qg).
struct FxGrid {
    double sx, sy, sz;       // 2^32 / Lx, 2^32 / Ly, 2^32 / (H + 2 r_c)
    long long zoff, zstep;   // r_c and 2H in units of the z fraction
    float rx, ry, rz;        // cell sizes / 2^32
    float gt, gb;
};

template <typename TIn, typename F>
__device__ __forceinline__ void for_each_source32(const CellGrid& g, const FxGrid& X, const TIn* pos, const TIn* q,
                                                  int64_t j, F f) {
    double x = (double)pos[3 * j], y = (double)pos[3 * j + 1], z = (double)pos[3 * j + 2];
    x = isfinite(x) ? x : 0.0;
    y = isfinite(y) ? y : 0.0;
    z = isfinite(z) ? z : 0.0;
    const uint32_t ux = (uint32_t)(unsigned long long)__double2ll_rn(x * X.sx);
    const uint32_t uy = (uint32_t)(unsigned long long)__double2ll_rn(y * X.sy);
    const long long A = __double2ll_rn(z * X.sz);
    const unsigned long long px = (unsigned long long)ux * (unsigned)g.ncx;
    const unsigned long long py = (unsigned long long)uy * (unsigned)g.ncy;
    const int cx = (int)(px >> 32), cy = (int)(py >> 32);
    const float xl = (float)(uint32_t)px * X.rx, yl = (float)(uint32_t)py * X.ry;
    const float qj = (float)q[j];
    auto emit = [&](int slot, long long uz, float w) {
        const unsigned long long pz = (unsigned long long)uz * (unsigned)g.ncz;
        const int cz = (int)(pz >> 32);
        f(slot, (cz * g.ncy + cy) * g.ncx + cx, xl, yl, (float)(uint32_t)pz * X.rz, w);
    };
    const long long top = 1LL << 32;
    long long u0 = A + X.zoff;  // the charge itself: always kept, clamped into the grid
    u0 = u0 < 0 ? 0 : (u0 >= top ? top - 1 : u0);
    emit(0, u0, qj);
    float gp_up = 1.f, gp_dn = 1.f;
    for (int l = 1; l <= g.lmax; l++) {
        if (l & 1) { gp_up *= X.gt; gp_dn *= X.gb; }
        else { gp_up *= X.gb; gp_dn *= X.gt; }
        const long long sA = (l & 1) ? -A : A;
        const long long up = sA + (long long)((l + 1) / 2) * X.zstep + X.zoff;
        const long long dn = sA - (long long)(l / 2) * X.zstep + X.zoff;
        if (gp_up != 0.f && up > 0 && up < top) emit(2 * l - 1, up, qj * gp_up);
        if (gp_dn != 0.f && dn > 0 && dn < top) emit(2 * l, dn, qj * gp_dn);
    }
}

// gate != NULL: the cell-list kernels return at once unless *gate != 0 (a pair-list
// rebuild decided on the device).  count_real != NULL: also count the real charges per cell.
__device__ __forceinline__ bool gated_off(const int* gate) { return gate && *gate == 0; }

__global__ void rs_clear_kernel(int* __restrict__ count, int* __restrict__ count_real, int ncell,
                                const int* __restrict__ gate) {
    if (gated_off(gate)) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        count[c] = 0;
        if (count_real) count_real[c] = 0;
    }
}

template <typename TIn, typename T>
__global__ void rs_count_kernel(DevParams dp, CellGrid g, FxGrid X, const TIn* __restrict__ pos,
                                const TIn* __restrict__ q, int64_t N, int* __restrict__ count,
                                int* __restrict__ count_real, const int* __restrict__ gate) {
    if (gated_off(gate)) return;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        if (sizeof(T) == 4) {
            for_each_source32(g, X, pos, q, j, [&](int slot, int c, float, float, float, float) {
                atomicAdd(&count[c], 1);
                if (count_real && slot == 0) atomicAdd(&count_real[c], 1);
            });
        } else {
            for_each_source(dp, g, pos, q, j, [&](int, double x, double y, double z, double) {
                double xl, yl, zl;
                atomicAdd(&count[cell_of(g, x, y, z, &xl, &yl, &zl)], 1);
            });
        }
    }
}

// Exclusive scan of the cell counts in tiles of 1024 cells: the first kernel sums each
// tile, the second offsets each tile by the tiles before it and scans it in the block
// (coalesced loads, integer sums: exact); it also clears the fill counters.
constexpr int RS_SCAN = 1024;

__device__ __forceinline__ int block_excl_scan(int v, int* total, int* wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;  // inclusive warp prefix
    }
    __syncthreads();
    *total = wsum[(blockDim.x >> 5) - 1];
    return x - v + (warp > 0 ? wsum[warp - 1] : 0);
}

__global__ void __launch_bounds__(RS_SCAN) rs_tile_sum_kernel(const int* __restrict__ count, int ncell,
                                                              int* __restrict__ tile_sum, const int* __restrict__ gate) {
    if (gated_off(gate)) return;
    __shared__ int wsum[32];
    const int i = blockIdx.x * RS_SCAN + threadIdx.x;
    int total;
    block_excl_scan(i < ncell ? count[i] : 0, &total, wsum);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(RS_SCAN) rs_scan_kernel(const int* __restrict__ count, int ncell,
                                                          const int* __restrict__ tile_sum, int* __restrict__ start,
                                                          int* __restrict__ fill, const int* __restrict__ gate) {
    if (gated_off(gate)) return;
    __shared__ int wsum[32];
    __shared__ int base;
    // sum of the preceding tiles (integers: any order is exact)
    int pre = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += RS_SCAN) pre += tile_sum[b];
    int tot;
    block_excl_scan(pre, &tot, wsum);
    if (threadIdx.x == 0) base = tot;
    __syncthreads();
    const int i = blockIdx.x * RS_SCAN + threadIdx.x;
    const int v = i < ncell ? count[i] : 0;
    int total;
    const int ex = block_excl_scan(v, &total, wsum);
    if (i < ncell) {
        start[i] = base + ex;
        if (fill) fill[i] = 0;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) start[ncell] = base + total;
}

template <typename TIn, typename T>
__global__ void rs_fill_kernel(DevParams dp, CellGrid g, FxGrid X, const TIn* __restrict__ pos,
                               const TIn* __restrict__ q, int64_t N, const int* __restrict__ start,
                               int* __restrict__ fill, typename Vec4<T>::type* __restrict__ src,
                               long long* __restrict__ key, const int* __restrict__ gate) {
    if (gated_off(gate)) return;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        if (sizeof(T) == 4) {
            for_each_source32(g, X, pos, q, j, [&](int slot, int c, float xl, float yl, float zl, float qg) {
                const int at = start[c] + atomicAdd(&fill[c], 1);
                typename Vec4<T>::type v;
                v.x = (T)xl; v.y = (T)yl; v.z = (T)zl; v.w = (T)qg;
                src[at] = v;
                key[at] = j * 256 + slot;
            });
            continue;
        }
        for_each_source(dp, g, pos, q, j, [&](int slot, double x, double y, double z, double qg) {
            double xl, yl, zl;
            const int c = cell_of(g, x, y, z, &xl, &yl, &zl);
            const int at = start[c] + atomicAdd(&fill[c], 1);
            typename Vec4<T>::type v;
            v.x = (T)xl; v.y = (T)yl; v.z = (T)zl; v.w = (T)qg;
            src[at] = v;
            key[at] = j * 256 + slot;
        });
    }
}

// One warp per cell: each source's rank among the cell's keys (keys are unique) gives its
// place in the ordered copy.
template <typename T>
__global__ void rs_order_kernel(int ncell, const int* __restrict__ start,
                                const typename Vec4<T>::type* __restrict__ src, const long long* __restrict__ key,
                                typename Vec4<T>::type* __restrict__ src_out, long long* __restrict__ key_out,
                                int* __restrict__ status, const int* __restrict__ gate) {
    if (gated_off(gate)) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < ncell; c += nwarps) {
        const int b = start[c], n = start[c + 1] - b;
        if (n > kMaxOrderedCell) {  // too crowded to order in bounded time: keep scatter order
            for (int i = lane; i < n; i += 32) {
                src_out[b + i] = src[b + i];
                key_out[b + i] = key[b + i];
            }
            if (lane == 0) atomicAdd(&status[ST_CELL], 1);
            continue;
        }
        for (int i = lane; i < n; i += 32) {
            const long long ki = key[b + i];
            int r = 0;
            for (int m = 0; m < n; m++) r += key[b + m] < ki;
            src_out[b + r] = src[b + i];
            key_out[b + r] = ki;
        }
    }
}

}  // namespace
}  // namespace rbe2d
