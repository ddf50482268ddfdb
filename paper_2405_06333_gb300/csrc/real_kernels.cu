// Real-space part of the force with image charges (Eq. 3.12; force by reading A15):
//   F_i = q_i sum_src q_src g_src [erfc(a r)/r^2 + (2a/sqrt(pi)) e^{-a^2 r^2}/r] (r_i - r_src)/r
// over the real charges (without i itself in the home cell) and the image charges of
// every charge (its own included) within r_c, in every xy replica.  Only images whose
// height lies in (-r_c, H + r_c) can be within r_c of a charge in the slab.
//
// Cell list: cells of at least r_c in x, y (periodic) and in z over [-r_c, H + r_c].
// Sources are counted per cell, scattered with atomics, then every cell is put in key
// order (key = particle index, image slot) by a rank pass, so the sums run in a fixed
// order and the result is bitwise reproducible.  Coordinates are stored relative to the
// cell corner, so float32 keeps ~1e-7 r_c resolution for any box size.
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
    typedef double4 type;
};

// Screened-Coulomb pair factors for a pair at distance r (r2 = r^2, ax = alpha r):
//   ec = erfc(alpha r),  g = exp(-alpha^2 r^2),  ir = 1/r.
// float32: erfc by Abramowitz and Stegun's rational approximation 7.1.26
// (|error| <= 1.5e-7 for x >= 0), which shares its exponential with the Gaussian term;
// float64: the library erfc and exp.
__device__ __forceinline__ void screened(float r2, float a, float& ec, float& g, float& ir) {
    ir = rsqrtf(r2);
    const float x = a * r2 * ir;
    g = __expf(-x * x);
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    const float p = fmaf(fmaf(fmaf(fmaf(1.061405429f, t, -1.453152027f), t, 1.421413741f), t, -0.284496736f), t,
                         0.254829592f);
    ec = t * p * g;
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

template <typename TIn>
__global__ void rs_count_kernel(DevParams dp, CellGrid g, const TIn* __restrict__ pos, const TIn* __restrict__ q,
                                int64_t N, int* __restrict__ count) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        for_each_source(dp, g, pos, q, j, [&](int, double x, double y, double z, double) {
            double xl, yl, zl;
            atomicAdd(&count[cell_of(g, x, y, z, &xl, &yl, &zl)], 1);
        });
    }
}

// Exclusive scan of the cell counts (one CTA; each thread scans a contiguous segment);
// also clears the fill counters.
__global__ void __launch_bounds__(1024) rs_scan_kernel(const int* __restrict__ count, int ncell,
                                                       int* __restrict__ start, int* __restrict__ fill) {
    __shared__ int part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int seg = (ncell + T - 1) / T;
    const int b = t * seg, e = min(ncell, b + seg);
    int s = 0;
    for (int i = b; i < e; i++) s += count[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {  // inclusive Hillis-Steele scan of the segment sums
        int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int i = b; i < e; i++) {
        start[i] = run;
        run += count[i];
        fill[i] = 0;
    }
    if (t == T - 1) start[ncell] = part[T - 1];
}

template <typename TIn, typename T>
__global__ void rs_fill_kernel(DevParams dp, CellGrid g, const TIn* __restrict__ pos, const TIn* __restrict__ q,
                               int64_t N, const int* __restrict__ start, int* __restrict__ fill,
                               typename Vec4<T>::type* __restrict__ src, long long* __restrict__ key) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
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
                                int* __restrict__ status) {
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

// One CTA per cell; each thread owns one charge of the cell (in passes of blockDim).  The
// sources of the 27 neighbour cells (with their periodic shifts applied, relative to
// this cell's corner) stream through a shared-memory chunk, and every thread sums the
// screened field of the chunk on its charge.  Entries of the home cell carry a marker so
// a charge skips itself; image slots are sources only.  Sums run in a fixed order.
constexpr int RS_THREADS = 64;
constexpr int RS_CHUNK = 512;

template <typename T, bool LJ>
__global__ void __launch_bounds__(RS_THREADS) rs_cell_kernel(DevParams dp, CellGrid g,
                                                             const typename Vec4<T>::type* __restrict__ src,
                                                             const long long* __restrict__ key,
                                                             const int* __restrict__ start, T* __restrict__ force,
                                                             T* __restrict__ phi, int pot, int energy,
                                                             double* __restrict__ epart, double* __restrict__ scal,
                                                             unsigned* __restrict__ done, int* __restrict__ status) {
    typedef typename Vec4<T>::type V;
    __shared__ V buf[RS_CHUNK];
    __shared__ long long kbuf[RS_CHUNK];  // 2 key + 1 for home-cell entries
    __shared__ double red[RS_THREADS / 32];
    __shared__ bool last;
    const int c = blockIdx.x;
    const int cx = c % g.ncx, cy = (c / g.ncx) % g.ncy, cz = c / (g.ncx * g.ncy);
    const int b0 = start[c], nT = start[c + 1] - b0;
    const T a = (T)dp.alpha, rc2 = (T)(dp.r_c * dp.r_c), k2 = (T)(2.0 * dp.alpha / sqrt(M_PI));
    double e_local = 0.0;
    for (int tb = 0; tb < nT; tb += blockDim.x) {
        const int t = tb + threadIdx.x;
        const bool active = t < nT && (key[b0 + min(t, nT - 1)] & 255) == 0;
        V me = src[b0 + min(t, nT - 1)];
        const long long myself = key[b0 + min(t, nT - 1)] * 2 + 1;
        T fx = 0, fy = 0, fz = 0, ph = 0, lx = 0, ly = 0, lz = 0, elj = 0;
        int fill = 0, budget = kMaxCandidates;
        auto process = [&](int n) {
            if (active) {
                for (int i = 0; i < n; i++) {
                    const V o = buf[i];
                    const T dx = me.x - o.x, dy = me.y - o.y, dz = me.z - o.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 >= rc2) continue;
                    const long long kk = kbuf[i];
                    if (kk == myself) continue;
                    T ec, gs, ir;
                    screened(r2, a, ec, gs, ir);
                    const T fr = o.w * (ec * ir + k2 * gs) * ir * ir;
                    fx += fr * dx; fy += fr * dy; fz += fr * dz;
                    ph += o.w * ec * ir;
                    if (LJ && r2 < (T)dp.lj_rc2 && ((kk >> 1) & 255) == 0) {
                        const T s2 = (T)dp.lj_sig2 / r2, s6 = s2 * s2 * s2;
                        const T flj = (T)(24.0 * dp.lj_eps) * (2 * s6 * s6 - s6) / r2;
                        lx += flj * dx; ly += flj * dy; lz += flj * dz;
                        elj += (T)(4.0 * dp.lj_eps) * (s6 * s6 - s6 + (T)0.25);
                    }
                }
            }
        };
        for (int oz = -1; oz <= 1; oz++) {
            const int zc = cz + oz;
            if (zc < 0 || zc >= g.ncz) continue;
            for (int oy = -g.my; oy <= g.my; oy++) {
                const int yc = wrap_cell(cy + oy, g.ncy);
                for (int ox = -g.mx; ox <= g.mx; ox++) {
                    const int xc = wrap_cell(cx + ox, g.ncx);
                    const int cc = (zc * g.ncy + yc) * g.ncx + xc;
                    const T sx = (T)(ox * g.hx), sy = (T)(oy * g.hy), sz = (T)(oz * g.hz);
                    const long long home = (ox == 0 && oy == 0 && oz == 0) ? 1 : 0;
                    int m = start[cc];
                    int m1 = start[cc + 1];
                    if (m1 - m > budget) {  // bounded work per cell whatever the density
                        m1 = m + budget;
                        if (threadIdx.x == 0) atomicAdd(&status[ST_CELL], 1);
                    }
                    budget -= m1 - m;
                    while (m < m1) {
                        const int n = min(m1 - m, RS_CHUNK - fill);
                        for (int i = threadIdx.x; i < n; i += blockDim.x) {
                            V o = src[m + i];
                            o.x += sx; o.y += sy; o.z += sz;
                            buf[fill + i] = o;
                            kbuf[fill + i] = key[m + i] * 2 + home;
                        }
                        fill += n;
                        m += n;
                        if (fill == RS_CHUNK) {
                            __syncthreads();
                            process(fill);
                            __syncthreads();
                            fill = 0;
                        }
                    }
                }
            }
        }
        __syncthreads();
        process(fill);
        __syncthreads();
        if (active) {
            const int64_t j = key[b0 + t] >> 8;
            const T qi = me.w, kc = (T)dp.kc;
            force[3 * j + 0] += kc * qi * fx + lx;
            force[3 * j + 1] += kc * qi * fy + ly;
            force[3 * j + 2] += kc * qi * fz + lz;
            if (pot) phi[j] += kc * ph;
            e_local += 0.5 * (double)kc * (double)qi * (double)ph + 0.5 * (double)elj;
        }
    }
    if (!energy) return;
    // energy: fixed-order block sums, then the last CTA adds them in block order
    double v = e_local;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tsum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) tsum += red[w];
        epart[blockIdx.x] = tsum;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double tsum = cta_sum_ordered(epart, gridDim.x, red);
    if (threadIdx.x == 0) {
        scal[SC_UREAL] = tsum;
        *done = 0u;
    }
}

template <typename TIn>
cudaError_t launch_real_t(cudaStream_t st, const DevParams& dp, const CellGrid& g, const RealBuffers& rb,
                          int64_t N, const TIn* pos, const TIn* q, bool fp64, int* status) {
    cudaError_t e = cudaMemsetAsync(rb.count, 0, sizeof(int) * (size_t)g.ncell, st);
    if (e != cudaSuccess) return e;
    int64_t pbl = (N + 255) / 256;
    if (pbl < 1) pbl = 1;
    if (pbl > 4096) pbl = 4096;
    const int pb = (int)pbl;
    rs_count_kernel<TIn><<<pb, 256, 0, st>>>(dp, g, pos, q, N, rb.count);
    rs_scan_kernel<<<1, 1024, 0, st>>>(rb.count, g.ncell, rb.start, rb.fill);
    int64_t obl = ((int64_t)g.ncell * 32 + 255) / 256;
    if (obl > 8192) obl = 8192;
    const int ob = (int)obl;
    if (fp64) {
        rs_fill_kernel<TIn, double><<<pb, 256, 0, st>>>(dp, g, pos, q, N, rb.start, rb.fill, (double4*)rb.src,
                                                        rb.key);
        rs_order_kernel<double><<<ob, 256, 0, st>>>(g.ncell, rb.start, (const double4*)rb.src, rb.key,
                                                    (double4*)rb.src_sorted, rb.key_sorted, status);
    } else {
        rs_fill_kernel<TIn, float><<<pb, 256, 0, st>>>(dp, g, pos, q, N, rb.start, rb.fill, (float4*)rb.src,
                                                       rb.key);
        rs_order_kernel<float><<<ob, 256, 0, st>>>(g.ncell, rb.start, (const float4*)rb.src, rb.key,
                                                   (float4*)rb.src_sorted, rb.key_sorted, status);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launches(4);  // count, scan, fill, order
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_real(cudaStream_t st, const DevParams& dp, const CellGrid& g, const RealBuffers& rb, int64_t N,
                        const void* pos, const void* q, bool in_f32, bool fp64, void* force, void* phi, int pot,
                        int energy, double* scal, unsigned* done, int* status) {
    if (N <= 0) return cudaMemsetAsync(scal + SC_UREAL, 0, sizeof(double), st);
    cudaError_t e = in_f32 ? launch_real_t<float>(st, dp, g, rb, N, (const float*)pos, (const float*)q, fp64, status)
                           : launch_real_t<double>(st, dp, g, rb, N, (const double*)pos, (const double*)q, fp64,
                                                   status);
    if (e != cudaSuccess) return e;
    const bool lj = dp.lj_eps != 0.0 && dp.lj_sig2 > 0.0;
#define RS_LAUNCH(T, V, L)                                                                                      \
    rs_cell_kernel<T, L><<<g.ncell, RS_THREADS, 0, st>>>(dp, g, (const V*)rb.src_sorted, rb.key_sorted, rb.start, \
                                                         (T*)force, (T*)phi, pot, energy, rb.epart, scal, done,    \
                                                         status)
    if (fp64) {
        if (lj) RS_LAUNCH(double, double4, true);
        else RS_LAUNCH(double, double4, false);
    } else {
        if (lj) RS_LAUNCH(float, float4, true);
        else RS_LAUNCH(float, float4, false);
    }
#undef RS_LAUNCH
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rbe2d
