// Device helpers of the k sampler shared by the single-system and batched kernels:
// Philox4x64-10, the guide-table search of the per-dimension cumulative tables, and
// the per-k coefficients of the re-calibrated image series (Sec. 3.4).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "rbe2d_internal.h"

namespace rbe2d {
namespace kdetail {

constexpr double kTwoPiK = 6.283185307179586476925286766559;

// ---------------------------------------------------------------- per-k coefficients
// Fill one KCoef record for the index triple n: the wave vector, c = -coef/k^2 and the
// re-calibration factors of Sec. 3.4 for the reflection series truncated at M:
//   E(kz) = sum_{m=1}^{M/2} 2 (gt gb)^m Re(z^m)                                  (l = 2m)
//   O(kz) = sum_{m=0}^{(M-1)/2} [gt^{m+1} gb^m conj(z)^{m+1} + gb^{m+1} gt^m z^m]   (l = 2m+1)
// with z = e^{2 i kz H}, and their derivatives with respect to gt, gb.  The powers of z
// and of the contrasts are built by running products (one sincospi per k).
static __device__ __noinline__ void fill_kcoef(const DevParams& dp, int nx, int ny, int nz, KCoef* out) {
    KCoef r;
    r.nx = nx; r.ny = ny; r.nz = nz; r.ok = 1;
    r.kx = kTwoPiK * nx * dp.inv_Lx;
    r.ky = kTwoPiK * ny * dp.inv_Ly;
    r.kz = kTwoPiK * nz * dp.inv_Lz;
    double k2 = r.kx * r.kx + r.ky * r.ky + r.kz * r.kz;
    r.c = -dp.coef / k2;
    double E = 0, Ore = 0, Oim = 0, dEt = 0, dEb = 0, dOrt = 0, dOit = 0, dOrb = 0, dOib = 0;
    const double gt = dp.gt, gb = dp.gb;
    const double hz = (double)nz * (dp.H * dp.inv_Lz);  // kz H / (2 pi), in turns
    double s1, c1;
    sincospi(4.0 * hz, &s1, &c1);  // z = e^{2 i kz H}
    double zr = 1.0, zi = 0.0;     // z^m
    double ptm = 1.0, pbm = 1.0;   // gt^m, gb^m
    double ptm1 = 0.0, pbm1 = 0.0; // gt^(m-1), gb^(m-1) (only used multiplied by m)
    for (int m = 0; 2 * m <= dp.M; m++) {
        const double nr = zr * c1 - zi * s1, ni = zr * s1 + zi * c1;  // z^(m+1)
        if (m >= 1) {
            E += 2.0 * ptm * pbm * zr;
            dEt += 2.0 * m * ptm1 * pbm * zr;
            dEb += 2.0 * m * ptm * pbm1 * zr;
        }
        if (2 * m + 1 <= dp.M) {
            const double a1 = ptm * gt * pbm, a2 = pbm * gb * ptm;
            Ore += a1 * nr + a2 * zr;
            Oim += -a1 * ni + a2 * zi;
            const double a1t = (m + 1) * ptm * pbm, a1b = m * ptm * gt * pbm1;
            const double a2t = m * pbm * gb * ptm1, a2b = (m + 1) * pbm * ptm;
            dOrt += a1t * nr + a2t * zr;
            dOit += -a1t * ni + a2t * zi;
            dOrb += a1b * nr + a2b * zr;
            dOib += -a1b * ni + a2b * zi;
        }
        ptm1 = ptm; pbm1 = pbm;
        ptm *= gt; pbm *= gb;
        zr = nr; zi = ni;
    }
    r.E = E; r.Ore = Ore; r.Oim = Oim;
    r.dE_t = dEt; r.dE_b = dEb; r.dOre_t = dOrt; r.dOim_t = dOit; r.dOre_b = dOrb; r.dOim_b = dOib;
    *out = r;
}

// The nine image-series sums of one kz (E, Re O, Im O and their gt, gb derivatives)
// split over a segment of W lanes (W a power of two dividing 32; lane m of the segment
// takes the terms m, m + W, ..., each from its own sincospi and contrast powers), added
// over the segment in a fixed shuffle order; the segment's lane 0 holds the totals in v.
// Every lane of the warp must call it (the shuffles span the warp).  On GB300 a float64
// instruction costs its scheduler the same time for one lane as for 32, so a warp serves
// 32 / W values of kz with each of its float64 instructions.
static __device__ __forceinline__ void image_series_seg(const DevParams& dp, int nz, int W, double v[9]) {
    const int sl = threadIdx.x & (W - 1);
    const double gt = dp.gt, gb = dp.gb;
    const double hz = (double)nz * (dp.H * dp.inv_Lz);  // kz H / (2 pi), in turns
    for (int c = 0; c < 9; c++) v[c] = 0.0;  // E, Ore, Oim, dEt, dEb, dOrt, dOit, dOrb, dOib
    for (int m = sl; 2 * m <= dp.M; m += W) {
        double ptm = 1.0, pbm = 1.0, ptm1 = 0.0, pbm1 = 0.0;
        for (int i = 0; i < m; i++) { ptm1 = ptm; pbm1 = pbm; ptm *= gt; pbm *= gb; }
        double zi, zr, ni, nr;
        sincospi(4.0 * hz * m, &zi, &zr);        // z^m, z = e^{2 i kz H}
        sincospi(4.0 * hz * (m + 1), &ni, &nr);  // z^(m+1)
        if (m >= 1) {
            v[0] += 2.0 * ptm * pbm * zr;
            v[3] += 2.0 * m * ptm1 * pbm * zr;
            v[4] += 2.0 * m * ptm * pbm1 * zr;
        }
        if (2 * m + 1 <= dp.M) {
            const double a1 = ptm * gt * pbm, a2 = pbm * gb * ptm;
            v[1] += a1 * nr + a2 * zr;
            v[2] += -a1 * ni + a2 * zi;
            const double a1t = (m + 1) * ptm * pbm, a1b = m * ptm * gt * pbm1;
            const double a2t = m * pbm * gb * ptm1, a2b = (m + 1) * pbm * ptm;
            v[5] += a1t * nr + a2t * zr;
            v[6] += -a1t * ni + a2t * zi;
            v[7] += a1b * nr + a2b * zr;
            v[8] += -a1b * ni + a2b * zi;
        }
    }
#pragma unroll
    for (int c = 0; c < 9; c++)
        for (int o = W >> 1; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o, W);
}

// One KCoef record from the wave-vector indices, c = -cnum / k^2 and the nine image-series
// sums v (one lane); a zero record when !valid.
static __device__ __forceinline__ void kcoef_record(const DevParams& dp, int nx, int ny, int nz, double cnum,
                                                    const double* v, bool valid, KCoef* out) {
    KCoef r = {};
    if (valid) {
        r.nx = nx; r.ny = ny; r.nz = nz; r.ok = 1;
        r.kx = kTwoPiK * nx * dp.inv_Lx;
        r.ky = kTwoPiK * ny * dp.inv_Ly;
        r.kz = kTwoPiK * nz * dp.inv_Lz;
        r.c = -cnum / (r.kx * r.kx + r.ky * r.ky + r.kz * r.kz);
        r.E = v[0]; r.Ore = v[1]; r.Oim = v[2];
        r.dE_t = v[3]; r.dE_b = v[4]; r.dOre_t = v[5]; r.dOim_t = v[6]; r.dOre_b = v[7]; r.dOim_b = v[8];
    }
    *out = r;
}

// The record with the series computed by a segment of W lanes (see image_series_seg);
// the segment's lane 0 writes *out (NULL: nothing).
static __device__ __noinline__ void fill_kcoef_seg(const DevParams& dp, int nx, int ny, int nz, double cnum, int W,
                                                   KCoef* out, bool valid) {
    double v[9];
    image_series_seg(dp, nz, W, v);
    if ((threadIdx.x & (W - 1)) == 0 && out) kcoef_record(dp, nx, ny, nz, cnum, v, valid, out);
}

// The record with the series read from the per-kz table built at set-up (row nz + half,
// nine float64).  A kz outside the table (a Metropolis chain started outside the box)
// takes the one-thread series instead, with c = -coef / k^2.  One lane.
static __device__ __forceinline__ void fill_kcoef_row(const DevParams& dp, const double* __restrict__ eo, int half,
                                                      int nx, int ny, int nz, double cnum, KCoef* out, bool valid) {
    if (valid && (nz < -half || nz > half)) {
        fill_kcoef(dp, nx, ny, nz, out);
        return;
    }
    double v[9];
    const double* row = eo + (size_t)((valid ? nz : 0) + half) * 9;
    for (int c = 0; c < 9; c++) v[c] = row[c];
    kcoef_record(dp, nx, ny, nz, cnum, v, valid, out);
}

// First index whose cumulative value exceeds u.  guide[g] is the first index whose value
// exceeds g/len.  With g = floor(u len) (the product may round across an integer by one),
// the answer lies in [guide[g-1], guide[g+2]]: the entry before guide[g-1] is at most
// (g-1)/len <= u and the entry at guide[g+2] exceeds (g+2)/len > u (the last entry is 1 > u).
// A binary search there needs at most log2(len) + 1 dependent loads, also in the flat
// tails of the distribution where one bucket spans hundreds of entries.
static __device__ __forceinline__ int first_above(const double* __restrict__ cdf, const int* __restrict__ guide, int len,
                                           double u) {
    int g = (int)(u * (double)len);
    if (g >= len) g = len - 1;
    if (g < 0) g = 0;
    int lo = guide[g > 0 ? g - 1 : 0];
    int hi = g + 2 < len ? guide[g + 2] : len - 1;
    while (lo < hi) {  // first index in [lo, hi] with cdf > u; cdf[hi] > u
        const int mid = (lo + hi) >> 1;
        if (cdf[mid] > u) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Philox4x64-10 (Salmon et al., SC'11): 10 rounds of the 4x64 S-box with the Weyl key
// schedule.
static __device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += W0; k1 += W1; }
        unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

}  // namespace kdetail
}  // namespace rbe2d
