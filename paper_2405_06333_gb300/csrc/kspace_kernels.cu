// k-space kernels of the RBE2D force (sm_103a).
//
// One force evaluation is: sample (or set) the batch -> pack -> structure factor ->
// fold -> finalize -> force (the last in force_kernels.cu).  The path is bound by sin/cos issue (MUFU) and FP32
// issue, not by HBM or tensor cores: every (particle, k) pair costs one sincos per
// angle and a few FMAs, and there is no dense contraction to put on tcgen05.
//
// Exact phase reduction: coordinates are packed once into fixed-point fractions
// u = frac(x/L) 2^32 (FP64 mode: 2^64), so k.r / 2pi mod 1 = (nx ux + ny uy + nz uz) / 2^32
// is computed exactly in wrapping integer arithmetic; only the final turn -> radians
// conversion and the sin/cos are rounded.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kcoef.cuh"
#include "pair32.cuh"
#include "phase.cuh"
#include "rbe2d_internal.h"
#include "sf32.cuh"

namespace rbe2d {

namespace {

using kdetail::fill_kcoef;
using kdetail::philox4x64_10;
using pair32::sincos_turn32x2;
using phase::sincos_poly32;
using phase::sincos_turn32;
using phase::sincos_turn64;
using sf32k::block_pack_sums;
using sf32k::dkey;
using sf32k::dunkey;
using sf32k::cp_async_commit;
using sf32k::cp_async_wait;
using sf32k::sf32_kernel;


// ---------------------------------------------------------------- small helpers
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
constexpr int SAMPLE_WAYS = 10;  // lanes per table search: ten probes, an 11-way split

// Bits of the float64 m 2^-53 for m < 2^53, by integer operations: m converts exactly and
// the scaling only lowers the exponent, so this equals (double)m * 0x1p-53 (float64
// instructions take 64 cycles each on this part; these are a few integer ones).
__device__ __forceinline__ unsigned long long u53_bits(unsigned long long m) {
    if (m == 0ull) return 0ull;
    const int e = 63 - __clzll((long long)m);  // position of the leading one, 0..52
    const unsigned long long mant = (m << (52 - e)) & ((1ull << 52) - 1ull);
    return ((unsigned long long)(1023 - 53 + e) << 52) | mant;
}

// One warp per wave vector.  Every lane runs Philox4x64-10 on counter (l, attempt, step, 0)
// and key (seed, 0); u_d = (word_d >> 11) 2^-53 (Sec. 2.3's draw from the product of the
// three 1-D factors by inverse CDF).  Lanes 10 d .. 10 d + 9 find the first entry of
// table d whose cumulative value exceeds u_d together: starting from the guide-table
// bracket, each step probes ten evenly spaced entries of [lo, hi] at once and keeps the
// sub-range where the table first exceeds u_d (about three dependent loads instead of a
// binary search's ten).  Non-negative float64 values order like their bit patterns, so
// the comparisons are integer ones.  k = 0 is rejected up to 64 times; lane 0 then reads
// the image-series sums of the drawn kz from the set-up table and writes the record.
__global__ void __launch_bounds__(128) sample_kernel(DevParams dp, SamplerTables tb, unsigned long long seed,
                                                     unsigned long long step_arg,
                                                     const unsigned long long* __restrict__ step_dev,
                                                     KCoef* __restrict__ kc, int32_t* __restrict__ kidx_out,
                                                     int* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int l = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);  // this warp's k slot
    if (l >= dp.P_pad) return;                                          // the whole warp
    const unsigned long long step = step_dev ? *step_dev : step_arg;
    const bool real = l < dp.P;  // slots [P, P_pad) get zero records
    const int d = lane < 3 * SAMPLE_WAYS ? lane / SAMPLE_WAYS : 2;  // lanes 30, 31 repeat lane 29
    const int sp = lane < 3 * SAMPLE_WAYS ? lane - SAMPLE_WAYS * d : SAMPLE_WAYS - 1;
    const double* cdf = tb.cdf[d];
    const int* guide = tb.guide[d];
    const int len = tb.len[d];
    int n[3] = {1, 0, 0};
    bool ok = !real;
    for (int a = 0; a < 64 && !ok; a++) {  // warp-uniform: every lane holds the same draw
        unsigned long long c[4] = {(unsigned long long)l, (unsigned long long)a, step, 0ULL};
        philox4x64_10(c, seed, 0ULL);
        const unsigned long long m = (d == 0 ? c[0] : (d == 1 ? c[1] : c[2])) >> 11;
        const long long ub = (long long)u53_bits(m);
        // bracket: g = floor(u len) exactly; the answer lies in [guide[g-1], guide[g+2]]
        const int g = (int)__umul64hi(m << 11, (unsigned long long)len);
        int lo = guide[g > 0 ? g - 1 : 0];
        int hi = g + 2 < len ? guide[g + 2] : len - 1;
        for (int it = 0; it < 32; it++) {  // each step shrinks hi - lo about elevenfold
            const bool active = lo < hi;
            if (!__any_sync(0xffffffffu, active)) break;
            const int r = hi - lo;
            const int p = lo + (int)(((long long)r * (sp + 1)) / (SAMPLE_WAYS + 1));
            const bool above = active && __double_as_longlong(cdf[p]) > ub;
            const unsigned bits = (__ballot_sync(0xffffffffu, above) >> (SAMPLE_WAYS * d)) & ((1u << SAMPLE_WAYS) - 1u);
            if (active) {
                if (bits) {  // probe f is the first above u: the answer is in (probe f-1, probe f]
                    const int f = __ffs(bits) - 1;
                    const int pf = lo + (int)(((long long)r * (f + 1)) / (SAMPLE_WAYS + 1));
                    if (f > 0) lo = lo + (int)(((long long)r * f) / (SAMPLE_WAYS + 1)) + 1;
                    hi = pf;
                } else {  // every probe at or below u: the answer is past the last one
                    lo = lo + (int)(((long long)r * SAMPLE_WAYS) / (SAMPLE_WAYS + 1)) + 1;
                }
            }
        }
        const int mine = lo - len / 2;
        const int ix = __shfl_sync(0xffffffffu, mine, 0);
        const int iy = __shfl_sync(0xffffffffu, mine, SAMPLE_WAYS);
        const int iz = __shfl_sync(0xffffffffu, mine, 2 * SAMPLE_WAYS);
        if (ix != 0 || iy != 0 || iz != 0) {
            n[0] = ix; n[1] = iy; n[2] = iz;
            ok = true;
        }
    }
    if (lane != 0) return;
    if (real) {
        if (!ok) atomicAdd(&status[ST_SAMPLER], 1);
        if (kidx_out) {
            kidx_out[3 * l] = n[0]; kidx_out[3 * l + 1] = n[1]; kidx_out[3 * l + 2] = n[2];
        }
    }
    // the image-series sums of the drawn kz come from the set-up table
    kdetail::fill_kcoef_row(dp, tb.eo, tb.eo_half, n[0], n[1], n[2], dp.coef, &kc[l], real);
}

// Set-up: the nine image-series sums for every kz index of the sampler's table box, one
// segment of dp.kseg lanes per kz (the same arithmetic as a per-draw evaluation).
__global__ void eo_table_kernel(DevParams dp, int half, double* __restrict__ eo) {
    const int W = dp.kseg, lane = threadIdx.x & 31;
    const int r = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / W) + lane / W;  // table row
    const int nz = min(r, 2 * half) - half;
    double v[9];
    kdetail::image_series_seg(dp, nz, W, v);
    if ((lane & (W - 1)) == 0 && r <= 2 * half)
        for (int c = 0; c < 9; c++) eo[(size_t)r * 9 + c] = v[c];
}

// Metropolis variant of the sampler (Sec. 2.3 names a Metropolis procedure; the
// proposal is this library's reading): chain l is a random walk on Z^3 \ {0} inside the
// table box, proposal n' = n + delta with delta_d uniform on {-hw_d, ..., hw_d}, accepted
// when u w(n) < w(n'), w the product of the three 1-D factors (0 at k = 0 and outside
// the box).  Update `it` of step `step` uses Philox4x64-10 with counter
// (l, it, step, 1) and key (seed, 0): delta_d from the top 32 bits of word d by a
// multiply-shift, u = (word_3 >> 11) 2^-53.  Lane 0 of a warp runs the chain; the warp
// then fills the batch record like the i.i.d. sampler.
__device__ __forceinline__ double mh_weight(const SamplerTables& tb, int nx, int ny, int nz) {
    const int hx = tb.len[0] / 2, hy = tb.len[1] / 2, hz = tb.len[2] / 2;
    if ((nx | ny | nz) == 0) return 0.0;
    if (nx < -hx || nx > hx || ny < -hy || ny > hy || nz < -hz || nz > hz) return 0.0;
    return tb.w[0][nx + hx] * tb.w[1][ny + hy] * tb.w[2][nz + hz];
}

__global__ void metropolis_kernel(DevParams dp, SamplerTables tb, unsigned long long seed, unsigned long long step,
                                  int sweeps, int32_t* __restrict__ state, KCoef* __restrict__ kc,
                                  int32_t* __restrict__ kidx_out, unsigned long long* __restrict__ accepted) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;  // one chain per thread
    const bool real = l < dp.P;
    int n[3] = {1, 0, 0};
    if (real) {
        n[0] = state[3 * l]; n[1] = state[3 * l + 1]; n[2] = state[3 * l + 2];
        double wn = mh_weight(tb, n[0], n[1], n[2]);
        unsigned long long acc = 0;
        for (int it = 0; it < sweeps; it++) {
            unsigned long long c[4] = {(unsigned long long)l, (unsigned long long)it, step, 1ULL};
            philox4x64_10(c, seed, 0ULL);
            int m[3];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const unsigned long long span = (unsigned long long)(2 * tb.hw[d] + 1);
                m[d] = n[d] + (int)(((c[d] >> 32) * span) >> 32) - tb.hw[d];
            }
            const double u = (double)(c[3] >> 11) * 0x1p-53;
            const double wm = mh_weight(tb, m[0], m[1], m[2]);
            if (u * wn < wm) {
                n[0] = m[0]; n[1] = m[1]; n[2] = m[2];
                wn = wm;
                acc++;
            }
        }
        state[3 * l] = n[0]; state[3 * l + 1] = n[1]; state[3 * l + 2] = n[2];
        if (kidx_out) {
            kidx_out[3 * l] = n[0]; kidx_out[3 * l + 1] = n[1]; kidx_out[3 * l + 2] = n[2];
        }
        if (accepted && acc) atomicAdd(accepted, acc);
    }
    if (l < dp.P_pad) kdetail::fill_kcoef_row(dp, tb.eo, tb.eo_half, n[0], n[1], n[2], dp.coef, &kc[l], real);
}

// Deterministic lattice sum (the k-space sum of Eq. 3.16 over every k != 0 of a box
// |n_d| <= nm[d], the quantity the random batch estimates): slot l holds entry t0 + l of
// the half lattice, the indices above (0, 0, 0) in the lexicographic order of
// (nz, ny, nx).  k and -k give the same real term (reading A13), so each half-lattice
// entry carries the weight 2 w(k), w(k) = exp(-k^2/4alpha^2) (Eq. 2.21), in place of S/P.
// Slots past the end of the half lattice get weight 0.  One warp per slot.
__global__ void lattice_k_kernel(DevParams dp, int nmx, int nmy, int nmz, long long t0, long long n_half,
                                 KCoef* __restrict__ kc) {
    const int W = dp.kseg, lane = threadIdx.x & 31;
    const int l = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / W) + lane / W;  // this segment's slot
    const bool real = l < dp.P;
    const long long t = t0 + l;
    int nx = 1, ny = 0, nz = 0;
    double cnum = 0.0;
    if (real && t < n_half) {
        const long long wx = 2LL * nmx + 1, wy = 2LL * nmy + 1;
        long long u = n_half + 1 + t;  // n_half is the lexicographic index of (0, 0, 0)
        nx = (int)(u % wx) - nmx;
        u /= wx;
        ny = (int)(u % wy) - nmy;
        nz = (int)(u / wy) - nmz;
        const double kx = kdetail::kTwoPiK * nx * dp.inv_Lx, ky = kdetail::kTwoPiK * ny * dp.inv_Ly;
        const double kz = kdetail::kTwoPiK * nz * dp.inv_Lz;
        const double k2 = kx * kx + ky * ky + kz * kz;
        cnum = 2.0 * dp.coef_unit * exp(-k2 / (4.0 * dp.alpha * dp.alpha));
    }
    kdetail::fill_kcoef_seg(dp, nx, ny, nz, cnum, W, l < dp.P_pad ? &kc[l] : nullptr, real);
}

__global__ void accum_uk_kernel(double* __restrict__ scal, int first, int last) {
    if (threadIdx.x == 0) {
        const double a = (first ? 0.0 : scal[SC_UK_ACC]) + scal[SC_UK];
        scal[SC_UK_ACC] = a;
        if (last) scal[SC_UK] = a;
    }
}

__global__ void set_k_kernel(DevParams dp, const int32_t* __restrict__ kidx, KCoef* __restrict__ kc,
                             int* __restrict__ status) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= dp.P_pad) return;
    if (l >= dp.P) {
        KCoef z = {};
        kc[l] = z;
        return;
    }
    int nx = kidx[3 * l], ny = kidx[3 * l + 1], nz = kidx[3 * l + 2];
    if (nx == 0 && ny == 0 && nz == 0) {  // k = 0 is not part of the sum: flag it, keep finite
        atomicAdd(&status[ST_SAMPLER], 1);
        nx = 1;
    }
    fill_kcoef(dp, nx, ny, nz, &kc[l]);
}

// ---------------------------------------------------------------- pack (a3)
template <typename TIn, bool FP64>
__global__ void __launch_bounds__(256) pack_kernel(DevParams dp, int64_t N, const TIn* __restrict__ pos,
                                                   const TIn* __restrict__ q, void* __restrict__ part,
                                                   double* __restrict__ pack_part) {
    double sQ = 0, sQ2 = 0, sMu = 0, sQa = 0, zmin = 1e300, zmax = -1e300;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double x = (double)pos[3 * i], y = (double)pos[3 * i + 1], z = (double)pos[3 * i + 2];
        double qi = (double)q[i];
        double fx = x * dp.inv_Lx; fx -= floor(fx);
        double fy = y * dp.inv_Ly; fy -= floor(fy);
        double fz = z * dp.inv_Lz; fz -= floor(fz);
        if (FP64) {
            Part64 p;
            p.ux = __double2ull_rz(fx * 18446744073709551616.0);
            p.uy = __double2ull_rz(fy * 18446744073709551616.0);
            p.uz = __double2ull_rz(fz * 18446744073709551616.0);
            p.q = qi;
            reinterpret_cast<Part64*>(part)[i] = p;
        } else {
            uint4 p;
            p.x = (uint32_t)(unsigned long long)__double2ll_rn(fx * 4294967296.0);
            p.y = (uint32_t)(unsigned long long)__double2ll_rn(fy * 4294967296.0);
            p.z = (uint32_t)(unsigned long long)__double2ll_rn(fz * 4294967296.0);
            p.w = __float_as_uint((float)qi);
            reinterpret_cast<uint4*>(part)[i] = p;
        }
        sQ += qi; sQ2 += qi * qi; sMu += qi * z; sQa += fabs(qi);
        zmin = fmin(zmin, z); zmax = fmax(zmax, z);
    }
    block_pack_sums(sQ, sQ2, sMu, sQa, zmin, zmax, pack_part + (size_t)blockIdx.x * PACK_STRIDE);
}

// ---------------------------------------------------------------- structure factor (a4)
// The FP32-mixed kernel, sf32_kernel, is in sf32.cuh; the FP64 kernel follows.

constexpr int SF_TILE64 = 256;
constexpr int SF_KR64 = 2;

template <bool SIG>
__global__ void __launch_bounds__(128) sf64_kernel(const Part64* __restrict__ part, int64_t N,
                                                   const KCoef* __restrict__ kc, int P,
                                                   double* __restrict__ sf_part, int nblk) {
    __shared__ Part64 tile[2][SF_TILE64];
    const int KT = blockDim.x;
    const int kbase = blockIdx.y * KT * SF_KR64;
    long long nx[SF_KR64], ny[SF_KR64], nz[SF_KR64];
#pragma unroll
    for (int j = 0; j < SF_KR64; j++) {
        int k = kbase + threadIdx.x + j * KT;
        if (k < P) { nx[j] = kc[k].nx; ny[j] = kc[k].ny; nz[j] = kc[k].nz; }
        else { nx[j] = 0; ny[j] = 0; nz[j] = 0; }
    }
    const int64_t b = blockIdx.x;
    const int64_t p0 = (N * b) / nblk, p1 = (N * (b + 1)) / nblk;
    const int64_t ntiles = (p1 - p0 + SF_TILE64 - 1) / SF_TILE64;
    double ar[SF_KR64], ai[SF_KR64], br[SF_KR64], bi[SF_KR64];
#pragma unroll
    for (int j = 0; j < SF_KR64; j++) ar[j] = ai[j] = br[j] = bi[j] = 0.0;
    auto issue = [&](int64_t t) {
        int64_t s = p0 + t * SF_TILE64;
        int n = (int)min((int64_t)SF_TILE64, p1 - s);
        Part64* dst = tile[t & 1];
        for (int i = threadIdx.x; i < 2 * n; i += KT)
            cp_async16(reinterpret_cast<uint4*>(dst) + i, reinterpret_cast<const uint4*>(part + s) + i);
        cp_async_commit();
    };
    if (ntiles > 0) issue(0);
    for (int64_t t = 0; t < ntiles; t++) {
        if (t + 1 < ntiles) { issue(t + 1); cp_async_wait<1>(); }
        else { cp_async_wait<0>(); }
        __syncthreads();
        const int n = (int)min((int64_t)SF_TILE64, p1 - (p0 + t * SF_TILE64));
        const Part64* tb = tile[t & 1];
        for (int p = 0; p < n; p++) {
            const Part64 u = tb[p];
#pragma unroll
            for (int j = 0; j < SF_KR64; j++) {
                const unsigned long long txy = (unsigned long long)nx[j] * u.ux + (unsigned long long)ny[j] * u.uy;
                const unsigned long long tz = (unsigned long long)nz[j] * u.uz;
                double s1, c1;
                sincos_turn64(txy + tz, &s1, &c1);
                ar[j] = fma(u.q, c1, ar[j]);
                ai[j] = fma(u.q, s1, ai[j]);
                if (SIG) {
                    double s2, c2;
                    sincos_turn64(txy - tz, &s2, &c2);
                    br[j] = fma(u.q, c2, br[j]);
                    bi[j] = fma(u.q, s2, bi[j]);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < SF_KR64; j++) {
        int k = kbase + threadIdx.x + j * KT;
        if (k < P) {
            double* o = sf_part + ((size_t)k * nblk + b) * 4;
            o[0] = ar[j]; o[1] = ai[j]; o[2] = br[j]; o[3] = bi[j];
        }
    }
}

// ---------------------------------------------------------------- fold (a5) + finalize
// Fixed-order sums over k and over the pack partials; energies and IBC factors
// (Eq. 3.18, general form):  U_IBC = (2pi/V) kc mu (cM mu + Q H dM).  Called by one CTA.
constexpr int FOLD_THREADS = 128;  // one CTA per k
constexpr int FIN_VALUES = 7;      // shared-memory rows of the trees (fold: 4, finalize: 7)

// -x by flipping the sign bit (integer pipe; float64 instructions are scarce on GB300)
__device__ __forceinline__ double neg(double x) { return __longlong_as_double(__double_as_longlong(x) ^ (1LL << 63)); }

// Sum the FOLD_THREADS values of rows 0 .. nv-1 of S into S[c][0], in a fixed binary tree
// whose levels spread all additions of all rows over the threads: each float64
// instruction adds for as many lanes as there are pairs left.  All threads call it.
__device__ __forceinline__ void tree_sum(double (*S)[FOLD_THREADS], int nv) {
    for (int h = FOLD_THREADS / 2; h > 0; h >>= 1) {
        for (int i = threadIdx.x; i < nv * h; i += FOLD_THREADS) {
            const int c = i / h, j = i - c * h;
            S[c][j] += S[c][j + h];
        }
        // threads below nv * h wrote this level: beyond warp 0 the block must sync
        if (nv * h > 32) __syncthreads();
        else __syncwarp();
    }
}

// Pack rows summed in groups of 32 by the fold CTAs: one row per group, six values
// (sum q, sum q^2, sum q z, sum |q|, min z, max z), fixed order.
constexpr int PACK_GROUP = 32;

__device__ void reduce_pack_group(const double* __restrict__ pack_part, int pack_blocks, int g,
                                  double* __restrict__ pack2) {
    const int lane = threadIdx.x & 31;
    const int b = g * PACK_GROUP + lane;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0, mn = 1e300, mx = -1e300;
    if (b < pack_blocks) {
        const double* o = pack_part + (size_t)b * PACK_STRIDE;
        s0 = __ldcg(&o[0]); s1 = __ldcg(&o[1]); s2 = __ldcg(&o[2]); s3 = __ldcg(&o[3]);
        mn = __ldcg(&o[4]); mx = __ldcg(&o[5]);
    }
    const double v = sf32k::warp_sums4(s0, s1, s2, s3);
    long long kmn, kmx;
    sf32k::warp_minmax(mn, mx, &kmn, &kmx);
    double* o = pack2 + (size_t)g * PACK_STRIDE;
    if ((lane & 7) == 0) o[lane >> 3] = v;  // the four sums (lanes 0, 8, 16, 24)
    if (lane == 0) { o[4] = sf32k::dunkey(kmn); o[5] = sf32k::dunkey(kmx); }
}


// Totals of one evaluation: k-space energy and its gamma derivatives over the P k-terms,
// charge sums over the pack groups (fixed shared-memory tree), z extrema through integer
// keys, then the energies and IBC factors from host-side constants.  All threads call
// it; the lanes of warp 0 write scal.
__device__ void finalize_block(const DevParams& dp, const double* __restrict__ pack2, int ngroups,
                               const double* __restrict__ kterm, double* __restrict__ scal,
                               double (*S)[FOLD_THREADS]) {
    __shared__ long long zk[FOLD_THREADS / 32][2];
    double v[7] = {0, 0, 0, 0, 0, 0, 0};  // u, gt, gb, Q, Q2, mu, Qa
    long long kmin = 0x7fffffffffffffffLL, kmax = -0x7fffffffffffffffLL - 1;
    // the k-terms of this thread: the first four rows loaded before any is added (one
    // memory round trip instead of four), the same order of additions
    double kt[4][3];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int l = threadIdx.x + i * FOLD_THREADS;
#pragma unroll
        for (int c = 0; c < 3; c++) kt[i][c] = l < dp.P ? __ldcg(&kterm[3 * l + c]) : 0.0;
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
        if (threadIdx.x + i * FOLD_THREADS < dp.P) { v[0] += kt[i][0]; v[1] += kt[i][1]; v[2] += kt[i][2]; }
    for (int l = threadIdx.x + 4 * FOLD_THREADS; l < dp.P; l += FOLD_THREADS) {
        v[0] += __ldcg(&kterm[3 * l]); v[1] += __ldcg(&kterm[3 * l + 1]); v[2] += __ldcg(&kterm[3 * l + 2]);
    }
    for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
        const double* o = pack2 + (size_t)g * PACK_STRIDE;
        v[3] += __ldcg(&o[0]); v[4] += __ldcg(&o[1]); v[5] += __ldcg(&o[2]); v[6] += __ldcg(&o[3]);
        kmin = min(kmin, dkey(__ldcg(&o[4]))); kmax = max(kmax, dkey(__ldcg(&o[5])));
    }
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_down_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_down_sync(0xffffffffu, kmax, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { zk[warp][0] = kmin; zk[warp][1] = kmax; }
    for (int c = 0; c < 7; c++) S[c][threadIdx.x] = v[c];
    __syncthreads();
    tree_sum(S, 7);
    if (threadIdx.x >= 32) return;
    kmin = zk[0][0];
    kmax = zk[0][1];
    for (int w = 1; w < FOLD_THREADS / 32; w++) {
        kmin = min(kmin, zk[w][0]);
        kmax = max(kmax, zk[w][1]);
    }
    // The outputs in one instruction stream, lane j writing scal[j]: with
    //   inner = cM mu + Q H dM  (sum_j q_j Z_j),  t_j = X_j mu + Z_j W_j Y_j,
    // every derived slot is base_j + M_j t_j (pre = 2 pi kc / V):
    //   SC_USELF = self_c Q2                        (X = 0, Z W Y = Q2)
    //   SC_UIBC = pre mu inner                      (X = cM, Z W Y = Q H dM)
    //   SC_FIBC = -pre (cM mu + inner),  SC_DQ_IBC_Z = pre (cM mu + inner)   (X = 2 cM)
    //   SC_DQ_IBC_C = pre mu H dM                   (X = 0, Z W Y = H dM)
    //   SC_DG_t/b = g_t/b + pre mu (dcM mu + Q H ddM)
    // and the rest are copies (U_k, Q, Q2, mu, sum|q|, the z range, U_real = 0).
    const double u = S[0][0], gt = S[1][0], gb = S[2][0], Q = S[3][0], Q2 = S[4][0], mu = S[5][0], Qa = S[6][0];
    const double pre = dp.coef_unit;
    const int j = threadIdx.x;
    const bool tb = j == SC_DG_B;
    const double X = (j == SC_UIBC) ? dp.cM : (j == SC_FIBC || j == SC_DQ_IBC_Z) ? 2.0 * dp.cM
                     : (j == SC_DG_T || j == SC_DG_B) ? (tb ? dp.dcM_b : dp.dcM_t) : 0.0;
    const double Z = j == SC_USELF ? Q2 : (j == SC_DQ_IBC_C ? 1.0 : Q);
    const double W = j == SC_USELF ? 1.0 : dp.H;
    const double Y = j == SC_USELF ? 1.0 : (j == SC_DG_T || j == SC_DG_B) ? (tb ? dp.ddM_b : dp.ddM_t) : dp.dM;
    const double M = j == SC_USELF ? dp.self_c : (j == SC_FIBC ? neg(pre) : (j == SC_DQ_IBC_Z ? pre : pre * mu));
    const double base = j == SC_DG_T ? gt : (j == SC_DG_B ? gb : 0.0);
    const double t = fma(X, mu, Z * W * Y);
    double out = fma(M, t, base);
    out = j == SC_UK ? u : j == SC_Q ? Q : j == SC_Q2 ? Q2 : j == SC_MU ? mu : j == SC_QABS ? Qa : out;
    out = j == SC_ZMIN ? dunkey(kmin) : j == SC_ZMAX ? dunkey(kmax) : j == SC_UREAL ? 0.0 : out;
    if (j <= SC_ZMAX) scal[j] = out;  // a real-space pass on these particles sets SC_UREAL afterwards
}

// One CTA per k: fixed-order strided sums of the per-chunk partials and a fixed
// shared-memory tree, then warp 0 computes per k
//   A = (2 + 2E) rho + conj(O) sigma,  B = O rho          (Eq. 3.25 via Sec. 3.4)
//   U term  = -c [(1+E)|rho|^2 + Re(O rho conj(sigma))]   (Eq. 3.16)
//   dU/dgamma terms with dE, dO in place of E, O,
// while warp 1 of the first CTAs reduces the pack rows in groups of 32.  The last CTA to
// finish (counted in `done`) runs the finalize step and re-arms the counter, so every
// launch leaves it at zero.  Float64 instructions take 64 cycles each on GB300 (one
// warp, dependent or not), so the per-k and final outputs are computed by lanes side by
// side in one short instruction stream rather than by one thread in turn.

__global__ void __launch_bounds__(FOLD_THREADS) fold_kernel(DevParams dp, const double* __restrict__ sf_part,
                                                               int nblk, const KCoef* __restrict__ kc, int fp64,
                                                               double* __restrict__ rs, double* __restrict__ kterm,
                                                               void* __restrict__ krec,
                                                               const double* __restrict__ pack_part, int pack_blocks,
                                                               double* __restrict__ pack2, double* __restrict__ scal,
                                                               unsigned* __restrict__ done) {
    __shared__ double S[FIN_VALUES][FOLD_THREADS];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int l = blockIdx.x;
    // the coefficients of this k (15 words of 8 bytes) copied to shared memory by warp 3
    // under the partial sums (cp.async: no register waits for them); the tree's first
    // barrier publishes them to warp 0
    __shared__ __align__(16) KCoef kq;
    static_assert(sizeof(KCoef) == 120, "KCoef is 15 words of 8 bytes");
    static_assert(FOLD_THREADS >= 128, "warp 3 stages the coefficients, warp 1 the pack rows");
    if (warp == 3 && lane < 15)
        sf32k::cp_async_small<8>(reinterpret_cast<unsigned long long*>(&kq) + lane,
                                 reinterpret_cast<const unsigned long long*>(kc + l) + lane);
    sf32k::cp_async_commit();
    const int j = lane;
    const int ngroups = (pack_blocks + PACK_GROUP - 1) / PACK_GROUP;
    {
        // thread t adds partials t, t + 128, ... (all loads issued before the adds); the
        // 128 per-thread sums of each component then go through a fixed shared-memory tree
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        const double2* base = reinterpret_cast<const double2*>(sf_part + (size_t)l * nblk * 4);
#pragma unroll 8
        for (int b = threadIdx.x; b < nblk; b += FOLD_THREADS) {
            const double2 u = base[2 * b], v = base[2 * b + 1];
            a0 += u.x; a1 += u.y; a2 += v.x; a3 += v.y;
        }
        S[0][threadIdx.x] = a0; S[1][threadIdx.x] = a1; S[2][threadIdx.x] = a2; S[3][threadIdx.x] = a3;
        sf32k::cp_async_wait<0>();
        __syncthreads();
        tree_sum(S, 4);
        if (warp == 0) {
            // the seven outputs of this k in one instruction stream, lane j computing
            //   scale_j (A_j u_j + B_j v_j + C_j w_j):  0..3: c A_r, c A_i, c B_r, c B_i
            //   (A = (2 + 2E) rho + conj(O) sigma, B = O rho);  4..6: the k-space energy term
            //   and its gamma_t, gamma_b derivatives, -c [e |rho|^2 + Re(o rho conj(sigma))]
            const double rr = S[0][0], ri = S[1][0], sr = S[2][0], si = S[3][0];
            const double E = kq.E, Ore = kq.Ore, Oim = kq.Oim, c = kq.c;
            const double dA = j == 5 ? kq.dE_t : kq.dE_b, dB = j == 5 ? kq.dOre_t : kq.dOre_b;
            const double dC = j == 5 ? kq.dOim_t : kq.dOim_b;
            const double kxyz = j == 4 ? kq.kx : (j == 5 ? kq.ky : kq.kz);
            const int knx = kq.nx, kny = kq.ny, knz = kq.nz;
            const double rho2 = fma(rr, rr, ri * ri), pr = fma(rr, sr, ri * si), pim = fma(ri, sr, -(rr * si));
            const double twoE = fma(2.0, E, 2.0), oneE = 1.0 + E;
            const double Aj = j < 2 ? twoE : (j < 4 ? Ore : (j == 4 ? oneE : dA));
            const double uj = (j == 0 || j == 2) ? rr : ((j == 1 || j == 3) ? ri : rho2);
            const double Bj = j < 2 ? Ore : (j == 2 ? neg(Oim) : (j == 3 ? Oim : (j == 4 ? Ore : dB)));
            const double vj = j == 0 ? sr : (j == 1 ? si : (j == 2 ? ri : (j == 3 ? rr : pr)));
            const double Cj = j == 0 ? Oim : (j == 1 ? neg(Oim) : (j < 4 ? 0.0 : (j == 4 ? neg(Oim) : neg(dC))));
            const double wj = j == 0 ? si : (j == 1 ? sr : pim);
            const double val = (j < 4 ? c : neg(c)) * fma(Aj, uj, fma(Bj, vj, Cj * wj));
            if (j < 4) rs[4 * l + j] = j == 0 ? rr : (j == 1 ? ri : (j == 2 ? sr : si));
            if (j >= 4 && j < 7) kterm[3 * l + (j - 4)] = val;
            if (fp64) {
                KRec64* r = reinterpret_cast<KRec64*>(krec) + l;
                if (j < 4) (&r->Ar)[j] = val;
                else if (j < 7) (&r->kx)[j - 4] = kxyz;
                else if (j == 7) { r->nx = knx; r->ny = kny; r->nz = knz; r->pad0 = 0; r->pad1 = 0.0; }
            } else {
                // half h of record l / 2 (KPair32: x components for even k, y for odd k), as
                // 32-bit words: lanes 0-6 write A'_r, A'_i, B'_r, B'_i, kx, ky, kz, lanes 0
                // and 2 also -A'_r and -B'_r, lanes 7-9 the indices nx, ny, nz
                static_assert(offsetof(KPair32, nx) == 0 && offsetof(KPair32, ny) == 8 && offsetof(KPair32, nz) == 16 &&
                                  offsetof(KPair32, kz) == 24 && offsetof(KPair32, kx) == 32 && offsetof(KPair32, ky) == 40 &&
                                  offsetof(KPair32, nAr) == 48 && offsetof(KPair32, Ai) == 56 && offsetof(KPair32, nBr) == 64 &&
                                  offsetof(KPair32, Bi) == 72 && offsetof(KPair32, Ar) == 80 && offsetof(KPair32, Br) == 88,
                              "word offsets of the fold's stores");
                uint32_t* r = reinterpret_cast<uint32_t*>(reinterpret_cast<KPair32*>(krec) + (l >> 1)) + (l & 1);
                const float f = (float)(j < 4 ? val : kxyz);  // one conversion instruction for all lanes
                // word of lane j's value (pairs of words: x half, y half): Ar 20, Ai 14, Br 22,
                // Bi 18, kx 8, ky 10, kz 6, 5 bits per lane
                constexpr unsigned long long kWord = 20ull | 14ull << 5 | 22ull << 10 | 18ull << 15 | 8ull << 20 |
                                                     10ull << 25 | 6ull << 30;
                if (j < 7) r[(kWord >> (5 * j)) & 31] = __float_as_uint(f);
                if (j == 0 || j == 2) r[j == 0 ? 12 : 16] = __float_as_uint(-f);
                if (j >= 7 && j < 10) r[2 * (j - 7)] = (uint32_t)(j == 7 ? knx : (j == 8 ? kny : knz));
            }
        } else if (warp == 1) {
            // meanwhile the pack rows in groups of 32, one group per pass (lanes 0, 8, 16, 24 write)
            for (int g = blockIdx.x; g < ngroups; g += gridDim.x) reduce_pack_group(pack_part, pack_blocks, g, pack2);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    finalize_block(dp, pack2, ngroups, kterm, scal, S);
    if (threadIdx.x == 0) *done = 0u;
}

// Totals of a sharded evaluation -> the fold's inputs: one partial row per k and one
// pack row (Q, Q2, mu, sum|q|; the z range is not known and is left open).
__global__ void inject_totals_kernel(int P, const double* __restrict__ rho, const double* __restrict__ sums,
                                     double* __restrict__ sf_part, double* __restrict__ pack_part) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < P; l += gridDim.x * blockDim.x)
        for (int c = 0; c < 4; c++) sf_part[4 * l + c] = rho[4 * l + c];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        pack_part[0] = sums[0]; pack_part[1] = sums[1]; pack_part[2] = sums[2]; pack_part[3] = sums[3];
        pack_part[4] = 0.0; pack_part[5] = 0.0;
    }
}

__global__ void copy_sums_kernel(const double* __restrict__ scal, double* __restrict__ out) {
    if (threadIdx.x == 0) {
        out[0] = scal[SC_Q]; out[1] = scal[SC_Q2]; out[2] = scal[SC_MU]; out[3] = scal[SC_QABS];
    }
}

__global__ void dgamma_kernel(const double* __restrict__ scal, double g, double* __restrict__ dgamma) {
    if (threadIdx.x == 0) {
        dgamma[0] = g * scal[SC_DG_T];
        dgamma[1] = g * scal[SC_DG_B];
    }
}

}  // namespace

// ====================================================================== launchers
cudaError_t launch_sample(cudaStream_t st, const DevParams& dp, const SamplerTables& tb, uint64_t seed,
                          uint64_t step, const unsigned long long* step_dev, KCoef* kc, int32_t* kidx_out,
                          int* status) {
    const int threads = 128;  // 4 warps, one wave vector each
    const int blocks = (dp.P_pad * 32 + threads - 1) / threads;
    sample_kernel<<<blocks, threads, 0, st>>>(dp, tb, seed, step, step_dev, kc, kidx_out, status);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lattice_k(cudaStream_t st, const DevParams& dp, const int nm[3], int64_t t0, int64_t n_half,
                             KCoef* kc) {
    const int threads = 64;  // 2 warps, each serving 32 / W wave vectors
    const int blocks = (dp.P_pad * dp.kseg + threads - 1) / threads;
    lattice_k_kernel<<<blocks, threads, 0, st>>>(dp, nm[0], nm[1], nm[2], (long long)t0, (long long)n_half, kc);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_metropolis(cudaStream_t st, const DevParams& dp, const SamplerTables& tb, uint64_t seed,
                              uint64_t step, int sweeps, int32_t* state, KCoef* kc, int32_t* kidx_out,
                              unsigned long long* accepted) {
    const int threads = 64;  // one chain per thread
    const int blocks = (dp.P_pad + threads - 1) / threads;
    metropolis_kernel<<<blocks, threads, 0, st>>>(dp, tb, seed, step, sweeps, state, kc, kidx_out, accepted);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_eo_table(cudaStream_t st, const DevParams& dp, int half, double* eo) {
    const int threads = 64;
    const long long rows = 2LL * half + 1;
    const int blocks = (int)((rows * dp.kseg + threads - 1) / threads);
    eo_table_kernel<<<blocks, threads, 0, st>>>(dp, half, eo);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_accum_uk(cudaStream_t st, double* scal, int first, int last) {
    accum_uk_kernel<<<1, 32, 0, st>>>(scal, first, last);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_set_k(cudaStream_t st, const DevParams& dp, const int32_t* kidx, KCoef* kc, int* status) {
    int threads = 32, blocks = (dp.P_pad + threads - 1) / threads;
    set_k_kernel<<<blocks, threads, 0, st>>>(dp, kidx, kc, status);
    note_launches(1);
    return cudaGetLastError();
}

int pack_blocks_for(int64_t N) {
    int64_t b = (N + 255) / 256;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return (int)b;
}

cudaError_t launch_pack(cudaStream_t st, const DevParams& dp, int64_t N, const void* pos, const void* q,
                        bool in_f32, bool fp64, void* part, double* pack_part, int pack_blocks) {
    if (in_f32) {
        if (fp64) pack_kernel<float, true><<<pack_blocks, 256, 0, st>>>(dp, N, (const float*)pos, (const float*)q, part, pack_part);
        else pack_kernel<float, false><<<pack_blocks, 256, 0, st>>>(dp, N, (const float*)pos, (const float*)q, part, pack_part);
    } else {
        if (fp64) pack_kernel<double, true><<<pack_blocks, 256, 0, st>>>(dp, N, (const double*)pos, (const double*)q, part, pack_part);
        else pack_kernel<double, false><<<pack_blocks, 256, 0, st>>>(dp, N, (const double*)pos, (const double*)q, part, pack_part);
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sf64(cudaStream_t st, const DevParams& dp, int64_t N, const void* part, bool want_sigma,
                        const KCoef* kc, double* sf_part, int nblk, int kthreads, int kchunks) {
    dim3 grid(nblk, kchunks);
    if (want_sigma) sf64_kernel<true><<<grid, kthreads, 0, st>>>((const Part64*)part, N, kc, dp.P, sf_part, nblk);
    else sf64_kernel<false><<<grid, kthreads, 0, st>>>((const Part64*)part, N, kc, dp.P, sf_part, nblk);
    note_launches(1);
    return cudaGetLastError();
}

// The variant that skips empty wave-vector groups runs when the k slots of the launch
// (k chunks x threads x wave vectors per thread) exceed P by at least one warp's group
// of 32 (built in sf32_live.cu); otherwise every group holds wave vectors and the plain
// variant runs (the same code without the per-warp dispatch, which costs registers).
template <typename TIn, bool SIG, bool PIECED, int SHAPE>
void launch_sf32_poly(cudaStream_t st, dim3 grid, int kthreads, int npoly, const DevParams& dp, const TIn* p,
                      const TIn* qq, int64_t N, const KCoef* kc, double* sf_part, int nblk, uint4* po,
                      double* pack_part) {
    const bool live = !PIECED && (int64_t)grid.y * kthreads * kSfKR[SHAPE] - dp.P >= 32;
    if (live) launch_sf32_live(st, grid, kthreads, npoly, SHAPE, sizeof(TIn) == 4, SIG, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
    else sf32k::launch_sf32_npoly<TIn, SIG, PIECED, SHAPE, false>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
}

// Shapes 1 and 2 are built for float64 device inputs only.
template <typename TIn, bool SIG>
void launch_sf32_in(cudaStream_t st, dim3 grid, int kthreads, int npoly, bool pieced, int shape, const DevParams& dp,
                    const TIn* p, const TIn* qq, int64_t N, const KCoef* kc, double* sf_part, int nblk, uint4* po,
                    double* pack_part) {
    if (pieced) launch_sf32_poly<TIn, SIG, true, 0>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
    else if (sizeof(TIn) == 8 && shape == 1) launch_sf32_poly<TIn, SIG, false, 1>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
    else if (sizeof(TIn) == 8 && shape == 2) launch_sf32_poly<TIn, SIG, false, 2>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
    else launch_sf32_poly<TIn, SIG, false, 0>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
}

cudaError_t launch_sf32(cudaStream_t st, const DevParams& dp, int64_t N, const void* pos, const void* q, bool in_f32,
                        bool want_sigma, const KCoef* kc, double* sf_part, int nblk, int kthreads, int kchunks,
                        void* part, double* pack_part, int npoly, bool host_inputs, int shape) {
    dim3 grid(nblk, kchunks);
    uint4* po = (uint4*)part;
    const bool pc = host_inputs;
    if (in_f32) {
        const float* p = (const float*)pos; const float* qq = (const float*)q;
        if (want_sigma) launch_sf32_in<float, true>(st, grid, kthreads, npoly, pc, 0, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
        else launch_sf32_in<float, false>(st, grid, kthreads, npoly, pc, 0, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
    } else {
        const double* p = (const double*)pos; const double* qq = (const double*)q;
        if (want_sigma) launch_sf32_in<double, true>(st, grid, kthreads, npoly, pc, shape, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
        else launch_sf32_in<double, false>(st, grid, kthreads, npoly, pc, shape, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fold(cudaStream_t st, const DevParams& dp, const double* sf_part, int nblk, const KCoef* kc,
                        bool fp64, double* rs, double* kterm, void* krec, const double* pack_part,
                        int pack_blocks, double* pack2, double* scal, unsigned* done) {
    fold_kernel<<<dp.P, FOLD_THREADS, 0, st>>>(
        dp, sf_part, nblk, kc, fp64 ? 1 : 0, rs, kterm, krec, pack_part, pack_blocks, pack2, scal, done);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_inject_totals(cudaStream_t st, int P, const double* rho, const double* sums, double* sf_part,
                                double* pack_part) {
    inject_totals_kernel<<<(P + 127) / 128, 128, 0, st>>>(P, rho, sums, sf_part, pack_part);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_copy_sums(cudaStream_t st, const double* scal, double* out) {
    copy_sums_kernel<<<1, 32, 0, st>>>(scal, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dgamma(cudaStream_t st, const double* scal, double g, double* dgamma) {
    dgamma_kernel<<<1, 32, 0, st>>>(scal, g, dgamma);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_copy_energy(cudaStream_t st, const double* scal, double* energy_out) {
    return cudaMemcpyAsync(energy_out, scal, 4 * sizeof(double), cudaMemcpyDeviceToDevice, st);
}

cudaError_t query_shapes(int device, int P_pad, Shapes* sh) {
    cudaError_t e = cudaDeviceGetAttribute(&sh->sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    for (int v = 0; v < kSfShapes; v++) {
        int kt32 = (P_pad + kSfKR[v] - 1) / kSfKR[v];
        kt32 = ((kt32 + 31) / 32) * 32;
        sh->sf_threads32[v] = kt32 < 32 ? 32 : (kt32 > 128 ? 128 : kt32);
    }
    int kt64 = (P_pad + SF_KR64 - 1) / SF_KR64;
    kt64 = ((kt64 + 31) / 32) * 32;
    sh->sf_threads64 = kt64 < 32 ? 32 : (kt64 > 128 ? 128 : kt64);
    sh->force_threads = 256;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &sh->sf_occ32[0], sf32_kernel<double, true, 2, false, kSfKR[0], kSfTile[0], kSfMinBlocks[0]>, sh->sf_threads32[0], 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &sh->sf_occ32[1], sf32_kernel<double, true, 2, false, kSfKR[1], kSfTile[1], kSfMinBlocks[1]>, sh->sf_threads32[1], 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &sh->sf_occ32[2], sf32_kernel<double, true, 2, false, kSfKR[2], kSfTile[2], kSfMinBlocks[2]>, sh->sf_threads32[2], 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sh->sf_occ64, sf64_kernel<true>, sh->sf_threads64, 0);
    if (e != cudaSuccess) return e;
    e = force_occupancy(P_pad, sh->force_occ32, &sh->force_occ64);
    if (e != cudaSuccess) return e;
    e = pot_occupancy(P_pad, sh->pot_occ32);
    if (e != cudaSuccess) return e;
    for (int v = 0; v < kSfShapes; v++)
        if (sh->sf_occ32[v] < 1) sh->sf_occ32[v] = 1;
    for (int v = 0; v < kForceShapes; v++)
        if (sh->force_occ32[v] < 1) sh->force_occ32[v] = 1;
    for (int v = 0; v < kPotShapes; v++)
        if (sh->pot_occ32[v] < 1) sh->pot_occ32[v] = 1;
    if (sh->sf_occ64 < 1) sh->sf_occ64 = 1;
    if (sh->force_occ64 < 1) sh->force_occ64 = 1;
    return cudaSuccess;
}

}  // namespace rbe2d

