// Structure factor of the FP32-mixed mode (row a4, with the packing step a3 fused in):
// the kernel template shared by kspace_kernels.cu (the variants whose wave-vector groups
// are all live) and sf32_live.cu (the variants that skip empty groups), so that the two
// sets of instantiations compile in parallel.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "pair32.cuh"
#include "phase.cuh"
#include "rbe2d_internal.h"

namespace rbe2d {
namespace sf32k {

using pair32::sincos_turn32x2;
using phase::sincos_poly32;
using phase::sincos_turn32;

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(n) : "memory");
}

// Order-preserving integer key of a float64 (integer compares give float64 order).
__device__ __forceinline__ long long dkey(double x) {
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dunkey(long long k) { return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL)); }

// Warp totals of four float64 sums by a butterfly that halves the sums each lane
// carries: after the xor-16 step lanes 0-15 carry (s0, s1) and lanes 16-31 (s2, s3),
// after xor-8 one sum each, and three more steps complete it, so lanes 8 s .. 8 s + 7
// end with the warp's total of sum s (each step adds two values that are the same pair
// on both lanes: every lane of a group gets the same bits, in a fixed order).  Six
// float64 additions per lane instead of twenty for four separate shuffle trees; float64
// instructions take 64 cycles each on GB300.
__device__ __forceinline__ double warp_sums4(double s0, double s1, double s2, double s3) {
    const int lane = threadIdx.x & 31;
    const bool up = (lane & 16) != 0;
    double a = up ? s2 : s0, b = up ? s3 : s1;
    a += __shfl_xor_sync(0xffffffffu, up ? s0 : s2, 16);
    b += __shfl_xor_sync(0xffffffffu, up ? s1 : s3, 16);
    const bool odd = (lane & 8) != 0;
    double v = odd ? b : a;
    v += __shfl_xor_sync(0xffffffffu, odd ? a : b, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

// Warp minimum and maximum of two float64 values through their integer keys.
__device__ __forceinline__ void warp_minmax(double mn, double mx, long long* kmn, long long* kmx) {
    long long a = dkey(mn), b = dkey(mx);
    for (int d = 16; d > 0; d >>= 1) {
        a = min(a, __shfl_xor_sync(0xffffffffu, a, d));
        b = max(b, __shfl_xor_sync(0xffffffffu, b, d));
    }
    *kmn = a;
    *kmx = b;
}

// Block-wide sums of four values and min / max of two more: warp totals (warp_sums4,
// warp_minmax), then the warps in order; lanes 0-5 of warp 0 write the six results to o
// (sums of q, q^2, q z, |q|, then min z, max z).  Every thread of the block must call it.
__device__ inline void block_pack_sums(double s0, double s1, double s2, double s3, double mn, double mx, double* o) {
    __shared__ double wv[8][4];  // up to 256 threads
    __shared__ long long wk[8][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const double v = warp_sums4(s0, s1, s2, s3);
    long long kmn, kmx;
    warp_minmax(mn, mx, &kmn, &kmx);
    if ((lane & 7) == 0) wv[warp][lane >> 3] = v;
    if (lane == 0) { wk[warp][0] = kmn; wk[warp][1] = kmx; }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = wv[0][threadIdx.x];
        for (int w = 1; w < nw; w++) t += wv[w][threadIdx.x];
        o[threadIdx.x] = t;
    } else if (threadIdx.x < 6) {
        const int c = threadIdx.x - 4;
        long long k = wk[0][c];
        for (int w = 1; w < nw; w++) k = c == 0 ? min(k, wk[w][0]) : max(k, wk[w][1]);
        o[threadIdx.x] = dunkey(k);
    }
}

// Grid: x = particle chunks (contiguous, equal +-1 particle), y = k chunks of
// blockDim.x * KR wave vectors; thread t owns k = kbase + t + j blockDim.x.
// Particles are staged through shared memory in double-buffered tiles with cp.async;
// every thread reads the same particle (broadcast).  FP32 sums run over one tile
// (<= 512 terms) and are then added into FP64 accumulators.
// Shapes (kSfKR wave vectors per thread, kSfTile particles per tile, kSfMinBlocks CTAs per
// SM) are chosen by the tuner; shape 0: 4 wave vectors, 224-particle tiles, 8 CTAs per SM.
static_assert(kSfKR[0] % 2 == 0 && kSfKR[1] % 2 == 0 && kSfKR[2] % 2 == 0,
              "the host-input variant sums wave-vector pairs");
constexpr int SF_THREADS32 = 128;  // upper bound of blockDim.x
constexpr int SF_PIECES0 = 4;      // pieces of the first tile when the inputs are in host memory

template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}

// 32-bit fixed-point turn fraction: round(v / L 2^32) mod 2^32 (the low 32 bits of the
// nearest integer; negative and out-of-cell values wrap periodically).
__device__ __forceinline__ uint32_t turn32(double v, double scale) {
    return (uint32_t)(unsigned long long)__double2ll_rn(v * scale);
}

// Structure factor, FP32-mixed mode, with the packing step fused in.  The raw positions
// and charges of tile t + 1 are copied to shared memory with cp.async while tile t is
// summed; each tile is converted once to {ux, uy, uz, q} (written to `part` for the force
// kernel by the first k-chunk) and read by every thread (broadcast).  FP32 sums run over
// one tile (<= 224 terms) and are then added into float64 accumulators kept in shared
// memory, which leaves registers and shared memory for 8 CTAs of 128 threads per SM.
template <typename TIn, bool SIG, int NPOLY, bool PIECED, int SF_KR32, int SF_TILE32, int MINB, bool LIVE = false>
__global__ void __launch_bounds__(SF_THREADS32, MINB) sf32_kernel(DevParams dp, const TIn* __restrict__ pos,
                                                   const TIn* __restrict__ q, int64_t N,
                                                   const KCoef* __restrict__ kc, int P,
                                                   double* __restrict__ sf_part, int nblk,
                                                   uint4* __restrict__ part_out, double* __restrict__ pack_part) {
    __shared__ __align__(16) TIn raw[4 * SF_TILE32];  // [3 * TILE positions | TILE charges]
    __shared__ uint4 tile[SF_TILE32];
    __shared__ double acc[4 * SF_KR32][SF_THREADS32];  // [component][thread]
    const int KT = blockDim.x;
    const int kbase = blockIdx.y * KT * SF_KR32;
    const bool writer = blockIdx.y == 0;
    uint32_t nx[SF_KR32], ny[SF_KR32], nz[SF_KR32];
#pragma unroll
    for (int j = 0; j < SF_KR32; j++) {
        int k = kbase + threadIdx.x + j * KT;
        if (k < P) { nx[j] = (uint32_t)kc[k].nx; ny[j] = (uint32_t)kc[k].ny; nz[j] = (uint32_t)kc[k].nz; }
        else { nx[j] = 0u; ny[j] = 0u; nz[j] = 0u; }
    }
#pragma unroll
    for (int c = 0; c < 4 * SF_KR32; c++) acc[c][threadIdx.x] = 0.0;
    const double sx = 4294967296.0 * dp.inv_Lx, sy = 4294967296.0 * dp.inv_Ly, sz = 4294967296.0 * dp.inv_Lz;
    const int64_t b = blockIdx.x;
    const int64_t p0 = (N * b) / nblk, p1 = (N * (b + 1)) / nblk;
    const int64_t ntiles = (p1 - p0 + SF_TILE32 - 1) / SF_TILE32;
    // charge sums in float64: mu = sum q z cancels heavily, and the neutrality check
    // compares |sum q| with 1e-10 sum |q|
    double sQ = 0.0, sQ2 = 0.0, sMu = 0.0, sQa = 0.0;
    double zmin = 1e300, zmax = -1e300;  // exact, for the z-range check
    // PIECED (inputs in host memory, which cross NVLink-C2C at a fraction of HBM speed):
    // tile 0 is staged in pieces of 16, 32 and 64 particles and the rest, each issued once
    // the previous one has been converted, so the first sums start when 16 particles have
    // arrived and each transfer (piece k + 1, then tile 1) runs under the sums of piece k.
    // Pieces issued all at once would arrive interleaved, not in order.  Later tiles are
    // prefetched whole during the previous tile.  The pieces change neither the order of
    // the float32 sums nor which thread converts which particle: both variants give the
    // same bits.
    auto piece_end = [](int k, int n) { return k == SF_PIECES0 - 1 ? n : min(n, 16 * ((2 << k) - 1)); };
    auto tile_len = [&](int64_t t) { return (int)min((int64_t)SF_TILE32, p1 - (p0 + t * SF_TILE32)); };
    // stage entries [lo, hi) of tile t as one cp.async group (empty when lo == hi)
    auto issue = [&](int64_t t, int lo, int hi) {
        const int64_t s0 = p0 + t * SF_TILE32;
        const TIn* gp = pos + 3 * (s0 + lo);
        for (int i = threadIdx.x; i < 3 * (hi - lo); i += KT) cp_async_small<sizeof(TIn)>(&raw[3 * lo + i], &gp[i]);
        for (int i = threadIdx.x; i < hi - lo; i += KT)
            cp_async_small<sizeof(TIn)>(&raw[3 * SF_TILE32 + lo + i], &q[s0 + lo + i]);
        cp_async_commit();
    };
    // raw -> fixed-point tile entries [lo, hi) (thread t takes the entries = t mod KT),
    // the packed output and the pack sums
    auto convert = [&](int64_t s0, int lo, int hi) {
        for (int i = threadIdx.x; i < hi; i += KT) {
            if (i < lo) continue;
            const double x = (double)raw[3 * i], y = (double)raw[3 * i + 1], z = (double)raw[3 * i + 2];
            const float qv = (float)raw[3 * SF_TILE32 + i];
            uint4 u;
            u.x = turn32(x, sx); u.y = turn32(y, sy); u.z = turn32(z, sz);
            u.w = __float_as_uint(qv);
            tile[i] = u;
            if (writer) {
                part_out[s0 + i] = u;
                const double qd = (double)raw[3 * SF_TILE32 + i];
                sQ += qd; sQ2 = fma(qd, qd, sQ2); sMu = fma(qd, z, sMu); sQa += fabs(qd);
                zmin = fmin(zmin, z); zmax = fmax(zmax, z);
            }
        }
    };
    // The float32 sums over tile entries [lo, hi), in entry order, one per wave vector
    // and component.  PIECED keeps them as float2 pairs of wave vectors (2h, 2h + 1) and
    // runs the scalings and fused multiply-adds of a pair as one paired instruction; each
    // component takes the same operations in the same order as the scalar sums, so both
    // give the same bits (measured: the paired sums are faster on host inputs, 0.443 ->
    // 0.430 ms, and slower on device inputs, 0.424 -> 0.430 ms).
    float ar[SF_KR32], ai[SF_KR32], br[SF_KR32], bi[SF_KR32];
    float2 ar2[SF_KR32 / 2], ai2[SF_KR32 / 2], br2[SF_KR32 / 2], bi2[SF_KR32 / 2];
    // The scalar sums over the first JL wave vectors of each thread (a warp's groups past
    // its live count jl hold no wave vector below P and are skipped).
    auto sums_live = [&](auto jlc, int lo, int hi) {
        constexpr int JL = decltype(jlc)::value;
#pragma unroll 2
        for (int p = lo; p < hi; p++) {
            const uint4 u = tile[p];
            const float qf = __uint_as_float(u.w);
#pragma unroll
            for (int j = 0; j < JL; j++) {
                const uint32_t txy = nx[j] * u.x + ny[j] * u.y;
                const uint32_t tz = nz[j] * u.z;
                float s1, c1;
                // the first NPOLY wave vectors take one angle on the FMA pipe, the rest on MUFU
                if (!SIG && j < NPOLY) sincos_poly32(txy + tz, &s1, &c1);
                else sincos_turn32(txy + tz, &s1, &c1);
                ar[j] = fmaf(qf, c1, ar[j]);
                ai[j] = fmaf(qf, s1, ai[j]);
                if (SIG) {
                    float s2, c2;
                    if (j < NPOLY) sincos_poly32(txy - tz, &s2, &c2);
                    else sincos_turn32(txy - tz, &s2, &c2);
                    br[j] = fmaf(qf, c2, br[j]);
                    bi[j] = fmaf(qf, s2, bi[j]);
                }
            }
        }
    };
    auto sums = [&](int lo, int hi) {
        if constexpr (PIECED) {
#pragma unroll 2
            for (int p = lo; p < hi; p++) {
                const uint4 u = tile[p];
                const float qf = __uint_as_float(u.w);
                const float2 q2 = make_float2(qf, qf);
#pragma unroll
                for (int h = 0; h < SF_KR32 / 2; h++) {
                    const int ja = 2 * h, jb = 2 * h + 1;
                    const uint32_t txya = nx[ja] * u.x + ny[ja] * u.y, tza = nz[ja] * u.z;
                    const uint32_t txyb = nx[jb] * u.x + ny[jb] * u.y, tzb = nz[jb] * u.z;
                    float2 s1, c1;
                    sincos_turn32x2(txya + tza, txyb + tzb, !SIG && ja < NPOLY, !SIG && jb < NPOLY, s1, c1);
                    ar2[h] = __ffma2_rn(q2, c1, ar2[h]);
                    ai2[h] = __ffma2_rn(q2, s1, ai2[h]);
                    if (SIG) {
                        float2 s2, c2;
                        sincos_turn32x2(txya - tza, txyb - tzb, ja < NPOLY, jb < NPOLY, s2, c2);
                        br2[h] = __ffma2_rn(q2, c2, br2[h]);
                        bi2[h] = __ffma2_rn(q2, s2, bi2[h]);
                    }
                }
            }
        } else if constexpr (LIVE) {
            // warp w holds the groups k = kbase + j KT + 32 w + lane (j < SF_KR32); those
            // with their first k at or beyond P hold no wave vector and are skipped: the
            // live groups of a warp are a prefix of length jl
            const int kw = P - (kbase + 32 * (int)(threadIdx.x >> 5));
            const int jl = kw <= 0 ? 0 : min(SF_KR32, (kw + KT - 1) / KT);
            if (jl == SF_KR32) sums_live(std::integral_constant<int, SF_KR32>(), lo, hi);
            else if (jl == 3) sums_live(std::integral_constant<int, (SF_KR32 > 3 ? 3 : 1)>(), lo, hi);
            else if (jl == 2) sums_live(std::integral_constant<int, (SF_KR32 > 2 ? 2 : 1)>(), lo, hi);
            else if (jl == 1) sums_live(std::integral_constant<int, 1>(), lo, hi);
        } else {
            sums_live(std::integral_constant<int, SF_KR32>(), lo, hi);
        }
    };
    if (ntiles > 0) issue(0, 0, PIECED ? piece_end(0, tile_len(0)) : tile_len(0));
    for (int64_t t = 0; t < ntiles; t++) {
        const int64_t s0 = p0 + t * SF_TILE32;
        const int n = tile_len(t);
#pragma unroll
        for (int j = 0; j < SF_KR32; j++) ar[j] = ai[j] = br[j] = bi[j] = 0.f;
#pragma unroll
        for (int h = 0; h < SF_KR32 / 2; h++) ar2[h] = ai2[h] = br2[h] = bi2[h] = make_float2(0.f, 0.f);
        int lo = 0;
        if (PIECED && t == 0) {
            for (int k = 0; k < SF_PIECES0 - 1; k++) {
                const int hi = piece_end(k, n);
                cp_async_wait<0>();
                __syncthreads();  // raw holds piece k
                convert(s0, lo, hi);
                __syncthreads();
                issue(0, hi, piece_end(k + 1, n));
                sums(lo, hi);
                lo = hi;
            }
        }
        cp_async_wait<0>();
        __syncthreads();  // raw holds tile t (the rest of it); every thread is done with the previous tile
        convert(s0, lo, n);
        __syncthreads();  // tile ready, raw free
        if (t + 1 < ntiles) issue(t + 1, 0, tile_len(t + 1));
        sums(lo, n);
        if constexpr (PIECED) {
#pragma unroll
            for (int j = 0; j < SF_KR32; j++) {
                const int h = j >> 1;
                ar[j] = (j & 1) ? ar2[h].y : ar2[h].x;
                ai[j] = (j & 1) ? ai2[h].y : ai2[h].x;
                br[j] = (j & 1) ? br2[h].y : br2[h].x;
                bi[j] = (j & 1) ? bi2[h].y : bi2[h].x;
            }
        }
#pragma unroll
        for (int j = 0; j < SF_KR32; j++) {
            acc[4 * j + 0][threadIdx.x] += ar[j];
            acc[4 * j + 1][threadIdx.x] += ai[j];
            acc[4 * j + 2][threadIdx.x] += br[j];
            acc[4 * j + 3][threadIdx.x] += bi[j];
        }
    }
#pragma unroll
    for (int j = 0; j < SF_KR32; j++) {
        int k = kbase + threadIdx.x + j * KT;
        if (k < P) {
            double* o = sf_part + ((size_t)k * nblk + b) * 4;
            o[0] = acc[4 * j][threadIdx.x]; o[1] = acc[4 * j + 1][threadIdx.x];
            o[2] = acc[4 * j + 2][threadIdx.x]; o[3] = acc[4 * j + 3][threadIdx.x];
        }
    }
    if (writer)  // per-chunk sums for the self and IBC terms and the input checks
        block_pack_sums(sQ, sQ2, sMu, sQa, zmin, zmax, pack_part + (size_t)b * PACK_STRIDE);
}

template <typename TIn, bool SIG, bool PIECED, int SHAPE, bool LIVE>
inline void launch_sf32_npoly(cudaStream_t st, dim3 grid, int kthreads, int npoly, const DevParams& dp, const TIn* p,
                              const TIn* qq, int64_t N, const KCoef* kc, double* sf_part, int nblk, uint4* po,
                              double* pack_part) {
    constexpr int KR = kSfKR[SHAPE], TL = kSfTile[SHAPE], MB = kSfMinBlocks[SHAPE];
    // tuner level 0, 1, 2, 3: NPOLY = 0, 1, 2, 4 wave vectors per thread with one angle on the FMA pipe
    if (npoly <= 0) sf32_kernel<TIn, SIG, 0, PIECED, KR, TL, MB, LIVE><<<grid, kthreads, 0, st>>>(dp, p, qq, N, kc, dp.P, sf_part, nblk, po, pack_part);
    else if (npoly == 1) sf32_kernel<TIn, SIG, 1, PIECED, KR, TL, MB, LIVE><<<grid, kthreads, 0, st>>>(dp, p, qq, N, kc, dp.P, sf_part, nblk, po, pack_part);
    else if (npoly == 2) sf32_kernel<TIn, SIG, 2, PIECED, KR, TL, MB, LIVE><<<grid, kthreads, 0, st>>>(dp, p, qq, N, kc, dp.P, sf_part, nblk, po, pack_part);
    else sf32_kernel<TIn, SIG, 4, PIECED, KR, TL, MB, LIVE><<<grid, kthreads, 0, st>>>(dp, p, qq, N, kc, dp.P, sf_part, nblk, po, pack_part);
}

}  // namespace sf32k
}  // namespace rbe2d
