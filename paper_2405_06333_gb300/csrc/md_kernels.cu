// Langevin MD step (Eq. 2.27) in the BAOAB splitting (Leimkuhler and Matthews, 2013):
//   B: v += dt/2 F/m;  A: x += dt/2 v;  O: v = c1 v + c2 sqrt(kT/m) xi;  A: x += dt/2 v;
//   [force at the new positions];  B: v += dt/2 F/m
// with c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2) and xi standard normals from Philox4x32-10
// (counter = (particle, step, 0, 0), key = noise seed) through the Box-Muller transform.
// The confining walls at z = 0 and z = H are purely repulsive shifted Lennard-Jones
// (WCA) walls, as in the paper's first electrolyte test (Sec. 4.1).  The step counter
// lives in device memory, so replaying a captured graph advances both the k sampler and
// the noise.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rbe2d_internal.h"

namespace rbe2d {

namespace {

// Philox4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k.x += W0; k.y += W1; }
        const unsigned hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const unsigned hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// WCA wall force on a particle at distance d from a wall (positive: away from the wall),
// evaluated no closer than d = sigma/2, where it is already ~1e5 eps/sigma.  In the
// precision of the force array: float32 beside a float32 k-space + real-space force,
// float64 in the float64 mode.
__device__ __forceinline__ float wall_force(float d, const MdParams& md) {
    if (!(md.w_sig > 0.f) || d >= md.w_rcut) return 0.f;
    const float dd = fmaxf(d, 0.5f * md.w_sig);
    const float s = __fdividef(md.w_sig, dd), s2 = s * s, s6 = s2 * s2 * s2;
    return __fdividef(md.w_f * (2.f * s6 * s6 - s6), dd);
}
__device__ __forceinline__ double wall_force(double d, const MdParams& md) {
    if (!(md.w_sig_d > 0.0) || d >= md.w_rcut_d) return 0.0;
    const double dd = fmax(d, 0.5 * md.w_sig_d);
    const double s = md.w_sig_d / dd, s2 = s * s, s6 = s2 * s2 * s2;
    return md.w_f_d * (2.0 * s6 * s6 - s6) / dd;
}

// Range tests on the bits of a float64 (integer compares on the ALU pipe; GB300's float64
// pipe runs at 1/64 of float32): for b >= 0 the bit patterns of non-negative doubles are
// ordered like the values, negative values (and -0.0) have b < 0, NaN and infinity have
// all exponent bits set.
__device__ __forceinline__ bool finite_bits(double x) {
    return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}
__device__ __forceinline__ bool in_range_bits(double x, long long lo_bits, long long hi_bits_excl) {
    const long long b = __double_as_longlong(x);
    return b >= lo_bits && b < hi_bits_excl;
}

// z force of both walls in the precision T of the force array; a height in
// [w_in_lo, w_in_hi) (bits in_lo .. in_hi) is out of both walls' reach with a margin, so
// the test on its bits returns the 0 that both evaluations would give.
template <typename T>
__device__ __forceinline__ double walls(double z, double H, const MdParams& md, long long in_lo, long long in_hi) {
    if (in_range_bits(z, in_lo, in_hi)) return 0.0;
    const T zt = (T)z;
    return (double)(wall_force(zt, md) - wall_force((T)H - zt, md));
}

// x into [0, L): an x outside (or at L, or -0.0) takes the floor path, then the rounding
// at the edges is corrected (x + L can round to L for x just below 0).
__device__ __forceinline__ double wrap_periodic(double x, double L, double inv_L, long long L_bits) {
    if (in_range_bits(x, 0LL, L_bits)) return x;
    x -= floor(x * inv_L) * L;
    if (x >= L) x -= L;
    if (x < 0.0) x += L;
    return x;
}

template <typename TF>
__global__ void md_baoa_kernel(DevParams dp, MdParams md, int64_t N, double* __restrict__ pos,
                               double* __restrict__ vel, const TF* __restrict__ force,
                               const unsigned long long* __restrict__ step, int* __restrict__ status) {
    const unsigned long long s = *step;
    const double h = md.hd, hk = md.hk, c1 = md.c1, c2 = md.c2s;
    const long long Lx_bits = __double_as_longlong(dp.Lx), Ly_bits = __double_as_longlong(dp.Ly);
    const long long H_bits_incl = __double_as_longlong(dp.H) + 1;  // z in [0, H]
    const long long in_lo = __double_as_longlong(md.w_in_lo), in_hi = __double_as_longlong(md.w_in_hi);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
        const double fw = walls<TF>(z, dp.H, md, in_lo, in_hi);
        vx += hk * (double)force[3 * i];
        vy += hk * (double)force[3 * i + 1];
        vz += hk * ((double)force[3 * i + 2] + fw);
        x += h * vx; y += h * vy; z += h * vz;
        const uint4 r = philox4x32_10(make_uint4((unsigned)i, (unsigned)(i >> 32), (unsigned)s, (unsigned)(s >> 32)),
                                      make_uint2((unsigned)md.noise_seed, (unsigned)(md.noise_seed >> 32)));
        // Box-Muller in float32 (thermostat noise needs no more): u in (0, 1], angle in [0, 2 pi)
        const float u1 = ((float)(r.x >> 8) + 0.5f) * 0x1p-24f, u2 = (float)(r.y >> 8) * 0x1p-24f;
        const float u3 = ((float)(r.z >> 8) + 0.5f) * 0x1p-24f, u4 = (float)(r.w >> 8) * 0x1p-24f;
        const float c2f = (float)c2;
        const float ra = c2f * sqrtf(-2.0f * logf(u1)), rb = c2f * sqrtf(-2.0f * logf(u3));
        float sa, ca, sb, cb;
        sincospif(2.0f * u2, &sa, &ca);
        sincospif(2.0f * u4, &sb, &cb);
        vx = fma(c1, vx, (double)(ra * ca));
        vy = fma(c1, vy, (double)(ra * sa));
        vz = fma(c1, vz, (double)(rb * cb));
        x += h * vx; y += h * vy; z += h * vz;
        // keep x, y in the cell; reflect at the walls should a step overshoot them
        x = wrap_periodic(x, dp.Lx, dp.inv_Lx, Lx_bits);
        y = wrap_periodic(y, dp.Ly, dp.inv_Ly, Ly_bits);
        if (!in_range_bits(z, 0LL, H_bits_incl)) {
            if (z < 0.0) { z = -z; vz = -vz; }
            if (z > dp.H) { z = 2.0 * dp.H - z; vz = -vz; }
            z = fmin(fmax(z, 0.0), dp.H);
        }
        if (!(finite_bits(x) && finite_bits(y) && finite_bits(z) && finite_bits(vx) && finite_bits(vy) &&
              finite_bits(vz))) {
            // an exploded particle: flag it and park it at rest in the slab centre plane
            atomicAdd(&status[ST_MD], 1);
            x = isfinite(x) ? x : 0.0; y = isfinite(y) ? y : 0.0; z = 0.5 * dp.H;
            vx = vy = vz = 0.0;
        }
        pos[3 * i] = x; pos[3 * i + 1] = y; pos[3 * i + 2] = z;
        vel[3 * i] = vx; vel[3 * i + 1] = vy; vel[3 * i + 2] = vz;
    }
}

// Final half kick with the new force; kinetic energy by fixed-order block sums (the last
// CTA adds them in block order) and the step counter advanced by that CTA.
template <typename TF>
__global__ void __launch_bounds__(256) md_b_kernel(DevParams dp, MdParams md, int64_t N,
                                                   const double* __restrict__ pos, double* __restrict__ vel,
                                                   const TF* __restrict__ force,
                                                   unsigned long long* __restrict__ step,
                                                   double* __restrict__ kpart, double* __restrict__ stats,
                                                   unsigned* __restrict__ done) {
    __shared__ double red[8];
    __shared__ bool last;
    const double hk = md.hk;
    const long long in_lo = __double_as_longlong(md.w_in_lo), in_hi = __double_as_longlong(md.w_in_hi);
    double ke = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double fw = walls<TF>(pos[3 * i + 2], dp.H, md, in_lo, in_hi);
        const double vx = vel[3 * i] + hk * (double)force[3 * i];
        const double vy = vel[3 * i + 1] + hk * (double)force[3 * i + 1];
        const double vz = vel[3 * i + 2] + hk * ((double)force[3 * i + 2] + fw);
        vel[3 * i] = vx; vel[3 * i + 1] = vy; vel[3 * i + 2] = vz;
        ke += 0.5 * md.mass * (vx * vx + vy * vy + vz * vz);
    }
    for (int o = 16; o > 0; o >>= 1) ke += __shfl_down_sync(0xffffffffu, ke, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ke;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        kpart[blockIdx.x] = t;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // all threads of the last CTA: fixed-order strided sums, then warps in order
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) t += __ldcg(&kpart[b]);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += red[w];
    if (stats) stats[0] = tot;
    *step += 1ull;
    *done = 0u;
}

}  // namespace

int md_blocks(int64_t N) {
    int64_t b = (N + 255) / 256;
    if (b < 1) b = 1;
    if (b > 2048) b = 2048;
    return (int)b;
}

cudaError_t launch_md_baoa(cudaStream_t st, const DevParams& dp, const MdParams& md, int64_t N, double* pos,
                           double* vel, const void* force, bool f64, const unsigned long long* step, int* status) {
    if (f64)
        md_baoa_kernel<double><<<md_blocks(N), 256, 0, st>>>(dp, md, N, pos, vel, (const double*)force, step, status);
    else
        md_baoa_kernel<float><<<md_blocks(N), 256, 0, st>>>(dp, md, N, pos, vel, (const float*)force, step, status);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_md_b(cudaStream_t st, const DevParams& dp, const MdParams& md, int64_t N, const double* pos,
                        double* vel, const void* force, bool f64, unsigned long long* step, double* kpart,
                        double* stats, unsigned* done) {
    if (f64)
        md_b_kernel<double><<<md_blocks(N), 256, 0, st>>>(dp, md, N, pos, vel, (const double*)force, step, kpart,
                                                           stats, done);
    else
        md_b_kernel<float><<<md_blocks(N), 256, 0, st>>>(dp, md, N, pos, vel, (const float*)force, step, kpart,
                                                          stats, done);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rbe2d
