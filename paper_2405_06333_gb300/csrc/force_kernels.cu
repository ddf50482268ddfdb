// Force and potential kernels of the RBE2D k-space term (sm_103a): Eq. 3.26 for the
// force on every particle from the P sampled wave vectors, plus dU/dq (the adjoint of
// Eq. 3.18) when asked.  They run after the fold has turned the structure factors into
// per-k records.  Each (particle, k) pair costs one sincos per angle and a few FMAs, so
// the kernels are bound by MUFU and FP32 issue.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pair32.cuh"
#include "phase.cuh"
#include "rbe2d_internal.h"

namespace rbe2d {

namespace {

using pair32::force_pair32;
using phase::sincos_turn64;

// The k records (A' = c A, B' = c B) are staged in shared memory in tiles of KTILE and
// read by all threads (broadcast); a particle's k-sum stays in one thread (or in S
// adjacent threads of one warp, see the split shapes below).  Per pair:
//   g1 = Im(e^{-i theta1} A') = A'i cos t1 - A'r sin t1,  theta1 = k.r
//   g2 = Im(e^{-i theta2} B'),                             theta2 = khat.r
//   F += (kx (g1+g2), ky (g1+g2), kz (g1-g2));  phi -= Re(e^{-i t1} A') + Re(e^{-i t2} B')
// and at the end F *= q_i, plus the IBC and self terms.  The FP32 kernel takes the wave
// vectors two at a time (KPair32): the float32 arithmetic of k0 and k1 runs as paired
// instructions (one issue slot for two results), the sums over even and odd k are kept
// apart and added at the end; the sin/cos stay one per angle.
constexpr int F_KTILE32 = 1000;  // wave vectors per shared-memory tile (500 records, even)
// a full tile plus the kernel's static shared memory (16 bytes) must fit the 48 KB that a
// block may use without opting in to more
static_assert(sizeof(KPair32) * (F_KTILE32 / 2) + 64 <= 48 * 1024 && F_KTILE32 % 2 == 0, "force32 tile too large");
constexpr int F_KTILE64 = 512;

// Store v, or add it to what is there (RBE2D_ACCUMULATE).
template <typename T>
__device__ __forceinline__ void put(T* p, T v, int acc) {
    if (acc) v += *p;
    *p = v;
}

// Persistent CTAs take rounds of R x THREADS / S particles from an atomic counter
// (counters[1]); each thread owns R particles of a round, so one shared-memory record
// load serves 2 R pairs.  A particle's k-sum stays in one thread (S = 1) or in S adjacent
// threads added in a fixed order, so the result does not depend on which CTA takes which
// round (it depends on S only through that order).  The last CTA to finish re-arms the
// counters (counters[2] counts finished CTAs).
//
// Launch shapes the tuner chooses from (rbe2d_autotune): {THREADS, R, MINB, S} =
// kForceThreads, kForceR, kForceMinBlocks, kForceSplit (rbe2d_internal.h).  S > 1 splits
// each particle's k-sum over S adjacent threads (thread s takes records s, s + S, ...),
// whose partial sums a fixed shuffle butterfly adds: rounds of THREADS R / S particles
// and S times shorter dependency chains, for systems too small to fill the GPU.

// FPOLY = number of the 2 R (particle, k) terms of a record (R particles x two wave
// vectors: (u0, k0), (u0, k1), (u1, k0), (u1, k1)) that evaluate one angle on the FMA pipe.
template <bool DIEL, bool POT, int FPOLY, int THREADS, int R, int MINB, int S>
__global__ void __launch_bounds__(THREADS, MINB) force32_kernel(DevParams dp, const uint4* __restrict__ part, int64_t N,
                                                          const KPair32* __restrict__ krec,
                                                          const double* __restrict__ scal, int ibc,
                                                          float* __restrict__ force, float* __restrict__ phi,
                                                          float fscale, float pscale, unsigned* __restrict__ counters) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    KPair32* ks = reinterpret_cast<KPair32*>(smem_raw);
    __shared__ unsigned round_sh;
    const int P = dp.P;
    const int ntile = (P + F_KTILE32 - 1) / F_KTILE32;  // 0 when only IBC/self terms are wanted
    static_assert(S == 1 || S == 2 || S == 4, "the k-split stays within a warp");
    constexpr int PT = THREADS / S;  // particles per R-slice of a round
    const int64_t per_round = (int64_t)PT * R;
    const int sub = (int)(threadIdx.x % S), pid = (int)(threadIdx.x / S);
    const unsigned nrounds = (unsigned)((N + per_round - 1) / per_round);
    const float fibc = ibc ? (float)scal[SC_FIBC] : 0.f;
    const double dqz = ibc ? scal[SC_DQ_IBC_Z] : 0.0, dqc = ibc ? scal[SC_DQ_IBC_C] : 0.0;
    const double self2 = -2.0 * dp.alpha / sqrt(M_PI) * dp.kc;
    // records of tile t: (n + 1) / 2 for its n wave vectors, six 16-byte words each
    auto load_tile = [&](int t) {
        const int k0 = t * F_KTILE32, n = min(F_KTILE32, P - k0);
        const uint4* src = reinterpret_cast<const uint4*>(krec + k0 / 2);
        uint4* dst = reinterpret_cast<uint4*>(ks);
        for (int i = threadIdx.x; i < 6 * ((n + 1) / 2); i += THREADS) dst[i] = src[i];
    };
    if (ntile == 1) load_tile(0);
    for (;;) {
        if (threadIdx.x == 0) round_sh = atomicAdd(&counters[1], 1u);
        __syncthreads();  // also publishes the k tile on the first pass
        const unsigned rnd = round_sh;
        __syncthreads();
        if (rnd >= nrounds) break;
        int64_t i[R];
        bool act[R];
        uint4 u[R];
        const float2 zero2 = make_float2(0.f, 0.f);
        float2 fx[R], fy[R], fz[R], ph[R];  // x: even k, y: odd k
#pragma unroll
        for (int j = 0; j < R; j++) {
            i[j] = (int64_t)rnd * per_round + pid + j * PT;
            act[j] = i[j] < N;
            u[j] = act[j] ? part[i[j]] : make_uint4(0, 0, 0, 0);
            fx[j] = fy[j] = fz[j] = ph[j] = zero2;
        }
        for (int t = 0; t < ntile; t++) {
            if (ntile > 1) { __syncthreads(); load_tile(t); __syncthreads(); }
            const int nrec = (min(F_KTILE32, P - t * F_KTILE32) + 1) / 2;
            for (int l = sub; l < nrec; l += S) {
                const KPair32 r = ks[l];
#pragma unroll
                for (int j = 0; j < R; j++)
                    force_pair32<DIEL, POT>(r, u[j], FPOLY >= 2 * j + 1, FPOLY >= 2 * j + 2, fx[j], fy[j], fz[j], ph[j]);
            }
        }
        if (S > 1) {  // every lane takes part; lane sub 0 of each particle ends with the sums
            auto add_xor = [](float2& v, int o) {
                v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
            };
#pragma unroll
            for (int j = 0; j < R; j++)
                for (int o = 1; o < S; o <<= 1) {
                    add_xor(fx[j], o); add_xor(fy[j], o); add_xor(fz[j], o);
                    if (POT) add_xor(ph[j], o);
                }
        }
#pragma unroll
        for (int j = 0; j < R; j++) {
            if (!act[j] || sub != 0) continue;
            const int64_t ii = i[j];
            const float qf = __uint_as_float(u[j].w);
            put(&force[3 * ii + 0], fscale * qf * (fx[j].x + fx[j].y), dp.acc);
            put(&force[3 * ii + 1], fscale * qf * (fy[j].x + fy[j].y), dp.acc);
            put(&force[3 * ii + 2], fscale * qf * ((fz[j].x + fz[j].y) + fibc), dp.acc);
            if (POT) {
                const double z = (double)u[j].z * 0x1p-32 * dp.Lz;
                put(&phi[ii], pscale * ((ph[j].x + ph[j].y) + (float)(z * dqz + dqc + self2 * (double)qf)), dp.acc);
            }
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&counters[2], 1u) == gridDim.x - 1) {  // every CTA is past its last fetch
            counters[1] = 0u;
            counters[2] = 0u;
            __threadfence();
        }
    }
}

template <bool DIEL, bool POT>
__global__ void __launch_bounds__(256) force64_kernel(DevParams dp, const Part64* __restrict__ part, int64_t N,
                                                      const KRec64* __restrict__ krec,
                                                      const double* __restrict__ scal, int ibc,
                                                      double* __restrict__ force, double* __restrict__ phi,
                                                      double fscale, double pscale) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    KRec64* ks = reinterpret_cast<KRec64*>(smem_raw);
    const int P = dp.P;
    const int ntile = (P + F_KTILE64 - 1) / F_KTILE64;
    const int64_t b = blockIdx.x, nb = gridDim.x;
    const int64_t p0 = (N * b) / nb, p1 = (N * (b + 1)) / nb;
    const double fibc = ibc ? scal[SC_FIBC] : 0.0;
    const double dqz = ibc ? scal[SC_DQ_IBC_Z] : 0.0, dqc = ibc ? scal[SC_DQ_IBC_C] : 0.0;
    const double self2 = -2.0 * dp.alpha / sqrt(M_PI) * dp.kc;
    auto load_tile = [&](int t) {
        const int k0 = t * F_KTILE64, n = min(F_KTILE64, P - k0);
        const uint4* src = reinterpret_cast<const uint4*>(krec + k0);
        uint4* dst = reinterpret_cast<uint4*>(ks);
        for (int i = threadIdx.x; i < 6 * n; i += blockDim.x) dst[i] = src[i];
    };
    if (ntile == 1) { load_tile(0); __syncthreads(); }
    for (int64_t base = p0; base < p1; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool active = i < p1;
        Part64 u = {0, 0, 0, 0.0};
        if (active) u = part[i];
        double fx = 0, fy = 0, fz = 0, ph = 0;
        for (int t = 0; t < ntile; t++) {
            if (ntile > 1) { __syncthreads(); load_tile(t); __syncthreads(); }
            const int n = min(F_KTILE64, P - t * F_KTILE64);
            if (active) {
                for (int l = 0; l < n; l++) {
                    const KRec64 r = ks[l];
                    const unsigned long long txy = (unsigned long long)r.nx * u.ux + (unsigned long long)r.ny * u.uy;
                    const unsigned long long tz = (unsigned long long)r.nz * u.uz;
                    double s1, c1;
                    sincos_turn64(txy + tz, &s1, &c1);
                    const double g1 = r.Ai * c1 - r.Ar * s1;
                    if (DIEL) {
                        double s2, c2;
                        sincos_turn64(txy - tz, &s2, &c2);
                        const double g2 = r.Bi * c2 - r.Br * s2;
                        fx += r.kx * (g1 + g2);
                        fy += r.ky * (g1 + g2);
                        fz += r.kz * (g1 - g2);
                        if (POT) ph -= r.Ar * c1 + r.Ai * s1 + r.Br * c2 + r.Bi * s2;
                    } else {
                        fx += r.kx * g1;
                        fy += r.ky * g1;
                        fz += r.kz * g1;
                        if (POT) ph -= r.Ar * c1 + r.Ai * s1;
                    }
                }
            }
        }
        if (active) {
            put(&force[3 * i + 0], fscale * u.q * fx, dp.acc);
            put(&force[3 * i + 1], fscale * u.q * fy, dp.acc);
            put(&force[3 * i + 2], fscale * u.q * (fz + fibc), dp.acc);
            if (POT) {
                const double z = (double)u.uz * 0x1p-64 * dp.Lz;
                put(&phi[i], pscale * (ph + z * dqz + dqc + self2 * u.q), dp.acc);
            }
        }
    }
}

}  // namespace

template <bool DIEL, bool POT, int SHAPE>
void launch_force32_shape(cudaStream_t st, int grid, size_t sm, int fpoly, const DevParams& d, const uint4* part,
                          int64_t N, const KPair32* krec, const double* scal, int ibc, float* force, float* phi,
                          float fs, float ps, unsigned* counters) {
    constexpr int T = kForceThreads[SHAPE], R = kForceR[SHAPE], MB = kForceMinBlocks[SHAPE], S = kForceSplit[SHAPE];
    // tuner level 0, 1, 2, 3: FPOLY = 0, 1, 2, 4 (2: the pair of particle 0, paired on the FMA pipe)
    switch (fpoly) {
        case 1: force32_kernel<DIEL, POT, 1, T, R, MB, S><<<grid, T, sm, st>>>(d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        case 2: force32_kernel<DIEL, POT, 2, T, R, MB, S><<<grid, T, sm, st>>>(d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        case 3: force32_kernel<DIEL, POT, 4, T, R, MB, S><<<grid, T, sm, st>>>(d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        default: force32_kernel<DIEL, POT, 0, T, R, MB, S><<<grid, T, sm, st>>>(d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
    }
}

// The potential variant (the adjoint and RBE2D_POTENTIAL) in its own shapes, kPot* in
// rbe2d_internal.h (its extra sums need more registers: 256 x 2 takes 76 without a cut;
// cut to 64 for 4 CTAs per SM it has no spills).
template <bool DIEL, int SHAPE>
void launch_force32_pot_shape(cudaStream_t st, int grid, size_t sm, int fpoly, const DevParams& d,
                              const uint4* part, int64_t N, const KPair32* krec, const double* scal, int ibc,
                              float* force, float* phi, float fs, float ps, unsigned* counters) {
    constexpr int T = kPotThreads[SHAPE], R = kPotR[SHAPE], MB = kPotMinBlocks[SHAPE], S = kPotSplit[SHAPE];
    switch (fpoly) {
        case 1: force32_kernel<DIEL, true, 1, T, R, MB, S><<<grid, T, sm, st>>>(d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        case 2: force32_kernel<DIEL, true, 2, T, R, MB, S><<<grid, T, sm, st>>>(d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        case 3: force32_kernel<DIEL, true, 4, T, R, MB, S><<<grid, T, sm, st>>>(d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        default: force32_kernel<DIEL, true, 0, T, R, MB, S><<<grid, T, sm, st>>>(d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
    }
}

template <bool DIEL>
void launch_force32_pot(cudaStream_t st, int grid, size_t sm, int fpoly, int shape, const DevParams& d,
                        const uint4* part, int64_t N, const KPair32* krec, const double* scal, int ibc, float* force,
                        float* phi, float fs, float ps, unsigned* counters) {
    switch (shape) {
        case 1: launch_force32_pot_shape<DIEL, 1>(st, grid, sm, fpoly, d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        case 2: launch_force32_pot_shape<DIEL, 2>(st, grid, sm, fpoly, d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        case 3: launch_force32_pot_shape<DIEL, 3>(st, grid, sm, fpoly, d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        default: launch_force32_pot_shape<DIEL, 0>(st, grid, sm, fpoly, d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
    }
}

template <bool DIEL, bool POT>
void launch_force32_poly(cudaStream_t st, int grid, size_t sm, int fpoly, int shape, const DevParams& d,
                         const uint4* part, int64_t N, const KPair32* krec, const double* scal, int ibc, float* force,
                         float* phi, float fs, float ps, unsigned* counters) {
    if constexpr (POT) {
        launch_force32_pot<DIEL>(st, grid, sm, fpoly, shape, d, part, N, krec, scal, ibc, force, phi, fs, ps, counters);
    } else {
    switch (shape) {
        case 1: launch_force32_shape<DIEL, POT, 1>(st, grid, sm, fpoly, d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        case 2: launch_force32_shape<DIEL, POT, 2>(st, grid, sm, fpoly, d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        case 3: launch_force32_shape<DIEL, POT, 3>(st, grid, sm, fpoly, d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        case 4: launch_force32_shape<DIEL, POT, 4>(st, grid, sm, fpoly, d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        case 5: launch_force32_shape<DIEL, POT, 5>(st, grid, sm, fpoly, d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        case 6: launch_force32_shape<DIEL, POT, 6>(st, grid, sm, fpoly, d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
        default: launch_force32_shape<DIEL, POT, 0>(st, grid, sm, fpoly, d, part, N, krec, scal, ibc, force, phi, fs, ps, counters); break;
    }
    }
}

size_t force32_smem(int P) { return sizeof(KPair32) * (size_t)((max(1, min(P, F_KTILE32)) + 1) / 2); }
size_t force64_smem(int P) { return sizeof(KRec64) * (size_t)max(1, min(P, F_KTILE64)); }

cudaError_t launch_force(cudaStream_t st, const DevParams& dp, int64_t N, const void* part, bool fp64,
                         const void* krec, const double* scal, int flags, void* force, void* phi,
                         double fscale, double pscale, const Shapes& sh, unsigned* counters, int fpoly, int fshape) {
    const bool pot = (flags & RBE2D_POTENTIAL) && phi;
    if (fp64 || fshape < 0 || fshape >= (pot ? kPotShapes : kForceShapes)) fshape = 0;
    // one full wave of resident CTAs, no more than there are rounds
    const int64_t per_cta = fp64  ? 256
                            : pot ? (int64_t)kPotThreads[fshape] / kPotSplit[fshape] * kPotR[fshape]
                                  : (int64_t)kForceThreads[fshape] / kForceSplit[fshape] * kForceR[fshape];
    int grid = sh.sms * (fp64 ? sh.force_occ64 : pot ? sh.pot_occ32[fshape] : sh.force_occ32[fshape]);
    const int64_t need = (N + per_cta - 1) / per_cta;
    if (need < grid) grid = (int)(need > 0 ? need : 1);
    const int ibc = (flags & RBE2D_IBC) ? 1 : 0;
    const bool diel = dp.diel != 0;
    DevParams d = dp;
    if (!(flags & RBE2D_KSPACE)) {
        d.P = 0;        // no k-space term
        d.alpha = 0.0;  // and no self term in dU/dq (it belongs to the k-space part, Eq. 2.7)
    }
    if (flags & kForceNoSelf) d.alpha = 0.0;
    d.acc = (flags & RBE2D_ACCUMULATE) ? 1 : 0;
    if (fp64) {
        size_t sm = force64_smem(dp.P);
        double fs = fscale, ps = pscale;
        if (diel) {
            if (pot) force64_kernel<true, true><<<grid, 256, sm, st>>>(d, (const Part64*)part, N, (const KRec64*)krec, scal, ibc, (double*)force, (double*)phi, fs, ps);
            else force64_kernel<true, false><<<grid, 256, sm, st>>>(d, (const Part64*)part, N, (const KRec64*)krec, scal, ibc, (double*)force, (double*)phi, fs, ps);
        } else {
            if (pot) force64_kernel<false, true><<<grid, 256, sm, st>>>(d, (const Part64*)part, N, (const KRec64*)krec, scal, ibc, (double*)force, (double*)phi, fs, ps);
            else force64_kernel<false, false><<<grid, 256, sm, st>>>(d, (const Part64*)part, N, (const KRec64*)krec, scal, ibc, (double*)force, (double*)phi, fs, ps);
        }
    } else {
        size_t sm = force32_smem(dp.P);
        float fs = (float)fscale, ps = (float)pscale;
        const uint4* pp = (const uint4*)part;
        const KPair32* kr = (const KPair32*)krec;
        if (diel) {
            if (pot) launch_force32_poly<true, true>(st, grid, sm, fpoly, fshape, d, pp, N, kr, scal, ibc, (float*)force, (float*)phi, fs, ps, counters);
            else launch_force32_poly<true, false>(st, grid, sm, fpoly, fshape, d, pp, N, kr, scal, ibc, (float*)force, (float*)phi, fs, ps, counters);
        } else {
            if (pot) launch_force32_poly<false, true>(st, grid, sm, fpoly, fshape, d, pp, N, kr, scal, ibc, (float*)force, (float*)phi, fs, ps, counters);
            else launch_force32_poly<false, false>(st, grid, sm, fpoly, fshape, d, pp, N, kr, scal, ibc, (float*)force, (float*)phi, fs, ps, counters);
        }
    }
    note_launches(1);
    return cudaGetLastError();
}

template <int SHAPE>
static cudaError_t occ32_shape(int* occ, size_t sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        occ, force32_kernel<true, false, 0, kForceThreads[SHAPE], kForceR[SHAPE], kForceMinBlocks[SHAPE], kForceSplit[SHAPE]>,
        kForceThreads[SHAPE], sm);
}

template <int SHAPE>
static cudaError_t occ32_pot_shape(int* occ, size_t sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        occ, force32_kernel<true, true, 0, kPotThreads[SHAPE], kPotR[SHAPE], kPotMinBlocks[SHAPE], kPotSplit[SHAPE]>,
        kPotThreads[SHAPE], sm);
}

cudaError_t pot_occupancy(int P_pad, int* occ32) {
    const size_t sm32 = force32_smem(P_pad);
    cudaError_t e = occ32_pot_shape<0>(&occ32[0], sm32);
    if (e == cudaSuccess) e = occ32_pot_shape<1>(&occ32[1], sm32);
    if (e == cudaSuccess) e = occ32_pot_shape<2>(&occ32[2], sm32);
    if (e == cudaSuccess) e = occ32_pot_shape<3>(&occ32[3], sm32);
    return e;
}

cudaError_t force_occupancy(int P_pad, int* occ32, int* occ64) {
    // the dielectric force without potential (the MD and benchmark launch) in each shape;
    // variants with more registers get a grid above their resident capacity, which the
    // work counter absorbs (late CTAs take what is left)
    const size_t sm32 = force32_smem(P_pad);
    cudaError_t e = occ32_shape<0>(&occ32[0], sm32);
    if (e == cudaSuccess) e = occ32_shape<1>(&occ32[1], sm32);
    if (e == cudaSuccess) e = occ32_shape<2>(&occ32[2], sm32);
    if (e == cudaSuccess) e = occ32_shape<3>(&occ32[3], sm32);
    if (e == cudaSuccess) e = occ32_shape<4>(&occ32[4], sm32);
    if (e == cudaSuccess) e = occ32_shape<5>(&occ32[5], sm32);
    if (e == cudaSuccess) e = occ32_shape<6>(&occ32[6], sm32);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ64, force64_kernel<true, true>, 256, force64_smem(P_pad));
}

}  // namespace rbe2d
