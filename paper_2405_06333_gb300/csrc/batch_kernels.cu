// Batched k-space force for many independent slab systems in one persistent launch.
//
// Work queue (one atomic head): all structure-factor items (system, particle chunk) come
// before all force items (system, particle chunk).  A structure-factor item sums
// q e^{i k.r}, q e^{i khat.r} over its chunk for every k of its system and writes the
// partial sums; the CTA that completes a system's last chunk folds that system (fixed
// chunk order, so bitwise reproducible), writes its force records and energies and
// publishes a ready flag.  A force item waits for its system's flag with a bounded spin
// (%globaltimer, ~2 s), then evaluates Eq. 3.26 for its chunk.  Waiting cannot deadlock:
// every structure-factor item has been taken, before any force item, by a running CTA
// that never waits.  The last CTA to leave re-arms the queue, counters and flags.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kcoef.cuh"
#include "rbe2d_internal.h"

namespace rbe2d {

namespace {

constexpr double kTwoPiB = 6.283185307179586476925286766559;

__device__ __forceinline__ void sincos_turn(uint32_t t, float* s, float* c) {
    __sincosf((float)(int32_t)t * 1.46291807926715968e-09f, s, c);
}

__device__ __forceinline__ uint32_t turn(double v, double scale) {
    return (uint32_t)(unsigned long long)__double2ll_rn(v * scale);
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ double bsum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
    return t;
}

// Fold of one system by one CTA: partial sums in chunk order -> A, B, force records,
// energies and IBC factors (as the single-system fold and finalize).
__device__ void fold_system(const BatchArgs& a, int s, double* red) {
    const BatchSys& bs = a.sys[s];
    const DevParams& dp = bs.dp;
    double u = 0.0;
    for (int l = threadIdx.x; l < dp.P; l += blockDim.x) {
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        const double* pp = a.partial + bs.part_base + (size_t)l * bs.nsf * 4;
        for (int c = 0; c < bs.nsf; c++) {
            a0 += __ldcg(&pp[4 * c]); a1 += __ldcg(&pp[4 * c + 1]);
            a2 += __ldcg(&pp[4 * c + 2]); a3 += __ldcg(&pp[4 * c + 3]);
        }
        const KCoef k = a.kc[(size_t)s * a.P_max + l];
        const double Ar = (2.0 + 2.0 * k.E) * a0 + (k.Ore * a2 + k.Oim * a3);
        const double Ai = (2.0 + 2.0 * k.E) * a1 + (k.Ore * a3 - k.Oim * a2);
        const double Br = k.Ore * a0 - k.Oim * a1;
        const double Bi = k.Ore * a1 + k.Oim * a0;
        const double pr = a0 * a2 + a1 * a3, pi_ = a1 * a2 - a0 * a3;
        u += -k.c * ((1.0 + k.E) * (a0 * a0 + a1 * a1) + (k.Ore * pr - k.Oim * pi_));
        KRec32 r;
        r.nx = k.nx; r.ny = k.ny; r.nz = k.nz; r.pad0 = 0;
        r.kx = (float)k.kx; r.ky = (float)k.ky; r.kz = (float)k.kz; r.pad1 = 0.f;
        r.Ar = (float)(k.c * Ar); r.Ai = (float)(k.c * Ai); r.Br = (float)(k.c * Br); r.Bi = (float)(k.c * Bi);
        a.krec[(size_t)s * a.P_max + l] = r;
    }
    double Q = 0, Q2 = 0, mu = 0;
    for (int c = threadIdx.x; c < bs.nsf; c += blockDim.x) {
        const double* o = a.pack + (size_t)(bs.sf_base + c) * 4;
        Q += __ldcg(&o[0]); Q2 += __ldcg(&o[1]); mu += __ldcg(&o[2]);
    }
    u = bsum(u, red); Q = bsum(Q, red); Q2 = bsum(Q2, red); mu = bsum(mu, red);
    if (threadIdx.x == 0) {
        const double pre = kTwoPiB / dp.V * dp.kc;
        const double inner = dp.cM * mu + Q * dp.H * dp.dM;
        double* sc = a.scal + (size_t)s * 4;
        sc[0] = u;
        sc[1] = -dp.alpha / sqrt(M_PI) * Q2 * dp.kc;
        sc[2] = pre * mu * inner;
        sc[3] = -pre * (dp.cM * mu + inner);  // F_IBC,z = q_i * sc[3]
    }
}

template <int KR>
__global__ void __launch_bounds__(128) batch_persistent_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[4];
    __shared__ int item_sh;
    __shared__ int flag_sh;
    uint4* tile = reinterpret_cast<uint4*>(smem);    // structure-factor items: particle tile
    KRec32* ks = reinterpret_cast<KRec32*>(smem);    // force items: the system's k records
    const int n_items = a.n_sf_items + a.n_f_items;
    for (;;) {
        if (threadIdx.x == 0) item_sh = atomicAdd(a.head, 1);
        __syncthreads();
        const int item = item_sh;
        __syncthreads();
        if (item >= n_items) break;
        if (item < a.n_sf_items) {
            // ---------------------------------------------------------------- structure factor
            const int s = a.item_sys[item];
            const BatchSys& bs = a.sys[s];
            const DevParams& dp = bs.dp;
            const int c = item - bs.sf_base;
            const int64_t p0 = bs.off + (int64_t)c * a.sf_chunk;
            const int64_t p1 = min((long long)(bs.off + bs.N), (long long)(p0 + a.sf_chunk));
            int nx[KR], ny[KR], nz[KR];
            for (int j = 0; j < KR; j++) {
                const int k = threadIdx.x + j * blockDim.x;
                const bool ok = k < dp.P;
                const KCoef* kk = a.kc + (size_t)s * a.P_max + (ok ? k : 0);
                nx[j] = ok ? kk->nx : 0; ny[j] = ok ? kk->ny : 0; nz[j] = ok ? kk->nz : 0;
            }
            const double sx = 4294967296.0 * dp.inv_Lx, sy = 4294967296.0 * dp.inv_Ly, sz = 4294967296.0 * dp.inv_Lz;
            double ar[KR], ai[KR], br[KR], bi[KR];
            for (int j = 0; j < KR; j++) ar[j] = ai[j] = br[j] = bi[j] = 0.0;
            double sQ = 0, sQ2 = 0, sMu = 0;
            for (int64_t t0 = p0; t0 < p1; t0 += blockDim.x) {
                const int n = (int)min((int64_t)blockDim.x, p1 - t0);
                __syncthreads();
                if (threadIdx.x < n) {
                    const int64_t i = t0 + threadIdx.x;
                    const double x = a.pos[3 * i], y = a.pos[3 * i + 1], z = a.pos[3 * i + 2], qv = a.q[i];
                    tile[threadIdx.x] = make_uint4(turn(x, sx), turn(y, sy), turn(z, sz), __float_as_uint((float)qv));
                    sQ += qv; sQ2 += qv * qv; sMu += qv * z;
                }
                __syncthreads();
                float fr[KR], fi[KR], gr[KR], gi[KR];
                for (int j = 0; j < KR; j++) fr[j] = fi[j] = gr[j] = gi[j] = 0.f;
                for (int p = 0; p < n; p++) {
                    const uint4 u = tile[p];
                    const float qf = __uint_as_float(u.w);
#pragma unroll
                    for (int j = 0; j < KR; j++) {
                        const uint32_t txy = (uint32_t)nx[j] * u.x + (uint32_t)ny[j] * u.y;
                        const uint32_t tz = (uint32_t)nz[j] * u.z;
                        float s1, c1, s2, c2;
                        sincos_turn(txy + tz, &s1, &c1);
                        sincos_turn(txy - tz, &s2, &c2);
                        fr[j] = fmaf(qf, c1, fr[j]); fi[j] = fmaf(qf, s1, fi[j]);
                        gr[j] = fmaf(qf, c2, gr[j]); gi[j] = fmaf(qf, s2, gi[j]);
                    }
                }
                for (int j = 0; j < KR; j++) { ar[j] += fr[j]; ai[j] += fi[j]; br[j] += gr[j]; bi[j] += gi[j]; }
            }
            for (int j = 0; j < KR; j++) {
                const int k = threadIdx.x + j * blockDim.x;
                if (k < dp.P) {
                    double* o = a.partial + bs.part_base + ((size_t)k * bs.nsf + c) * 4;
                    o[0] = ar[j]; o[1] = ai[j]; o[2] = br[j]; o[3] = bi[j];
                }
            }
            sQ = bsum(sQ, red); sQ2 = bsum(sQ2, red); sMu = bsum(sMu, red);
            if (threadIdx.x == 0) {
                double* o = a.pack + (size_t)item * 4;
                o[0] = sQ; o[1] = sQ2; o[2] = sMu; o[3] = 0.0;
                __threadfence();
                flag_sh = atomicAdd(&a.sf_done[s], 1) == bs.nsf - 1;
            }
            __syncthreads();
            if (flag_sh) {  // this CTA finished the system's last chunk: fold it
                __threadfence();
                fold_system(a, s, red);
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    atomicExch(&a.ready[s], 1);
                }
            }
        } else {
            // ---------------------------------------------------------------- force
            const int fi_ = item - a.n_sf_items;
            const int s = a.item_sys[item];
            const BatchSys& bs = a.sys[s];
            const DevParams& dp = bs.dp;
            const int c = fi_ - bs.f_base;
            if (threadIdx.x == 0) {  // bounded wait for the system's fold
                int ok = 1;
                const unsigned long long t_start = globaltimer();
                while (atomicAdd(&a.ready[s], 0) == 0) {
                    if (globaltimer() - t_start > 2000000000ull) {
                        atomicAdd(&a.status[ST_TIMEOUT], 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(200);
                }
                flag_sh = ok;
            }
            __syncthreads();
            if (!flag_sh) continue;  // timed out: this chunk is left unwritten, the host is told
            __threadfence();
            for (int l = threadIdx.x; l < dp.P; l += blockDim.x) ks[l] = a.krec[(size_t)s * a.P_max + l];
            __syncthreads();
            const double sx = 4294967296.0 * dp.inv_Lx, sy = 4294967296.0 * dp.inv_Ly, sz = 4294967296.0 * dp.inv_Lz;
            const float fibc = a.ibc ? (float)__ldcg(&a.scal[(size_t)s * 4 + 3]) : 0.f;
            const int64_t p0 = bs.off + (int64_t)c * a.f_chunk;
            const int64_t p1 = min((long long)(bs.off + bs.N), (long long)(p0 + a.f_chunk));
            for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
                const uint32_t ux = turn(a.pos[3 * i], sx), uy = turn(a.pos[3 * i + 1], sy), uz = turn(a.pos[3 * i + 2], sz);
                const float qf = (float)a.q[i];
                float fx = 0.f, fy = 0.f, fz = 0.f;
                for (int l = 0; l < dp.P; l++) {
                    const KRec32 r = ks[l];
                    const uint32_t txy = (uint32_t)r.nx * ux + (uint32_t)r.ny * uy;
                    const uint32_t tz = (uint32_t)r.nz * uz;
                    float s1, c1, s2, c2;
                    sincos_turn(txy + tz, &s1, &c1);
                    sincos_turn(txy - tz, &s2, &c2);
                    const float g1 = fmaf(r.Ai, c1, -r.Ar * s1), g2 = fmaf(r.Bi, c2, -r.Br * s2);
                    fx = fmaf(r.kx, g1 + g2, fx);
                    fy = fmaf(r.ky, g1 + g2, fy);
                    fz = fmaf(r.kz, g1 - g2, fz);
                }
                a.force[3 * i + 0] = qf * fx;
                a.force[3 * i + 1] = qf * fy;
                a.force[3 * i + 2] = qf * (fz + fibc);
            }
            __syncthreads();
        }
    }
    // leave: the last CTA re-arms the queue, the per-system counters and flags
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        flag_sh = atomicAdd(a.exit_count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!flag_sh) return;
    __threadfence();
    for (int s = threadIdx.x; s < a.n_sys; s += blockDim.x) {
        a.sf_done[s] = 0;
        a.ready[s] = 0;
    }
    if (threadIdx.x == 0) {
        *a.head = 0;
        *a.exit_count = 0u;
    }
}

// Batched k sampler: one thread per (system, k); the same draws as rbe2d_sample_k would
// make for the system alone (Philox key = the system's seed).
__global__ void batch_sample_kernel(BatchArgs a, const double* __restrict__ cdf, const int* __restrict__ guide,
                                    unsigned long long step) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int s = (int)(g / a.P_max), l = (int)(g % a.P_max);
    if (s >= a.n_sys) return;
    const BatchSys& bs = a.sys[s];
    KCoef* out = const_cast<KCoef*>(a.kc) + (size_t)s * a.P_max + l;
    if (l >= bs.dp.P) return;
    int n[3] = {1, 0, 0};
    bool ok = false;
    for (int att = 0; att < 64 && !ok; att++) {
        unsigned long long c[4] = {(unsigned long long)l, (unsigned long long)att, step, 0ULL};
        kdetail::philox4x64_10(c, bs.seed, 0ULL);
        int m[3];
        for (int d = 0; d < 3; d++) {
            const int len = bs.tab_len[d];
            m[d] = kdetail::first_above(cdf + bs.tab_off[d], guide + bs.tab_off[d], len,
                                        (double)(c[d] >> 11) * 0x1p-53) - len / 2;
        }
        if (m[0] != 0 || m[1] != 0 || m[2] != 0) {
            n[0] = m[0]; n[1] = m[1]; n[2] = m[2];
            ok = true;
        }
    }
    if (!ok) atomicAdd(&a.status[ST_SAMPLER], 1);
    kdetail::fill_kcoef(bs.dp, n[0], n[1], n[2], out);
}

}  // namespace

cudaError_t launch_batch_sample(cudaStream_t st, const BatchArgs& a, const double* cdf, const int* guide,
                                uint64_t step) {
    const long long total = (long long)a.n_sys * a.P_max;
    batch_sample_kernel<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(a, cdf, guide, step);
    note_launches(1);
    return cudaGetLastError();
}

size_t batch_smem_bytes(int P_max) {
    size_t a = sizeof(uint4) * 128, b = sizeof(KRec32) * (size_t)P_max;
    return a > b ? a : b;
}

// Wave vectors per thread: the smallest of 1, 2, 4 with 128 KR >= P_max.
cudaError_t launch_batch(cudaStream_t st, const BatchArgs& a, int grid) {
    const size_t sm = batch_smem_bytes(a.P_max);
    if (a.P_max <= 128) batch_persistent_kernel<1><<<grid, 128, sm, st>>>(a);
    else if (a.P_max <= 256) batch_persistent_kernel<2><<<grid, 128, sm, st>>>(a);
    else batch_persistent_kernel<4><<<grid, 128, sm, st>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t batch_occupancy(int P_max, int* per_sm) {
    const size_t sm = batch_smem_bytes(P_max);
    if (P_max <= 128) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_persistent_kernel<1>, 128, sm);
    if (P_max <= 256) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_persistent_kernel<2>, 128, sm);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_persistent_kernel<4>, 128, sm);
}

}  // namespace rbe2d
