// Batched k-space force for many independent slab systems in one persistent launch.
//
// Work queue (one atomic head): all structure-factor items (system, particle chunk) come
// before all force items (system, particle chunk).  A structure-factor item converts its
// particles once to 16-byte fixed-point records {ux, uy, uz, q} (kept in `part` for the
// force items), sums q e^{i k.r}, q e^{i khat.r} over its chunk for every k of its system
// and writes the partial sums; the CTA that completes a system's last chunk folds that system (fixed
// chunk order, so bitwise reproducible), writes its force records and energies and
// publishes a ready flag.  A force item waits for its system's flag with a bounded spin
// (%globaltimer, 2 s unless set otherwise), then evaluates Eq. 3.26 for its chunk; a wait
// that runs out raises the timeout status and leaves the chunk unwritten.  Waiting cannot deadlock:
// every structure-factor item has been taken, before any force item, by a running CTA
// that never waits.  The last CTA to leave re-arms the queue, counters and flags.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kcoef.cuh"
#include "pair32.cuh"
#include "rbe2d_internal.h"

namespace rbe2d {

namespace {

constexpr double kTwoPiB = 6.283185307179586476925286766559;

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
    KPair32* rec = a.krec + (size_t)s * a.KP;
    // an odd P: the k1 half of the last record is zero (it adds exactly nothing)
    if ((dp.P & 1) && threadIdx.x == 0) pair32::set_half(&rec[dp.P >> 1], 1, 0, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
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
        pair32::set_half(&rec[l >> 1], l & 1, k.nx, k.ny, k.nz, (float)k.kx, (float)k.ky, (float)k.kz,
                         (float)(k.c * Ar), (float)(k.c * Ai), (float)(k.c * Br), (float)(k.c * Bi));
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

// The float32 sums of one structure-factor tile for the first JL of a thread's KR k slots:
// particles taken two at a time (x halves: entry 2m, y halves: entry 2m + 1; an odd tile
// ends with a zero-charge record).
template <int KR, int JL, bool POLY>
__device__ __forceinline__ void sf_tile_sums(const uint4* tile, int n, const uint32_t* nx, const uint32_t* ny,
                                             const uint32_t* nz, float2* fr, float2* fi, float2* gr, float2* gi) {
    for (int p = 0; p < n; p += 2) {
        const uint4 ua = tile[p], ub = tile[p + 1];
        const float2 q2 = make_float2(__uint_as_float(ua.w), __uint_as_float(ub.w));
#pragma unroll
        for (int j = 0; j < JL; j++) {
            const uint32_t txya = nx[j] * ua.x + ny[j] * ua.y, tza = nz[j] * ua.z;
            const uint32_t txyb = nx[j] * ub.x + ny[j] * ub.y, tzb = nz[j] * ub.z;
            float2 s1, c1, s2, c2;
            pair32::sincos_turn32x2(txya + tza, txyb + tzb, false, false, s1, c1);
            // POLY: one angle in 2 JL x 2 (the first slot's k-hat angle of particle a) on the FMA pipe
            pair32::sincos_turn32x2(txya - tza, txyb - tzb, POLY && j == 0, false, s2, c2);
            fr[j] = __ffma2_rn(q2, c1, fr[j]); fi[j] = __ffma2_rn(q2, s1, fi[j]);
            gr[j] = __ffma2_rn(q2, c2, gr[j]); gi[j] = __ffma2_rn(q2, s2, gi[j]);
        }
    }
}

// Particles per structure-factor tile (two per thread) and per force pass (two per thread).
constexpr int kBatchThreads = 128;
constexpr int kBatchSfTile = 2 * kBatchThreads;
constexpr int kBatchFPass = 2 * kBatchThreads;

// MINB: resident CTAs per SM the compiler must allow (1: registers as needed; 8: at most
// 64 registers per thread, which can spill a little); POLY: one angle of each group in
// the structure-factor items on the FMA-pipe polynomial -- choices of the batch autotuner.
template <int KR, int MINB, bool POLY>
__global__ void __launch_bounds__(kBatchThreads, MINB) batch_persistent_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[4];
    __shared__ uint32_t tail_n[3][16];  // structure-factor items: the split last group's nx, ny, nz
    __shared__ double tail_acc[4][16];  // and its float64 sums (warp 3 only)
    __shared__ int item_sh;
    __shared__ int flag_sh;
    uint4* tile = reinterpret_cast<uint4*>(smem);    // structure-factor items: particle tile
    KPair32* ks = reinterpret_cast<KPair32*>(smem);  // force items: the system's k records
    const int n_items = a.n_sf_items + a.n_f_items;
    const float2 zero2 = make_float2(0.f, 0.f);
    for (;;) {
        if (threadIdx.x == 0) item_sh = atomicAdd(a.head, 1);
        __syncthreads();
        const int item = item_sh;
        __syncthreads();
        if (item >= n_items) break;
        if (item < a.n_sf_items) {
            // ---------------------------------------------------------------- structure factor
            // thread t owns k = t + j 128 (j < KR); the particles of a tile are taken two at
            // a time, particle 2m in the x halves and 2m + 1 in the y halves of paired
            // float32 sums (an odd tile ends with a zero-charge record, which adds nothing)
            const int s = a.item_sys[item];
            const BatchSys& bs = a.sys[s];
            const DevParams& dp = bs.dp;
            const int c = item - bs.sf_base;
            const int64_t p0 = bs.off + (int64_t)c * a.sf_chunk;
            const int64_t p1 = min((long long)(bs.off + bs.N), (long long)(p0 + a.sf_chunk));
            uint32_t nx[KR], ny[KR], nz[KR];
#pragma unroll
            for (int j = 0; j < KR; j++) {
                const int k = threadIdx.x + j * kBatchThreads;
                const bool ok = k < dp.P;
                const KCoef* kk = a.kc + (size_t)s * a.P_max + (ok ? k : 0);
                nx[j] = ok ? (uint32_t)kk->nx : 0u; ny[j] = ok ? (uint32_t)kk->ny : 0u; nz[j] = ok ? (uint32_t)kk->nz : 0u;
            }
            // groups of 32 wave vectors: group g is warp g % 4's slot g / 4.  A last group with
            // at most 16 live wave vectors goes to warp 3 (the fewest groups) with its lanes
            // split over the particles -- L wave vectors x 32 / 2^lg particle phases -- instead
            // of a slot with 32 - L idle lanes.
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            const int G = (dp.P + 31) >> 5, L = dp.P - 32 * (G - 1);
            const bool split = L <= 16;
            const int Greg = G - (split ? 1 : 0);
            int lg = 0;
            while ((1 << lg) < L) lg++;
            if (split && warp == 3) {
                if (lane < L) {
                    const KCoef* kk = a.kc + (size_t)s * a.P_max + 32 * (G - 1) + lane;
                    tail_n[0][lane] = (uint32_t)kk->nx; tail_n[1][lane] = (uint32_t)kk->ny;
                    tail_n[2][lane] = (uint32_t)kk->nz;
                }
                if (lane < 16) tail_acc[0][lane] = tail_acc[1][lane] = tail_acc[2][lane] = tail_acc[3][lane] = 0.0;
                __syncwarp();
            }
            const double sx = 4294967296.0 * dp.inv_Lx, sy = 4294967296.0 * dp.inv_Ly, sz = 4294967296.0 * dp.inv_Lz;
            double ar[KR], ai[KR], br[KR], bi[KR];
#pragma unroll
            for (int j = 0; j < KR; j++) ar[j] = ai[j] = br[j] = bi[j] = 0.0;
            double sQ = 0, sQ2 = 0, sMu = 0;
            for (int64_t t0 = p0; t0 < p1; t0 += kBatchSfTile) {
                const int n = (int)min((int64_t)kBatchSfTile, p1 - t0);
                __syncthreads();
                for (int e = threadIdx.x; e < ((n + 1) & ~1); e += kBatchThreads) {
                    uint4 u = make_uint4(0u, 0u, 0u, 0u);
                    if (e < n) {
                        const int64_t i = t0 + e;
                        const double x = a.pos[3 * i], y = a.pos[3 * i + 1], z = a.pos[3 * i + 2], qv = a.q[i];
                        u = make_uint4(turn(x, sx), turn(y, sy), turn(z, sz), __float_as_uint((float)qv));
                        a.part[i] = u;  // the force items read this record
                        sQ += qv; sQ2 += qv * qv; sMu += qv * z;
                    }
                    tile[e] = u;
                }
                __syncthreads();
                float2 fr[KR], fi[KR], gr[KR], gi[KR];
#pragma unroll
                for (int j = 0; j < KR; j++) fr[j] = fi[j] = gr[j] = gi[j] = zero2;
                // a warp whose last k slots all lie past P (or hold the split group) runs a
                // loop without them (one warp-uniform choice per tile, outside the particle loop)
                const int jlive = min(KR, (Greg - warp + 3) >> 2);
                if (jlive >= KR) sf_tile_sums<KR, KR, POLY>(tile, n, nx, ny, nz, fr, fi, gr, gi);
                else if (KR >= 4 && jlive == 3) sf_tile_sums<KR, (KR >= 4 ? 3 : 1), POLY>(tile, n, nx, ny, nz, fr, fi, gr, gi);
                else if (KR >= 3 && jlive == 2) sf_tile_sums<KR, (KR >= 3 ? 2 : 1), POLY>(tile, n, nx, ny, nz, fr, fi, gr, gi);
                else if (jlive == 1) sf_tile_sums<KR, 1, POLY>(tile, n, nx, ny, nz, fr, fi, gr, gi);
#pragma unroll
                for (int j = 0; j < KR; j++) {
                    ar[j] += fr[j].x + fr[j].y; ai[j] += fi[j].x + fi[j].y;
                    br[j] += gr[j].x + gr[j].y; bi[j] += gi[j].x + gi[j].y;
                }
                if (split && warp == 3) {
                    // lane: wave vector kk of the last group, particle pairs ph, ph + 32 / 2^lg, ...;
                    // the phases' float sums are added by a fixed butterfly, lane kk keeps them
                    const int kk = lane & ((1 << lg) - 1), ph = lane >> lg;
                    const bool live = kk < L;
                    const uint32_t tx = live ? tail_n[0][kk] : 0u, ty = live ? tail_n[1][kk] : 0u,
                                   tz = live ? tail_n[2][kk] : 0u;
                    float2 tr = zero2, ti = zero2, ur = zero2, ui = zero2;
                    for (int m = ph; 2 * m < n; m += 32 >> lg) {
                        const uint4 ua = tile[2 * m], ub = tile[2 * m + 1];
                        const float2 q2 = make_float2(__uint_as_float(ua.w), __uint_as_float(ub.w));
                        const uint32_t txya = tx * ua.x + ty * ua.y, tza = tz * ua.z;
                        const uint32_t txyb = tx * ub.x + ty * ub.y, tzb = tz * ub.z;
                        float2 s1, c1, s2, c2;
                        pair32::sincos_turn32x2(txya + tza, txyb + tzb, false, false, s1, c1);
                        pair32::sincos_turn32x2(txya - tza, txyb - tzb, false, false, s2, c2);
                        tr = __ffma2_rn(q2, c1, tr); ti = __ffma2_rn(q2, s1, ti);
                        ur = __ffma2_rn(q2, c2, ur); ui = __ffma2_rn(q2, s2, ui);
                    }
                    float v0 = tr.x + tr.y, v1 = ti.x + ti.y, v2 = ur.x + ur.y, v3 = ui.x + ui.y;
                    for (int o = 1 << lg; o < 32; o <<= 1) {
                        v0 += __shfl_xor_sync(0xffffffffu, v0, o); v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                        v2 += __shfl_xor_sync(0xffffffffu, v2, o); v3 += __shfl_xor_sync(0xffffffffu, v3, o);
                    }
                    if (ph == 0 && live) {
                        tail_acc[0][kk] += v0; tail_acc[1][kk] += v1;
                        tail_acc[2][kk] += v2; tail_acc[3][kk] += v3;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < KR; j++) {
                const int k = threadIdx.x + j * kBatchThreads;
                if (k < 32 * Greg && k < dp.P) {
                    double* o = a.partial + bs.part_base + ((size_t)k * bs.nsf + c) * 4;
                    o[0] = ar[j]; o[1] = ai[j]; o[2] = br[j]; o[3] = bi[j];
                }
            }
            if (split && warp == 3 && lane < L) {  // lane kk of warp 3 holds wave vector 32 (G - 1) + kk
                double* o = a.partial + bs.part_base + ((size_t)(32 * (G - 1) + lane) * bs.nsf + c) * 4;
                o[0] = tail_acc[0][lane]; o[1] = tail_acc[1][lane]; o[2] = tail_acc[2][lane]; o[3] = tail_acc[3][lane];
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
                if (threadIdx.x == 0 && s != a.withhold) {  // a withheld system is never published
                    __threadfence();
                    atomicExch(&a.ready[s], 1);
                }
            }
        } else {
            // ---------------------------------------------------------------- force
            // passes of 256 particles, two per thread, against the system's records of two
            // wave vectors each: one shared-memory record serves four (particle, k) pairs
            const int fi_ = item - a.n_sf_items;
            const int s = a.item_sys[item];
            const BatchSys& bs = a.sys[s];
            const DevParams& dp = bs.dp;
            const int c = fi_ - bs.f_base;
            if (threadIdx.x == 0) {  // bounded wait for the system's fold
                int ok = 1;
                const unsigned long long t_start = globaltimer();
                while (atomicAdd(&a.ready[s], 0) == 0) {
                    if (globaltimer() - t_start > a.wait_ns) {
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
            const int nrec = (dp.P + 1) >> 1;
            {
                const uint4* src = reinterpret_cast<const uint4*>(a.krec + (size_t)s * a.KP);
                uint4* dst = reinterpret_cast<uint4*>(ks);
                for (int w = threadIdx.x; w < 6 * nrec; w += kBatchThreads) dst[w] = __ldcg(&src[w]);
            }
            __syncthreads();
            const float fibc = a.ibc ? (float)__ldcg(&a.scal[(size_t)s * 4 + 3]) : 0.f;
            const int64_t p0 = bs.off + (int64_t)c * a.f_chunk;
            const int64_t p1 = min((long long)(bs.off + bs.N), (long long)(p0 + a.f_chunk));
            for (int64_t b0 = p0; b0 < p1; b0 += kBatchFPass) {
                const int64_t i0 = b0 + threadIdx.x, i1 = i0 + kBatchThreads;
                const bool a0 = i0 < p1, a1 = i1 < p1;
                const uint4 u0 = a0 ? __ldcg(&a.part[i0]) : make_uint4(0u, 0u, 0u, 0u);
                const uint4 u1 = a1 ? __ldcg(&a.part[i1]) : make_uint4(0u, 0u, 0u, 0u);
                float2 fx0 = zero2, fy0 = zero2, fz0 = zero2, fx1 = zero2, fy1 = zero2, fz1 = zero2, ph = zero2;
                for (int l = 0; l < nrec; l++) {
                    const KPair32 r = ks[l];
                    pair32::force_pair32<true, false>(r, u0, false, false, fx0, fy0, fz0, ph);
                    pair32::force_pair32<true, false>(r, u1, false, false, fx1, fy1, fz1, ph);
                }
                if (a0) {
                    const float qf = __uint_as_float(u0.w);
                    a.force[3 * i0 + 0] = qf * (fx0.x + fx0.y);
                    a.force[3 * i0 + 1] = qf * (fy0.x + fy0.y);
                    a.force[3 * i0 + 2] = qf * ((fz0.x + fz0.y) + fibc);
                }
                if (a1) {
                    const float qf = __uint_as_float(u1.w);
                    a.force[3 * i1 + 0] = qf * (fx1.x + fx1.y);
                    a.force[3 * i1 + 1] = qf * (fy1.x + fy1.y);
                    a.force[3 * i1 + 2] = qf * ((fz1.x + fz1.y) + fibc);
                }
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
// make for the system alone (Philox key = the system's seed), with the image-series sums
// of the drawn kz read from the system's table built at set-up.
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
    kdetail::fill_kcoef_row(bs.dp, a.eo + bs.eo_off, bs.eo_half, n[0], n[1], n[2], bs.dp.coef, out, true);
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
    size_t a = sizeof(uint4) * kBatchSfTile, b = sizeof(KPair32) * (size_t)((P_max + 1) / 2);
    return a > b ? a : b;
}

// Wave vectors per thread: the smallest of 1, 2, 4 with 128 KR >= P_max.  Variant bit 0
// caps the registers for 8 resident CTAs per SM (KR <= 2 only; KR = 4 would spill
// heavily), bit 1 moves one angle in 8 (KR = 2) of the structure-factor items to the FMA pipe.
template <int KR, int MINB>
static void launch_kr_poly(cudaStream_t st, const BatchArgs& a, int grid, size_t sm, bool poly) {
    if (poly) batch_persistent_kernel<KR, MINB, true><<<grid, kBatchThreads, sm, st>>>(a);
    else batch_persistent_kernel<KR, MINB, false><<<grid, kBatchThreads, sm, st>>>(a);
}

template <int KR>
static cudaError_t launch_kr(cudaStream_t st, const BatchArgs& a, int grid, size_t sm, int variant) {
    const bool poly = (variant & 2) != 0;
    if constexpr (KR <= 2) {
        if (variant & 1) {
            launch_kr_poly<KR, 8>(st, a, grid, sm, poly);
            return cudaSuccess;
        }
    }
    launch_kr_poly<KR, 1>(st, a, grid, sm, poly);
    return cudaSuccess;
}

cudaError_t launch_batch(cudaStream_t st, const BatchArgs& a, int grid, int variant) {
    const size_t sm = batch_smem_bytes(a.P_max);
    if (a.P_max <= 128) launch_kr<1>(st, a, grid, sm, variant);
    else if (a.P_max <= 256) launch_kr<2>(st, a, grid, sm, variant);
    else launch_kr<4>(st, a, grid, sm, variant);
    note_launches(1);
    return cudaGetLastError();
}

template <int KR>
static cudaError_t occ_kr(int* per_sm, size_t sm, int variant) {
    if constexpr (KR <= 2) {
        if (variant & 1)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_persistent_kernel<KR, 8, false>,
                                                                 kBatchThreads, sm);
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_persistent_kernel<KR, 1, false>, kBatchThreads,
                                                         sm);
}

cudaError_t batch_occupancy(int P_max, int variant, int* per_sm) {
    const size_t sm = batch_smem_bytes(P_max);
    if (P_max <= 128) return occ_kr<1>(per_sm, sm, variant);
    if (P_max <= 256) return occ_kr<2>(per_sm, sm, variant);
    return occ_kr<4>(per_sm, sm, variant);
}

}  // namespace rbe2d
