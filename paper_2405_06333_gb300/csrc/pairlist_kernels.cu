// Real-space pair lists for the MD loop (Eq. 3.12; force by reading A15), FP32-mixed mode.
//
// The cell scan (real_kernels.cu) tests every source of the 27 neighbour cells for
// every charge on every call: ~810 candidates for ~110 sources within r_c at the MD
// workload.  Between MD steps the charges move little, so here a Verlet list per charge
// holds the sources (real charges and images) within r_c + skin, built by a scan of
// cells of at least r_c + skin, and every step evaluates only the listed pairs (those
// within r_c at the current positions).  The lists stay exact while no charge has moved
// more than skin / 2 since the build: every source within r_c now was within
// r_c + skin then.  A prep kernel checks that on the device every step and raises a
// flag; the build kernels run every step but return at once unless the flag is set, so a
// captured CUDA graph rebuilds exactly when needed.
//
// Positions enter as 32-bit fixed-point records {ux, uy, A, q}: ux, uy turn fractions of
// the cell (the periodic minimum-image difference is an int32 subtraction; the lists
// need Lx, Ly >= 2 (r_c + 2 skin)), A = round(z 2^32 / zext) with zext = H + 2 (r_c + skin);
// an image of slot s has z turn +-A + off_s, the integers the cell-list build uses,
// so the build and the pair evaluation place every image identically.  A charge's sum
// runs over its list in list order (the cell scan's source order): bitwise reproducible.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "cells.cuh"
#include "rbe2d_internal.h"

namespace rbe2d {

namespace {

constexpr int NL_THREADS = 128;
constexpr int NL_WARPS = NL_THREADS / 32;
constexpr int NL_TG = 2;          // charges per warp at a time in the build scan
constexpr int NL_TARGETS = 128;   // charges per pass over the neighbourhood
constexpr int NL_NB = 64;         // neighbour cells described per staging group
constexpr int NL_CH = 1024;       // staged sources per chunk

// Per-launch constants of the list kernels (computed on the host).
struct NlConst {
    float a, rc2, k2, kc;          // alpha, r_c^2, 2 alpha / sqrt(pi), Coulomb prefactor
    float lj_rc2, lj_sig2, lj_f, lj_e;
    float xturn, yturn, zturn;     // Lx / 2^32, Ly / 2^32, zext / 2^32
    float hs2;                     // (skin / 2)^2: the displacement that forces a rebuild
    float rcs2;                    // (r_c + skin)^2: the build's cutoff
    float hx, hy, hz;              // cell sizes of the list grid
    double sx, sy, sz;             // 2^32 / Lx, 2^32 / Ly, 2^32 / zext
    long long zoff;                // (r_c + skin) in z turns
    int nslot;                     // image slots 0 .. nslot-1 (2 lmax + 1)
    long long off[kNlMaxSlots];    // z turn of slot s: A + off[s], mirrored (-A + off[s]) on odd levels
    float coef[kNlMaxSlots];       // image coefficient of slot s (1 for the charge itself)
};

__device__ __forceinline__ uint32_t turn(double v, double scale) {
    return (uint32_t)(unsigned long long)__double2ll_rn(v * scale);
}

// Every charge: its fixed-point record for this step (also at its slot of the last build,
// srec[inv[j]], for the pair kernel), and whether it has moved more than skin / 2 since
// the last build, which sets flag[0].  With the flag already set (set-up, another N) the
// slots are not valid yet and the rebuild writes srec instead.
template <typename TIn>
__global__ void rs_list_prep_kernel(NlConst K, const TIn* __restrict__ pos, const TIn* __restrict__ q, int64_t N,
                                    uint4* __restrict__ rec, const uint4* __restrict__ ref, int* __restrict__ flag,
                                    const int* __restrict__ inv, uint4* __restrict__ srec) {
    const bool check = flag[0] == 0;
    bool moved = false;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const double x = (double)pos[3 * j], y = (double)pos[3 * j + 1], z = (double)pos[3 * j + 2];
        const uint4 r = make_uint4(turn(x, K.sx), turn(y, K.sy), (uint32_t)__double2ll_rn(z * K.sz),
                                   __float_as_uint((float)q[j]));
        rec[j] = r;
        if (check) {  // the lists of the last build stand unless a charge has moved too far
            const int t = inv[j];
            if ((uint64_t)t < (uint64_t)N) srec[t] = r;
            const uint4 o = ref[j];
            const float dx = (float)(int32_t)(r.x - o.x) * K.xturn, dy = (float)(int32_t)(r.y - o.y) * K.yturn;
            const float dz = (float)((long long)r.z - (long long)o.z) * K.zturn;
            moved |= !(dx * dx + dy * dy + dz * dz <= K.hs2);  // a non-finite step counts as moved
        }
    }
    if (__any_sync(0xffffffffu, moved) && (threadIdx.x & 31) == 0) atomicOr(&flag[0], 1);
}

// One CTA per cell of the list grid at a time (cells of at least r_c + skin; a bounded
// grid loops over the cells, so that a skipped build costs one short launch), built like
// the cell scan: the 27 neighbour cells' sources stream through shared memory; each warp takes
// two charges at a time and appends, by ballot in source order, the sources within
// r_c + skin to their lists.  Charge t of the cell (in key order) owns list slot
// real_start[cell] + t.  A charge skips its own entry; its images are sources.
__global__ void __launch_bounds__(NL_THREADS) rs_list_build_kernel(
    NlConst K, CellGrid g, const float4* __restrict__ src, const long long* __restrict__ key,
    const int* __restrict__ start, const int* __restrict__ real_start, PairLists L, const int* __restrict__ gate,
    int* __restrict__ status) {
    if (*gate == 0) return;
    __shared__ float4 buf[NL_CH];
    __shared__ int benc[NL_CH];                 // list entry of each staged source: its slot * 64 + image slot
    __shared__ int tcount[NL_TARGETS];           // entries found so far per charge of this pass
    __shared__ unsigned char tlist[NL_TARGETS];  // this pass's real charges (entry offsets)
    __shared__ int wcount[NL_WARPS];
    __shared__ int home_lo, home_hi, home_g0;
    __shared__ int nb_start[NL_NB], nb_count[NL_NB], nb_off[NL_NB + 1];
    __shared__ float4 nb_shift[NL_NB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    for (int c = blockIdx.x; c < g.ncell; c += gridDim.x) {
        const int cx = c % g.ncx, cy = (c / g.ncx) % g.ncy, cz = c / (g.ncx * g.ncy);
        const int b0 = start[c], nT = start[c + 1] - b0;
        const int slot0 = real_start[c];
        int real_before = 0;  // real charges of this cell in earlier passes
        const int64_t nslots = L.n_slots;
        for (int tb = 0; tb < nT; tb += NL_TARGETS) {
            const int nt = min(NL_TARGETS, nT - tb);
            {
                const bool real = threadIdx.x < nt && (key[b0 + tb + threadIdx.x] & 255) == 0;
                const unsigned m = __ballot_sync(0xffffffffu, real);
                if (lane == 0) wcount[warp] = __popc(m);
                __syncthreads();
                int off = __popc(m & below);
                for (int w = 0; w < warp; w++) off += wcount[w];
                if (real) tlist[off] = (unsigned char)threadIdx.x;
            }
            int nreal = 0;
            for (int w = 0; w < NL_WARPS; w++) nreal += wcount[w];
            for (int i = threadIdx.x; i < NL_TARGETS; i += NL_THREADS) tcount[i] = 0;
            if (threadIdx.x == 0) { home_lo = 0; home_hi = 0; home_g0 = 0; }
            int fill = 0, budget = kMaxCandidates;
            auto process = [&](int n) {
                for (int t0 = warp * NL_TG; t0 < nreal; t0 += NL_WARPS * NL_TG) {
                    float4 me[NL_TG];
                    bool act[NL_TG];
                    int self[NL_TG], cnt[NL_TG];
                    int64_t slot[NL_TG];
    #pragma unroll
                    for (int u = 0; u < NL_TG; u++) {
                        act[u] = t0 + u < nreal;
                        const int tt = min(t0 + u, nreal - 1);
                        const int e = b0 + tb + tlist[tt];
                        me[u] = src[e];
                        const int si = home_lo + (e - home_g0);
                        self[u] = (si >= home_lo && si < home_hi) ? si : -1;
                        cnt[u] = tcount[tt];
                        slot[u] = (int64_t)slot0 + real_before + tt;
                    }
                    for (int i0 = 0; i0 < n; i0 += 32) {
                        const int i = i0 + lane;
                        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (i < n) o = buf[i];
    #pragma unroll
                        for (int u = 0; u < NL_TG; u++) {
                            bool in = false;
                            if (i < n && act[u] && i != self[u]) {
                                const float dx = me[u].x - o.x, dy = me[u].y - o.y, dz = me[u].z - o.z;
                                in = dx * dx + dy * dy + dz * dz < K.rcs2;
                            }
                            const unsigned m = __ballot_sync(0xffffffffu, in);
                            const int at = cnt[u] + __popc(m & below);
                            if (in && at < L.cap) L.nl[(int64_t)at * nslots + slot[u]] = benc[i];
                            cnt[u] += __popc(m);
                        }
                    }
                    if (lane == 0) {
    #pragma unroll
                        for (int u = 0; u < NL_TG; u++)
                            if (act[u]) tcount[t0 + u] = cnt[u];
                    }
                    __syncwarp();
                }
            };
            const int nbx = 2 * g.mx + 1, nby = 2 * g.my + 1, nnb = 3 * nbx * nby;
            for (int q0 = 0; q0 < nnb; q0 += NL_NB) {
                const int qn = min(NL_NB, nnb - q0);
                if (threadIdx.x < qn) {
                    const int k = q0 + threadIdx.x;
                    const int ox = k % nbx - g.mx, oy = (k / nbx) % nby - g.my, oz = k / (nbx * nby) - 1;
                    const int zc = cz + oz;
                    int st = 0, ct = 0;
                    if (zc >= 0 && zc < g.ncz) {
                        const int cc = (zc * g.ncy + wrap_cell(cy + oy, g.ncy)) * g.ncx + wrap_cell(cx + ox, g.ncx);
                        st = start[cc];
                        ct = start[cc + 1] - st;
                    }
                    nb_start[threadIdx.x] = st;
                    nb_count[threadIdx.x] = ct;
                    nb_shift[threadIdx.x] = make_float4((float)ox, (float)oy, (float)oz, 0.f);
                }
                __syncthreads();
                if (threadIdx.x == 0) {  // exclusive prefix in staging order, within the work budget
                    int run = 0;
                    for (int k = 0; k < qn; k++) {
                        int ct = nb_count[k];
                        if (ct > budget) {
                            ct = budget;
                            atomicAdd(&status[ST_CELL], 1);
                        }
                        budget -= ct;
                        nb_off[k] = run;
                        run += ct;
                    }
                    nb_off[qn] = run;
                }
                __syncthreads();
                const int gtotal = nb_off[qn];
                const int khome = nbx * nby + g.my * nbx + g.mx;
                const int hk = (khome >= q0 && khome < q0 + qn) ? khome - q0 : -1;
                for (int gdone = 0; gdone < gtotal;) {
                    const int n = min(gtotal - gdone, NL_CH - fill);
                    for (int i = threadIdx.x; i < n; i += NL_THREADS) {
                        const int f = gdone + i;
                        int lo = 0, hi = qn - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (nb_off[mid] <= f) lo = mid;
                            else hi = mid - 1;
                        }
                        const int gi = nb_start[lo] + (f - nb_off[lo]);
                        const float4 sh = nb_shift[lo];
                        float4 o = src[gi];
                        o.x += sh.x * K.hx; o.y += sh.y * K.hy; o.z += sh.z * K.hz;
                        buf[fill + i] = o;
                        const long long kk = key[gi];
                        benc[fill + i] = L.inv[kk >> 8] * kNlMaxSlots + (int)(kk & 255);
                    }
                    if (threadIdx.x == 0 && hk >= 0) {
                        const int a0 = max(nb_off[hk], gdone), a1 = min(nb_off[hk + 1], gdone + n);
                        if (a0 < a1) {
                            home_lo = fill + (a0 - gdone);
                            home_hi = fill + (a1 - gdone);
                            home_g0 = nb_start[hk] + (a0 - nb_off[hk]);
                        }
                    }
                    fill += n;
                    gdone += n;
                    if (fill == NL_CH) {
                        __syncthreads();
                        process(fill);
                        __syncthreads();
                        fill = 0;
                        if (threadIdx.x == 0) { home_lo = 0; home_hi = 0; home_g0 = 0; }
                        __syncthreads();
                    }
                }
                __syncthreads();
            }
            __syncthreads();
            process(fill);
            __syncthreads();
            for (int t = threadIdx.x; t < nreal; t += NL_THREADS) {
                const int e = b0 + tb + tlist[t];
                const int64_t s = (int64_t)slot0 + real_before + t;
                const int j = (int)(key[e] >> 8);
                const int n_e = tcount[t];
                if (n_e > L.cap) atomicAdd(&status[ST_CELL], 1);  // entries past the capacity were dropped
                L.cnt[s] = min(n_e, L.cap);
                L.tgt[s] = j;
                L.ref[j] = L.rec[j];
                L.srec[s] = L.rec[j];
            }
            real_before += nreal;
            __syncthreads();
        }
    }
}

// Before a build (gated like it): the list slot of every charge, inv[j] = real_start[cell]
// + its rank among the cell's real charges in key order -- the slot the build gives it --
// so that the build can name every source (a charge or one of its images) by its slot.
// One warp per cell.
__global__ void rs_list_slots_kernel(int ncell, const int* __restrict__ start, const int* __restrict__ real_start,
                                     const long long* __restrict__ key, int* __restrict__ inv,
                                     const int* __restrict__ gate) {
    if (*gate == 0) return;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < ncell; c += nwarps) {
        const int b = start[c], n = start[c + 1] - b;
        int run = real_start[c];
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            const long long k = i < n ? key[b + i] : 1;
            const bool real = i < n && (k & 255) == 0;
            const unsigned m = __ballot_sync(0xffffffffu, real);
            if (real) inv[k >> 8] = run + __popc(m & below);
            run += __popc(m);
        }
    }
}

// After a build: count it and clear the flag (one thread).
__global__ void rs_list_done_kernel(int* __restrict__ flag, unsigned long long* __restrict__ builds) {
    if (threadIdx.x == 0 && flag[0] != 0) {
        flag[0] = 0;
        *builds += 1ull;
    }
}

// Every listed pair within r_c at the current positions: one thread per list slot (charges
// in cell order, so a warp's sources overlap in cache), the sum in list order; the force
// (screened Coulomb and, between charges, WCA) is added to force.  All position
// arithmetic is 32-bit: differences of turn fractions wrap to the minimum image (in z
// the true difference is far below 2^31 turns), and image slots come from a shared-memory
// table {mask, z offset, coefficient}: the image's z turn is (A xor mask) + offset, where
// an odd (mirrored) level has mask = ~0 and offset off_s + 1, since -A = (A xor ~0) + 1
// modulo 2^32, and slot 0 and even levels have mask 0 and offset off_s.  Entries are taken four at a time so that their loads
// overlap.
constexpr int NL_UNROLL = 4;

template <bool LJ>
__global__ void __launch_bounds__(NL_THREADS) rs_list_pair_kernel(NlConst K, PairLists L, int64_t N,
                                                                  float* __restrict__ force) {
    __shared__ uint4 slot_tab[kNlMaxSlots];  // {mask, z turn offset (mod 2^32), coefficient bits, 0}
    for (int i = threadIdx.x; i < K.nslot; i += NL_THREADS) {
        const bool mirror = ((i + 1) >> 1) & 1;  // slot 0 and even levels keep z, odd levels mirror it
        slot_tab[i] = make_uint4(mirror ? 0xffffffffu : 0u, (uint32_t)(unsigned long long)K.off[i] + (mirror ? 1u : 0u),
                                 __float_as_uint(K.coef[i]), 0u);
    }
    __syncthreads();
    const int64_t t = blockIdx.x * (int64_t)NL_THREADS + threadIdx.x;
    if (t >= N) return;
    const int j = L.tgt[t];
    const uint4 ri = L.srec[t];
    const uint32_t zi = ri.z + (uint32_t)K.zoff;
    const int n = L.cnt[t];
    float f0 = 0.f, f1 = 0.f, f2 = 0.f, l0 = 0.f, l1 = 0.f, l2 = 0.f;
    const int* __restrict__ col = L.nl + t;
    const int64_t ns = L.n_slots;
    auto term = [&](int enc, const uint4& rs) {
        const int sl = enc & (kNlMaxSlots - 1);
        const uint4 tab = slot_tab[sl];
        const uint32_t zs = (rs.z ^ tab.x) + tab.y;
        const float dx = (float)(int32_t)(ri.x - rs.x) * K.xturn;
        const float dy = (float)(int32_t)(ri.y - rs.y) * K.yturn;
        const float dz = (float)(int32_t)(zi - zs) * K.zturn;
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < K.rc2)) return;
        float ec, gs, ir;
        screened(r2, K.a, ec, gs, ir);
        const float w = __uint_as_float(rs.w) * __uint_as_float(tab.z);
        const float fr = w * (ec * ir + K.k2 * gs) * ir * ir;
        f0 += fr * dx; f1 += fr * dy; f2 += fr * dz;
        if (LJ && sl == 0 && r2 < K.lj_rc2) {
            const float s2 = K.lj_sig2 / r2, s6 = s2 * s2 * s2;
            const float flj = K.lj_f * (2 * s6 * s6 - s6) / r2;
            l0 += flj * dx; l1 += flj * dy; l2 += flj * dz;
        }
    };
    // two entries at once: the float32 arithmetic of both on paired instructions (x
    // halves: entry a, y halves: entry b), an entry beyond r_c weighted 0 (its terms stay
    // finite: |d| <= L / 2, exp(-x^2) underflows to 0), the sums kept per half
    const float2 zero2 = make_float2(0.f, 0.f);
    float2 g0 = zero2, g1 = zero2, g2 = zero2;
    auto term2 = [&](int ea, const uint4& ra, int eb, const uint4& rb) {
        const int sa = ea & (kNlMaxSlots - 1), sb = eb & (kNlMaxSlots - 1);
        const uint4 ta = slot_tab[sa], tb = slot_tab[sb];
        const uint32_t za = (ra.z ^ ta.x) + ta.y;
        const uint32_t zb = (rb.z ^ tb.x) + tb.y;
        const float2 dx = __fmul2_rn(make_float2((float)(int32_t)(ri.x - ra.x), (float)(int32_t)(ri.x - rb.x)),
                                     make_float2(K.xturn, K.xturn));
        const float2 dy = __fmul2_rn(make_float2((float)(int32_t)(ri.y - ra.y), (float)(int32_t)(ri.y - rb.y)),
                                     make_float2(K.yturn, K.yturn));
        const float2 dz = __fmul2_rn(make_float2((float)(int32_t)(zi - za), (float)(int32_t)(zi - zb)),
                                     make_float2(K.zturn, K.zturn));
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        const bool ina = r2.x < K.rc2, inb = r2.y < K.rc2;
        if (!(ina || inb)) return;
        float2 ec, gs, ir;
        screened2(r2, K.a, ec, gs, ir);
        const float2 w = make_float2(ina ? __uint_as_float(ra.w) * __uint_as_float(ta.z) : 0.f,
                                     inb ? __uint_as_float(rb.w) * __uint_as_float(tb.z) : 0.f);
        const float2 fr = __fmul2_rn(
            __fmul2_rn(__fmul2_rn(w, __ffma2_rn(ec, ir, __fmul2_rn(make_float2(K.k2, K.k2), gs))), ir), ir);
        g0 = __ffma2_rn(fr, dx, g0); g1 = __ffma2_rn(fr, dy, g1); g2 = __ffma2_rn(fr, dz, g2);
        // nearly every pair lies beyond the WCA range, so one test of the nearer entry
        // skips both entries' checks (each check below implies it)
        if (LJ && fminf(r2.x, r2.y) < K.lj_rc2) {
            if (sa == 0 && ina && r2.x < K.lj_rc2) {
                const float s2 = K.lj_sig2 / r2.x, s6 = s2 * s2 * s2;
                const float flj = K.lj_f * (2 * s6 * s6 - s6) / r2.x;
                l0 += flj * dx.x; l1 += flj * dy.x; l2 += flj * dz.x;
            }
            if (sb == 0 && inb && r2.y < K.lj_rc2) {
                const float s2 = K.lj_sig2 / r2.y, s6 = s2 * s2 * s2;
                const float flj = K.lj_f * (2 * s6 * s6 - s6) / r2.y;
                l0 += flj * dx.y; l1 += flj * dy.y; l2 += flj * dz.y;
            }
        }
    };
    int e = 0;
    for (; e + NL_UNROLL <= n; e += NL_UNROLL) {
        int enc[NL_UNROLL];
        uint4 rs[NL_UNROLL];
#pragma unroll
        for (int k = 0; k < NL_UNROLL; k++) enc[k] = __ldg(&col[(int64_t)(e + k) * ns]);
#pragma unroll
        for (int k = 0; k < NL_UNROLL; k++) rs[k] = __ldg(&L.srec[enc[k] >> 6]);
#pragma unroll
        for (int k = 0; k < NL_UNROLL; k += 2) term2(enc[k], rs[k], enc[k + 1], rs[k + 1]);
    }
    for (; e < n; e++) {
        const int enc = __ldg(&col[(int64_t)e * ns]);
        term(enc, __ldg(&L.srec[enc >> 6]));
    }
    f0 += g0.x + g0.y; f1 += g1.x + g1.y; f2 += g2.x + g2.y;
    const float qi = __uint_as_float(ri.w), kc = K.kc;
    force[3 * (int64_t)j + 0] += kc * qi * f0 + l0;
    force[3 * (int64_t)j + 1] += kc * qi * f1 + l1;
    force[3 * (int64_t)j + 2] += kc * qi * f2 + l2;
}

}  // namespace

cudaError_t launch_real_lists(cudaStream_t st, const DevParams& dp, const PairLists& L, const RealBuffers& rb,
                              int64_t N, const double* pos, const double* q, float* force, int* status) {
    if (N <= 0) return cudaSuccess;
    const double rcs = dp.r_c + L.skin;
    const double zext = dp.H + 2.0 * rcs;
    NlConst K = {};
    K.a = (float)dp.alpha;
    K.rc2 = (float)(dp.r_c * dp.r_c);
    K.k2 = (float)(2.0 * dp.alpha / sqrt(M_PI));
    K.kc = (float)dp.kc;
    K.lj_rc2 = (float)dp.lj_rc2; K.lj_sig2 = (float)dp.lj_sig2;
    K.lj_f = (float)(24.0 * dp.lj_eps); K.lj_e = (float)(4.0 * dp.lj_eps);
    K.xturn = (float)(dp.Lx / 4294967296.0); K.yturn = (float)(dp.Ly / 4294967296.0);
    K.zturn = (float)(zext / 4294967296.0);
    K.hs2 = (float)(0.25 * L.skin * L.skin);
    K.rcs2 = (float)(rcs * rcs);
    K.hx = (float)L.g.hx; K.hy = (float)L.g.hy; K.hz = (float)L.g.hz;
    K.sx = 4294967296.0 / dp.Lx; K.sy = 4294967296.0 / dp.Ly; K.sz = 4294967296.0 / zext;
    K.zoff = llrint(rcs * K.sz);
    const long long zstep = llrint(2.0 * dp.H * K.sz);
    K.nslot = 2 * L.g.lmax + 1;
    K.off[0] = K.zoff; K.coef[0] = 1.f;
    double gp_up = 1.0, gp_dn = 1.0;
    for (int l = 1; l <= L.g.lmax; l++) {  // the slots of the cell-list build (for_each_source32)
        if (l & 1) { gp_up *= dp.gt; gp_dn *= dp.gb; }
        else { gp_up *= dp.gb; gp_dn *= dp.gt; }
        K.off[2 * l - 1] = (long long)((l + 1) / 2) * zstep + K.zoff;
        K.off[2 * l] = -(long long)(l / 2) * zstep + K.zoff;
        K.coef[2 * l - 1] = (float)gp_up;
        K.coef[2 * l] = (float)gp_dn;
    }
    // 1. records and the displacement check
    int64_t pbl = (N + 255) / 256;
    if (pbl > 4096) pbl = 4096;
    rs_list_prep_kernel<double><<<(int)pbl, 256, 0, st>>>(K, pos, q, N, L.rec, L.ref, L.flag, L.inv, L.srec);
    // 2. the cell list of the list grid and the lists, when the flag is set
    DevParams d = dp;
    d.r_c = rcs;  // sources (and images) within r_c + skin of the slab, cells of at least r_c + skin
    cudaError_t e = launch_cells(st, d, L.g, rb, N, pos, q, false, false, status, L.flag, L.count_real,
                                 L.real_start, L.tile_sum2, L.build_blocks);
    if (e != cudaSuccess) return e;
    const int bblocks = (int)(L.g.ncell < L.build_blocks ? L.g.ncell : L.build_blocks);
    rs_list_slots_kernel<<<L.build_blocks, 256, 0, st>>>((int)L.g.ncell, rb.start, L.real_start, rb.key_sorted,
                                                         L.inv, L.flag);
    rs_list_build_kernel<<<bblocks, NL_THREADS, 0, st>>>(K, L.g, (const float4*)rb.src_sorted, rb.key_sorted,
                                                          rb.start, L.real_start, L, L.flag, status);
    rs_list_done_kernel<<<1, 32, 0, st>>>(L.flag, L.builds);
    // 3. the pairs
    const bool lj = dp.lj_eps != 0.0 && dp.lj_sig2 > 0.0;
    const int blocks = (int)((N + NL_THREADS - 1) / NL_THREADS);
    if (lj) rs_list_pair_kernel<true><<<blocks, NL_THREADS, 0, st>>>(K, L, N, force);
    else rs_list_pair_kernel<false><<<blocks, NL_THREADS, 0, st>>>(K, L, N, force);
    note_launches(5);  // prep, slots, build, done, pairs (the cell-list kernels count themselves)
    return cudaGetLastError();
}

}  // namespace rbe2d
