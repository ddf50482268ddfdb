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

#include "cells.cuh"
#include "rbe2d_internal.h"

namespace rbe2d {

namespace {

// One CTA per cell.  The sources of the 27 neighbour cells (with their periodic shifts
// applied, relative to this cell's corner) stream through a shared-memory chunk; each
// warp takes the cell's charges RS_TG (two) at a time.  The warp scans the chunk 32 sources at
// a time (one shared-memory load per source serves those charges), appends, per
// charge, the indices of the sources within r_c to a queue (in source order, by ballot),
// and evaluates the screened pair terms only in full rounds of 32 queued pairs, so the
// erfc / exp work runs with every lane busy.  A lane's sums and the warp's shuffle tree
// run in a fixed order, and chunk results are added per charge in chunk order: the
// result is bitwise reproducible.  A charge skips itself (the same entry of the home
// cell, unshifted); image slots are sources only.
constexpr int RS_THREADS = 128;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_TG = 2;          // charges per warp at a time
constexpr int RS_TARGETS = 128;   // charges per pass over the neighbourhood
constexpr int RS_NB = 64;         // neighbour cells described per staging group

// Per-launch constants of the pair kernel in its own precision, computed on the host
// (float64 arithmetic on GB300 is 1/64 of float32, so the kernel does none per CTA).
template <typename T>
struct RsConst {
    T a, rc2, k2, kc;       // alpha, r_c^2, 2 alpha / sqrt(pi), Coulomb prefactor
    T hx, hy, hz;           // cell sizes (periodic shifts of neighbour cells)
    T lj_rc2, lj_sig2, lj_f, lj_e;  // WCA: cutoff^2, sigma^2, 24 eps, 4 eps
};

template <typename T>
struct RsChunk;
template <>
struct RsChunk<float> {
    static constexpr int n = 1024;
};
template <>
struct RsChunk<double> {
    static constexpr int n = 512;
};

template <typename T, bool LJ>
__global__ void __launch_bounds__(RS_THREADS) rs_cell_kernel(RsConst<T> K, CellGrid g,
                                                             const typename Vec4<T>::type* __restrict__ src,
                                                             const long long* __restrict__ key,
                                                             const int* __restrict__ start, T* __restrict__ force,
                                                             T* __restrict__ phi, int pot, int energy,
                                                             double* __restrict__ epart, double* __restrict__ scal,
                                                             unsigned* __restrict__ done, int* __restrict__ status) {
    typedef typename Vec4<T>::type V;
    constexpr int CH = RsChunk<T>::n;
    __shared__ V buf[CH];
    __shared__ unsigned realbits[CH / 32];   // bit i: staged source i is a real charge
    __shared__ T tacc[RS_TARGETS][8];        // per charge: f (3), phi, LJ force (3), LJ energy
    __shared__ unsigned short queue[RS_WARPS][RS_TG][64];
    __shared__ unsigned char tlist[RS_TARGETS];  // this pass's real charges (entry offsets)
    __shared__ int wcount[RS_WARPS];
    __shared__ int home_lo, home_hi, home_g0;  // the unshifted home cell in this chunk
    __shared__ int nb_start[RS_NB], nb_count[RS_NB], nb_off[RS_NB + 1];
    __shared__ float4 nb_shift[RS_NB];
    __shared__ double red[RS_WARPS];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const int c = blockIdx.x;
    const int cx = c % g.ncx, cy = (c / g.ncx) % g.ncy, cz = c / (g.ncx * g.ncy);
    const int b0 = start[c], nT = start[c + 1] - b0;
    const T a = K.a, rc2 = K.rc2, k2 = K.k2;
    double e_local = 0.0;
    for (int tb = 0; tb < nT; tb += RS_TARGETS) {
        const int nt = min(RS_TARGETS, nT - tb);
        // the real charges of this pass, in entry order (image entries are sources only)
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
        for (int w = 0; w < RS_WARPS; w++) nreal += wcount[w];
        for (int i = threadIdx.x; i < RS_TARGETS * 8; i += RS_THREADS) (&tacc[0][0])[i] = (T)0;
        for (int i = threadIdx.x; i < CH / 32; i += RS_THREADS) realbits[i] = 0u;
        if (threadIdx.x == 0) { home_lo = 0; home_hi = 0; home_g0 = 0; }
        int fill = 0, budget = kMaxCandidates;
        // sum the staged chunk on every real charge of this pass
        auto process = [&](int n) {
            for (int t0 = warp * RS_TG; t0 < nreal; t0 += RS_WARPS * RS_TG) {
                V me[RS_TG];
                bool act[RS_TG];
                int self[RS_TG];  // staged index of the charge itself, or -1
#pragma unroll
                for (int u = 0; u < RS_TG; u++) {
                    act[u] = t0 + u < nreal;
                    const int e = b0 + tb + tlist[min(t0 + u, nreal - 1)];
                    me[u] = src[e];
                    const int si = home_lo + (e - home_g0);
                    self[u] = (si >= home_lo && si < home_hi) ? si : -1;
                }
                T acc[RS_TG][8];
#pragma unroll
                for (int u = 0; u < RS_TG; u++)
#pragma unroll
                    for (int k = 0; k < 8; k++) acc[u][k] = (T)0;
                auto pair = [&](int u, int i) {
                    if (i == self[u]) return;
                    const V o = buf[i];
                    const T dx = me[u].x - o.x, dy = me[u].y - o.y, dz = me[u].z - o.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    T ec, gs, ir;
                    screened(r2, a, ec, gs, ir);
                    const T fr = o.w * (ec * ir + k2 * gs) * ir * ir;
                    acc[u][0] += fr * dx; acc[u][1] += fr * dy; acc[u][2] += fr * dz;
                    acc[u][3] += o.w * ec * ir;
                    if (LJ && r2 < K.lj_rc2 && ((realbits[i >> 5] >> (i & 31)) & 1u)) {
                        const T s2 = K.lj_sig2 / r2, s6 = s2 * s2 * s2;
                        const T flj = K.lj_f * (2 * s6 * s6 - s6) / r2;
                        acc[u][4] += flj * dx; acc[u][5] += flj * dy; acc[u][6] += flj * dz;
                        acc[u][7] += K.lj_e * (s6 * s6 - s6 + (T)0.25);
                    }
                };
                int qn[RS_TG];
#pragma unroll
                for (int u = 0; u < RS_TG; u++) qn[u] = 0;
                for (int i0 = 0; i0 < n; i0 += 32) {
                    const int i = i0 + lane;
                    V o;
                    if (i < n) o = buf[i];
#pragma unroll
                    for (int u = 0; u < RS_TG; u++) {
                        bool in = false;
                        if (i < n && act[u]) {
                            const T dx = me[u].x - o.x, dy = me[u].y - o.y, dz = me[u].z - o.z;
                            in = dx * dx + dy * dy + dz * dz < rc2;
                        }
                        const unsigned m = __ballot_sync(0xffffffffu, in);
                        if (in) queue[warp][u][qn[u] + __popc(m & below)] = (unsigned short)i;
                        qn[u] += __popc(m);
                    }
                    __syncwarp();
#pragma unroll
                    for (int u = 0; u < RS_TG; u++) {
                        if (qn[u] >= 32) {  // a full round: one pair per lane
                            pair(u, queue[warp][u][lane]);
                            const int rest = qn[u] - 32;
                            __syncwarp();
                            if (lane < rest) queue[warp][u][lane] = queue[warp][u][32 + lane];
                            __syncwarp();
                            qn[u] = rest;
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < RS_TG; u++) {
                    if (lane < qn[u]) pair(u, queue[warp][u][lane]);
#pragma unroll
                    for (int k = 0; k < 8; k++)
                        for (int o = 16; o > 0; o >>= 1) acc[u][k] += __shfl_down_sync(0xffffffffu, acc[u][k], o);
                    if (lane == 0 && act[u])
#pragma unroll
                        for (int k = 0; k < 8; k++) tacc[t0 + u][k] += acc[u][k];
                }
                __syncwarp();
            }
        };
        // stage the neighbour cells in groups of up to 64: one thread describes each cell
        // (start, count, periodic shift), a prefix sum makes the group one flat range,
        // and all threads copy it, so each group costs two dependent loads, not two per cell
        const int nbx = 2 * g.mx + 1, nby = 2 * g.my + 1, nnb = 3 * nbx * nby;
        for (int q0 = 0; q0 < nnb; q0 += RS_NB) {
            const int qn = min(RS_NB, nnb - q0);
            if (threadIdx.x < qn) {
                const int k = q0 + threadIdx.x;
                const int ox = k % nbx - g.mx, oy = (k / nbx) % nby - g.my, oz = k / (nbx * nby) - 1;
                const int zc = cz + oz;
                int st = 0, cnt = 0;
                if (zc >= 0 && zc < g.ncz) {
                    const int cc = (zc * g.ncy + wrap_cell(cy + oy, g.ncy)) * g.ncx + wrap_cell(cx + ox, g.ncx);
                    st = start[cc];
                    cnt = start[cc + 1] - st;
                }
                nb_start[threadIdx.x] = st;
                nb_count[threadIdx.x] = cnt;
                nb_shift[threadIdx.x] = make_float4((float)ox, (float)oy, (float)oz, 0.f);
            }
            __syncthreads();
            if (threadIdx.x == 0) {  // exclusive prefix in staging order, within the work budget
                int run = 0;
                for (int k = 0; k < qn; k++) {
                    int cnt = nb_count[k];
                    if (cnt > budget) {  // bounded work per cell whatever the density
                        cnt = budget;
                        atomicAdd(&status[ST_CELL], 1);
                    }
                    budget -= cnt;
                    nb_off[k] = run;
                    run += cnt;
                }
                nb_off[qn] = run;
            }
            __syncthreads();
            const int gtotal = nb_off[qn];
            const int khome = nbx * nby + g.my * nbx + g.mx;  // the unshifted home cell
            const int hk = (khome >= q0 && khome < q0 + qn) ? khome - q0 : -1;
            for (int gdone = 0; gdone < gtotal;) {
                const int n = min(gtotal - gdone, CH - fill);
                for (int i = threadIdx.x; i < n; i += RS_THREADS) {
                    const int f = gdone + i;
                    int lo = 0, hi = qn - 1;  // the cell k with nb_off[k] <= f < nb_off[k + 1]
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (nb_off[mid] <= f) lo = mid;
                        else hi = mid - 1;
                    }
                    const int gi = nb_start[lo] + (f - nb_off[lo]);
                    const float4 sh = nb_shift[lo];
                    V o = src[gi];
                    o.x += (T)sh.x * K.hx; o.y += (T)sh.y * K.hy; o.z += (T)sh.z * K.hz;
                    buf[fill + i] = o;
                    if ((key[gi] & 255) == 0) atomicOr(&realbits[(fill + i) >> 5], 1u << ((fill + i) & 31));
                }
                if (threadIdx.x == 0 && hk >= 0) {  // the part of the home cell in this piece
                    const int a0 = max(nb_off[hk], gdone), a1 = min(nb_off[hk + 1], gdone + n);
                    if (a0 < a1) {
                        home_lo = fill + (a0 - gdone);
                        home_hi = fill + (a1 - gdone);
                        home_g0 = nb_start[hk] + (a0 - nb_off[hk]);
                    }
                }
                fill += n;
                gdone += n;
                if (fill == CH) {
                    __syncthreads();
                    process(fill);
                    __syncthreads();
                    fill = 0;
                    for (int i = threadIdx.x; i < CH / 32; i += RS_THREADS) realbits[i] = 0u;
                    if (threadIdx.x == 0) { home_lo = 0; home_hi = 0; home_g0 = 0; }
                    __syncthreads();
                }
            }
            __syncthreads();  // the group's descriptors are read until here
        }
        __syncthreads();
        process(fill);
        __syncthreads();
        for (int t = threadIdx.x; t < nreal; t += RS_THREADS) {
            const int e = b0 + tb + tlist[t];
            const int64_t j = key[e] >> 8;
            const T qi = src[e].w, kc = K.kc;
            force[3 * j + 0] += kc * qi * tacc[t][0] + tacc[t][4];
            force[3 * j + 1] += kc * qi * tacc[t][1] + tacc[t][5];
            force[3 * j + 2] += kc * qi * tacc[t][2] + tacc[t][6];
            if (pot) phi[j] += kc * tacc[t][3];
            e_local += 0.5 * (double)kc * (double)qi * (double)tacc[t][3] + 0.5 * (double)tacc[t][7];
        }
        __syncthreads();
    }
    if (!energy) return;
    // energy: fixed-order block sums, then the last CTA adds them in block order
    double v = e_local;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tsum = 0.0;
        for (int w = 0; w < RS_WARPS; w++) tsum += red[w];
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
cudaError_t launch_cells_t(cudaStream_t st, const DevParams& dp, const CellGrid& g, const RealBuffers& rb, int64_t N,
                           const TIn* pos, const TIn* q, bool fp64, int* status, const int* gate, int* count_real,
                           int* real_start, int* tile_sum2, int max_blocks) {
    cudaError_t e = cudaSuccess;
    if (gate) rs_clear_kernel<<<(g.ncell + 255) / 256, 256, 0, st>>>(rb.count, count_real, g.ncell, gate);
    else e = cudaMemsetAsync(rb.count, 0, sizeof(int) * (size_t)g.ncell, st);
    if (e != cudaSuccess) return e;
    int64_t pbl = (N + 255) / 256;
    if (pbl < 1) pbl = 1;
    if (pbl > 4096) pbl = 4096;
    if (max_blocks > 0 && pbl > max_blocks) pbl = max_blocks;
    const int pb = (int)pbl;
    FxGrid X;
    const double zext = dp.H + 2.0 * dp.r_c;
    X.sx = 4294967296.0 / dp.Lx; X.sy = 4294967296.0 / dp.Ly; X.sz = 4294967296.0 / zext;
    X.zoff = llrint(dp.r_c * X.sz); X.zstep = llrint(2.0 * dp.H * X.sz);
    X.rx = (float)(g.hx / 4294967296.0); X.ry = (float)(g.hy / 4294967296.0); X.rz = (float)(g.hz / 4294967296.0);
    X.gt = (float)dp.gt; X.gb = (float)dp.gb;
    if (fp64) rs_count_kernel<TIn, double><<<pb, 256, 0, st>>>(dp, g, X, pos, q, N, rb.count, count_real, gate);
    else rs_count_kernel<TIn, float><<<pb, 256, 0, st>>>(dp, g, X, pos, q, N, rb.count, count_real, gate);
    const int ntile = (g.ncell + RS_SCAN - 1) / RS_SCAN;
    rs_tile_sum_kernel<<<ntile, RS_SCAN, 0, st>>>(rb.count, g.ncell, rb.tile_sum, gate);
    rs_scan_kernel<<<ntile, RS_SCAN, 0, st>>>(rb.count, g.ncell, rb.tile_sum, rb.start, rb.fill, gate);
    int launched = 5;
    if (count_real) {
        rs_tile_sum_kernel<<<ntile, RS_SCAN, 0, st>>>(count_real, g.ncell, tile_sum2, gate);
        rs_scan_kernel<<<ntile, RS_SCAN, 0, st>>>(count_real, g.ncell, tile_sum2, real_start, nullptr, gate);
        launched += 2;
    }
    int64_t obl = ((int64_t)g.ncell * 32 + 255) / 256;
    if (obl > 8192) obl = 8192;
    if (max_blocks > 0 && obl > max_blocks) obl = max_blocks;
    const int ob = (int)obl;
    if (fp64) {
        rs_fill_kernel<TIn, double><<<pb, 256, 0, st>>>(dp, g, X, pos, q, N, rb.start, rb.fill, (double4_32a*)rb.src,
                                                        rb.key, gate);
        rs_order_kernel<double><<<ob, 256, 0, st>>>(g.ncell, rb.start, (const double4_32a*)rb.src, rb.key,
                                                    (double4_32a*)rb.src_sorted, rb.key_sorted, status, gate);
    } else {
        rs_fill_kernel<TIn, float><<<pb, 256, 0, st>>>(dp, g, X, pos, q, N, rb.start, rb.fill, (float4*)rb.src,
                                                       rb.key, gate);
        rs_order_kernel<float><<<ob, 256, 0, st>>>(g.ncell, rb.start, (const float4*)rb.src, rb.key,
                                                   (float4*)rb.src_sorted, rb.key_sorted, status, gate);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launches(launched + (gate ? 1 : 0));  // (clear,) count, tile sums, scan(s), fill, order
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_cells(cudaStream_t st, const DevParams& dp, const CellGrid& g, const RealBuffers& rb, int64_t N,
                         const void* pos, const void* q, bool in_f32, bool fp64, int* status, const int* gate,
                         int* count_real, int* real_start, int* tile_sum2, int max_blocks) {
    return in_f32 ? launch_cells_t<float>(st, dp, g, rb, N, (const float*)pos, (const float*)q, fp64, status, gate,
                                          count_real, real_start, tile_sum2, max_blocks)
                  : launch_cells_t<double>(st, dp, g, rb, N, (const double*)pos, (const double*)q, fp64, status, gate,
                                           count_real, real_start, tile_sum2, max_blocks);
}

cudaError_t launch_real(cudaStream_t st, const DevParams& dp, const CellGrid& g, const RealBuffers& rb, int64_t N,
                        const void* pos, const void* q, bool in_f32, bool fp64, void* force, void* phi, int pot,
                        int energy, double* scal, unsigned* done, int* status) {
    if (N <= 0) return cudaMemsetAsync(scal + SC_UREAL, 0, sizeof(double), st);
    cudaError_t e = launch_cells(st, dp, g, rb, N, pos, q, in_f32, fp64, status, nullptr, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    const bool lj = dp.lj_eps != 0.0 && dp.lj_sig2 > 0.0;
    auto consts = [&](auto zero) {
        typedef decltype(zero) T;
        RsConst<T> K;
        K.a = (T)dp.alpha; K.rc2 = (T)(dp.r_c * dp.r_c); K.k2 = (T)(2.0 * dp.alpha / sqrt(M_PI)); K.kc = (T)dp.kc;
        K.hx = (T)g.hx; K.hy = (T)g.hy; K.hz = (T)g.hz;
        K.lj_rc2 = (T)dp.lj_rc2; K.lj_sig2 = (T)dp.lj_sig2; K.lj_f = (T)(24.0 * dp.lj_eps); K.lj_e = (T)(4.0 * dp.lj_eps);
        return K;
    };
#define RS_LAUNCH(T, V, L)                                                                                      \
    rs_cell_kernel<T, L><<<g.ncell, RS_THREADS, 0, st>>>(consts((T)0), g, (const V*)rb.src_sorted, rb.key_sorted, \
                                                         rb.start, (T*)force, (T*)phi, pot, energy, rb.epart, scal, \
                                                         done, status)
    if (fp64) {
        if (lj) RS_LAUNCH(double, double4_32a, true);
        else RS_LAUNCH(double, double4_32a, false);
    } else {
        if (lj) RS_LAUNCH(float, float4, true);
        else RS_LAUNCH(float, float4, false);
    }
#undef RS_LAUNCH
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rbe2d
