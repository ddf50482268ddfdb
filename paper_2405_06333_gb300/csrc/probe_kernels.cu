// Throughput probes of the three pipes that bound this library's kernels: the MUFU
// (special-function) pipe that evaluates __sinf / __cosf, the float32 FMA pipe and the
// float64 FMA pipe.  They measure the roofline denominators of the sin/cos-bound k-space
// kernels (results per clock per SM) instead of taking them from a table.  No
// counterpart in the paper; a measurement aid (rbe2d_pipe_probe in include/rbe2d.h).
//
// Each kernel runs eight independent dependency chains per thread in every resident
// warp of every SM; thread 0 of each CTA records the SM cycles (clock64) its CTA spent.
// All CTAs of an SM run at the same time (the grid is one full wave), so the results of
// one SM per clock are (operations per CTA x resident CTAs) / cycles.
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/rbe2d.h"

namespace rbe2d {
void note_launches(int n);  // the library's kernel-launch counter (rbe2d_api.cu)
}

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

template <int KIND>  // 0: __sinf / __cosf (MUFU), 1: float32 FMA, 2: float64 FMA
__global__ void __launch_bounds__(kProbeThreads) probe_kernel(int iters, float seed, long long* cycles,
                                                              double* sink) {
    float f[kProbeChains];
    double d[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) {
        f[c] = seed * (float)(threadIdx.x + c + 1);
        d[c] = (double)f[c];
    }
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < kProbeChains; c++) {
            if (KIND == 0) f[c] = (c & 1) ? __cosf(f[c]) : __sinf(f[c]);  // one MUFU result each
            else if (KIND == 1) f[c] = fmaf(f[c], 0.999999f, 1e-7f);
            else d[c] = fma(d[c], 0.9999999999, 1e-12);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) acc += KIND == 2 ? d[c] : (double)f[c];
    if (acc == 12345.678) sink[0] = acc;  // keeps the chains alive; never true in practice
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" int rbe2d_pipe_probe(double* out) {
    if (!out) return RBE2D_EINVAL;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RBE2D_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RBE2D_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_kernel<0>, kProbeThreads, 0) != cudaSuccess)
        return RBE2D_ECUDA;
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 4) per_sm = 4;  // 32 warps per SM: enough chains to cover every pipe's latency
    const int grid = sms * per_sm;
    long long* cyc = nullptr;
    double* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = RBE2D_OK;
    if (cudaMalloc(&cyc, sizeof(long long) * grid) != cudaSuccess || cudaMalloc(&sink, sizeof(double)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = RBE2D_ECUDA;
    }
    const int iters[3] = {2048, 8192, 256};
    std::vector<long long> h(grid);
    for (int kind = 0; kind < 3 && rc == RBE2D_OK; kind++) {
        double best = 0.0, mhz = 0.0;
        for (int rep = 0; rep < 3 && rc == RBE2D_OK; rep++) {
            cudaEventRecord(e0, 0);
            if (kind == 0) probe_kernel<0><<<grid, kProbeThreads>>>(iters[0], 0.37f, cyc, sink);
            else if (kind == 1) probe_kernel<1><<<grid, kProbeThreads>>>(iters[1], 0.37f, cyc, sink);
            else probe_kernel<2><<<grid, kProbeThreads>>>(iters[2], 0.37f, cyc, sink);
            cudaEventRecord(e1, 0);
            rbe2d::note_launches(1);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
                cudaMemcpy(h.data(), cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = RBE2D_ECUDA;
                break;
            }
            long long cmax = 1;
            for (long long c : h) cmax = c > cmax ? c : cmax;
            const double ops_per_cta = (double)iters[kind] * kProbeChains * kProbeThreads;
            const double rate = ops_per_cta * per_sm / (double)cmax;  // per clock per SM
            if (rate > best) {
                best = rate;
                mhz = ms > 0.f ? (double)cmax / (ms * 1e3) : 0.0;  // cycles per microsecond
            }
        }
        out[kind] = best;
        if (kind == 0) out[3] = mhz;
    }
    cudaFree(cyc);
    cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess && rc == RBE2D_OK) rc = RBE2D_ECUDA;
    return rc;
}
