// rbe2d_structure_factor_noalloc: structure factors without any device allocation.
//
// Some callers cannot allocate device memory on their call path: code that runs while
// a stream is being captured in global capture mode (where cudaMalloc is refused as an
// unsafe call), host programs that hand all device memory to their own pool and forbid
// allocations outside it, and plugins that must not create a per-call context.  This
// entry point serves them: it needs no rbe2d_ctx, and its scratch (the per-chunk
// partial sums) lives in a file-scope __device__ array of fixed size that every GPU
// loading the library holds until the process exits.
//
// The scratch array is shared by every call on a device and keeps the contents of the
// last call.  Each call writes every scratch slot it reads before reading it, so
// nothing needs clearing; calls that overlap on the GPU (different streams, or
// different host threads) race on the array and must be serialised by the caller.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/rbe2d.h"

namespace rbe2d {
void note_launches(int n);  // the library's kernel-launch counter (rbe2d_api.cu)
}

namespace {

constexpr int kNoallocChunks = 256;                     // particle chunks (CTAs)
constexpr int kNoallocThreads = 128;                    // threads per CTA
constexpr int kNoallocKPerThread = 4;                   // wave vectors per thread
constexpr int kNoallocMaxP = kNoallocThreads * kNoallocKPerThread;  // 512

// [P][chunk][4] float64 partial sums: 512 * 256 * 4 * 8 B = 4 MiB.
static __device__ __align__(256) double g_noalloc_scratch[(size_t)kNoallocMaxP * kNoallocChunks * 4];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device
std::once_flag g_scratch_once[kMaxDevices];
cudaError_t g_scratch_status[kMaxDevices];

__device__ __forceinline__ uint32_t to_turn32(double v, double scale) {
    // round(v * 2^32 / L) mod 2^32: the low 32 bits of the nearest integer
    return (uint32_t)(unsigned long long)__double2ll_rn(v * scale);
}

// One CTA per particle chunk; thread t owns k = t + j * blockDim.x (j < JMAX, the slots a
// batch of P wave vectors reaches: JMAX = ceil(P / 128), so a small batch evaluates no
// idle slots).  Particles are converted to 32-bit fixed-point fractions in shared memory,
// one per thread, and every thread sums q e^{i k.r} and q e^{i khat.r} over them in
// float32, promoting the tile sums to float64.
template <int JMAX>
__global__ void __launch_bounds__(kNoallocThreads) noalloc_sf_kernel(
    const double* __restrict__ pos, const double* __restrict__ q, int64_t N, const int32_t* __restrict__ kidx,
    int P, double sx, double sy, double sz, double* __restrict__ scratch) {
    __shared__ uint4 tile[kNoallocThreads];
    int nx[kNoallocKPerThread], ny[kNoallocKPerThread], nz[kNoallocKPerThread];
    for (int j = 0; j < JMAX; j++) {
        int k = threadIdx.x + j * kNoallocThreads;
        nx[j] = k < P ? kidx[3 * k] : 0;
        ny[j] = k < P ? kidx[3 * k + 1] : 0;
        nz[j] = k < P ? kidx[3 * k + 2] : 0;
    }
    const int64_t b = blockIdx.x;
    const int64_t p0 = (N * b) / kNoallocChunks, p1 = (N * (b + 1)) / kNoallocChunks;
    double ar[kNoallocKPerThread] = {}, ai[kNoallocKPerThread] = {};
    double br[kNoallocKPerThread] = {}, bi[kNoallocKPerThread] = {};
    const float k2pi = 1.46291807926715968e-09f;  // 2 pi / 2^32
    for (int64_t s = p0; s < p1; s += kNoallocThreads) {
        const int n = (int)min((int64_t)kNoallocThreads, p1 - s);
        __syncthreads();
        if (threadIdx.x < n) {
            const int64_t i = s + threadIdx.x;
            uint4 u;
            u.x = to_turn32(pos[3 * i], sx);
            u.y = to_turn32(pos[3 * i + 1], sy);
            u.z = to_turn32(pos[3 * i + 2], sz);
            u.w = __float_as_uint((float)q[i]);
            tile[threadIdx.x] = u;
        }
        __syncthreads();
        float fr[kNoallocKPerThread] = {}, fi[kNoallocKPerThread] = {};
        float gr[kNoallocKPerThread] = {}, gi[kNoallocKPerThread] = {};
        for (int p = 0; p < n; p++) {
            const uint4 u = tile[p];
            const float qf = __uint_as_float(u.w);
#pragma unroll
            for (int j = 0; j < JMAX; j++) {
                const uint32_t txy = (uint32_t)nx[j] * u.x + (uint32_t)ny[j] * u.y;
                const uint32_t tz = (uint32_t)nz[j] * u.z;
                float s1, c1, s2, c2;
                __sincosf((float)(int32_t)(txy + tz) * k2pi, &s1, &c1);
                __sincosf((float)(int32_t)(txy - tz) * k2pi, &s2, &c2);
                fr[j] = fmaf(qf, c1, fr[j]);
                fi[j] = fmaf(qf, s1, fi[j]);
                gr[j] = fmaf(qf, c2, gr[j]);
                gi[j] = fmaf(qf, s2, gi[j]);
            }
        }
        for (int j = 0; j < JMAX; j++) {
            ar[j] += fr[j]; ai[j] += fi[j]; br[j] += gr[j]; bi[j] += gi[j];
        }
    }
    for (int j = 0; j < JMAX; j++) {
        const int k = threadIdx.x + j * kNoallocThreads;
        if (k < P) {
            double* o = scratch + ((size_t)k * kNoallocChunks + b) * 4;
            o[0] = ar[j]; o[1] = ai[j]; o[2] = br[j]; o[3] = bi[j];
        }
    }
}

// One CTA per k: the chunk partials summed in a fixed order (bitwise reproducible).
__global__ void __launch_bounds__(kNoallocChunks) noalloc_fold_kernel(const double* __restrict__ scratch,
                                                                      double* __restrict__ out) {
    __shared__ double red[4][kNoallocChunks];
    const int k = blockIdx.x, t = threadIdx.x;
    const double* src = scratch + ((size_t)k * kNoallocChunks + t) * 4;
    for (int c = 0; c < 4; c++) red[c][t] = src[c];
    __syncthreads();
    for (int w = kNoallocChunks / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int c = 0; c < 4; c++) red[c][t] += red[c][t + w];
        __syncthreads();
    }
    if (t < 4) out[4 * k + t] = red[t][0];
}

// Device address of the scratch array for the current device, looked up once.
cudaError_t scratch_for_current_device(double** ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(g_scratch_once[dev], [dev]() {
        void* p = nullptr;
        g_scratch_status[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        g_scratch_addr[dev] = p;
    });
    if (g_scratch_status[dev] != cudaSuccess) return g_scratch_status[dev];
    *ptr = static_cast<double*>(g_scratch_addr[dev]);
    return cudaSuccess;
}

}  // namespace

extern "C" {

int rbe2d_structure_factor_noalloc(double Lx, double Ly, double Lz, int64_t N, const double* pos, const double* q,
                                   int P, const int32_t* k_idx, double* rho_out, void* stream) {
    if (!(Lx > 0) || !(Ly > 0) || !(Lz > 0) || N < 0) return RBE2D_EINVAL;
    // the fixed scratch holds 512 x 256 partial sums: a larger batch is refused
    if (P < 1 || P > kNoallocMaxP) return RBE2D_EINVAL;
    if ((N > 0 && (!pos || !q)) || !k_idx || !rho_out) return RBE2D_EINVAL;
    double* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return RBE2D_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const double two32 = 4294967296.0;
    const double sx = two32 / Lx, sy = two32 / Ly, sz = two32 / Lz;
    const int jmax = (P + kNoallocThreads - 1) / kNoallocThreads;  // 1 .. 4 slots per thread
    auto* kern = jmax == 1 ? noalloc_sf_kernel<1> : jmax == 2 ? noalloc_sf_kernel<2>
                                                  : jmax == 3 ? noalloc_sf_kernel<3> : noalloc_sf_kernel<4>;
    kern<<<kNoallocChunks, kNoallocThreads, 0, st>>>(pos, q, N, k_idx, P, sx, sy, sz, scratch);
    noalloc_fold_kernel<<<P, kNoallocChunks, 0, st>>>(scratch, rho_out);
    rbe2d::note_launches(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return RBE2D_ECUDA;
    return RBE2D_OK;
}

}  // extern "C"
