// The structure-factor variants that skip empty wave-vector groups (sf32.cuh, LIVE):
// launched when the k slots of a launch exceed P by at least one warp's group of 32,
// e.g. P = 300 with 96 threads x 4 wave vectors.  A separate translation unit so that
// these instantiations compile in parallel with kspace_kernels.cu.
#include "sf32.cuh"

namespace rbe2d {

void launch_sf32_live(cudaStream_t st, dim3 grid, int kthreads, int npoly, int shape, bool in_f32, bool sig,
                      const DevParams& dp, const void* pos, const void* q, int64_t N, const KCoef* kc,
                      double* sf_part, int nblk, uint4* po, double* pack_part) {
    using sf32k::launch_sf32_npoly;
    if (in_f32) {  // float inputs run shape 0
        const float* p = (const float*)pos; const float* qq = (const float*)q;
        if (sig) launch_sf32_npoly<float, true, false, 0, true>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
        else launch_sf32_npoly<float, false, false, 0, true>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
        return;
    }
    const double* p = (const double*)pos; const double* qq = (const double*)q;
    if (sig) {
        if (shape == 1) launch_sf32_npoly<double, true, false, 1, true>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
        else if (shape == 2) launch_sf32_npoly<double, true, false, 2, true>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
        else launch_sf32_npoly<double, true, false, 0, true>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
    } else {
        if (shape == 1) launch_sf32_npoly<double, false, false, 1, true>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
        else if (shape == 2) launch_sf32_npoly<double, false, false, 2, true>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
        else launch_sf32_npoly<double, false, false, 0, true>(st, grid, kthreads, npoly, dp, p, qq, N, kc, sf_part, nblk, po, pack_part);
    }
}

}  // namespace rbe2d
