// Paired float32 arithmetic of the FP32-mixed k-space kernels: two independent terms
// carried in the x and y halves of float2 values, so that each scaling and fused
// multiply-add is one paired instruction (__fmul2_rn, __ffma2_rn, __fadd2_rn: one issue
// slot for two results).  The sin/cos stay one MUFU operation per angle.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "phase.cuh"
#include "rbe2d_internal.h"

namespace rbe2d {
namespace pair32 {

// sin and cos of the turn fractions ta (x halves) and tb (y halves); the two scalings to
// radians in one paired multiplication; polya / polyb: that angle on the FMA pipe
// (phase::sincos_poly_pi32, the full-circle polynomial) instead of MUFU.
__device__ __forceinline__ void sincos_turn32x2(uint32_t ta, uint32_t tb, bool polya, bool polyb, float2& s,
                                                float2& c) {
    const float k = 1.46291807926715968e-09f;  // 2 pi / 2^32
    const float2 x = __fmul2_rn(make_float2((float)(int32_t)ta, (float)(int32_t)tb), make_float2(k, k));
    if (polya) phase::sincos_poly_pi32(x.x, &s.x, &c.x);
    else __sincosf(x.x, &s.x, &c.x);
    if (polyb) phase::sincos_poly_pi32(x.y, &s.y, &c.y);
    else __sincosf(x.y, &s.y, &c.y);
}

// The (particle u, k0) and (particle u, k1) terms of Eq. 3.26 for one record r of two
// wave vectors (x halves: k0, y halves: k1), added to the paired sums:
//   g1 = Im(e^{-i theta1} A') = A'i cos t1 - A'r sin t1,  theta1 = k.r
//   g2 = Im(e^{-i theta2} B'),                             theta2 = khat.r  (DIEL)
//   F += (kx (g1+g2), ky (g1+g2), kz (g1-g2));  phi -= Re(e^{-i t1} A') + Re(e^{-i t2} B')
// polya / polyb: the second angle (the first when there is only one) of k0 / k1 on the
// FMA pipe.
template <bool DIEL, bool POT>
__device__ __forceinline__ void force_pair32(const KPair32& r, const uint4& u, bool polya, bool polyb, float2& fx,
                                             float2& fy, float2& fz, float2& ph) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const uint32_t txya = (uint32_t)r.nx.x * u.x + (uint32_t)r.ny.x * u.y, tza = (uint32_t)r.nz.x * u.z;
    const uint32_t txyb = (uint32_t)r.nx.y * u.x + (uint32_t)r.ny.y * u.y, tzb = (uint32_t)r.nz.y * u.z;
    float2 s1, c1;
    sincos_turn32x2(txya + tza, txyb + tzb, !DIEL && polya, !DIEL && polyb, s1, c1);
    const float2 g1 = __ffma2_rn(r.Ai, c1, __fmul2_rn(r.nAr, s1));
    if (DIEL) {
        float2 s2, c2;
        sincos_turn32x2(txya - tza, txyb - tzb, polya, polyb, s2, c2);
        const float2 g2 = __ffma2_rn(r.Bi, c2, __fmul2_rn(r.nBr, s2));
        const float2 G = __fadd2_rn(g1, g2), D = __ffma2_rn(g2, m1, g1);
        fx = __ffma2_rn(r.kx, G, fx);
        fy = __ffma2_rn(r.ky, G, fy);
        fz = __ffma2_rn(r.kz, D, fz);
        if (POT) ph = __ffma2_rn(__ffma2_rn(r.Ar, c1, __ffma2_rn(r.Ai, s1, __ffma2_rn(r.Br, c2, __fmul2_rn(r.Bi, s2)))), m1, ph);
    } else {
        fx = __ffma2_rn(r.kx, g1, fx);
        fy = __ffma2_rn(r.ky, g1, fy);
        fz = __ffma2_rn(r.kz, g1, fz);
        if (POT) ph = __ffma2_rn(__ffma2_rn(r.Ar, c1, __fmul2_rn(r.Ai, s1)), m1, ph);
    }
}

// Half h (0: x, 1: y) of a KPair32 record from one wave vector's float64 values: the
// indices, the wave vector and A' = c A, B' = c B with their negations.
__device__ __forceinline__ void set_half(KPair32* r, int h, int nx, int ny, int nz, float kx, float ky, float kz,
                                         float Ar, float Ai, float Br, float Bi) {
    (&r->nx.x)[h] = nx; (&r->ny.x)[h] = ny; (&r->nz.x)[h] = nz;
    (&r->kx.x)[h] = kx; (&r->ky.x)[h] = ky; (&r->kz.x)[h] = kz;
    (&r->nAr.x)[h] = -Ar; (&r->Ai.x)[h] = Ai; (&r->nBr.x)[h] = -Br; (&r->Bi.x)[h] = Bi;
    (&r->Ar.x)[h] = Ar; (&r->Br.x)[h] = Br;
}

}  // namespace pair32
}  // namespace rbe2d
