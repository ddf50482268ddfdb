// Sine and cosine of a fixed-point turn fraction, shared by the structure-factor and
// force kernels.  A phase k.r / 2 pi mod 1 is carried as an unsigned 32-bit (FP32
// mode) or 64-bit (FP64 mode) fraction of a turn; these convert it to radians once and
// evaluate sin and cos.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace rbe2d {
namespace phase {

// sin and cos of 2 pi t / 2^32 (t read as a signed turn fraction, |angle| <= pi).
__device__ __forceinline__ void sincos_turn32(uint32_t t, float* s, float* c) {
    const float k = 1.46291807926715968e-09f;  // 2 pi / 2^32
    __sincosf((float)(int32_t)t * k, s, c);
}

// Minimax polynomials for sin and cos over the whole circle |x| <= pi (csrc/fit_sincos.py,
// Remez exchange on the absolute error; max error 2.0e-7 for sin, 4.9e-8 for cos with
// these float32 constants, about 4e-7 after float32 evaluation): sin x ~ x S(x^2),
// cos x ~ C(x^2).  Listed from the constant term up.
#define RBE2D_SIN_POLY 9.999995828e-01f, -1.666655391e-01f, 8.332408033e-03f, -1.980874076e-04f, \
                       2.699822744e-06f, -2.036623314e-08f
#define RBE2D_COS_POLY 1.000000000e+00f, -4.999998808e-01f, 4.166648909e-02f, -1.388780773e-03f, \
                       2.476996633e-05f, -2.707977558e-07f, 1.724760668e-09f
__device__ constexpr float kSinPoly[6] = {RBE2D_SIN_POLY};
__device__ constexpr float kCosPoly[7] = {RBE2D_COS_POLY};

// sin and cos of x (|x| <= pi) on the FMA pipe (no MUFU): 13 fused multiply-adds and
// multiplications, no quadrant bookkeeping, so a kernel can move any share of its
// angles off the MUFU unit for little extra issue.
__device__ __forceinline__ void sincos_poly_pi32(float x, float* s, float* c) {
    const float y = x * x;
    float p = kSinPoly[5];
#pragma unroll
    for (int i = 4; i >= 0; i--) p = fmaf(p, y, kSinPoly[i]);
    float q = kCosPoly[6];
#pragma unroll
    for (int i = 5; i >= 0; i--) q = fmaf(q, y, kCosPoly[i]);
    *s = x * p;
    *c = q;
}

// The same for the turn fraction t (2 pi t / 2^32, t read as signed).
__device__ __forceinline__ void sincos_poly32(uint32_t t, float* s, float* c) {
    sincos_poly_pi32((float)(int32_t)t * 1.46291807926715968e-09f, s, c);
}

// sin and cos of 2 pi t / 2^64.
__device__ __forceinline__ void sincos_turn64(unsigned long long t, double* s, double* c) {
    sincospi((double)(long long)t * 0x1p-63, s, c);
}

}  // namespace phase
}  // namespace rbe2d
