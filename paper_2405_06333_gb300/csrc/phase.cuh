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

// sin and cos of 2 pi t / 2^32 on the FMA pipe (no MUFU): the nearest quarter turn from
// the top bits, the remainder (|x| <= pi/4, converted exactly to within 16 units of
// 2^-32 turn) through minimax polynomials (coefficients from csrc/fit_sincos.py, max
// error 4.1e-9 for sin, 2.7e-9 for cos before float32 rounding), then a rotation by
// the quarter turns.
__device__ __forceinline__ void sincos_poly32(uint32_t t, float* s, float* c) {
    const uint32_t qd = (t + 0x20000000u) >> 30;
    const int32_t r = (int32_t)(t - (qd << 30));
    const float x = (float)r * 1.46291807926715968e-09f;
    const float y = x * x;
    const float sp = x * fmaf(fmaf(fmaf(-1.950402220e-04f, y, 8.332036436e-03f), y, -1.666665077e-01f), y, 1.0f);
    const float cp = fmaf(fmaf(fmaf(fmaf(2.437992953e-05f, y, -1.388661913e-03f), y, 4.166661575e-02f), y, -0.5f), y,
                          1.0f);
    const bool odd = (qd & 1u) != 0;
    const float ss = odd ? cp : sp, cc = odd ? sp : cp;
    *s = (qd & 2u) ? -ss : ss;
    *c = ((qd + 1u) & 2u) ? -cc : cc;
}

// sin and cos of 2 pi t / 2^64.
__device__ __forceinline__ void sincos_turn64(unsigned long long t, double* s, double* c) {
    sincospi((double)(long long)t * 0x1p-63, s, c);
}

}  // namespace phase
}  // namespace rbe2d
