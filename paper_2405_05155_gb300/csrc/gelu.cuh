// GELU in its erf form, GELU(z) = z Phi(z) with Phi(z) = (1 + erf(z / sqrt 2)) / 2,
// and its derivative Phi(z) + z phi(z), phi(z) = exp(-z^2 / 2) / sqrt(2 pi).
//
// erf is evaluated with the rational-exponential approximation of Abramowitz and
// Stegun (Handbook of Mathematical Functions, formula 7.1.26): for x >= 0,
//   erf x = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-x^2},  t = 1 / (1 + p x),
// with absolute error at most 1.5e-7, and erf(-x) = -erf x.  At x = |z| / sqrt 2,
//   s = (1 - erf x) / 2 = t (a1/2 + ... ) e^{-z^2/2},   Phi(z) = 1 - s (z >= 0), s (z < 0),
// so GELU(z) = max(z, 0) - |z| s without a branch.  The reciprocal and the power of
// two are the special-function unit's approximate instructions (rcp.approx,
// ex2.approx, relative errors near 2^-23); the activations are rounded to bfloat16
// (relative 2^-9) afterwards, far above these errors.
#pragma once

namespace gelu_as {

constexpr float kP = 0.3275911f;
constexpr float kA1 = 0.254829592f, kA2 = -0.284496736f, kA3 = 1.421413741f, kA4 = -1.453152027f,
                kA5 = 1.061405429f;
constexpr float kInvSqrt2 = 0.70710678118654752f;
constexpr float kInvSqrt2Pi = 0.39894228040143268f;
constexpr float kHalfLog2e = 0.72134752044448170f;   // log2(e) / 2

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// s(z) = (1 - erf(|z| / sqrt 2)) / 2 = Phi(-|z|), the normal tail beyond |z|.
__device__ __forceinline__ float normal_tail(float z) {
    const float t = rcp_approx(fmaf(kP * kInvSqrt2, fabsf(z), 1.0f));
    const float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 0.5f * kA5, 0.5f * kA4), 0.5f * kA3), 0.5f * kA2),
                                0.5f * kA1);
    return poly * ex2_approx(-(z * z) * kHalfLog2e);
}

__device__ __forceinline__ float gelu(float z) { return fmaf(-fabsf(z), normal_tail(z), fmaxf(z, 0.0f)); }

// Two activations at once on the paired float32 instructions (FFMA2 / FMUL2): the same
// operations in the same order as gelu per element, so the same bits; the reciprocal and
// the power of two stay per element on the special-function unit.
__device__ __forceinline__ float2 gelu2(float2 z) {
    const float2 az = make_float2(fabsf(z.x), fabsf(z.y));
    const float2 d = __ffma2_rn(make_float2(kP * kInvSqrt2, kP * kInvSqrt2), az, make_float2(1.0f, 1.0f));
    const float2 t = make_float2(rcp_approx(d.x), rcp_approx(d.y));
    float2 q = __ffma2_rn(t, make_float2(0.5f * kA5, 0.5f * kA5), make_float2(0.5f * kA4, 0.5f * kA4));
    q = __ffma2_rn(t, q, make_float2(0.5f * kA3, 0.5f * kA3));
    q = __ffma2_rn(t, q, make_float2(0.5f * kA2, 0.5f * kA2));
    q = __ffma2_rn(t, q, make_float2(0.5f * kA1, 0.5f * kA1));
    const float2 poly = __fmul2_rn(t, q);
    const float2 zz = __fmul2_rn(z, z);
    const float2 arg = __fmul2_rn(make_float2(-zz.x, -zz.y), make_float2(kHalfLog2e, kHalfLog2e));
    const float2 s = __fmul2_rn(poly, make_float2(ex2_approx(arg.x), ex2_approx(arg.y)));
    return __ffma2_rn(make_float2(-az.x, -az.y), s, make_float2(fmaxf(z.x, 0.0f), fmaxf(z.y, 0.0f)));
}

__device__ __forceinline__ float gelu_grad(float z) {
    const float s = normal_tail(z);
    const float phi = z >= 0.0f ? 1.0f - s : s;
    return fmaf(z * kInvSqrt2Pi, ex2_approx(-(z * z) * kHalfLog2e), phi);
}

}  // namespace gelu_as
