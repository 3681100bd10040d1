// swe_gelu.cuh -- the corrector network's activation on the GPU: GELU in
// its erf form, with erf evaluated by a published rational approximation.
#pragma once

#include <cuda_bf16.h>

#include "swe_device.cuh"

namespace swe {

using bf16 = __nv_bfloat16;

// erf by Abramowitz & Stegun, Handbook of Mathematical Functions, eq. 7.1.26:
// erf(x) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-x^2),
// t = 1 / (1 + p x) for x >= 0 (odd extension), |error| <= 1.5e-7.  Also
// returns exp(-x^2), which the GELU derivative reuses.
__device__ __forceinline__ float erf_as(float x, float &gauss)
{
    const float ax = fabsf(x);
    const float t = rcp(fmaf(0.3275911f, ax, 1.0f));
    float poly = fmaf(1.061405429f, t, -1.453152027f);
    poly = fmaf(poly, t, 1.421413741f);
    poly = fmaf(poly, t, -0.284496736f);
    poly = fmaf(poly, t, 0.254829592f);
    poly *= t;
    gauss = __expf(-ax * ax);
    const float e = fmaf(-poly, gauss, 1.0f);
    return copysignf(e, x);
}

// GELU 0.5 z (1 + erf(z / sqrt 2)) for the forward passes, with erf from
// Abramowitz & Stegun eq. 7.1.27: erf(x) = 1 - 1 / (1 + a1 x + a2 x^2 +
// a3 x^3 + a4 x^4)^4, |error| <= 5e-4, a1..a4 = 0.278393, 0.230389,
// 0.000972, 0.078108.  With u = |z| (x = u / sqrt 2) and the polynomial
// divided by 2^(-1/4) -- coefficients c_k = a_k / (2^(-1/4) sqrt(2)^k),
// c_0 = 2^(1/4) -- the fourth power of its reciprocal is
// q = (1 - erf(x)) / 2, so GELU = z (1 - q) for z >= 0 and z q for z < 0:
// written without a branch as GELU = z/2 + |z| (1/2 - q): one reciprocal
// and eight other operations.  The GELU error is at most 6.9e-4
// (2.3e-4 |z| for |z| > 1), about one bf16 half-ulp of the output.
constexpr float kGeluC4 = 2.322164733e-02f, kGeluC3 = 4.086756578e-04f, kGeluC2 = 1.369901190e-01f,
                kGeluC1 = 2.340996757e-01f, kGeluC0 = 1.189207115e+00f;

__device__ __forceinline__ float gelu_f(float z)
{
    const float u = fabsf(z);
    float d = fmaf(kGeluC4, u, kGeluC3);
    d = fmaf(d, u, kGeluC2);
    d = fmaf(d, u, kGeluC1);
    d = fmaf(d, u, kGeluC0);
    const float r = rcp(d);
    const float r2 = __fmul_rn(r, r);
    const float q = __fmul_rn(r2, r2);
    return fmaf(u, fmaf(q, -1.0f, 0.5f), __fmul_rn(0.5f, z));
}

// Packed pairs of FP32 values (the sm_100-family f32x2 instructions: two
// lanes of the same IEEE operation in one instruction).
__device__ __forceinline__ unsigned long long f32x2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f32x2_split(unsigned long long v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long fma_x2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ unsigned long long mul_x2(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// gelu_f of two values, the polynomial and products done pairwise; the
// same operations in the same order, so the same bits as gelu_f.
__device__ __forceinline__ void gelu_f2(float z0, float z1, float &g0, float &g1)
{
    const unsigned long long u = f32x2(fabsf(z0), fabsf(z1));
    unsigned long long d = fma_x2(f32x2(kGeluC4, kGeluC4), u, f32x2(kGeluC3, kGeluC3));
    d = fma_x2(d, u, f32x2(kGeluC2, kGeluC2));
    d = fma_x2(d, u, f32x2(kGeluC1, kGeluC1));
    d = fma_x2(d, u, f32x2(kGeluC0, kGeluC0));
    float d0, d1;
    f32x2_split(d, d0, d1);
    const unsigned long long r = f32x2(rcp(d0), rcp(d1));
    const unsigned long long r2 = mul_x2(r, r);
    const unsigned long long q = mul_x2(r2, r2);
    const unsigned long long hz = mul_x2(f32x2(0.5f, 0.5f), f32x2(z0, z1));
    const unsigned long long g = fma_x2(u, fma_x2(q, f32x2(-1.0f, -1.0f), f32x2(0.5f, 0.5f)), hz);
    f32x2_split(g, g0, g1);
}

// Derivative 0.5 (1 + erf(z / sqrt 2)) + z phi(z) for the backward pass,
// with the more accurate erf of eq. 7.1.26.

__device__ __forceinline__ float gelu_grad_f(float z)
{
    float g;  // exp(-z^2 / 2)
    const float e = erf_as(z * 0.70710678118654752f, g);
    return fmaf(z * g, 0.39894228040143268f, 0.5f * (1.0f + e));
}

}  // namespace swe
