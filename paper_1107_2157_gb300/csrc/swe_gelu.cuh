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
// one reciprocal and nine other operations.  The GELU error is at most
// 6.9e-4 (2.3e-4 |z| for |z| > 1), about one bf16 half-ulp of the output.
__device__ __forceinline__ float gelu_f(float z)
{
    const float u = fabsf(z);
    float d = fmaf(2.322164733e-02f, u, 4.086756578e-04f);
    d = fmaf(d, u, 1.369901190e-01f);
    d = fmaf(d, u, 2.340996757e-01f);
    d = fmaf(d, u, 1.189207115e+00f);
    const float r = rcp(d);
    const float r2 = r * r;
    const float q = r2 * r2;
    return z * (z >= 0.0f ? 1.0f - q : q);
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
