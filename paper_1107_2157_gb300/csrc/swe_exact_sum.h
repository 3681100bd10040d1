// swe_exact_sum.h -- exact sum of binary32 values in 64-bit integers, the
// accumulator of the FP32 mass reduction (the mass of Sec. 3 is the sum of
// the depths times dx dy).  Plain C++ that nvcc compiles for the device and a
// host compiler for the host, so the same code is checked on the CPU.
//
// A finite binary32 value x with biased exponent e and fraction f is
// m * 2^(max(e,1) - 150) with the integer m = f (+ 2^23 if e > 0), m < 2^24.
// The accumulator holds an integer count of units 2^(R - 155), R being the
// largest exponent met so far: a value whose exponent lies within 5 binades
// below R contributes m * 2^(5 - (R - e)) units exactly.  A larger exponent
// first flushes the accumulator to the FP64 total (exactly: it stays below
// 2^53) and makes itself the reference.  Values more than 5 binades below R
// and non-finite values are added to the FP64 total directly; zeros add
// nothing.  The result is total + acc * 2^(R - 155): every value reaches it
// exactly, and FP64 rounding enters only where flushed parts and the small
// values are added to the total.
//
// Fast path: four positive, normal, finite values whose exponents all lie in
// [R - 5, R] (R >= 6) cost a few integer shifts, masks and additions.  Each
// such group adds less than 4 * 2^24 * 2^5 = 2^31 units, so the
// accumulator stays below 2^53 for up to 2^22 groups between flushes (a
// thread of the mass kernel meets at most 2^12 for the largest grid, 65536^2
// over 1024 blocks of 256 threads).
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define SWE_HD __host__ __device__ __forceinline__
#else
#define SWE_HD inline
#endif

namespace swe {

SWE_HD uint32_t f32_bits(float x)
{
    uint32_t b;
    memcpy(&b, &x, sizeof b);
    return b;
}

// 2^e as a double, for -1022 <= e <= 1023.
SWE_HD double pow2_f64(int e)
{
    const long long b = (long long)(e + 1023) << 52;
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
}

struct ExactSum32 {
    long long acc = 0;
    int R = 0;  // reference biased exponent (0: none yet)
    double total = 0.0;

    SWE_HD void flush_to(int newR)
    {
        total += (double)acc * pow2_f64(R - 155);
        acc = 0;
        R = newR;
    }
    SWE_HD void add1(float x)
    {
        const uint32_t b = f32_bits(x);
        const int e = (int)((b >> 23) & 0xffu);
        uint32_t m = b & 0x7fffffu;
        if (e == 255) {  // Inf or NaN: propagates as in an FP64 sum
            total += (double)x;
            return;
        }
        if (e != 0) m |= 0x800000u;
        if (m == 0) return;
        const int ee = e > 0 ? e : 1;
        if (ee > R) flush_to(ee);
        const int d = R - ee;
        if (d <= 5) {
            const long long c = (long long)(m << (5 - d));
            acc += (b >> 31) ? -c : c;
        } else {
            total += (double)x;
        }
    }
    SWE_HD void add4(float x0, float x1, float x2, float x3)
    {
        const uint32_t b0 = f32_bits(x0), b1 = f32_bits(x1), b2 = f32_bits(x2), b3 = f32_bits(x3);
        // shift of each value's significand: its exponent - (R - 5), in [0, 5]
        // on the fast path; a set sign bit or a larger exponent gives more
        // than 5, a smaller exponent wraps around to a large unsigned value
        const uint32_t base = (uint32_t)R - 5u;
        const uint32_t s0 = (b0 >> 23) - base, s1 = (b1 >> 23) - base, s2 = (b2 >> 23) - base,
                       s3 = (b3 >> 23) - base;
        const uint32_t smax = s0 > s1 ? s0 : s1, smax2 = s2 > s3 ? s2 : s3;
        if (R >= 6 && (smax > smax2 ? smax : smax2) <= 5u) {
            const uint32_t s = (((b0 & 0x7fffffu) | 0x800000u) << s0) + (((b1 & 0x7fffffu) | 0x800000u) << s1) +
                               (((b2 & 0x7fffffu) | 0x800000u) << s2) + (((b3 & 0x7fffffu) | 0x800000u) << s3);
            acc += (long long)s;
        } else {
            add1(x0);
            add1(x1);
            add1(x2);
            add1(x3);
        }
    }
    SWE_HD double value() const { return total + (double)acc * pow2_f64(R - 155); }
};

}  // namespace swe
