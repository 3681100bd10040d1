/*
 * fma_negzero.c -- host check of the identity behind the packed unfused
 * product of the FP32 step kernels: with round-to-nearest binary32,
 *
 *     fma(a, b, -0) == RN(a * b)   bit for bit,
 *
 * for every a and b (the exact product plus -0 is the exact product, except
 * that an exact zero product keeps its own sign: +0 + -0 = +0, -0 + -0 = -0;
 * NaN inputs give NaN either way).  A +0 addend would not do: it turns a -0
 * product into +0.  Checked on all pairs of a set of special values (signed
 * zeros, subnormals, the smallest and largest normals, infinities, NaN,
 * values whose product underflows or overflows), on 2^24 random pairs of
 * bit patterns and on 2^21 pairs whose products lie near the subnormal and
 * overflow thresholds, against the product computed by the C multiply
 * (binary32, round to nearest, no contraction); a control checks that a +0
 * addend fails.  Prints "ok <count>" or the first failures; exit status
 * 0 = ok.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

static float f_of(uint32_t u)
{
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}
static uint32_t u_of(float f)
{
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
}

static uint64_t rng = 0x9E3779B97F4A7C15ull;
static uint32_t next32(void)
{
    /* SplitMix64 (Steele, Lea, Flood 2014), upper half */
    uint64_t z = (rng += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (uint32_t)(z >> 32);
}

static long long checked = 0, bad = 0;

static void check(float a, float b)
{
    volatile float va = a, vb = b;
    const float prod = va * vb;
    const float viaf = fmaf(va, vb, -0.0f);
    ++checked;
    const int both_nan = isnan(prod) && isnan(viaf);
    if (!both_nan && u_of(prod) != u_of(viaf)) {
        if (bad < 10)
            printf("mismatch a=%08x b=%08x mul=%08x fma=%08x\n", (unsigned)u_of(a), (unsigned)u_of(b),
                   (unsigned)u_of(prod), (unsigned)u_of(viaf));
        ++bad;
    }
}

int main(void)
{
    const uint32_t special[] = {
        0x00000000u, 0x80000000u,              /* +0, -0 */
        0x00000001u, 0x80000001u, 0x007fffffu, /* subnormals */
        0x00800000u, 0x80800000u,              /* smallest normals */
        0x3f800000u, 0xbf800000u, 0x3f800001u, /* +-1, 1 + ulp */
        0x1f800000u, 0x9f800000u,              /* 2^-64: products underflow */
        0x5f800000u, 0xdf800000u,              /* 2^64: products overflow */
        0x7f7fffffu, 0xff7fffffu,              /* largest normals */
        0x7f800000u, 0xff800000u,              /* infinities */
        0x7fc00000u,                           /* NaN */
        0x3eaaaaabu, 0x40490fdbu, 0x4b000001u, /* 1/3, pi, 2^23 + 1 */
    };
    const int ns = (int)(sizeof special / sizeof special[0]);
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) check(f_of(special[i]), f_of(special[j]));
    for (long k = 0; k < (1L << 24); ++k) check(f_of(next32()), f_of(next32()));
    /* products near zero and near the largest normal: exponents chosen */
    for (long k = 0; k < (1L << 20); ++k) {
        const uint32_t m = next32();
        const uint32_t ea = (m & 0xff) % 254 + 1, eb = (253 - ea + (m >> 8) % 9) % 254 + 1;
        const uint32_t a = ((m >> 31) << 31) | (ea << 23) | (next32() & 0x7fffffu);
        const uint32_t b = (((m >> 30) & 1u) << 31) | (eb << 23) | (next32() & 0x7fffffu);
        check(f_of(a), f_of(b));
        check(f_of(a), f_of(b ^ 0x3f000000u));
    }
    /* the check can fail: with a +0 addend a -0 product becomes +0 */
    {
        volatile float m1 = -1.0f, z = 0.0f, pz = 0.0f;
        if (u_of(fmaf(m1, z, pz)) == u_of(m1 * z)) {
            printf("FAIL control: fma(-1, 0, +0) kept the sign of -0\n");
            return 1;
        }
    }
    if (bad) {
        printf("FAIL %lld of %lld\n", bad, checked);
        return 1;
    }
    printf("ok %lld\n", checked);
    return 0;
}
