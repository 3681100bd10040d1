/*
 * region_division_math.c -- host check of the mathematics of the region
 * statements' FP32 division (P. Markstein, IBM J. Res. Dev. 34(1), 1990;
 * Muller et al., Handbook of Floating-Point Arithmetic, ch. 4), independent
 * of the GPU's rcp.approx: the steps are restated here with C's correctly
 * rounded fmaf and fed every starting value the hardware approximation may
 * return (relative error at most 2^-23).
 *
 *   y1 = y0 + y0 (1 - b y0),  y2 = y1 + y1 (1 - b y1),
 *   q0 = a y2,  q1 = q0 + (a - b q0) y2,  q = q1 + (a - b q1) y2
 *
 * Checks (b in [1, 2): the FMAs scale exactly by powers of two over the
 * division's fast range 2^-20 <= b < 2^20, and so does the relative bound):
 *   1. y2 = RN(1/b) for every significand but the all-ones one and every
 *      float y0 within the bound;
 *   2. the all-ones significand has a y0 within the bound for which it is
 *      not (why the division sends those divisors to the exact fallback);
 *   3. q = RN(a/b) for every 8th significand b and for all of the first and
 *      last 4096 significands (about 1.06 million b), a on both sides of
 *      several quotient midpoints and at random, y0 at both ends of the
 *      bound and in the middle.  The reference is the quotient in double
 *      rounded to float, which is correctly rounded (53 >= 2 * 24 + 2).
 * Prints one line "ok <counts>" or the first failures; exit status 0 = ok.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

static float f_of(uint32_t u)
{
    float f;
    memcpy(&f, &u, 4);
    return f;
}

static float newton(float b, float y) { return fmaf(fmaf(-b, y, 1.0f), y, y); }

/* the floats y0 with |y0 - 1/b| <= 2^-23 / b, from the lowest up */
static float first_y0(double r)
{
    float y = (float)(r - ldexp(r, -23));
    while ((double)y < r - ldexp(r, -23)) y = nextafterf(y, 2.0f);
    return y;
}

static uint64_t lcg = 0x9E3779B97F4A7C15ull;
static uint32_t next_u32(void)
{
    lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
    return (uint32_t)(lcg >> 32);
}

int main(void)
{
    long n1 = 0, bad1 = 0, n3 = 0, bad3 = 0;
    for (uint32_t s = 0; s < (1u << 23) - 1; ++s) {
        const float b = f_of((127u << 23) | s);
        const double r = 1.0 / (double)b;
        const float want = (float)r;
        for (float y0 = first_y0(r); (double)y0 <= r + ldexp(r, -23); y0 = nextafterf(y0, 2.0f)) {
            ++n1;
            if (newton(b, newton(b, y0)) != want && bad1++ < 5) printf("rcp b=%a y0=%a\n", b, y0);
        }
        /* check 3 on every 8th significand, plus all of the first and last 4096 */
        if ((s & 7u) && s >= 4096u && s < (1u << 23) - 4097u) continue;
        float y0s[3] = {first_y0(r), want, 0.0f};  /* lowest, RN(1/b), highest */
        float top = want;
        while ((double)nextafterf(top, 2.0f) <= r + ldexp(r, -23)) top = nextafterf(top, 2.0f);
        y0s[2] = top;
        for (int t = 0; t < 6; ++t) {
            float a;
            if (t < 4) {
                /* a = RN(b m) for a quotient midpoint m: the hardest rounding cases */
                const float q = f_of((uint32_t)(127 - 30 + (next_u32() % 60)) << 23 | (next_u32() & 0x7fffffu));
                const double m = ((double)q + (double)nextafterf(q, 3.0e38f)) / 2.0;
                a = (float)((double)b * m);
                if (t & 1) a = nextafterf(a, 3.0e38f);
            } else {
                a = f_of((uint32_t)(127 - 60 + (next_u32() % 120)) << 23 | (next_u32() & 0x7fffffu));
            }
            const float ref = (float)((double)a / (double)b);
            for (int k = 0; k < 3; ++k) {
                const float y2 = newton(b, newton(b, y0s[k]));
                const float q0 = a * y2;
                const float q1 = fmaf(fmaf(-b, q0, a), y2, q0);
                const float q = fmaf(fmaf(-b, q1, a), y2, q1);
                ++n3;
                if (q != ref && bad3++ < 5) printf("div a=%a b=%a y0=%a q=%a want=%a\n", a, b, y0s[k], q, ref);
            }
        }
    }
    /* check 2 */
    const float b1 = f_of((127u << 23) | 0x7fffffu);
    const double r1 = 1.0 / (double)b1;
    int miss = 0;
    for (float y0 = first_y0(r1); (double)y0 <= r1 + ldexp(r1, -23); y0 = nextafterf(y0, 2.0f))
        miss += newton(b1, newton(b1, y0)) != (float)r1;
    const int ok = bad1 == 0 && bad3 == 0 && miss > 0;
    printf("%s rcp %ld/%ld div %ld/%ld all-ones-misses %d\n", ok ? "ok" : "FAIL", n1 - bad1, n1, n3 - bad3, n3, miss);
    return ok ? 0 : 1;
}
