// Host harness for the FP32 mass accumulator (swe_exact_sum.h, the same
// code the mass kernel runs): reads binary32 values from the file argv[1],
// feeds them in groups of four (the kernel's vector path) and the remainder
// one by one (its row tail), and prints the result in hexadecimal
// floating-point notation.
#include <stdio.h>
#include <stdlib.h>

#include "swe_exact_sum.h"

int main(int argc, char **argv)
{
    if (argc < 2) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    fseek(f, 0, SEEK_END);
    const long bytes = ftell(f);
    fseek(f, 0, SEEK_SET);
    const long n = bytes / 4;
    float *x = (float *)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
    if (!x || fread(x, 4, (size_t)n, f) != (size_t)n) return 2;
    fclose(f);
    swe::ExactSum32 s;
    long i = 0;
    for (; i + 4 <= n; i += 4) s.add4(x[i], x[i + 1], x[i + 2], x[i + 3]);
    for (; i < n; ++i) s.add1(x[i]);
    printf("%a\n", s.value());
    free(x);
    return 0;
}
