/*
 * brute_force.c -- exhaustive check of the oracle's HC and SHC against its
 * naive matcher on every small input over a three-letter alphabet.
 *
 * Test code: compiled together with oracle/hc_oracle.c (or a mutated copy of
 * it) by tests/test_oracle_search.py and tests/test_oracle_mutants.py.
 *
 * Enumerates every pattern x over {0,1,2} with 1 <= m <= 4, every q in
 * [1, m], alpha in {1, 2, 3, 4, 6, 10}, and every text y over {0,1,2} with
 * 0 <= n <= 8.  Prints "cases=<c> hc_mismatch=<a> shc_mismatch=<b>".
 */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

size_t or_naive_search(const uint8_t *x, size_t m, const uint8_t *y, size_t n,
                       uint64_t *out, size_t cap);
size_t or_hc_search(const uint8_t *x, long m, const uint8_t *y, long n, int q,
                    int alpha, uint32_t *F, uint64_t *out, size_t cap);
size_t or_shc_search(const uint8_t *x, long m, uint8_t *ybuf, long n, int q,
                     int alpha, uint32_t *F, uint64_t *out, size_t cap);

static void decode(long code, int len, uint8_t *s) {
    for (int i = 0; i < len; i++) {
        s[i] = (uint8_t)(code % 3);
        code /= 3;
    }
}

int main(void) {
    static uint32_t F[1 << 10];
    uint8_t x[4], y[8], ybuf[16];
    uint64_t a[16], b[16], c[16];
    const int alphas[] = {1, 2, 3, 4, 6, 10};
    long cases = 0, hc_bad = 0, shc_bad = 0;
    for (int m = 1; m <= 4; m++) {
        long nx = 1;
        for (int i = 0; i < m; i++) nx *= 3;
        for (long cx = 0; cx < nx; cx++) {
            decode(cx, m, x);
            for (int q = 1; q <= m; q++) {
                for (unsigned ai = 0; ai < sizeof alphas / sizeof alphas[0]; ai++) {
                    int alpha = alphas[ai];
                    for (int n = 0; n <= 8; n++) {
                        long ny = 1;
                        for (int i = 0; i < n; i++) ny *= 3;
                        for (long cy = 0; cy < ny; cy++) {
                            decode(cy, n, y);
                            size_t k0 = or_naive_search(x, (size_t)m, y, (size_t)n, a, 16);
                            size_t k1 = or_hc_search(x, m, y, n, q, alpha, F, b, 16);
                            memcpy(ybuf, y, (size_t)n);
                            size_t k2 = or_shc_search(x, m, ybuf, n, q, alpha, F, c, 16);
                            cases++;
                            if (k1 != k0 || memcmp(a, b, k0 * sizeof(uint64_t)) != 0)
                                hc_bad++;
                            if (k2 != k0 || memcmp(a, c, k0 * sizeof(uint64_t)) != 0)
                                shc_bad++;
                        }
                    }
                }
            }
        }
    }
    printf("cases=%ld hc_mismatch=%ld shc_mismatch=%ld\n", cases, hc_bad, shc_bad);
    return 0;
}
