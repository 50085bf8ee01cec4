/*
 * markov.c -- seeded order-2 Markov text source for synthetic inputs.
 *
 * Input generation only: nothing of the string-matching method is computed
 * here.  Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), one stream per
 * block so that blocks can be generated in parallel and reproducibly.
 */
#include <stddef.h>
#include <stdint.h>

static uint64_t sm64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Draw a symbol index from a cumulative table of sigma uint32 thresholds
 * (the last one is 2^32 - 1): the first k with u <= cum[k]. */
static int draw(const uint32_t *cum, int sigma, uint32_t u) {
    for (int k = 0; k < sigma - 1; k++)
        if (u <= cum[k]) return k;
    return sigma - 1;
}

/*
 * Fill out[0..len) with block `block` of an order-2 Markov chain over
 * `sigma` symbols.  uni_cum: sigma cumulative thresholds for the first two
 * symbols; row_cum: sigma*sigma rows of sigma thresholds, row (a*sigma + b)
 * giving the distribution of the symbol after the pair (a, b).  Symbol k is
 * written as the byte lut[k].
 */
void hcgen_markov2_block(uint8_t *out, size_t len, int sigma,
                         const uint32_t *uni_cum, const uint32_t *row_cum,
                         const uint8_t *lut, uint64_t seed, uint64_t block) {
    uint64_t st = seed * 0x632be59bd9b4e019ULL + block * 0xd1b54a32d192ed03ULL;
    int a = 0, b = 0;
    for (size_t i = 0; i < len; i++) {
        uint32_t u = (uint32_t)(sm64_next(&st) >> 32);
        int c;
        if (i < 2)
            c = draw(uni_cum, sigma, u);
        else
            c = draw(row_cum + ((size_t)a * sigma + b) * sigma, sigma, u);
        out[i] = lut[c];
        a = b;
        b = c;
    }
}
