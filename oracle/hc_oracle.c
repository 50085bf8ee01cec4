/*
 * hc_oracle.c -- plain, slow, obviously-correct CPU oracle for the Hash Chain
 * (HC) exact string matcher of "Efficient Online String Matching through
 * Linked Weak Factors" (Palmer, Faro, Scafiti; arXiv 2310.15711).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker, not the product: only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg load
 * it.  It shares no code, header or table with the CUDA library, and it
 * imports nothing from it.
 *
 * Contents, each following one passage of the paper:
 *   or_naive_search   -- the problem statement itself (Sec. 1 and Sec. 2): every
 *                        window start p with y[p..p+m-1] = x, ascending.
 *   or_hash           -- the shift-then-add hash h (Eq. 3, Eq. 4), reading the
 *                        q-gram backwards from its last byte.
 *   or_link_hash      -- the link hash lambda (Eq. 5) with w = 32.
 *   or_preprocess     -- the preprocessing phase (Sec. 3.1, Eq. 1, Eq. 2): the
 *                        links of every chain, then the marks of the first
 *                        q-grams only where no link was set (Sec. 3.4, first
 *                        optimisation); returns F, s, F', H_v.
 *   or_window         -- one window after a passed first test: the back-walk
 *                        over linked q-grams (Sec. 3.3, Eq. 5), the H_v test
 *                        (Sec. 3.4, second optimisation) and verification.
 *   or_hc_search      -- the HC searching phase (Sec. 3.3).
 *   or_shc_search     -- the sentinel variant SHC (Sec. 3.4, third
 *                        optimisation).
 *
 * Readings taken where the paper is silent or garbled:
 *   - Verify/output position.  The paper's pseudocode (Fig. 5), after a
 *     window has been read in full, verifies and reports one position before
 *     the window's start (its first window would be checked at y[-1]).  The
 *     window that was read starts at end - m + 1, and the text of Sec. 3.3
 *     says the next window is the one starting one position further: the
 *     oracle verifies and reports the window's own start, end - m + 1, and
 *     then examines the window ending at end + 1.
 *   - w, the number of bits in a word of F, is 32 (Sec. 3.2 fixes w in the
 *     implementation without giving its value; the result set does not
 *     depend on it, F does).
 *   - Characters are unsigned bytes 0..255; hashes are computed in uint32.
 *     With alpha <= 15 the unmasked value stays below 2^24.
 *   - 1 <= q <= m and 1 <= alpha <= 15 are required; m = 0 is rejected.
 *   - n < m gives no windows and an empty result.
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define OR_W 32u /* bits per word of F */

/* ---------------------------------------------------------------------- */
/* Problem statement (Sec. 1, Sec. 2): all p in [0, n-m] with y[p..p+m-1] = x.
 * Writes up to cap positions into out and returns the total count. */
size_t or_naive_search(const uint8_t *x, size_t m, const uint8_t *y, size_t n,
                       uint64_t *out, size_t cap) {
    size_t count = 0;
    if (m == 0 || n < m) return 0;
    for (size_t p = 0; p + m <= n; p++) {
        size_t k = 0;
        while (k < m && y[p + k] == x[k]) k++;
        if (k == m) {
            if (count < cap) out[count] = (uint64_t)p;
            count++;
        }
    }
    return count;
}

/* ---------------------------------------------------------------------- */
/* Hash(x, p, q, s, F') of Fig. 4: read the q-gram that ENDS at position p
 * backwards, from x[p] down to x[p-q+1], shifting the running value left by
 * s before adding each character, and mask with F' = 2^alpha - 1 at the end.
 * This equals Eq. 3 (x[p-q+1] gets weight 1, x[p] weight 2^(s(q-1))),
 * taken mod 2^alpha. */
uint32_t or_hash(const uint8_t *x, long p, int q, int s, uint32_t mask) {
    uint32_t v = 0;
    for (long i = p; i >= p - q + 1; i--) v = (v << s) + (uint32_t)x[i];
    return v & mask;
}

/* LinkHash(v) of Fig. 4 / Eq. 5: a word with the single bit (v mod w) set. */
uint32_t or_link_hash(uint32_t v) { return 1u << (v & (OR_W - 1u)); }

/* ---------------------------------------------------------------------- */
/* Preprocessing(x, m, q, alpha) of Fig. 4 (Sec. 3.1).
 *   F      : caller buffer of 2^alpha words, overwritten.
 *   s_out, mask_out, hv_out : s = floor(alpha/q) (Eq. 4), F' = 2^alpha - 1,
 *            and H_v, the last hash computed in the chain phase, i.e. the
 *            hash of the first q-gram of the chain ending at m-1 (Sec. 3.4).
 *   trace  : if not NULL, receives the end position p of every Hash call in
 *            call order (chain phase first, then the marking phase), up to
 *            trace_cap entries; *trace_len gets the number of calls made and
 *            *chain_calls the number made in the chain phase.
 * Returns 0, or -1 on invalid arguments. */
int or_preprocess(const uint8_t *x, long m, int q, int alpha, uint32_t *F,
                  int *s_out, uint32_t *mask_out, uint32_t *hv_out,
                  long *trace, long trace_cap, long *trace_len,
                  long *chain_calls) {
    if (x == NULL || F == NULL || m < 1 || q < 1 || q > m || alpha < 1 ||
        alpha > 15)
        return -1;
    long calls = 0;
#define OR_TRACE(pos)                                                      \
    do {                                                                   \
        if (trace != NULL && calls < trace_cap) trace[calls] = (pos);      \
        calls++;                                                           \
    } while (0)

    int s = alpha / q;                   /* Eq. 4 */
    uint32_t mask = (1u << alpha) - 1u;  /* F' : mod 2^alpha as an AND */
    for (uint32_t i = 0; i <= mask; i++) F[i] = 0;

    /* Links (Sec. 3.1, Eq. 1).  A chain is a run of adjacent,
     * non-overlapping q-grams of x; the chain whose last q-gram ends at
     * pattern position e holds the q-grams ending at e, e - q, e - 2q, ...
     * down to q - 1.  Every q-gram belongs to exactly one chain, and the
     * chain ends are the last min(q, m - q + 1) positions of x.  The chains
     * are taken from the leftmost end to the one at m - 1, each from its
     * right end leftwards; for two neighbours of a chain, the right one's
     * word receives the link bit of the left one's hash. */
    long first_end = m - ((m - q + 1 < q) ? (m - q + 1) : q);
    uint32_t first_of_chain = 0;
    for (long e = first_end; e <= m - 1; e++) {
        uint32_t right = or_hash(x, e, q, s, mask);
        OR_TRACE(e);
        for (long p = e - q; p >= q - 1; p -= q) {
            uint32_t left = or_hash(x, p, q, s, mask);
            OR_TRACE(p);
            F[right] |= or_link_hash(left);    /* Eq. 1 */
            right = left;
        }
        first_of_chain = right;                /* hash of the chain's first q-gram */
    }
    /* H_v (Sec. 3.4, second optimisation): the hash of the first q-gram of
     * the chain that ends at m - 1, the last chain taken above. */
    uint32_t hv = first_of_chain;
    if (chain_calls != NULL) *chain_calls = calls;

    /* Marks (Eq. 2 with the first optimisation of Sec. 3.4): the first
     * q-gram of every chain -- those ending at q - 1 .. min(2q - 1, m) - 1,
     * which have no left neighbour -- gets the value 1, but only in a word
     * that no link has set. */
    long stop = (2 * q - 1 < m) ? (2 * q - 1) : m;
    for (long e = q - 1; e < stop; e++) {
        uint32_t u = or_hash(x, e, q, s, mask);
        OR_TRACE(e);
        if (F[u] == 0) F[u] = 1;
    }
#undef OR_TRACE
    if (trace_len != NULL) *trace_len = calls;
    *s_out = s;
    *mask_out = mask;
    *hv_out = hv;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* One window of the searching phase (Sec. 3.3, Eq. 5, Sec. 3.4), after its
 * first test has passed: the q-gram ending at the window's last position
 * `end` hashed to h, whose word F[h] is non-empty.  Going right to left,
 * each further q-gram that lies wholly inside the window must be linked to
 * its right neighbour: its link bit lambda(hash) must be set in the
 * neighbour's word.  At the first q-gram that is not, the window is left
 * and the next one examined ends m - q + 1 past that q-gram's end, the
 * first window that does not contain it.  A window read in full is an
 * occurrence candidate only if its leftmost hash equals H_v; it is then
 * compared with x, and the next window is the one starting one position
 * to the right.  Returns the end of the next window; *hit is 1 when the
 * window (starting at end - m + 1) is an occurrence. */
static long or_window(const uint8_t *x, long m, const uint8_t *t, long end,
                      int q, int s, uint32_t mask, const uint32_t *F,
                      uint32_t hv, uint32_t h, int *hit) {
    const long wstart = end - m + 1;
    uint32_t word = F[h];
    long last = end;                           /* end of the leftmost q-gram read */
    *hit = 0;
    while (last - 2 * q + 1 >= wstart) {       /* the next q-gram is inside */
        long left = last - q;
        uint32_t hl = or_hash(t, left, q, s, mask);
        if ((word & or_link_hash(hl)) == 0)
            return left + (m - q + 1);         /* not linked: leave the window */
        word = F[hl];
        h = hl;
        last = left;
    }
    if (h == hv && memcmp(t + wstart, x, (size_t)m) == 0) *hit = 1;
    return end + 1;
}

/* HC(x, m, y, n, q, alpha) of Sec. 3.3, using the filter built by
 * or_preprocess.  F must hold 2^alpha words.  Windows are examined left to
 * right by their last position; a window whose end q-gram hashes to an
 * empty word of F contains no factor of x ending there and is skipped by
 * m - q + 1 positions (the paper's shift), the others go through or_window.
 * Writes up to cap positions (0-based window starts, ascending) and returns
 * the total count; returns (size_t)-1 on invalid arguments. */
size_t or_hc_search(const uint8_t *x, long m, const uint8_t *y, long n,
                    int q, int alpha, uint32_t *F, uint64_t *out, size_t cap) {
    int s;
    uint32_t mask, hv;
    if (or_preprocess(x, m, q, alpha, F, &s, &mask, &hv, NULL, 0, NULL,
                      NULL) != 0)
        return (size_t)-1;
    size_t count = 0;
    long end = m - 1;                          /* the first window is y[0..m-1] */
    while (end < n) {
        uint32_t h = or_hash(y, end, q, s, mask);   /* first test */
        if (F[h] == 0) {
            end += m - q + 1;
            continue;
        }
        int hit;
        long next = or_window(x, m, y, end, q, s, mask, F, hv, h, &hit);
        if (hit) {
            if (count < cap) out[count] = (uint64_t)(end - m + 1);
            count++;
        }
        end = next;
    }
    return count;
}

/* ---------------------------------------------------------------------- */
/* SHC(x, m, y, n, q, alpha) of Sec. 3.4 (third optimisation): HC with a
 * copy of x placed right after the text, so that the loop of first tests
 * needs no test of the window position -- it stops at the latest on a
 * window inside the copy, every q-gram of which hits a non-empty word.
 * ybuf must be writable and hold n + m bytes; ybuf[n .. n+m-1] is
 * overwritten.  Same output convention as or_hc_search. */
size_t or_shc_search(const uint8_t *x, long m, uint8_t *ybuf, long n, int q,
                     int alpha, uint32_t *F, uint64_t *out, size_t cap) {
    int s;
    uint32_t mask, hv;
    if (or_preprocess(x, m, q, alpha, F, &s, &mask, &hv, NULL, 0, NULL,
                      NULL) != 0)
        return (size_t)-1;
    memcpy(ybuf + n, x, (size_t)m);            /* the sentinel */
    size_t count = 0;
    long end = m - 1;
    for (;;) {
        uint32_t h;
        while (F[h = or_hash(ybuf, end, q, s, mask)] == 0)
            end += m - q + 1;                  /* first tests only */
        if (end >= n) break;                   /* stopped in the sentinel */
        int hit;
        long next = or_window(x, m, ybuf, end, q, s, mask, F, hv, h, &hit);
        if (hit) {
            if (count < cap) out[count] = (uint64_t)(end - m + 1);
            count++;
        }
        end = next;
    }
    return count;
}
