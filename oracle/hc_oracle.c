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
 *   or_hash           -- the shift-then-add hash h (Eq. 3, Eq. 4) in the
 *                        backward-reading form of the Hash routine (Fig. 4).
 *   or_link_hash      -- the link hash lambda (Eq. 5) with w = 32.
 *   or_preprocess     -- the preprocessing phase (Sec. 3.1, Eq. 1, Eq. 2,
 *                        Fig. 4), chains walked backwards from the pattern end,
 *                        first q-grams marked last and only if empty
 *                        (Sec. 3.4, first optimisation); returns F, s, F', H_v.
 *   or_hc_search      -- the HC searching phase (Sec. 3.3, Fig. 5 left) with
 *                        the H_v early reject (Sec. 3.4, second optimisation).
 *   or_shc_search     -- the sentinel variant SHC (Sec. 3.4, third
 *                        optimisation, Fig. 5 right).
 *
 * Readings taken where the paper is silent or garbled:
 *   - Verify/output position.  Fig. 5 sets j <- i - q after a full pass, which
 *     puts j at (window end) - m + q, and then verifies and outputs at j - q.
 *     The window that was just scanned starts at (window end) - m + 1 =
 *     j - q + 1 (the first window is y[0..m-1] with j = m - 1, and Sec. 3.3
 *     says the window then advances by exactly one).  The oracle verifies the
 *     window y[j-q+1 .. j-q+m] and outputs j - q + 1; j itself is left as the
 *     paper sets it, so the next window is still one position to the right.
 *   - w, the number of bits in a word of F, is 32 (Sec. 3.2 leaves it
 *     "hard-coded"; the result set does not depend on it, F does).
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

    /* Chain phase.  There are min(m-q+1, q) chains (Sec. 3.1); chain i ends
     * at m-i and they are taken for i = min(m-q+1, q) down to 1, so the chain
     * ending at the pattern end comes last.  Each chain is walked from its
     * right end leftwards, one q-gram at a time; each (left, right) pair of
     * adjacent q-grams ORs lambda(h(left)) into F[h(right)] (Eq. 1). */
    uint32_t v = 0;
    long nchains = (m - q + 1 < q) ? (m - q + 1) : q;
    for (long i = nchains; i >= 1; i--) {
        v = or_hash(x, m - i, q, s, mask);     /* rightmost q-gram of chain */
        OR_TRACE(m - i);
        long j = m - i - q;                    /* end of its left neighbour */
        while (j >= q - 1) {                   /* left neighbour fits in x */
            uint32_t vr = v;                   /* right q-gram's hash */
            v = or_hash(x, j, q, s, mask);     /* left q-gram's hash */
            OR_TRACE(j);
            F[vr] |= or_link_hash(v);          /* Eq. 1 */
            j -= q;
        }
    }
    /* H_v: the last hash of the last chain, i.e. of the first q-gram of the
     * chain that ends at m-1 (Sec. 3.4, second optimisation). */
    uint32_t hv = v;
    if (chain_calls != NULL) *chain_calls = calls;

    /* Marking phase (Eq. 2 with the first optimisation of Sec. 3.4): the
     * q-grams ending at q-1 .. min(2q-1, m)-1 have no left neighbour; their
     * word gets the value 1 only if nothing has been set in it yet. */
    long last = (2 * q - 1 < m) ? (2 * q - 1) : m;
    for (long i = q - 1; i <= last - 1; i++) {
        uint32_t u = or_hash(x, i, q, s, mask);
        OR_TRACE(i);
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
/* HC(x, m, y, n, q, alpha) of Fig. 5 left (Sec. 3.3), using the filter built
 * by or_preprocess.  F must hold 2^alpha words.  Writes up to cap positions
 * (0-based window starts, ascending) and returns the total count; returns
 * (size_t)-1 on invalid arguments. */
size_t or_hc_search(const uint8_t *x, long m, const uint8_t *y, long n,
                    int q, int alpha, uint32_t *F, uint64_t *out, size_t cap) {
    int s;
    uint32_t mask, hv;
    if (or_preprocess(x, m, q, alpha, F, &s, &mask, &hv, NULL, 0, NULL,
                      NULL) != 0)
        return (size_t)-1;
    /* j is the text position aligned with the END of the current window;
     * the first window is y[0..m-1]. */
    size_t count = 0;
    long j = m - 1;
    while (j < n) {
        /* First test: the q-gram ending at the window end must hash to a
         * non-empty word of F, else no factor of x ends there (Sec. 3.3). */
        uint32_t v = or_hash(y, j, q, s, mask);
        uint32_t z = F[v];
        if (z != 0) {
            /* Back-walk: read the window's q-grams right to left; each must
             * be linked (Eq. 1) to the q-gram on its right, i.e. its bit
             * lambda(v) must be set in z = F[h(right q-gram)].  i bounds the
             * walk so that every q-gram read lies inside the window. */
            long i = j - m + 2 * q;
            int broke = 0;
            while (j >= i) {
                j -= q;
                v = or_hash(y, j, q, s, mask);
                if ((z & or_link_hash(v)) == 0) {
                    broke = 1;  /* not linked: shift past this q-gram */
                    break;
                }
                z = F[v];
            }
            if (!broke) {
                /* The whole window was read (the while loop's else branch).
                 * Reset j so the shift below advances the window by one, and
                 * verify only if the last hash equals H_v (Sec. 3.4). */
                j = i - q;
                long start = j - q + 1;         /* reading: window start */
                if (v == hv && memcmp(y + start, x, (size_t)m) == 0) {
                    if (count < cap) out[count] = (uint64_t)start;
                    count++;
                }
            }
        }
        /* Shift: m-q+1 past the window end on a first-test miss, past the
         * unlinked q-gram after a break, by one after a full read. */
        j += m - q + 1;
    }
    return count;
}

/* ---------------------------------------------------------------------- */
/* SHC(x, m, y, n, q, alpha) of Fig. 5 right (Sec. 3.4, sentinel).  ybuf must
 * be writable and hold n + m bytes: the pattern is copied into
 * ybuf[n .. n+m-1] so that the inner miss loop needs no position test.
 * Same output convention as or_hc_search. */
size_t or_shc_search(const uint8_t *x, long m, uint8_t *ybuf, long n, int q,
                     int alpha, uint32_t *F, uint64_t *out, size_t cap) {
    int s;
    uint32_t mask, hv;
    if (or_preprocess(x, m, q, alpha, F, &s, &mask, &hv, NULL, 0, NULL,
                      NULL) != 0)
        return (size_t)-1;
    /* Sentinel: a copy of x right after the text guarantees that the fast
     * miss loop below stops at the latest on the sentinel window. */
    for (long i = 0; i < m; i++) ybuf[n + i] = x[i];
    size_t count = 0;
    long j = m - 1;
    while (j < n) {
        /* Fast loop: first test only, no position check. */
        while (F[or_hash(ybuf, j, q, s, mask)] == 0)
            j += m - q + 1;
        /* The position check happens once the fast loop has stopped; the
         * rest is the HC back-walk and verification. */
        if (j < n) {
            uint32_t v = or_hash(ybuf, j, q, s, mask);
            uint32_t z = F[v];
            long i = j - m + 2 * q;
            int broke = 0;
            while (j >= i) {
                j -= q;
                v = or_hash(ybuf, j, q, s, mask);
                if ((z & or_link_hash(v)) == 0) {
                    broke = 1;
                    break;
                }
                z = F[v];
            }
            if (!broke) {
                j = i - q;
                long start = j - q + 1;         /* reading: window start */
                if (v == hv && memcmp(ybuf + start, x, (size_t)m) == 0) {
                    if (count < cap) out[count] = (uint64_t)start;
                    count++;
                }
            }
            j += m - q + 1;
        }
    }
    return count;
}
