/*
 * hc.h -- C ABI of the GB300 (sm_103a) Hash Chain (HC) exact string matcher.
 *
 * Method: "Efficient Online String Matching through Linked Weak Factors"
 * (M. N. Palmer, S. Faro, S. Scafiti; arXiv 2310.15711).  The problem (Sec. 1,
 * Sec. 2): report every occurrence of a pattern x of length m in a text y of
 * length n, i.e. every window start p in [0, n-m] with y[p..p+m-1] = x.
 *
 * Conventions shared by every entry point:
 *   - Bytes are unsigned (0..255).  A filter word has w = 32 bits.
 *   - Positions are 0-based window starts, uint64, strictly ascending.
 *   - Pointers named *_dev are CUDA device pointers (any allocation the
 *     current device can read/write); all others are host pointers.  The
 *     caller owns every buffer it passes; the library never frees them and
 *     never writes to the text.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *     work is enqueued on it; entry points without the _async suffix also wait
 *     for it.
 *   - Return value: HC_OK (0) or one of the HC_ERR_* codes below;
 *     hc_last_error() gives a message for the calling thread's last failure.
 *   - Parameter ranges: m >= 1, 1 <= q <= min(m, 8), 1 <= alpha <= 15.  The
 *     paper's experiments use 1 <= q <= 8 and 8 <= alpha <= 12 (Sec. 4).
 */
#ifndef HC_GB300_H
#define HC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hc_filter hc_filter;      /* opaque: F, s, F', H_v, q, alpha, x */
typedef struct CUstream_st *hc_stream_t; /* same type as cudaStream_t */

enum {
    HC_OK = 0,
    HC_ERR_ARG = 1,       /* null pointer or parameter out of range */
    HC_ERR_CAPACITY = 2,  /* more occurrences than the output buffer holds */
    HC_ERR_CUDA = 3,      /* a CUDA runtime call failed (see hc_last_error) */
    HC_ERR_NOMEM = 4,     /* host or device allocation failed */
    HC_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up */
    HC_ERR_ADMISSION = 6, /* server: request refused by the memory budget */
    HC_ERR_STATE = 7      /* object used in the wrong state */
};

/* Library version (major*10000 + minor*100 + patch). */
int hc_version(void);

/* Message describing the calling thread's most recent failure ("" if none). */
const char *hc_last_error(void);

/* ------------------------------------------------------------------------
 * Preprocessing phase (Sec. 3.1, Eq. 1-5, Fig. 4).
 *
 * hc_preprocess builds the filter of pattern x (host memory, m bytes) on the
 * host: F is a table of 2^alpha 32-bit words; for every pair u1.u2 of
 * adjacent non-overlapping q-grams of x, F[h(u2)] |= lambda(h(u1)) (Eq. 1);
 * then every first q-gram u (starting at 0 .. min(q, m-q+1)-1) whose word is
 * still empty gets F[h(u)] = 1 (Eq. 2 with the first optimisation of
 * Sec. 3.4).  h is the shift-then-add hash (Eq. 3) with s = floor(alpha/q)
 * (Eq. 4) taken mod 2^alpha; lambda(v) = 1 << (v mod 32) (Eq. 5).  H_v is
 * h of the first q-gram of the chain ending at m-1, i.e. of x[m mod q ..]
 * (Sec. 3.4, second optimisation).
 * On success *out receives a filter owned by the caller (free it with
 * hc_filter_free).  Needs no GPU.  Errors: HC_ERR_ARG, HC_ERR_NOMEM.
 */
int hc_preprocess(const uint8_t *x, size_t m, int q, int alpha,
                  hc_filter **out);

/* Frees a filter and its device copy (if one was made).  NULL is a no-op. */
void hc_filter_free(hc_filter *f);

/* Read-only view of the filter: *F receives a pointer to its 2^alpha words
 * (valid until hc_filter_free), *nwords = 2^alpha, *hv = H_v.  Any output
 * pointer may be NULL.  Errors: HC_ERR_ARG. */
int hc_filter_words(const hc_filter *f, const uint32_t **F, size_t *nwords,
                    uint32_t *hv);

/* Parameters of a filter: pattern length m, q, alpha and s = floor(alpha/q).
 * Any output pointer may be NULL.  Errors: HC_ERR_ARG. */
int hc_filter_params(const hc_filter *f, size_t *m, int *q, int *alpha,
                     int *s);

/* Copies the filter (F words and pattern bytes) to the current device, once
 * per filter; later calls are no-ops.  hc_search does this itself on first
 * use; call it beforehand when the first search must not allocate (e.g.
 * before capturing a CUDA graph).  Errors: HC_ERR_CUDA, HC_ERR_NOMEM. */
int hc_filter_to_device(hc_filter *f);

/* ------------------------------------------------------------------------
 * Searching phase (Sec. 3.3, Fig. 5 left, with the H_v early reject of
 * Sec. 3.4).  Each length-m window is read backwards q-gram by q-gram: the
 * q-gram at the window end must hit a non-empty word of F, every q-gram to
 * its left must be linked to its right neighbour (its lambda bit set in the
 * neighbour's word); the window shifts on the first miss (by m-q+1 on a
 * first-test miss, past the unlinked q-gram otherwise), and a window read in
 * full whose last hash equals H_v is verified byte by byte against x and then
 * advanced by one.  The result is exactly the set of occurrences.
 *
 * hc_search_async: y_dev is the text (n bytes, device memory, any alignment);
 * pos_dev receives the first min(count, cap) occurrence positions in
 * ascending order (may be NULL when cap = 0); count_dev (one uint64)
 * receives the total count; both may be device memory or mapped host memory
 * (hc_mapped_alloc).  Both must be 8-byte aligned (any
 * element of a uint64 array is), else HC_ERR_ARG.  Nothing is waited for.  The first call
 * with a filter copies it to the device (see hc_filter_to_device).  Each call
 * takes a stream-ordered workspace from the library's memory pool and gives
 * it back after its kernels: 16 bytes per warp plus 4 bytes per spilled
 * position (by default min(n-m+1, max(cap, 2^20)) of them), for the
 * dense form's bitmap (m = q, hc_search_opts.bitmap) 16 bytes per warp plus
 * one bit per window start, or for the single-pass dense form 8 bytes per
 * tile of 8192 window starts;
 * the pool keeps freed memory for reuse.  n < m is not an error: the count is 0.  Errors:
 * HC_ERR_ARG, HC_ERR_CUDA, HC_ERR_NOMEM; a device wait that gave up is
 * reported by the next hc_search/hc_check_status.
 */
int hc_search_async(const hc_filter *f, const uint8_t *y_dev, size_t n,
                    uint64_t *pos_dev, size_t cap, uint64_t *count_dev,
                    hc_stream_t stream);

/* Launch options of hc_search_ex (zero = automatic).
 *   mode: HC_MODE_STAGED -- each thread runs HC over its own run of window
 *         starts, the text staged in shared memory by bulk copies;
 *         HC_MODE_DIRECT -- the same, reading the text from global memory
 *         (long patterns: their shifts skip most of the text);
 *         HC_MODE_DENSE -- for m = q only, where HC tests every window in
 *         turn: the lanes of a warp test consecutive windows together.
 *         HC_MODE_AUTO picks DENSE when m = q, DIRECT when m - q + 1 >= 200,
 *         else STAGED.  Every mode returns the same positions.
 *   lane_bytes: window starts per thread and chunk (1..4096, a chunk holds
 *         256 of them; at most 256 in the dense mode);
 *   stages: text staging buffers per CTA (2..4);
 *   ctas_per_sm: upper bound on resident CTAs per SM;
 *   spill_entries: capacity, in positions, of the per-launch spill regions
 *         that hold occurrences until their output offsets are known
 *         (positions that do not fit are found again by a second scan of
 *         the affected chunks);
 *   speculate: 1 -- in the staged and direct modes, the lanes of a warp
 *         test the next 32 windows of HC's miss sequence together and
 *         finish the first one that hits, with the warp; -1 -- each lane
 *         runs HC over its own run of window starts; 0 -- automatic (the
 *         per-lane form, faster on every workload measured so far).
 * struct_size must be sizeof(hc_search_opts). */
enum { HC_MODE_AUTO = 0, HC_MODE_STAGED = 1, HC_MODE_DIRECT = 2, HC_MODE_DENSE = 3 };

typedef struct hc_search_opts {
    size_t struct_size;
    int lane_bytes;
    int stages;
    int ctas_per_sm;
    int mode;
    uint64_t spill_entries;
    int speculate;
    int pos32;              /* 1: positions written as uint32 (pos_dev holds cap
                               uint32 values, 4-byte aligned; needs
                               n - m + 1 <= 2^32); 0: uint64 */
    int single_pass;        /* dense mode: 1 -- one kernel writes the
                               positions in text order as it goes (tiles
                               claimed in order; a tile's output offset is
                               the sum of the counts of the tiles before it,
                               read from per-tile entries and a tree of group
                               totals), after a small kernel that zeroes
                               those counts; 0 or -1 -- the positions are
                               held in spill regions and a second kernel
                               (emit) writes them (the automatic choice: a
                               tile of the single pass waits for the slowest
                               earlier tile, which measured slower on GB300) */
    int tile_steps;         /* single pass: window steps of 512 per tile
                               (1..64, rounded up to whole chunks);
                               0 = automatic */
    int sentinel;           /* staged mode: 1 -- the GPU form of SHC's
                               sentinel (Sec. 3.4, third optimisation): the
                               staging buffers are padded so that a lane's
                               loop of first tests may read past its run of
                               window starts, and the window position is
                               tested once per round of four first tests and
                               once per test that passes, instead of for
                               every window; 0 -- HC's position test per
                               window */
    int bitmap;             /* dense mode: 1 -- the scan writes one bit per
                               window start (n / 8 bytes of workspace) and
                               each warp's count, and the emit kernel turns
                               the bits into positions: no work per
                               occurrence in the scan and no spill round
                               trip, for patterns with many occurrences;
                               0 -- spill regions (the automatic choice).
                               Excludes single_pass = 1. */
} hc_search_opts;

/* hc_search_ex: hc_search_async with explicit launch options (opts may be
 * NULL).  Same arguments, results and errors as hc_search_async, plus
 * HC_ERR_ARG for options out of range.  Used by the autotuner and tests. */
int hc_search_ex(const hc_filter *f, const uint8_t *y_dev, size_t n,
                 uint64_t *pos_dev, size_t cap, uint64_t *count_dev,
                 const hc_search_opts *opts, hc_stream_t stream);

/* hc_search: the synchronous form named after the paper's HC(x, m, y, n, q,
 * alpha).  x (host, the filter's m pattern bytes) must be the pattern the
 * filter was built from, else HC_ERR_ARG.  Runs hc_search_async, waits for
 * the stream and stores the total number of occurrences in *count (host).
 * Returns HC_ERR_CAPACITY (after writing the first cap positions) when the
 * total exceeds cap; call with cap = 0 to size the buffer.  Errors:
 * HC_ERR_ARG, HC_ERR_CAPACITY, HC_ERR_CUDA, HC_ERR_NOMEM, HC_ERR_TIMEOUT. */
int hc_search(const hc_filter *f, const uint8_t *x, const uint8_t *y_dev,
              size_t n, uint64_t *pos_dev, size_t cap, size_t *count,
              hc_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched search: many (pattern, text) queries in one set of launches.
 *
 * Each query is a search of hc_search_async (same results) with the pattern
 * already in device memory.  hc_batch_create checks and plans the table
 * once: it allocates the filters, the launch tables and the workspace on the
 * current device (cudaMalloc) and keeps the query table's pointers, which
 * must stay valid until hc_batch_destroy.  hc_batch_run then enqueues three
 * kernels on `stream` and allocates nothing, so it may be captured in a CUDA
 * graph and replayed: the preprocessing phase of every query on the device
 * (Sec. 3.1, Eq. 1-5; F equals hc_preprocess's word for word), one
 * persistent scan over a device-side work queue of (query, text range)
 * tiles, and the output of positions and counts.  Runs on the same batch
 * must not overlap on the GPU.  q and alpha are per query; lane_bytes and
 * mode (HC_MODE_AUTO, _STAGED or _DIRECT; m = q runs in the staged form) are
 * launch options, 0 = automatic.  A query with q = 0 takes q and alpha
 * (its launch options stay automatic: the tuner measures those on one query
 * alone, and in a batch of mixed queries the automatic ones ran faster)
 * from the autotuner given to hc_batch_create_tuned (from the
 * paper's Tables 1-3 without one) for its text's alphabet size: `sigma`, or
 * when sigma = 0 the effective alphabet size 1 / sum(p_c^2) of the byte
 * frequencies of a sample of the text, measured on the device at creation
 * (a nonzero lane_bytes or mode of the query still applies).
 */
typedef struct hc_batch_query {
    const uint8_t *x_dev;   /* pattern, m bytes, device memory */
    uint64_t m;
    const uint8_t *y_dev;   /* text, n bytes, device memory (any alignment) */
    uint64_t n;
    int q, alpha;           /* 1 <= q <= min(m, 8), 1 <= alpha <= 15 */
    uint64_t *pos_dev;      /* first min(count, cap) positions, ascending;
                               8-byte aligned, like count_dev */
    uint64_t cap;
    uint64_t *count_dev;    /* total occurrences (one uint64, device) */
    int lane_bytes;         /* window starts per lane and chunk, 0 = auto */
    int mode;               /* HC_MODE_AUTO, HC_MODE_STAGED or HC_MODE_DIRECT */
    int sigma;              /* alphabet size for q = 0 (0 = measure the text) */
    int reserved;           /* 0 */
} hc_batch_query;

typedef struct hc_batch hc_batch;

/* Search parameters of one (alphabet size, pattern length) cell: filter
 * parameters q and alpha, launch options lane_bytes and mode, and the text
 * rate measured for them (GB/s; 0 when not measured). */
typedef struct hc_tune_entry {
    int sigma;
    int q, alpha, lane_bytes, mode;
    int sentinel;           /* 1: the staged mode's sentinel form
                               (hc_search_opts.sentinel) */
    int bitmap;             /* 1: the dense mode's bitmap form
                               (hc_search_opts.bitmap) */
    uint64_t m;
    double gbps;
} hc_tune_entry;

typedef struct hc_tuner hc_tuner;

/* Errors: HC_ERR_ARG (null pointer or parameter out of range, with the query
 * index in hc_last_error), HC_ERR_NOMEM, HC_ERR_CUDA. */
int hc_batch_create(const hc_batch_query *queries, size_t nq, hc_batch **out);

/* hc_batch_create, with the parameters of q = 0 queries from `tuner` (NULL:
 * the paper's Tables 1-3).  Synchronous when some query has q = 0 and
 * sigma = 0 (the alphabet sizes are measured first).  Errors as
 * hc_batch_create. */
int hc_batch_create_tuned(const hc_batch_query *queries, size_t nq,
                          const hc_tuner *tuner, hc_batch **out);

/* The parameters query `query` runs with (q, alpha, resolved lane_bytes and
 * mode; sigma and gbps are 0).  Errors: HC_ERR_ARG. */
int hc_batch_params(const hc_batch *b, size_t query, hc_tune_entry *out);

/* Enqueues one run of every query.  Errors: HC_ERR_ARG, HC_ERR_STATE (other
 * device), HC_ERR_CUDA; a device wait that gave up is reported by
 * hc_check_status. */
int hc_batch_run(hc_batch *b, hc_stream_t stream);

/* Plan figures: work tiles, per-warp records, workspace bytes (any pointer
 * may be NULL).  Errors: HC_ERR_ARG. */
int hc_batch_info(const hc_batch *b, uint64_t *tiles, uint64_t *records,
                  uint64_t *workspace_bytes);

/* After a run has completed: copies query `query`'s filter (2^alpha words,
 * F must hold nwords >= 2^alpha) and H_v to host memory (either may be
 * NULL).  Synchronous.  Errors: HC_ERR_ARG, HC_ERR_CUDA. */
int hc_batch_filter(const hc_batch *b, size_t query, uint32_t *F, size_t nwords,
                    uint32_t *hv);

/* Frees a batch and its device memory.  NULL is a no-op. */
void hc_batch_destroy(hc_batch *b);

/* ------------------------------------------------------------------------
 * Autotuner: a table of search parameters per (alphabet size, pattern
 * length) cell, measured on this GPU.  The paper picks q and alpha per text
 * and pattern length from its measurements (Sec. 4, Tables 1-3); the tuner
 * measures the same choice, plus the window starts per lane and the scan
 * mode, on the batched kernels here.
 *
 * hc_tuner_create: an empty table; lookups then give the paper's choice
 *   (nearest of its three texts by alphabet size: <= 8 genome, <= 40
 *   protein, else English; nearest m on a log scale; q clamped to m).
 * hc_tuner_calibrate: for every sigma of `sigmas` a calibration text of
 *   text_bytes bytes drawn i.i.d. uniform over sigma symbols on the device
 *   (seeded), for every m of `ms` a pattern copied from it; each candidate
 *   (q in [1, min(8, m)], alpha in [8, 13]) is screened by one run on the
 *   first 8 MiB of the text; the 4 fastest, then for the best of them
 *   lane_bytes halved and doubled and each scan mode, are timed on the
 *   whole text, best of 3 runs after one untimed.  Path HC_TUNE_BATCHED
 *   runs a candidate as a one-query batch (the kernels of hc_batch_run),
 *   HC_TUNE_SINGLE as a single search (hc_search_ex, host-built filter; its
 *   dense mode for m = q).  The
 *   fastest fills the (sigma, m) cell, replacing an older one.  Synchronous
 *   on `stream`; allocates and frees device memory (text_bytes plus
 *   workspace).  A table from HC_TUNE_SINGLE may hold HC_MODE_DENSE cells
 *   (q = m); batches and servers run those in the automatic mode.
 * hc_tuner_lookup: the cell nearest to (sigma, m) on log scales, q clamped
 *   to m (the paper's choice when the table is empty).
 * hc_tuner_save / hc_tuner_load: the table as text, one cell per line
 *   ("sigma m q alpha lane_bytes mode gbps sentinel bitmap"; the last two
 *   columns are optional, 0 when absent); load adds to the table.
 * Errors: HC_ERR_ARG, HC_ERR_NOMEM, HC_ERR_CUDA; HC_ERR_STATE for an
 * unreadable or malformed file. */
enum { HC_TUNE_BATCHED = 0, HC_TUNE_SINGLE = 1 };
int hc_tuner_create(hc_tuner **out);
int hc_tuner_calibrate(hc_tuner *t, const int *sigmas, size_t nsigma,
                       const uint64_t *ms, size_t nm, uint64_t text_bytes,
                       uint64_t seed, int path, hc_stream_t stream);
int hc_tuner_lookup(const hc_tuner *t, double sigma, uint64_t m,
                    hc_tune_entry *out);
/* Number of cells, and cell i of the table (sorted by sigma, then m). */
int hc_tuner_size(const hc_tuner *t, size_t *count);
int hc_tuner_entry(const hc_tuner *t, size_t i, hc_tune_entry *out);
int hc_tuner_save(const hc_tuner *t, const char *path);
int hc_tuner_load(hc_tuner *t, const char *path);
void hc_tuner_free(hc_tuner *t);

/* Pinned host memory mapped into the current device's address space, for
 * outputs that the kernels write straight to the host (positions, counts:
 * pass *dev_ptr as pos_dev / count_dev; on a Grace-Blackwell node the
 * stores travel over NVLink-C2C, so no copy follows the search).  The host
 * reads the results at *host_ptr once the search has completed.  Errors:
 * HC_ERR_ARG, HC_ERR_CUDA.  hc_mapped_free releases it (NULL: no-op). */
int hc_mapped_alloc(size_t bytes, void **host_ptr, void **dev_ptr);
void hc_mapped_free(void *host_ptr);

/* Checked builds only (libhc_checked.so, compiled with HC_CHECKED, the
 * library's test variant): the number of device-side bounds violations
 * counted since the last call -- staged-buffer and text reads of the scan
 * kernels, spill-region and output accesses of the emit -- then reset.  A
 * violating access is skipped or clamped, not made.  Synchronous.  Errors:
 * HC_ERR_STATE in the regular build, HC_ERR_ARG, HC_ERR_CUDA. */
int hc_check_bounds(uint64_t *violations);

/* ------------------------------------------------------------------------
 * Served search: a request loop with continuous batching.
 *
 * A server keeps registered texts resident in device memory and runs
 * requests (a host pattern against one resident text) submitted from any
 * host thread.  Its worker thread takes queued requests in order into
 * batches (the batched search above: device preprocessing, persistent scan,
 * emit) and runs up to max_inflight batches at once, each on its own
 * stream: requests that arrive while earlier batches are on the GPU are
 * launched as soon as a stream and memory are free, and their work overlaps
 * with the earlier batches' on the device.  A request's result is the same
 * as that of hc_search on its pattern and text, alone or in any mix.
 *
 * Admission: resident texts plus the device bytes of every admitted request
 * (filter, pattern, launch tables, scan workspace) stay within mem_limit
 * (default 32 GiB).  A request that does not fit waits until completed
 * batches release memory; one that can never fit completes with
 * HC_ERR_ADMISSION.  Queue order is kept.  Results (counts, positions) are
 * written by the kernels into pinned host memory mapped into the device, so
 * no copy step follows a batch.  That memory is not counted in mem_limit:
 * each of the max_inflight slots holds 8 * (requests + sum of their caps)
 * bytes for its largest batch so far, kept until hc_server_destroy; a batch
 * whose results cannot be allocated completes with HC_ERR_NOMEM and the
 * server carries on.
 *
 * plain = 1 runs each request as one plain search launch (host-built filter,
 * the kernels of hc_search_async) instead: the comparison form.  Otherwise
 * the requests of a batch of at most 3, and in batches of at most 16 the
 * requests with m = q (served best by the dense single-search kernel), run
 * that way too, unless batch_only = 1.
 */
typedef struct hc_server hc_server;

typedef struct hc_server_config {
    size_t struct_size;     /* sizeof(hc_server_config) */
    uint64_t mem_limit;     /* device bytes: texts + admitted requests; 0 = 32 GiB */
    int max_inflight;       /* batches on the device at once, 1..16; 0 = 3 */
    int max_batch;          /* requests per batch, 1..2^20; 0 = 1024 */
    uint64_t default_cap;   /* positions kept per request when its cap is 0; 0 = 4096 */
    int plain;              /* 1: one plain search launch per request */
    int batch_only;         /* 1: every request runs the batched kernels (0:
                               batches of <= 3 requests, and m = q requests
                               in batches of <= 16, run the single-search
                               kernels) */
    uint64_t max_batch_bytes; /* text bytes per batch while the queue is
                               short (a single larger request still runs,
                               alone), so that a request arriving behind a
                               batch waits for little text; when more than
                               max_inflight times this much text is queued,
                               a batch may take queued text / max_inflight
                               instead, so that a backlog drains in few
                               large batches; 0 = 64 MiB */
} hc_server_config;

typedef struct hc_server_request {
    uint32_t text;          /* id from hc_server_add_text */
    int q, alpha;           /* q = 0: from the server's tuner for the text's sigma */
    int lane_bytes, mode;   /* launch options, 0 = tuned / automatic */
    const uint8_t *x;       /* pattern, host memory (copied at submission) */
    uint64_t m;             /* 1 .. 65536 */
    uint64_t cap;           /* positions kept; 0 = default_cap */
} hc_server_request;

typedef struct hc_server_result {
    uint64_t id;
    int status;             /* HC_OK; HC_ERR_CAPACITY: count > cap, the first cap
                               positions kept; HC_ERR_ADMISSION; HC_ERR_NOMEM (the
                               batch's pinned result memory could not be
                               allocated); HC_ERR_TIMEOUT (a device wait gave
                               up); HC_ERR_CUDA; HC_ERR_STATE (cancelled by
                               hc_server_destroy) */
    uint32_t text;
    int q, alpha;           /* the parameters it ran with */
    uint64_t count;         /* total occurrences */
    uint64_t npos;          /* positions in pos (ascending) */
    const uint64_t *pos;    /* host memory, valid until hc_server_release(id) */
    uint64_t submit_ns;     /* steady clock: submitted (replay: scheduled arrival) */
    uint64_t start_ns;      /* its batch launched */
    uint64_t done_ns;       /* its batch seen complete, results copied */
    uint64_t batch;         /* batch number, and requests in that batch */
    uint64_t batch_size;
} hc_server_result;

typedef struct hc_server_stats {
    uint64_t submitted, completed, batches, rejected, admission_waits;
    uint64_t max_batch, pending, inflight_bytes, peak_inflight_bytes;
    uint64_t text_bytes, mem_limit;
} hc_server_stats;

/* Creates a server on the current device with its worker thread.  cfg may
 * be NULL (defaults); tuner may be NULL (the paper's tables) and must
 * outlive the server.  Errors: HC_ERR_ARG, HC_ERR_NOMEM, HC_ERR_CUDA. */
int hc_server_create(const hc_server_config *cfg, const hc_tuner *tuner,
                     hc_server **out);

/* Registers a text: on_device = 0 copies n bytes from host memory into
 * device memory the server owns; 1 keeps the caller's device pointer (valid
 * until hc_server_destroy).  sigma = 0: the effective alphabet size is
 * measured on the device (see hc_batch_create_tuned).  Synchronous.
 * Errors: HC_ERR_ARG, HC_ERR_ADMISSION (texts beyond mem_limit),
 * HC_ERR_CUDA. */
int hc_server_add_text(hc_server *s, const uint8_t *y, uint64_t n,
                       int on_device, int sigma, uint32_t *text_id);
/* Length and (given or measured) alphabet size of a registered text. */
int hc_server_text_info(const hc_server *s, uint32_t text_id, uint64_t *n,
                        double *sigma);

/* Queues one request; *id identifies its result.  The pattern is copied.
 * Errors: HC_ERR_ARG (unknown text, parameters out of range), HC_ERR_STATE
 * (server stopped after a CUDA error), HC_ERR_NOMEM. */
int hc_server_submit(hc_server *s, const hc_server_request *r, uint64_t *id);

/* Load generation: validates all n requests, then submits request i at
 * arrival_ns[i] (non-decreasing) after the call started, from the calling
 * thread; its latency counts from that scheduled time.  Returns when all
 * are submitted.  Errors as hc_server_submit. */
int hc_server_replay(hc_server *s, const hc_server_request *r, size_t n,
                     const uint64_t *arrival_ns, uint64_t *ids);

/* Up to max completed results not yet polled, waiting up to wait_us
 * microseconds for the first (0: no wait, < 0: no limit). */
int hc_server_poll(hc_server *s, hc_server_result *out, size_t max,
                   size_t *got, int64_t wait_us);

/* Frees a polled result's positions.  Errors: HC_ERR_ARG (unknown id),
 * HC_ERR_STATE (not yet polled). */
int hc_server_release(hc_server *s, uint64_t id);

/* Waits until no request is queued or running (timeout_ms < 0: no limit).
 * Errors: HC_ERR_TIMEOUT; HC_ERR_CUDA when the server stopped on a CUDA
 * error. */
int hc_server_drain(hc_server *s, int64_t timeout_ms);

int hc_server_get_stats(const hc_server *s, hc_server_stats *out);

/* Stops the worker (queued requests are cancelled, running batches
 * finish), frees everything.  NULL is a no-op. */
void hc_server_destroy(hc_server *s);

/* ------------------------------------------------------------------------
 * hc_search_noalloc: the search of hc_search_async for callers that cannot
 * allocate device memory -- e.g. applications whose device memory is
 * planned in full by their own allocator or arena (a hidden cudaMalloc can
 * exceed the plan, and cudaFree synchronises the device), or latency-critical
 * paths that must not enter an allocator.  The paper has no counterpart: this
 * is an interface of this library only.
 *
 * It allocates nothing (no cudaMalloc, cudaFree or pool allocation): the
 * caller passes every buffer -- F_dev, the filter's 2^alpha words as returned
 * by hc_filter_words, and x_dev, its m pattern bytes, both copied by the
 * caller into device memory; the text y_dev; the output pos_dev (cap
 * positions, may be NULL when cap = 0) and count_dev (one uint64).  The
 * scratch that holds occurrences until their output offsets are known is a
 * fixed 8 MiB array inside the library, held by every GPU that loads the
 * library until the process exits.  Limit: min(cap, n-m+1) at most 2,000,000
 * positions; larger requests are rejected with HC_ERR_ARG (the count alone,
 * cap = 0, works for any n).  Results and the other errors are those of
 * hc_search_async; nothing is waited for.
 *
 * The first call on each device looks up the scratch's device address and
 * prepares the kernels; make that first call before capturing a stream.  All
 * calls on a device share the one scratch array and it keeps the last
 * call's contents: calls that overlap on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller.
 */
int hc_search_noalloc(const hc_filter *f, const uint32_t *F_dev,
                      const uint8_t *x_dev, const uint8_t *y_dev, size_t n,
                      uint64_t *pos_dev, size_t cap, uint64_t *count_dev,
                      hc_stream_t stream);

/* Waits for `stream` and reports (and clears) any device-side error flag
 * raised by the library's kernels on the current device: HC_ERR_TIMEOUT if a
 * bounded wait gave up, else HC_OK.  Errors: HC_ERR_CUDA. */
int hc_check_status(hc_stream_t stream);

/* Self-test of the failure path of the library's device-side waits:
 * enqueues on `stream` one kernel whose thread waits, with the same bounded
 * wait every bulk-copy wait of the search kernels uses, on an mbarrier that
 * nothing completes.  After about 2 s the wait gives up and sets the status
 * flag, as a copy that never landed would; the kernel then returns.  The
 * next hc_check_status on that stream returns HC_ERR_TIMEOUT (and clears the
 * flag); the context stays usable.  Errors: HC_ERR_CUDA. */
int hc_selftest_wait_timeout(hc_stream_t stream);

/* Number of launches of the library's own kernels issued so far by this
 * process (all devices, all entry points). */
uint64_t hc_kernel_launches(void);

/* Kernel timing, a profiling aid.  hc_timing_enable(1) makes every later
 * kernel launch of the library record a CUDA event pair around itself on its
 * stream (0 stops it).  hc_timing_report waits for the recorded launches and
 * writes, for kernel families 0..nkinds-1, the summed elapsed milliseconds
 * (ms[k]) and launch counts (launches[k]); either array may be NULL.  With
 * reset != 0 the recorded launches are then forgotten.  Families:
 * hc_timing_kind_name(k) for k = 0.. ("scan_staged", "scan_direct",
 * "scan_dense", "emit", "preprocess", "batch", "lb_init" -- the kernel that
 * zeroes a single-pass search's tile table; "" past the last).  Errors:
 * HC_ERR_CUDA. */
int hc_timing_enable(int on);
int hc_timing_report(double *ms, uint64_t *launches, int nkinds, int reset);
const char *hc_timing_kind_name(int kind);

#ifdef __cplusplus
}
#endif

#endif /* HC_GB300_H */
