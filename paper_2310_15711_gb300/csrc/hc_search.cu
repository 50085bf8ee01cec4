// hc_search.cu -- the HC searching phase (Sec. 3.3, Fig. 5 left, with the H_v
// early reject of Sec. 3.4) on sm_103a.
//
// Decomposition.  The window starts [0, n-m] are cut into chunks of C = 256*L
// consecutive starts; chunk k reads text bytes [kC, kC + C + m - 1).  A grid
// sized to fill the GPU (a whole number of CTAs per SM) gives each CTA a
// contiguous range of chunks.  Each CTA keeps F (2^alpha words) and x in
// shared memory and streams its chunks through 2-4 staging buffers: while it
// scans one chunk, the next ones are in flight from HBM into shared memory as
// 1-D bulk copies (TMA, cp.async.bulk, 16-byte aligned) completing on
// mbarriers.
//
// Inside a chunk, thread t runs the sequential HC loop over its own L window
// starts [tL, tL + L).  This is exact: HC started at any window reports every
// occurrence that starts at or after it (its shifts never pass over one), so
// it reports exactly the occurrences that start in [tL, tL+L) if it stops at
// the first window starting at or beyond tL + L.  L is 4 times an odd number,
// so the 32 lanes of a warp, whose windows advance in step while they miss,
// read 32 different shared-memory banks.
//
// Output in text order, without any wait between CTAs.  CTA b scans a
// contiguous range of chunks.  Per chunk, each thread counts its occurrences
// (keeping the first four in shared memory); when a chunk has any, a block
// scan orders them and they are appended, in text order, to CTA b's private
// spill region in global memory (as offsets from the start of its range).
// A second, light kernel gives CTA b its output offset (the sum of the
// totals of CTAs 0..b-1) and copies its region to the output.  A region that
// fills up is marked at the first chunk that did not fit; the second kernel
// re-scans the text from that chunk on and writes those positions itself.
//
// Every wait (bulk-copy completion) is bounded; a wait that gives up sets
// the status flag and the kernel returns.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <map>
#include <tuple>
#include <utility>

#include "hc_device.cuh"
#include "hc_internal.h"

namespace hc {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxStages = 4;
constexpr int kSlots = 4;
constexpr int kMaxSmemX = 4096;             // larger patterns verify from global memory
constexpr size_t kMaxStagedM = 16384;       // larger patterns use the unstaged kernel
constexpr unsigned long long kNoOverflow = ~0ull;
constexpr int kDirectShift = 200;
constexpr int kEmitSplit = 2;               // CTAs of the emit kernel per record group
constexpr int kMaxEmitGroup = 64;           // records per emit record group, at most           // shifts this long skip most 32-byte sectors

// bit 0: a bounded device-side wait gave up
__device__ unsigned int g_status;

struct SearchArgs {
  const uint8_t* y;          // text (device)
  unsigned long long n;      // text length
  unsigned long long nwin;   // number of window starts, n - m + 1
  const uint32_t* F;         // filter words (device), fwords of them
  const uint8_t* x;          // pattern (device)
  uint32_t fwords;
  int m, s;
  uint32_t mask, hv;
  unsigned long long* pos;   // output positions (device), cap of them
  unsigned long long cap;
  unsigned long long* count_out;
  // workspace (no zeroing needed: the scan kernel writes every entry it or
  // the emit kernel reads)
  unsigned long long* cta_total;     // [grid] occurrences in CTA b's range
  unsigned long long* cta_overflow;  // [grid] (first unstored chunk << 40) | stored, or kNoOverflow
  uint32_t* region;                  // [grid * region_entries] offsets from range start
  unsigned long long region_entries;
  unsigned long long num_chunks;
  unsigned long long chunks_per_cta;
  int L;                     // window starts per thread
  uint32_t C;                // window starts per chunk (kThreads * L)
  int head;                  // y mod 16: offset of y[kC] in its staged buffer
  uint32_t stage_bytes;      // bytes per staging buffer (16-byte multiple)
  uint32_t x_smem;           // bytes of shared memory for x (0: verify from global)
  int stages;                // staging buffers per CTA (2..kMaxStages)
  unsigned long long records;     // spill records (one per warp)
  int spec;                       // 1: warp-speculative HC per chunk (rare first-test hits)
  unsigned long long emit_group;  // records served by one emit CTA group
  // h as at most two byte-dot-products (see qgram_hash): bytes [0, g0) with
  // weights w0, bytes [g0, q) with weights w1, scaled by 2^(s*g0)
  uint32_t w0, w1;
  int g0;
};

// ---------------------------------------------------------------------------
// q-gram hash h (Eq. 3, Eq. 4): sum over the q bytes b_k (first byte k = 0)
// of b_k * 2^(s*k), mod 2^alpha.  The bytes are split into at most two
// groups, [0, g0) and [g0, q), chosen on the host so that every weight
// 2^(s*k) inside a group fits in one byte; each group is then one unsigned
// 4-byte dot product (dp4a), and h = dot0 + (dot1 << (s*g0)).  With
// alpha <= 15 and q <= 8 two groups always suffice (s*(q-1) <= 7 for q >= 4
// or a split after 2-4 bytes), and the value equals the Horner evaluation of
// Eq. 3 exactly, since no partial sum exceeds 32 bits.
// `lo` holds bytes 0-3 of the q-gram, `hi` bytes 4-7 (little-endian).
template <int Q>
__device__ __forceinline__ uint32_t hash_bytes(uint32_t lo, uint32_t hi, const SearchArgs& a) {
  uint32_t v = __dp4a(lo, a.w0, 0u);
  if constexpr (Q > 1) {
    if (Q > a.g0) {
      const uint32_t rest = __funnelshift_rc(lo, hi, 8u * static_cast<uint32_t>(a.g0));
      v += __dp4a(rest, a.w1, 0u) << (a.s * a.g0);
    }
  }
  return v & a.mask;
}

// The q bytes starting at byte offset o of `base`: staged -- `base` is a
// 16-byte aligned shared-memory buffer with at least 12 readable bytes past
// the q-gram, read as aligned 32-bit words and funnel-shifted; unstaged --
// byte loads from global memory (no read outside the q-gram).
template <int Q, bool STAGED>
__device__ __forceinline__ void load_qgram(const uint8_t* base, int o, uint32_t* lo, uint32_t* hi) {
  if constexpr (STAGED) {
    const uint32_t* W = reinterpret_cast<const uint32_t*>(base);
    const int wi = o >> 2;
    const uint32_t r = static_cast<uint32_t>(o & 3) * 8u;
    const uint32_t w0 = W[wi], w1 = W[wi + 1];
    *lo = __funnelshift_r(w0, w1, r);
    *hi = 0;
    if constexpr (Q > 4) *hi = __funnelshift_r(w1, W[wi + 2], r);
  } else {
    // the aligned 8-byte words that overlap the q-gram (one or two); an
    // aligned word holding a text byte never crosses a page
    const uintptr_t addr = reinterpret_cast<uintptr_t>(base + o);
    const unsigned long long* p8 = reinterpret_cast<const unsigned long long*>(addr & ~uintptr_t(7));
    const uint32_t off = static_cast<uint32_t>(addr & 7u);
    const unsigned long long d0 = __ldg(p8);
    const unsigned long long d1 = (off + Q > 8u) ? __ldg(p8 + 1) : 0ull;
    const uint32_t x0 = static_cast<uint32_t>(d0), x1 = static_cast<uint32_t>(d0 >> 32);
    const uint32_t x2 = static_cast<uint32_t>(d1), x3 = static_cast<uint32_t>(d1 >> 32);
    const uint32_t r = (off & 3u) * 8u;
    const bool up = off >= 4u;  // first byte in the second 32-bit word
    const uint32_t a0 = up ? x1 : x0, a1 = up ? x2 : x1, a2 = up ? x3 : x2;
    *lo = __funnelshift_r(a0, a1, r);
    *hi = Q > 4 ? __funnelshift_r(a1, a2, r) : 0u;
  }
}

template <int Q, bool STAGED>
__device__ __forceinline__ uint32_t qgram_hash(const uint8_t* base, int o, const SearchArgs& a) {
  uint32_t lo, hi;
  load_qgram<Q, STAGED>(base, o, &lo, &hi);
  return hash_bytes<Q>(lo, hi, a);
}

__device__ __forceinline__ bool verify_window(const uint8_t* w, const uint8_t* x, int m) {
  for (int k = 0; k < m; ++k)
    if (w[k] != x[k]) return false;
  return true;
}

enum SinkMode { kCount = 0, kToRegion = 1, kToPositions = 2 };

// Where a segment scan puts the occurrences it finds.
struct Sink {
  uint32_t* slot;            // kCount: first kSlots starts at slot[k * kThreads]
  uint32_t* region;          // kToRegion: region[obase + i] = vbase + start
  unsigned long long* pos;   // kToPositions: pos[obase + i] = vbase + start
  unsigned long long obase, vbase, limit;
};

// Records one occurrence (window start `start`, chunk-relative) as the
// cnt-th of this thread's segment.
template <int MODE>
__device__ __forceinline__ void record_match(const Sink& sink, int cnt, int start) {
  if constexpr (MODE == kCount) {
    if (cnt < kSlots) sink.slot[cnt * kThreads] = static_cast<uint32_t>(start);
  } else {
    const unsigned long long idx = sink.obase + static_cast<unsigned long long>(cnt);
    if (idx < sink.limit) {
      if constexpr (MODE == kToRegion)
        sink.region[idx] = static_cast<uint32_t>(sink.vbase + static_cast<unsigned>(start));
      else
        sink.pos[idx] = sink.vbase + static_cast<unsigned long long>(start);
    }
  }
}

template <bool STAGED>
__device__ __forceinline__ uint8_t text_byte(const uint8_t* base, int k) {
  if constexpr (STAGED) return base[k];
  else return __ldg(base + k);
}

// Finishes the HC test of the window ending at ew with the whole warp: the
// back-walk has reached q-gram end j, whose F word is z, with every link so
// far passing; vlast is the hash of that q-gram.  The lanes hash the next 32
// q-grams of the walk at once; lane t checks the link of q-gram t against
// the word of q-gram t-1 (passed along with a shuffle); a ballot finds the
// first unlinked q-gram, which is where the sequential walk would break.  A
// window read in full is checked against H_v and compared with x by the
// warp.  Returns the next window end; *match tells whether the window is an
// occurrence.  All 32 lanes must call it with the same arguments.
template <int Q, bool STAGED>
__device__ __forceinline__ int warp_finish_window(const uint8_t* base, int head, int ew, int j,
                                                  uint32_t z, uint32_t vlast, const SearchArgs& a,
                                                  const uint32_t* Fs, const uint8_t* xv,
                                                  bool* match) {
  const int lane = threadIdx.x & 31;
  const int m = a.m;
  const int shift = m - Q + 1;
  const int i = ew - m + 2 * Q;
  *match = false;
  while (j >= i) {
    const int T = (j - i) / Q + 1;      // walk steps left
    const bool valid = lane < T;
    const int p = j - (lane + 1) * Q;   // end of this lane's q-gram
    uint32_t v = 0, zt = 0;
    if (valid) {
      v = qgram_hash<Q, STAGED>(base, head + p - Q + 1, a);
      zt = Fs[v];
    }
    uint32_t zprev = __shfl_up_sync(0xffffffffu, zt, 1);
    if (lane == 0) zprev = z;
    const unsigned fails = __ballot_sync(0xffffffffu, valid && (zprev & (1u << (v & 31u))) == 0u);
    if (fails) return j - __ffs(fails) * Q + shift;  // shift past the unlinked q-gram
    const int last = min(T, 32) - 1;
    z = __shfl_sync(0xffffffffu, zt, last);
    vlast = __shfl_sync(0xffffffffu, v, last);
    j -= (last + 1) * Q;
  }
  // read in full: H_v test, then the warp compares the window with x
  if (vlast == a.hv) {
    const int start = ew - m + 1;
    const uint8_t* txt = base + head;
    bool eq = true;
    for (int k = lane; k < m; k += 32) eq &= text_byte<STAGED>(txt, start + k) == xv[k];
    *match = __all_sync(0xffffffffu, eq);
  }
  return ew + 1;
}

// HC over all window starts [0, wins) of a chunk by one warp, for patterns
// whose first test rarely hits: the lanes test the next 32 windows of the
// miss sequence e, e+S, ..., e+31S (S = m-q+1) at once; a ballot finds the
// first whose end q-gram hits a non-empty word of F -- every window before
// it is a miss that the sequential loop would visit and shift past -- and
// the warp finishes that window (warp_finish_window) and resumes after it.
// Occurrences are appended in order at sink.obase + count.  Returns the
// number found.  All 32 lanes must call it together.
template <int Q, bool STAGED, int MODE>
__device__ __forceinline__ int warp_scan_chunk(const uint8_t* base, int head, int wins,
                                               const SearchArgs& a, const uint32_t* Fs,
                                               const uint8_t* xv, const Sink& sink) {
  const int lane = threadIdx.x & 31;
  const int m = a.m;
  const int shift = m - Q + 1;
  const int e_end = wins + m - 1;
  int cnt = 0;
  int e = m - 1;
  while (e < e_end) {
    const int ek = e + lane * shift;
    const bool valid = ek < e_end;
    uint32_t v = 0, z = 0;
    if (valid) {
      v = qgram_hash<Q, STAGED>(base, head + ek - Q + 1, a);
      z = Fs[v];
    }
    const unsigned hits = __ballot_sync(0xffffffffu, z != 0u);
    if (hits == 0u) {
      e += 32 * shift;
      continue;
    }
    const int k = __ffs(hits) - 1;
    const int ew = e + k * shift;
    bool match;
    e = warp_finish_window<Q, STAGED>(base, head, ew, ew, __shfl_sync(0xffffffffu, z, k),
                                      __shfl_sync(0xffffffffu, v, k), a, Fs, xv, &match);
    if (match) {
      if (lane == 0) record_match<MODE>(sink, cnt, ew - m + 1);
      ++cnt;
    }
  }
  return cnt;
}

// Walk steps a lane takes on its own before handing the window to its warp.
constexpr int kShallowSteps = 3;

// HC (Fig. 5 left) over the window starts [lo, hi) of a chunk, one segment
// per thread; chunk-relative text byte k is base[head + k].  Returns the
// number of occurrences found and stores them according to MODE.
//
// Each lane runs the paper's loop on its own segment.  A window whose
// back-walk passes kShallowSteps links (rare, except for true occurrences of
// long patterns) is finished by the whole warp: the lanes hash the next 32
// q-grams of the walk at once, take the link test of each against its right
// neighbour's word (passed along with a shuffle), and a ballot finds the
// first unlinked q-gram -- the same break point the sequential walk reaches.
// A fully read window is then checked against H_v and verified by the warp.
// All 32 lanes of a warp must call this together (an empty range is fine).
template <int Q, bool STAGED, int MODE>
__device__ __forceinline__ int scan_segment(const uint8_t* base, int head, int lo, int hi,
                                            const SearchArgs& a, const uint32_t* Fs,
                                            const uint8_t* xv, const Sink& sink) {
  const int lane = threadIdx.x & 31;
  const int m = a.m;
  const uint32_t hv = a.hv;
  const int shift = m - Q + 1;
  const uint8_t* txt = base + head;
  int cnt = 0;
  int e = lo + m - 1;              // window end (chunk-relative)
  const int e_end = hi + m - 1;    // first window end past the segment
  bool deep = false;               // window at e waits for the warp
  int dj = 0;                      // walk position reached
  uint32_t dz = 0;                 // F word of the q-gram ending at dj
  while (true) {
    while (!deep && e < e_end) {
      // first test: the q-gram ending at the window end
      uint32_t v = qgram_hash<Q, STAGED>(base, head + e - Q + 1, a);
      uint32_t z = Fs[v];
      if (z == 0) {
        e += shift;
        continue;
      }
      // back-walk over the q-grams to the left, each linked to its right one
      int j = e;
      const int i = e - m + 2 * Q;
      bool broke = false;
      int steps = 0;
      while (j >= i) {
        if (steps == kShallowSteps) {
          deep = true;
          break;
        }
        j -= Q;
        v = qgram_hash<Q, STAGED>(base, head + j - Q + 1, a);
        if ((z & (1u << (v & 31u))) == 0) {
          broke = true;
          break;
        }
        z = Fs[v];
        ++steps;
      }
      if (deep) {
        dj = j;
        dz = z;
        break;
      }
      if (broke) {
        e = j + shift;             // shift past the unlinked q-gram
        continue;
      }
      // read in full (short window): H_v test, verification, advance by one
      const int start = e - m + 1;
      bool eq = v == hv;
      for (int k = 0; eq && k < m; ++k) eq = text_byte<STAGED>(txt, start + k) == xv[k];
      if (eq) record_match<MODE>(sink, cnt++, start);
      e += 1;
    }
    unsigned need = __ballot_sync(0xffffffffu, deep);
    if (need == 0u) break;
    for (; need; need &= need - 1u) {
      const int L0 = __ffs(need) - 1;
      const int ew = __shfl_sync(0xffffffffu, e, L0);
      const int j = __shfl_sync(0xffffffffu, dj, L0);
      const uint32_t z = __shfl_sync(0xffffffffu, dz, L0);
      bool match;
      const int e_next = warp_finish_window<Q, STAGED>(base, head, ew, j, z, 0u, a, Fs, xv, &match);
      if (lane == L0) {
        if (match) record_match<MODE>(sink, cnt++, ew - m + 1);
        e = e_next;
        deep = false;
      }
    }
  }
  return cnt;
}

// Block-wide exclusive scan of one count per thread; every thread gets its
// exclusive prefix and the block total.  Uses warp_sum (kWarps words).
__device__ __forceinline__ void block_scan(uint32_t cnt, uint32_t* warp_sum, uint32_t* excl,
                                           uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t incl = warp_incl_scan_u32(cnt);
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kWarps ? warp_sum[lane] : 0u;
    w = warp_incl_scan_u32(w);
    if (lane < kWarps) warp_sum[lane] = w;
  }
  __syncthreads();
  *excl = (warp ? warp_sum[warp - 1] : 0u) + incl - cnt;
  *total = warp_sum[kWarps - 1];
}

// ---------------------------------------------------------------------------
// Kernel 1: per-lane HC.  Every warp is an independent stream: record
// w = blockIdx.x * 8 + warp owns a contiguous range of chunks of 32*L window
// starts; lane l scans starts [lL, lL + L) of each chunk.  Staged: the warp
// brings its chunks into its own ring of shared-memory buffers with bulk
// copies on its own mbarriers; direct: the lanes read the text from global
// memory.  Occurrences go, in text order, to the warp's spill region; the
// total to cta_total[w].  No CTA-wide barrier in the loop.
template <int Q, bool STAGED>
__global__ void __launch_bounds__(kThreads) hc_scan_kernel(const SearchArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[kWarps][kMaxStages];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long w_id = static_cast<unsigned long long>(blockIdx.x) * kWarps + warp;
  uint32_t* Fs = reinterpret_cast<uint32_t*>(smem);
  const uint32_t f_bytes = (a.fwords * 4u + 15u) & ~15u;
  uint8_t* xs = smem + f_bytes;
  uint32_t* slots = reinterpret_cast<uint32_t*>(xs + a.x_smem);
  for (uint32_t i = tid; i < a.fwords; i += kThreads) Fs[i] = a.F[i];
  for (uint32_t i = tid; i < a.x_smem && i < static_cast<uint32_t>(a.m); i += kThreads)
    xs[i] = a.x[i];
  const uint8_t* xv = a.x_smem ? xs : a.x;
  __syncthreads();

  const unsigned long long c0 = w_id * a.chunks_per_cta;
  const unsigned long long c1 = min(c0 + a.chunks_per_cta, a.num_chunks);
  if (c0 >= c1) {
    if (lane == 0) {
      a.cta_total[w_id] = 0;
      a.cta_overflow[w_id] = kNoOverflow;
    }
    return;
  }
  const int nchunks = static_cast<int>(c1 - c0);
  const int nst = a.stages;
  uint8_t* stages = reinterpret_cast<uint8_t*>(slots + kSlots * kThreads) +
                    static_cast<size_t>(warp) * nst * a.stage_bytes;
  uint64_t* wb = bars[warp];
  auto issue = [&](int st, unsigned long long c) {
    const unsigned long long cs = c * a.C;
    const unsigned long long len = min(static_cast<unsigned long long>(a.C) + a.m - 1, a.n - cs);
    const uint32_t bytes = static_cast<uint32_t>((a.head + len + 15) & ~15ull);
    mbar_arrive_expect_tx(&wb[st], bytes);
    bulk_copy_g2s(stages + static_cast<size_t>(st) * a.stage_bytes, a.y + cs - a.head, bytes, &wb[st]);
  };
  if constexpr (STAGED) {
    if (lane == 0) {
      for (int k = 0; k < nst; ++k) mbar_init(&wb[k], 1);
      fence_mbar_init();
      for (int k = 0; k < nst && k < nchunks; ++k) issue(k, c0 + k);
    }
    __syncwarp();
  }

  const unsigned long long S = a.region_entries;
  uint32_t* region = a.region + w_id * S;
  unsigned long long T = 0;               // occurrences so far in this range
  unsigned long long overflow = kNoOverflow;
  Sink sink{};
  sink.slot = slots + tid;
  bool ok = true;
  int i = 0;
  for (; i < nchunks; ++i) {
    const int st = i % nst;
    const unsigned long long c = c0 + static_cast<unsigned long long>(i);
    if constexpr (STAGED) {
      if (lane == 0 && i > 0 && i + nst - 1 < nchunks) {
        // the buffer of chunk i-1 was released by the __syncwarp that ended it
        fence_proxy_async_smem();
        issue((i + nst - 1) % nst, c + nst - 1);
      }
      ok = __all_sync(0xffffffffu, mbar_wait_bounded(&wb[st], static_cast<uint32_t>(i / nst) & 1u));
      if (!ok) break;
    }
    const unsigned long long cs = c * a.C;
    const int wins = static_cast<int>(min(static_cast<unsigned long long>(a.C), a.nwin - cs));
    const uint8_t* base;
    int head;
    if constexpr (STAGED) {
      base = stages + static_cast<size_t>(st) * a.stage_bytes;
      head = a.head;
    } else {
      base = a.y + cs;
      head = 0;
    }
    if (a.spec) {
      // warp-speculative HC over the whole chunk; matches appended in order
      Sink w{};
      w.region = region;
      w.obase = T;
      w.vbase = static_cast<uint32_t>(static_cast<unsigned long long>(i) * a.C);
      w.limit = overflow == kNoOverflow ? S : 0ull;
      const unsigned long long found =
          static_cast<unsigned long long>(warp_scan_chunk<Q, STAGED, kToRegion>(base, head, wins, a, Fs, xv, w));
      if (overflow == kNoOverflow && T + found > S) overflow = (static_cast<unsigned long long>(i) << 40) | T;
      T += found;
      __syncwarp();
      continue;
    }
    const int lo = lane * a.L;
    const int hi = max(lo, min(lo + a.L, wins));
    const int cnt = scan_segment<Q, STAGED, kCount>(base, head, lo, hi, a, Fs, xv, sink);

    if (__any_sync(0xffffffffu, cnt != 0)) {
      const uint32_t incl = warp_incl_scan_u32(static_cast<uint32_t>(cnt));
      const uint32_t excl = incl - static_cast<uint32_t>(cnt);
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      if (overflow == kNoOverflow) {
        if (T + total <= S) {
          const uint32_t rel = static_cast<uint32_t>(static_cast<unsigned long long>(i) * a.C);
          const unsigned long long ob = T + excl;
          if (cnt <= kSlots)
            for (int k = 0; k < cnt; ++k) region[ob + k] = rel + sink.slot[k * kThreads];
          // lanes with more than kSlots occurrences scan their segment again,
          // writing them all (the whole warp takes part)
          Sink w{};
          w.region = region;
          w.obase = ob;
          w.vbase = rel;
          w.limit = S;
          scan_segment<Q, STAGED, kToRegion>(base, head, lo, cnt > kSlots ? hi : lo, a, Fs, xv, w);
        } else {
          overflow = (static_cast<unsigned long long>(i) << 40) | T;
        }
      }
      T += total;
    }
    __syncwarp();  // staging buffer st and the slots are free again
  }

  if (lane == 0) {
    a.cta_total[w_id] = T;
    a.cta_overflow[w_id] = overflow;
    if constexpr (STAGED) {
      if (!ok) {
        atomicOr(&g_status, 1u);
        // let the copies still in flight land before the CTA's shared memory goes
        for (int j = i; j < nchunks && j < i + nst; ++j)
          (void)mbar_wait_bounded(&wb[j % nst], static_cast<uint32_t>(j / nst) & 1u);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Kernel 1, dense form for m = q.  With m = q the window is a single q-gram,
// the back-walk is empty and every shift is one position, so HC tests every
// window in turn: a window w is reported iff F[h(w)] != 0, h(w) = H_v and
// w = x.  Where w = x, h(w) = h(x), so the first two tests have the same
// value for every window that passes the third: the kernel evaluates
// F[h(x)] != 0 and h(x) = H_v once per warp and the byte comparison per
// window -- 16 consecutive windows per lane, read with 16-byte shared-memory
// loads, compared with word-wide XOR/OR and an exact zero-byte test.
//
// Every warp is an independent stream: it owns a contiguous range of chunks
// (record w = blockIdx.x * 8 + warp), stages them through its own ring of
// shared-memory buffers with bulk copies on its own mbarriers, and appends
// its matches -- compacted in order with ballots -- straight to its own
// spill region.  There is no CTA-wide barrier in the loop.
template <int Q>
__global__ void __launch_bounds__(kThreads) hc_scan_dense_kernel(const SearchArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[kWarps][kMaxStages];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long w_id = static_cast<unsigned long long>(blockIdx.x) * kWarps + warp;
  uint32_t* Fs = reinterpret_cast<uint32_t*>(smem);
  for (uint32_t i = tid; i < a.fwords; i += kThreads) Fs[i] = a.F[i];
  __syncthreads();

  const unsigned long long c0 = w_id * a.chunks_per_cta;
  const unsigned long long c1 = min(c0 + a.chunks_per_cta, a.num_chunks);
  if (c0 >= c1) {
    if (lane == 0) {
      a.cta_total[w_id] = 0;
      a.cta_overflow[w_id] = kNoOverflow;
    }
    return;
  }
  const int nst = a.stages;
  const uint32_t f_bytes = (a.fwords * 4u + 15u) & ~15u;
  uint8_t* stages = smem + f_bytes + static_cast<size_t>(warp) * nst * a.stage_bytes;
  uint64_t* wb = bars[warp];
  const int nchunks = static_cast<int>(c1 - c0);

  // the chunk's bytes go to stage (i % nst); the warp's lane 0 drives the copies
  auto issue = [&](int st, unsigned long long c) {
    const unsigned long long cs = c * a.C;
    const unsigned long long len = min(static_cast<unsigned long long>(a.C) + a.m - 1, a.n - cs);
    const uint32_t bytes = static_cast<uint32_t>((a.head + len + 15) & ~15ull);
    mbar_arrive_expect_tx(&wb[st], bytes);
    bulk_copy_g2s(stages + static_cast<size_t>(st) * a.stage_bytes, a.y + cs - a.head, bytes, &wb[st]);
  };
  if (lane == 0) {
    for (int k = 0; k < nst; ++k) mbar_init(&wb[k], 1);
    fence_mbar_init();
    for (int k = 0; k < nst && k < nchunks; ++k) issue(k, c0 + k);
  }
  __syncwarp();

  // pattern byte c replicated into the 4 bytes of a word
  uint32_t xrep[Q];
  uint32_t xlo = 0, xhi = 0;
#pragma unroll
  for (int c = 0; c < Q; ++c) {
    const uint32_t xb = a.x[c];
    xrep[c] = 0x01010101u * xb;
    if (c < 4) xlo |= xb << (8 * c); else xhi |= xb << (8 * (c - 4));
  }
  // HC's first test and H_v test, evaluated on x itself (see above)
  const uint32_t hx = hash_bytes<Q>(xlo, xhi, a);
  const bool filter_passes = Fs[hx] != 0u && hx == a.hv;

  const unsigned long long S = a.region_entries;
  uint32_t* region = a.region + w_id * S;
  unsigned long long T = 0;                 // matches so far in this warp's range
  unsigned long long overflow = kNoOverflow;
  bool ok = true;
  int i = 0;
  for (; i < nchunks; ++i) {
    const int st = i % nst;
    const unsigned long long c = c0 + static_cast<unsigned long long>(i);
    if (lane == 0 && i > 0 && i + nst - 1 < nchunks) {
      // the buffer of chunk i-1 was released by the __syncwarp that ended it
      fence_proxy_async_smem();
      issue((i + nst - 1) % nst, c + nst - 1);
    }
    ok = __all_sync(0xffffffffu, mbar_wait_bounded(&wb[st], static_cast<uint32_t>(i / nst) & 1u));
    if (!ok) break;
    const unsigned long long cs = c * a.C;
    const int wins = static_cast<int>(min(static_cast<unsigned long long>(a.C), a.nwin - cs));
    const uint8_t* sb = stages + static_cast<size_t>(st) * a.stage_bytes;
    const uint32_t rel = static_cast<uint32_t>(static_cast<unsigned long long>(i) * a.C);
    const bool store = overflow == kNoOverflow;
    unsigned long long t = T;  // matches of the range before this step
    // window grid shifted by -head so that every lane's 16 windows start at a
    // 16-byte aligned shared-memory offset; windows outside [0, wins) are
    // masked
    for (int base = -a.head; base < wins; base += 512) {
      const int w0 = base + 16 * lane;      // first window of this lane
      uint32_t mbits = 0;
      if (w0 < wins) {  // lanes past the chunk's end read nothing
        const uint32_t o = static_cast<uint32_t>(a.head + w0);
        const uint4 A = *reinterpret_cast<const uint4*>(sb + o);
        const uint2 B = *reinterpret_cast<const uint2*>(sb + o + 16);
        const uint32_t Tw[6] = {A.x, A.y, A.z, A.w, B.x, B.y};  // bytes o .. o+23
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          // byte k of d stays 0 while window w0+4g+k agrees with x
          uint32_t d = Tw[g] ^ xrep[0];
#pragma unroll
          for (int cc = 1; cc < Q; ++cc) {
            const int wq = g + (cc >> 2);
            const uint32_t col = (cc & 3) ? __funnelshift_r(Tw[wq], Tw[wq + 1], 8u * (cc & 3)) : Tw[wq];
            d |= col ^ xrep[cc];
          }
          // exact zero-byte test: bit 7 of a byte set iff the byte is 0
          const uint32_t z = ~(((d & 0x7f7f7f7fu) + 0x7f7f7f7fu) | d | 0x7f7f7f7fu);
          // gather the four bit-7 flags into bits 4g .. 4g+3
          mbits |= (((z >> 7) & 0x01010101u) * 0x01020408u >> 24) << (4 * g);
        }
        // windows outside [0, wins)
        if (w0 < 0) mbits &= 0xffffu << min(-w0, 16);
        if (w0 + 16 > wins) mbits &= 0xffffu >> (16 - (wins - w0));
        if (!filter_passes) mbits = 0;
      }
      if (__ballot_sync(0xffffffffu, mbits != 0u) == 0u) continue;
      // in-order compaction (lanes in order, a lane's windows in order),
      // written straight to the spill region
      const uint32_t mine = static_cast<uint32_t>(__popc(mbits));
      const uint32_t incl = warp_incl_scan_u32(mine);
      if (store) {
        unsigned long long out = t + (incl - mine);
        while (mbits) {
          const int k = __ffs(mbits) - 1;
          if (out < S) region[out] = rel + static_cast<uint32_t>(w0 + k);
          ++out;
          mbits &= mbits - 1u;
        }
      }
      t += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (store && t > S) overflow = (static_cast<unsigned long long>(i) << 40) | T;
    T = t;
    __syncwarp();  // staging buffer st is free again
  }

  if (lane == 0) {
    a.cta_total[w_id] = T;
    a.cta_overflow[w_id] = overflow;
    if (!ok) {
      atomicOr(&g_status, 1u);
      // let the copies still in flight land before the CTA's shared memory goes
      for (int j = i; j < nchunks && j < i + nst; ++j)
        (void)mbar_wait_bounded(&wb[j % nst], static_cast<uint32_t>(j / nst) & 1u);
    }
  }
}

// ---------------------------------------------------------------------------
// Kernel 2: record r's output offset is the sum of cta_total[0..r); copy its
// region to the output; re-scan (from global memory) the chunks whose
// occurrences did not fit in the region.  A CTA serves a group of
// emit_group consecutive records (so the sums over earlier records are made
// once per group), and kEmitSplit CTAs share each group's copying; the first
// of them writes the count (last record) and does the re-scans.
template <int Q>
__global__ void __launch_bounds__(kThreads) hc_emit_kernel(const SearchArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ unsigned long long red[kWarps];
  __shared__ uint32_t warp_sum[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long g = blockIdx.x / kEmitSplit;
  const unsigned part = blockIdx.x % kEmitSplit;
  const unsigned long long r0 = g * a.emit_group;
  const unsigned long long r1 = min(r0 + a.emit_group, a.records);

  __shared__ unsigned long long s_tot[kMaxEmitGroup], s_ovf[kMaxEmitGroup];
  // sum of the earlier records' totals: loads issued 8 at a time
  unsigned long long p = 0;
  for (unsigned long long k0 = tid; k0 < r0; k0 += 8ull * kThreads) {
    unsigned long long v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const unsigned long long k = k0 + static_cast<unsigned long long>(u) * kThreads;
      v[u] = k < r0 ? a.cta_total[k] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) p += v[u];
  }
  p = warp_sum_u64(p);
  if (lane == 0) red[warp] = p;
  if (static_cast<unsigned long long>(tid) < r1 - r0) {
    s_tot[tid] = a.cta_total[r0 + tid];
    s_ovf[tid] = a.cta_overflow[r0 + tid];
  }
  __syncthreads();
  unsigned long long P = 0;  // output offset of record b (updated below)
  for (int w = 0; w < kWarps; ++w) P += red[w];

  bool f_loaded = false;
  for (unsigned long long b = r0; b < r1; ++b) {
    const unsigned long long T = s_tot[b - r0];
    const unsigned long long ovf = s_ovf[b - r0];
    if (part == 0 && b == a.records - 1 && tid == 0) *a.count_out = P + T;
    if (T == 0) continue;  // nothing to copy, nothing overflowed
    const unsigned long long stored = ovf == kNoOverflow ? T : (ovf & ((1ull << 40) - 1));
    const unsigned long long c0 = b * a.chunks_per_cta;
    const unsigned long long vbase = c0 * a.C;
    const uint32_t* region = a.region + b * a.region_entries;
    // copy: 16-byte region loads (regions are 16-byte aligned), four of them
    // in flight per thread; 16-byte stores when the output offset is even
    const unsigned long long ncopy = a.cap > P ? min(stored, a.cap - P) : 0ull;
    const uint4* r4 = reinterpret_cast<const uint4*>(region);
    const unsigned long long nvec = (ncopy + 3) / 4;
    const unsigned long long stride = static_cast<unsigned long long>(kThreads) * kEmitSplit;
    const bool even = (P & 1ull) == 0ull;
    for (unsigned long long k0 = part * kThreads + tid; k0 < nvec; k0 += 4 * stride) {
      uint4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned long long k = k0 + static_cast<unsigned long long>(u) * stride;
        if (k < nvec) v[u] = __ldcs(r4 + k);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned long long k = (k0 + static_cast<unsigned long long>(u) * stride) * 4;
        if (k < ncopy) {
          unsigned long long* o = a.pos + P + k;
          if (even && k + 4 <= ncopy) {
            __stcs(reinterpret_cast<ulonglong2*>(o), make_ulonglong2(vbase + v[u].x, vbase + v[u].y));
            __stcs(reinterpret_cast<ulonglong2*>(o + 2), make_ulonglong2(vbase + v[u].z, vbase + v[u].w));
          } else {
            __stcs(o, vbase + v[u].x);
            if (k + 1 < ncopy) __stcs(o + 1, vbase + v[u].y);
            if (k + 2 < ncopy) __stcs(o + 2, vbase + v[u].z);
            if (k + 3 < ncopy) __stcs(o + 3, vbase + v[u].w);
          }
        }
      }
    }
    if (part == 0) {
      if (ovf != kNoOverflow && P + stored < a.cap) {
        // re-scan the chunks from the first unstored one on
        uint32_t* Fs = reinterpret_cast<uint32_t*>(smem);
        uint32_t* slots = Fs + ((a.fwords + 3u) & ~3u);
        if (!f_loaded) {
          for (uint32_t k = tid; k < a.fwords; k += kThreads) Fs[k] = a.F[k];
          __syncthreads();
          f_loaded = true;
        }
        const unsigned long long c1 = min(c0 + a.chunks_per_cta, a.num_chunks);
        unsigned long long out = P + stored;
        Sink cs_sink{};
        cs_sink.slot = slots + tid;
        for (unsigned long long c = c0 + (ovf >> 40); c < c1 && out < a.cap; ++c) {
          const unsigned long long cs = c * a.C;
          const int wins = static_cast<int>(min(static_cast<unsigned long long>(a.C), a.nwin - cs));
          const int lo = tid * a.L;
          const int hi = max(lo, min(lo + a.L, wins));
          const uint8_t* base = a.y + cs;
          const int cnt = scan_segment<Q, false, kCount>(base, 0, lo, hi, a, Fs, a.x, cs_sink);
          uint32_t excl, total;
          block_scan(static_cast<uint32_t>(cnt), warp_sum, &excl, &total);
          Sink w{};
          w.pos = a.pos;
          w.obase = out + excl;
          w.vbase = cs;
          w.limit = a.cap;
          scan_segment<Q, false, kToPositions>(base, 0, lo, cnt > 0 ? hi : lo, a, Fs, a.x, w);
          out += total;
          __syncthreads();
        }
      }
    }
    P += T;
  }
}

// ---------------------------------------------------------------------------
// host side
namespace {

template <bool STAGED>
KernelFn scan_kernel_for_q(int q) {
  switch (q) {
    case 1: return hc_scan_kernel<1, STAGED>;
    case 2: return hc_scan_kernel<2, STAGED>;
    case 3: return hc_scan_kernel<3, STAGED>;
    case 4: return hc_scan_kernel<4, STAGED>;
    case 5: return hc_scan_kernel<5, STAGED>;
    case 6: return hc_scan_kernel<6, STAGED>;
    case 7: return hc_scan_kernel<7, STAGED>;
    default: return hc_scan_kernel<8, STAGED>;
  }
}

KernelFn dense_kernel_for_q(int q) {
  switch (q) {
    case 1: return hc_scan_dense_kernel<1>;
    case 2: return hc_scan_dense_kernel<2>;
    case 3: return hc_scan_dense_kernel<3>;
    case 4: return hc_scan_dense_kernel<4>;
    case 5: return hc_scan_dense_kernel<5>;
    case 6: return hc_scan_dense_kernel<6>;
    case 7: return hc_scan_dense_kernel<7>;
    default: return hc_scan_dense_kernel<8>;
  }
}

KernelFn emit_kernel_for_q(int q) {
  switch (q) {
    case 1: return hc_emit_kernel<1>;
    case 2: return hc_emit_kernel<2>;
    case 3: return hc_emit_kernel<3>;
    case 4: return hc_emit_kernel<4>;
    case 5: return hc_emit_kernel<5>;
    case 6: return hc_emit_kernel<6>;
    case 7: return hc_emit_kernel<7>;
    default: return hc_emit_kernel<8>;
  }
}

std::mutex g_attr_mu;
std::map<std::pair<int, const void*>, size_t> g_attr_set;  // dynamic smem opted in

// Raises the kernel's dynamic shared-memory limit to at least `smem` bytes.
int ensure_smem_attr(int dev, KernelFn fn, size_t smem) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  auto key = std::make_pair(dev, reinterpret_cast<const void*>(fn));
  auto it = g_attr_set.find(key);
  if (it != g_attr_set.end() && it->second >= smem) return HC_OK;
  cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(fn),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
  g_attr_set[key] = smem;
  return HC_OK;
}

// Static shared memory of a kernel (counts against the per-block limit).
size_t static_smem(KernelFn fn) {
  static std::mutex mu;
  static std::map<const void*, size_t> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(reinterpret_cast<const void*>(fn));
  if (it != cache.end()) return it->second;
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(fn)) != cudaSuccess) return 1024;
  cache[reinterpret_cast<const void*>(fn)] = fa.sharedSizeBytes;
  return fa.sharedSizeBytes;
}

// Resident CTAs per SM of a kernel at a given dynamic shared memory size.
int occupancy(int dev, KernelFn fn, size_t smem, int* per_sm) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, size_t>, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_tuple(dev, reinterpret_cast<const void*>(fn), smem);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *per_sm = it->second;
    return HC_OK;
  }
  int v = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fn, kThreads, smem);
  if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  cache[key] = v;
  *per_sm = v;
  return HC_OK;
}

}  // namespace

// Chooses the launch shape for one search (see SearchPlan in hc_internal.h).
// Kinds: dense (m = q: every window in turn, warp-cooperative), staged
// (per-lane HC over text staged in shared memory) and direct (per-lane HC
// reading the text from global memory: long patterns, whose large shifts
// skip most of the text, and patterns too long to stage).
int plan_search(const Filter* f, size_t n, size_t cap, const hc_search_opts* o, int dev,
                SearchPlan* out) {
  SearchPlan p{};
  const DeviceInfo& di = device_info(dev);
  const int m = static_cast<int>(std::min<size_t>(f->m, size_t(1) << 30));
  const int shift = m - f->q + 1;
  const int mode = o ? o->mode : HC_MODE_AUTO;
  if (mode < HC_MODE_AUTO || mode > HC_MODE_DENSE)
    return set_error(HC_ERR_ARG, "hc_search: unknown mode");
  if (mode == HC_MODE_DENSE && f->m != static_cast<size_t>(f->q))
    return set_error(HC_ERR_ARG, "hc_search: the dense mode needs m = q");
  int kind = mode;
  const int L_req = o ? o->lane_bytes : 0;
  if (kind == HC_MODE_AUTO) {
    if (f->m == static_cast<size_t>(f->q) && L_req <= 256) kind = HC_MODE_DENSE;
    else if (shift >= kDirectShift || f->m > kMaxStagedM) kind = HC_MODE_DIRECT;
    else kind = HC_MODE_STAGED;
  }
  int L = L_req;
  if (L == 0) {
    if (kind == HC_MODE_DENSE) {
      L = 8;
    } else if (kind == HC_MODE_DIRECT) {
      L = std::min(4096, std::max(64, shift));
    } else {
      // 4 * (odd number of words) >= max(64, 4 * shift), at most 188 bytes:
      // lanes that advance in step read 32 different banks
      const int lw = std::max(16, shift) | 1;
      L = 4 * std::min(lw, 47);
    }
  }
  if (L < 1 || L > 4096) return set_error(HC_ERR_ARG, "hc_search: lane_bytes out of [1, 4096]");
  if (kind == HC_MODE_DENSE && L > 256)
    return set_error(HC_ERR_ARG, "hc_search: the dense mode needs lane_bytes <= 256");
  const int stages = o && o->stages ? o->stages : (kind == HC_MODE_STAGED ? 2 : 3);
  if (stages < 2 || stages > kMaxStages) return set_error(HC_ERR_ARG, "hc_search: stages out of [2, 4]");
  p.kind = kind;
  p.L = L;
  // a chunk holds 256*L window starts in the dense kernel (a warp covers it in
  // L/2 steps of 16 windows per lane) and 32*L otherwise (one segment of L
  // starts per lane of the warp that owns it)
  p.C = static_cast<uint32_t>(kind == HC_MODE_DENSE ? kThreads : 32) * static_cast<uint32_t>(L);
  p.stages = stages;
  p.x_smem = f->m <= static_cast<size_t>(kMaxSmemX) ? static_cast<uint32_t>((f->m + 15) & ~size_t(15)) : 0u;
  const size_t fbytes = (f->F.size() * 4 + 15) & ~size_t(15);
  const size_t slot_bytes = size_t(kSlots) * kThreads * 4;
  // staged text: head (< 16) + C + m - 1 bytes, rounded to 16, plus slack for
  // the word loads that run past the last q-gram (at most 20 bytes past the
  // chunk's last window start in the dense kernel, 12 in the others)
  p.stage_bytes = static_cast<uint32_t>(((16 + p.C + f->m - 1 + 15) & ~size_t(15)) + 64);
  if (kind == HC_MODE_DENSE) {
    // one ring of `stages` buffers per warp
    p.scan = dense_kernel_for_q(f->q);
    p.smem_scan = fbytes + size_t(kWarps) * stages * p.stage_bytes;
    if (mode == HC_MODE_AUTO && p.smem_scan + static_smem(p.scan) > di.smem_optin) {
      kind = HC_MODE_STAGED;  // caller's lane_bytes too large for per-warp rings
      p.C = 32u * static_cast<uint32_t>(L);
      p.stage_bytes = static_cast<uint32_t>(((16 + p.C + f->m - 1 + 15) & ~size_t(15)) + 64);
    }
  }
  p.kind = kind;
  if (kind == HC_MODE_STAGED) {
    p.scan = scan_kernel_for_q<true>(f->q);
    p.smem_scan = fbytes + p.x_smem + slot_bytes + size_t(kWarps) * stages * p.stage_bytes;
    if (p.smem_scan + static_smem(p.scan) > di.smem_optin) {
      if (mode == HC_MODE_STAGED)
        return set_error(HC_ERR_ARG, "hc_search: staging buffers exceed shared memory");
      p.kind = kind = HC_MODE_DIRECT;
    }
  }
  if (kind == HC_MODE_DIRECT) {
    p.scan = scan_kernel_for_q<false>(f->q);
    p.smem_scan = fbytes + p.x_smem + slot_bytes;
  }
  if (p.smem_scan + static_smem(p.scan) > di.smem_optin)
    return set_error(HC_ERR_ARG, "hc_search: filter and buffers exceed shared memory");
  p.emit = emit_kernel_for_q(f->q);
  p.smem_emit = (((f->F.size() + 3) & ~size_t(3)) * 4) + slot_bytes;
  // warp-speculative HC only on request: measured on GB300 it loses to the
  // per-lane form on every sweep cell (each first-test hit serialises the
  // warp), so the automatic choice is the per-lane form
  if (kind != HC_MODE_DENSE) p.spec = o != nullptr && o->speculate > 0;

  int rc = ensure_smem_attr(dev, p.scan, p.smem_scan);
  if (rc != HC_OK) return rc;
  rc = ensure_smem_attr(dev, p.emit, p.smem_emit);
  if (rc != HC_OK) return rc;
  int per_sm = 0;
  rc = occupancy(dev, p.scan, p.smem_scan, &per_sm);
  if (rc != HC_OK) return rc;
  per_sm = std::max(per_sm, 1);
  if (o && o->ctas_per_sm > 0) per_sm = std::min(per_sm, o->ctas_per_sm);

  const unsigned long long nwin = n - f->m + 1;
  p.num_chunks = (nwin + p.C - 1) / p.C;
  // one record (total, overflow mark, spill region) per warp, each owning a
  // contiguous range of chunks
  const unsigned long long per_record = kWarps;
  unsigned long long records = std::min<unsigned long long>(
      p.num_chunks, static_cast<unsigned long long>(per_sm) * di.sm_count * per_record);
  p.chunks_per_cta = (p.num_chunks + records - 1) / records;
  if (p.chunks_per_cta * p.C >= (1ull << 32))
    return set_error(HC_ERR_ARG, "hc_search: text too long for one launch");
  p.records = (p.num_chunks + p.chunks_per_cta - 1) / p.chunks_per_cta;
  p.grid = (p.records + per_record - 1) / per_record;
  p.records = p.grid * per_record;
  unsigned long long spill = o ? o->spill_entries : 0;
  if (spill == 0)
    spill = cap == 0 ? 0 : std::min<unsigned long long>(nwin, std::max<unsigned long long>(cap, 1ull << 20));
  p.region_entries = (std::max<unsigned long long>(1, (spill + p.records - 1) / p.records) + 3) & ~3ull;
  // emit: about 2 record groups per SM, kEmitSplit CTAs each
  const unsigned long long groups = std::max<unsigned long long>(
      (p.records + kMaxEmitGroup - 1) / kMaxEmitGroup,
      std::min<unsigned long long>(p.records, 2ull * di.sm_count));
  p.emit_group = (p.records + groups - 1) / groups;
  p.emit_ctas = ((p.records + p.emit_group - 1) / p.emit_group) * kEmitSplit;
  p.ws_bytes = p.records * 16 + p.records * p.region_entries * 4;
  *out = p;
  return HC_OK;
}

void fill_args(const Filter* f, const SearchPlan& p, const uint8_t* y, size_t n, uint64_t* pos,
               size_t cap, uint64_t* count_dev, void* ws, void* args_out) {
  SearchArgs& a = *static_cast<SearchArgs*>(args_out);
  a = SearchArgs{};
  a.y = y;
  a.n = n;
  a.nwin = n - f->m + 1;
  a.F = f->dev_F();
  a.x = f->dev_x();
  a.fwords = static_cast<uint32_t>(f->F.size());
  a.m = static_cast<int>(f->m);
  a.s = f->s;
  a.mask = f->mask;
  a.hv = f->hv;
  a.pos = reinterpret_cast<unsigned long long*>(pos);
  a.cap = pos ? cap : 0;
  a.count_out = reinterpret_cast<unsigned long long*>(count_dev);
  a.cta_total = static_cast<unsigned long long*>(ws);
  a.cta_overflow = a.cta_total + p.records;
  a.region = reinterpret_cast<uint32_t*>(a.cta_overflow + p.records);
  a.region_entries = p.region_entries;
  a.num_chunks = p.num_chunks;
  a.chunks_per_cta = p.chunks_per_cta;
  a.L = p.L;
  a.C = p.C;
  a.head = static_cast<int>(reinterpret_cast<uintptr_t>(y) & 15u);
  a.stage_bytes = p.stage_bytes;
  a.x_smem = p.x_smem;
  a.stages = p.stages;
  a.records = p.records;
  a.spec = p.spec ? 1 : 0;
  a.emit_group = p.emit_group;
  // byte groups of h: the longest prefix whose weights 2^(s*k) fit in a byte
  const int s = f->s, q = f->q;
  int g = 1;
  while (g < 4 && g < q && s * g <= 7) ++g;
  a.g0 = g;
  a.w0 = 0;
  for (int k = 0; k < g; ++k) a.w0 |= (1u << (s * k)) << (8 * k);
  a.w1 = 0;
  for (int k = 0; k < q - g && k < 4; ++k) a.w1 |= (1u << (s * k)) << (8 * k);
}

// Enqueues the two kernels of one search with a caller-supplied workspace.
int launch_planned(const Filter* f, const SearchPlan& p, const uint8_t* y, size_t n, uint64_t* pos,
                   size_t cap, uint64_t* count_dev, void* ws, cudaStream_t stream) {
  SearchArgs a;
  fill_args(f, p, y, n, pos, cap, count_dev, ws, &a);
  const int kind = p.kind == HC_MODE_DENSE ? kKindScanDense
                   : (p.kind == HC_MODE_DIRECT ? kKindScanDirect : kKindScanStaged);
  TimingToken t0 = timing_begin(kind, stream);
  p.scan<<<static_cast<unsigned>(p.grid), kThreads, p.smem_scan, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  timing_end(t0, stream);
  if (e != cudaSuccess) return cuda_error(e, "hc_scan_kernel launch");
  TimingToken t1 = timing_begin(kKindEmit, stream);
  p.emit<<<static_cast<unsigned>(p.emit_ctas), kThreads, p.smem_emit, stream>>>(a);
  e = cudaGetLastError();
  timing_end(t1, stream);
  g_launches.fetch_add(2);
  if (e != cudaSuccess) return cuda_error(e, "hc_emit_kernel launch");
  return HC_OK;
}

// Enqueues the two kernels of one search reading the filter words and the
// pattern from caller-supplied device copies instead of the filter's own.
int launch_planned_filter_ptrs(const Filter* f, const SearchPlan& p, const uint32_t* F_dev,
                               const uint8_t* x_dev, const uint8_t* y, size_t n, uint64_t* pos,
                               size_t cap, uint64_t* count_dev, void* ws, cudaStream_t stream) {
  SearchArgs a;
  fill_args(f, p, y, n, pos, cap, count_dev, ws, &a);
  a.F = F_dev;
  a.x = x_dev;
  const int kind = p.kind == HC_MODE_DENSE ? kKindScanDense
                   : (p.kind == HC_MODE_DIRECT ? kKindScanDirect : kKindScanStaged);
  TimingToken t0 = timing_begin(kind, stream);
  p.scan<<<static_cast<unsigned>(p.grid), kThreads, p.smem_scan, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  timing_end(t0, stream);
  if (e != cudaSuccess) return cuda_error(e, "hc_scan_kernel launch");
  TimingToken t1 = timing_begin(kKindEmit, stream);
  p.emit<<<static_cast<unsigned>(p.emit_ctas), kThreads, p.smem_emit, stream>>>(a);
  e = cudaGetLastError();
  timing_end(t1, stream);
  g_launches.fetch_add(2);
  if (e != cudaSuccess) return cuda_error(e, "hc_emit_kernel launch");
  return HC_OK;
}

// Enqueues one search; the workspace comes from the library's stream-ordered
// pool and goes back to it after the kernels.
int launch_search(Filter* f, const uint8_t* y, size_t n, uint64_t* pos, size_t cap,
                  uint64_t* count_dev, const hc_search_opts* o, cudaStream_t stream) {
  int rc = filter_to_device(f);
  if (rc != HC_OK) return rc;
  cudaError_t e;
  if (n < f->m) {
    e = cudaMemsetAsync(count_dev, 0, sizeof(uint64_t), stream);
    return e == cudaSuccess ? HC_OK : cuda_error(e, "cudaMemsetAsync(count)");
  }
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  SearchPlan p;
  rc = plan_search(f, n, pos ? cap : 0, o, dev, &p);
  if (rc != HC_OK) return rc;
  void* ws = nullptr;
  e = cudaMallocFromPoolAsync(&ws, p.ws_bytes, device_pool(dev), stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocFromPoolAsync(workspace)");
  rc = launch_planned(f, p, y, n, pos, cap, count_dev, ws, stream);
  cudaFreeAsync(ws, stream);
  return rc;
}

int read_and_clear_status(cudaStream_t stream) {
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  unsigned int st = 0;
  e = cudaMemcpyFromSymbol(&st, g_status, sizeof st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyFromSymbol(status)");
  if (st != 0) {
    const unsigned int zero = 0;
    cudaMemcpyToSymbol(g_status, &zero, sizeof zero);
    return set_error(HC_ERR_TIMEOUT, "a bounded device-side wait gave up (status flag set)");
  }
  return HC_OK;
}

}  // namespace hc

using namespace hc;

namespace {
int check_search_args(const char* who, Filter* f, const uint8_t* y_dev, size_t n,
                      const uint64_t* pos_dev, size_t cap) {
  if (f == nullptr) return set_error(HC_ERR_ARG, std::string(who) + ": invalid filter");
  if (y_dev == nullptr && n > 0) return set_error(HC_ERR_ARG, std::string(who) + ": y_dev is NULL");
  if (pos_dev == nullptr && cap > 0)
    return set_error(HC_ERR_ARG, std::string(who) + ": pos_dev is NULL with cap > 0");
  return HC_OK;
}
}  // namespace

extern "C" {

int hc_search_ex(const hc_filter* fp, const uint8_t* y_dev, size_t n, uint64_t* pos_dev,
                 size_t cap, uint64_t* count_dev, const hc_search_opts* opts,
                 hc_stream_t stream) {
  clear_error();
  Filter* f = as_filter(fp);
  int rc = check_search_args("hc_search_ex", f, y_dev, n, pos_dev, cap);
  if (rc != HC_OK) return rc;
  if (count_dev == nullptr) return set_error(HC_ERR_ARG, "hc_search_ex: count_dev is NULL");
  if (opts != nullptr && opts->struct_size != sizeof(hc_search_opts))
    return set_error(HC_ERR_ARG, "hc_search_ex: opts->struct_size mismatch");
  return launch_search(f, y_dev, n, pos_dev, cap, count_dev, opts,
                       reinterpret_cast<cudaStream_t>(stream));
}

int hc_search_async(const hc_filter* fp, const uint8_t* y_dev, size_t n, uint64_t* pos_dev,
                    size_t cap, uint64_t* count_dev, hc_stream_t stream) {
  clear_error();
  Filter* f = as_filter(fp);
  int rc = check_search_args("hc_search_async", f, y_dev, n, pos_dev, cap);
  if (rc != HC_OK) return rc;
  if (count_dev == nullptr) return set_error(HC_ERR_ARG, "hc_search_async: count_dev is NULL");
  return launch_search(f, y_dev, n, pos_dev, cap, count_dev, nullptr,
                       reinterpret_cast<cudaStream_t>(stream));
}

int hc_search(const hc_filter* fp, const uint8_t* x, const uint8_t* y_dev, size_t n,
              uint64_t* pos_dev, size_t cap, size_t* count, hc_stream_t stream_) {
  clear_error();
  Filter* f = as_filter(fp);
  int rc = check_search_args("hc_search", f, y_dev, n, pos_dev, cap);
  if (rc != HC_OK) return rc;
  if (x == nullptr || count == nullptr) return set_error(HC_ERR_ARG, "hc_search: x or count is NULL");
  if (std::memcmp(x, f->x.data(), f->m) != 0)
    return set_error(HC_ERR_ARG, "hc_search: x is not the pattern the filter was built from");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  void* cnt_dev = nullptr;
  e = cudaMallocFromPoolAsync(&cnt_dev, sizeof(uint64_t), device_pool(dev), stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocFromPoolAsync(count)");
  rc = launch_search(f, y_dev, n, pos_dev, cap, static_cast<uint64_t*>(cnt_dev), nullptr, stream);
  unsigned long long host_count = 0;
  if (rc == HC_OK) {
    e = cudaMemcpyAsync(&host_count, cnt_dev, sizeof host_count, cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) rc = cuda_error(e, "cudaMemcpyAsync(count)");
  }
  cudaFreeAsync(cnt_dev, stream);
  const int st = read_and_clear_status(stream);
  if (rc != HC_OK) return rc;
  if (st != HC_OK) return st;
  *count = static_cast<size_t>(host_count);
  if (host_count > cap) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "hc_search: %llu occurrences, output holds %zu", host_count, cap);
    return set_error(HC_ERR_CAPACITY, buf);
  }
  return HC_OK;
}

int hc_check_status(hc_stream_t stream) {
  clear_error();
  return read_and_clear_status(reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
