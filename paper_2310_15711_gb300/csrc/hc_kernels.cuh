// hc_kernels.cuh -- device-side building blocks of the HC search shared by
// the single-search kernels (hc_search.cu) and the batched kernels
// (hc_batch.cu): launch arguments, the q-gram hash, the per-lane and
// warp-cooperative forms of the HC loop, the per-warp streaming loop and the
// emit logic.
#pragma once

#include <cstdint>

#include "hc_device.cuh"
#include "hc_internal.h"

namespace hc {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxStages = 4;
constexpr int kSlots = 2;
constexpr int kMaxSmemX = 4096;             // larger patterns verify from global memory
constexpr size_t kMaxStagedM = 16384;       // larger patterns use the unstaged kernel
constexpr unsigned long long kNoOverflow = ~0ull;
constexpr int kDirectShift = 200;           // shifts this long skip most 32-byte sectors
constexpr int kEmitSplit = 2;               // CTAs of the emit kernel per record group
constexpr int kMaxEmitGroup = 64;           // records per emit record group, at most
constexpr int kEmitUnits = 8;               // 8-byte region loads in flight per emit thread
constexpr int kSinglePassMaxSteps = 64;     // 512-window steps per single-pass tile (a u64 of flags)
constexpr int kSinglePassTileSteps = 16;    // default steps per single-pass tile
constexpr unsigned long long kSinglePassGroup = 64;  // tiles per group of the single-pass counts
constexpr int kQueueCap = 256;              // dense scan: candidate lanes queued per warp (u16 each)
constexpr int kDirectLanes = 16;            // dense scan: candidate lanes from which a step is finished at once
constexpr int kTwoStageLanes = 6;           // dense scan, q >= 5: mean candidate lanes per step above which one stage


// Bytes of one staging buffer: head (< 16) + C + m - 1 bytes of text rounded
// up to 16, plus 16 bytes of slack for the per-lane kernels (their word loads
// end at most 11 bytes past the last q-gram's first byte) or 32 for the dense
// kernel (its 16-byte loads end at most 20 bytes past the last window start).
inline uint32_t stage_bytes_for(uint32_t C, uint64_t m, bool dense) {
  return static_cast<uint32_t>(((16 + C + m - 1 + 15) & ~uint64_t(15)) + (dense ? 32 : 16));
}

struct SearchArgs {
  unsigned int* status;      // device status word: bit 0 set when a bounded wait gave up
  const uint8_t* y;          // text (device)
  unsigned long long n;      // text length
  unsigned long long nwin;   // number of window starts, n - m + 1
  const uint32_t* F;         // filter words (device), fwords of them
  const uint8_t* x;          // pattern (device)
  uint32_t fwords;
  int m, q, s;
  uint32_t mask, hv;
  unsigned long long* pos;   // output positions (device), cap of them
  unsigned long long cap;
  int pos32;                 // 1: positions are uint32 values at pos (cap of them)
  unsigned long long* count_out;
  // workspace (no zeroing needed: the scan kernel writes every entry it or
  // the emit kernel reads)
  unsigned long long* cta_total;     // [records] occurrences in record (warp) w's range
  unsigned long long* blk_total;     // [grid] sum over CTA b's kWarps records (NULL: not kept)
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
  int unchecked;                  // 1: staged, padded buffers: no position test per first test
  unsigned long long emit_group;  // records served by one emit CTA group
  // h as at most two byte-dot-products (see qgram_hash): bytes [0, g0) with
  // weights w0, bytes [g0, q) with weights w1, scaled by 2^(s*g0)
  uint32_t w0, w1;
  int g0;
  // single-pass dense form (m = q): tiles of tile_chunks consecutive chunks
  // are claimed from the kWarps counters at lb_ticket; lb_desc[t] holds tile
  // t's match count, lb_gpack[g] the total of group g (64 tiles) and
  // lb_gtree[1..G] a Fenwick tree of the group totals (see hc_dense.cu);
  // flag_steps is the number of 512-window steps per tile
  unsigned int* lb_ticket;
  unsigned int* lb_desc;
  unsigned long long* lb_gpack;
  unsigned long long* lb_gtree;
  unsigned long long num_tiles, num_groups;
  int tile_chunks;
  int flag_steps;
  // bitmap form of the dense scan (m = q): bit j of bitmap[g] is set iff
  // window 16g + j is an occurrence (chunk c's groups start at c * C / 16);
  // the emit kernel turns the bits into positions.  NULL: spill regions.
  uint16_t* bitmap;
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
// When q <= g0 the second group is empty and w1 = 0, so the second dot
// product adds nothing: the evaluation has no branch.
template <int Q>
__device__ __forceinline__ uint32_t hash_bytes(uint32_t lo, uint32_t hi, const SearchArgs& a) {
  uint32_t v = __dp4a(lo, a.w0, 0u);
  if constexpr (Q > 1) {
    const uint32_t rest = __funnelshift_rc(lo, hi, 8u * static_cast<uint32_t>(a.g0));
    v += __dp4a(rest, a.w1, 0u) << (a.s * a.g0);
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
  // staged: the three words read from o's word lie in the staging buffer;
  // unstaged: the q-gram lies in the text
  if constexpr (STAGED) {
    if (!HC_IN_BOUNDS(o >= 0 && o + 12 <= static_cast<int>(a.stage_bytes))) o = 0;
  } else {
    if (!HC_IN_BOUNDS(base + o >= a.y && base + o + Q <= a.y + a.n)) o = 0;
  }
  uint32_t lo, hi;
  load_qgram<Q, STAGED>(base, o, &lo, &hi);
  return hash_bytes<Q>(lo, hi, a);
}

// The hash constants of a search, held in registers by the per-lane scan
// (read from the kernel's parameters once instead of inside its loops).
struct HashK {
  uint32_t w0, w1, mask, g8, sg;  // weights of the two byte groups, mask, 8*g0, s*g0
};

__device__ __forceinline__ HashK hash_consts(const SearchArgs& a) {
  return HashK{a.w0, a.w1, a.mask, 8u * static_cast<uint32_t>(a.g0), static_cast<uint32_t>(a.s * a.g0)};
}

// hash_bytes with the constants in registers
template <int Q>
__device__ __forceinline__ uint32_t hash_k(uint32_t lo, uint32_t hi, const HashK& k) {
  uint32_t v = __dp4a(lo, k.w0, 0u);
  if constexpr (Q > 1) v += __dp4a(__funnelshift_rc(lo, hi, k.g8), k.w1, 0u) << k.sg;
  return v & k.mask;
}

// qgram_hash with the constants in registers
template <int Q, bool STAGED>
__device__ __forceinline__ uint32_t qgram_hash_k(const uint8_t* base, int o, const SearchArgs& a,
                                                 const HashK& k) {
  if constexpr (STAGED) {
    if (!HC_IN_BOUNDS(o >= 0 && o + 12 <= static_cast<int>(a.stage_bytes))) o = 0;
  } else {
    if (!HC_IN_BOUNDS(base + o >= a.y && base + o + Q <= a.y + a.n)) o = 0;
  }
  uint32_t lo, hi;
  load_qgram<Q, STAGED>(base, o, &lo, &hi);
  return hash_k<Q>(lo, hi, k);
}

// ---------------------------------------------------------------------------
// Byte tests of the dense (m = q) scans: 16 consecutive windows per lane,
// four per 32-bit word (byte k of a word belongs to window 4g + k).

// Bytes at lane-relative offset off .. off+3 of the 24 bytes Tw holds.
template <int OFF>
__device__ __forceinline__ uint32_t text_word(const uint32_t (&Tw)[6]) {
  if constexpr ((OFF & 3) == 0) return Tw[OFF >> 2];
  else return __funnelshift_r(Tw[OFF >> 2], Tw[(OFF >> 2) + 1], 8u * (OFF & 3));
}

// Column set of the byte test: 0 = every column c < Q; 1 = the first
// stage of the two-stage test (columns 0, 1, 4, 5: the cheapest four, two
// of them word-aligned); 2 = the remaining columns.
template <int SET>
__device__ __forceinline__ constexpr bool in_set(int c) {
  return SET == 0 || ((SET == 1) == ((c & 2) == 0));
}

// d[g] |= OR over the columns c of SET of (text bytes at 4g + c) ^ x[c]
// replicated: byte k of d[g] stays 0 while window 4g + k agrees with x on
// those columns.
template <int Q, int SET, int G, int C>
__device__ __forceinline__ void or_columns(const uint32_t (&Tw)[6], const uint32_t (&xrep)[Q],
                                           uint32_t (&d)[4]) {
  if constexpr (C < Q) {
    if constexpr (in_set<SET>(C)) d[G] |= text_word<4 * G + C>(Tw) ^ xrep[C];
    or_columns<Q, SET, G, C + 1>(Tw, xrep, d);
  } else if constexpr (G < 3) {
    or_columns<Q, SET, G + 1, 0>(Tw, xrep, d);
  }
}

// Bit 7 of byte k of the result is set iff byte k of d is zero (exact for
// every byte).
__device__ __forceinline__ uint32_t zero_bytes(uint32_t d) {
  return ~(((d & 0x7f7f7f7fu) + 0x7f7f7f7fu) | d | 0x7f7f7f7fu);
}

// Nonzero iff d has a zero byte (the lowest zero byte is always flagged;
// bytes above it may be flagged wrongly, so only the test is used).
__device__ __forceinline__ uint32_t has_zero_byte(uint32_t d) {
  return (d - 0x01010101u) & ~d & 0x80808080u;
}

// Nonzero iff some word of d has a zero byte (the per-word test of
// has_zero_byte, the four words combined before the final mask).
__device__ __forceinline__ uint32_t any_zero_byte4(const uint32_t (&d)[4]) {
  uint32_t acc = 0;
#pragma unroll
  for (int g = 0; g < 4; ++g) acc |= (d[g] - 0x01010101u) & ~d[g];
  return acc & 0x80808080u;
}

// 16-bit mask, bit 4g + k set iff bit 8k + 7 of z[g] is set.
__device__ __forceinline__ uint32_t gather_mask(const uint32_t (&z)[4]) {
  uint32_t m = 0;
#pragma unroll
  for (int g = 0; g < 4; ++g) m |= (((z[g] >> 7) * 0x01020408u) >> 24) << (4 * g);
  return m;
}


// Whether the m bytes of a window starting at chunk-relative `start` may be
// read for verification (always true outside checked builds).
template <bool STAGED>
__device__ __forceinline__ bool window_in_bounds(const uint8_t* txt, int start, const SearchArgs& a,
                                                 int head) {
  if constexpr (STAGED) {
    return HC_IN_BOUNDS(start >= -head && head + start + a.m <= static_cast<int>(a.stage_bytes));
  } else {
    return HC_IN_BOUNDS(txt + start >= a.y && txt + start + a.m <= a.y + a.n);
  }
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
  int pos32;                 // kToPositions: pos holds uint32 values
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
      else if (sink.pos32)
        reinterpret_cast<uint32_t*>(sink.pos)[idx] = static_cast<uint32_t>(sink.vbase + static_cast<unsigned>(start));
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
    bool eq = window_in_bounds<STAGED>(txt, start, a, head);
    for (int k = lane; eq && k < m; k += 32) eq &= text_byte<STAGED>(txt, start + k) == xv[k];
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
// First tests a lane evaluates together (see scan_segment).
constexpr int kFirstTests = 4;

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
template <int Q, bool STAGED, int MODE, int FT = 1, bool UNCHECKED = false>
__device__ __forceinline__ int scan_segment(const uint8_t* base, int head, int lo, int hi,
                                            const SearchArgs& a, const uint32_t* Fs,
                                            const uint8_t* xv, const Sink& sink,
                                            int* tests = nullptr, int* hits = nullptr) {
  const int lane = threadIdx.x & 31;
  const int m = a.m;
  const uint32_t hv = a.hv;
  const int shift = m - Q + 1;
  const uint8_t* txt = base + head;
  const HashK hk = hash_consts(a);
  int cnt = 0;
  int e = lo + m - 1;              // window end (chunk-relative)
  const int e_end = hi + m - 1;    // first window end past the segment
  bool deep = false;               // window at e waits for the warp
  int dj = 0;                      // walk position reached
  uint32_t dz = 0;                 // F word of the q-gram ending at dj
  int n_tests = 0, n_hits = 0;      // first tests made and passed (FT > 1 only)
  while (true) {
    while (!deep && e < e_end) {
      // first tests of the next FT windows of the miss sequence e, e +
      // shift, ... at once (independent loads, one branch per run): each
      // window whose end q-gram hits an empty word is shifted past, as the
      // sequential loop does; the first window that hits a non-empty word
      // goes on to the back-walk.  Windows past the segment take no part
      // (their test reads window e's q-gram and is discarded).
      uint32_t v = 0, z = 0;
      {
        uint32_t vu[FT], zu[FT];
#pragma unroll
        for (int u = 0; u < FT; ++u) {
          const int ek = e + u * shift;
          // with UNCHECKED (padded buffers) windows past the segment are
          // tested too; a hit there ends the segment below
          const bool in = UNCHECKED || u == 0 || ek < e_end;
          vu[u] = qgram_hash_k<Q, STAGED>(base, head + (in ? ek : e) - Q + 1, a, hk);
          zu[u] = in ? Fs[vu[u]] : 0u;
        }
        int k = FT;
#pragma unroll
        for (int u = FT - 1; u >= 0; --u) {
          if (zu[u] != 0u) {
            k = u;
            v = vu[u];
            z = zu[u];
          }
        }
        if constexpr (FT > 1) {
          n_tests += k == FT ? FT : k + 1;
          n_hits += k < FT ? 1 : 0;
        }
        if (k == FT) {
          e += FT * shift;
          continue;
        }
        e += k * shift;
        if constexpr (UNCHECKED) {
          if (e >= e_end) continue;  // the first hit lies past the segment: done
        }
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
        v = qgram_hash_k<Q, STAGED>(base, head + j - Q + 1, a, hk);
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
      bool eq = v == hv && window_in_bounds<STAGED>(txt, start, a, head);
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
  if (tests != nullptr) *tests = n_tests;
  if (hits != nullptr) *hits = n_hits;
  return cnt;
}

// Copies `words` 32-bit words (F) from global to shared memory: 16-byte
// loads when both pointers are 16-byte aligned and `words` is a multiple of
// 4, else 4-byte loads.  (Keeping several loads of a thread in flight cost
// registers -- the batched scan kernel went from 64 to 128 -- and measured
// no faster: the copy overlaps the previous kernel's tail.)  Every thread of
// the CTA calls it; the caller synchronises before reading dst.
__device__ __forceinline__ void stage_words(uint32_t* dst, const uint32_t* src, uint32_t words) {
  const uint32_t tid = threadIdx.x;
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 && (words & 3u) == 0) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (uint32_t i = tid; i < (words >> 2); i += kThreads) d4[i] = __ldg(s4 + i);
    return;
  }
  for (uint32_t i = tid; i < words; i += kThreads) dst[i] = __ldg(src + i);
}

// Copies n bytes (the pattern x) from global to shared memory: 16-byte loads
// for the whole 16-byte blocks when both pointers are 16-byte aligned, bytes
// for the rest; nothing past src[n - 1] is read.  Called by every thread of
// the CTA; the caller synchronises.
__device__ __forceinline__ void stage_bytes(uint8_t* dst, const uint8_t* src, uint32_t n) {
  const uint32_t tid = threadIdx.x;
  uint32_t done = 0;
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
    const uint32_t n16 = n >> 4;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (uint32_t i = tid; i < n16; i += kThreads) d4[i] = __ldg(s4 + i);
    done = n16 << 4;
  }
  for (uint32_t i = done + tid; i < n; i += kThreads) dst[i] = src[i];
}

// End of a single-search scan CTA: the sum of its kWarps records' totals
// (each written by lane 0 of its warp) into blk_total[blockIdx.x], so that
// the emit kernel sums one total per CTA instead of one per warp.  Every
// thread of the CTA must call it.
__device__ __forceinline__ void block_total(const SearchArgs& a) {
  __shared__ unsigned long long s_wt[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_wt[warp] = a.cta_total[static_cast<unsigned long long>(blockIdx.x) * kWarps + warp];
  __syncthreads();
  if (threadIdx.x == 0 && a.blk_total != nullptr) {
    unsigned long long t = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += s_wt[w];
    a.blk_total[blockIdx.x] = t;
  }
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


// The per-warp stream of kernel 1 (per-lane HC): record w_id owns chunks
// [w_id*K, (w_id+1)*K) of a.  Fs / xv: F and x (shared memory); slots: the
// CTA's per-thread occurrence slots; stages / wb: this warp's ring of
// staging buffers and its mbarriers (staged form).  Writes cta_total[w_id]
// and cta_overflow[w_id].  Used by the single-search kernel and by the
// batched kernel, which calls it once per (query, record).
template <int Q, bool STAGED>
__device__ __forceinline__ void warp_stream(const SearchArgs& a, unsigned long long w_id,
                                            const uint32_t* Fs, const uint8_t* xv,
                                            uint32_t* slots, uint8_t* stages, uint64_t* wb) {
  const int lane = threadIdx.x & 31;
  const int tid = threadIdx.x;
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
  bool batch_first = true;                // first tests four at a time (warp-uniform)
  int probe_in = 0;                       // chunks until the batched form is tried again
  unsigned long long T = 0;               // occurrences so far in this range
  unsigned long long overflow = kNoOverflow;
  Sink sink{};
  sink.slot = slots + tid;
  bool ok = true;
  int i = 0;
  // ring slot and mbarrier phase of chunk i, kept incrementally (no runtime
  // division by the ring size in the loop)
  int st = 0, prev_st = nst - 1;
  uint32_t phase = 0;
  for (; i < nchunks; ++i, prev_st = st, st = (st + 1 == nst) ? 0 : st + 1, phase ^= (st == 0) ? 1u : 0u) {
    const unsigned long long c = c0 + static_cast<unsigned long long>(i);
    if constexpr (STAGED) {
      if (lane == 0 && i > 0 && i + nst - 1 < nchunks) {
        // the buffer of chunk i-1 was released by the __syncwarp that ended it
        fence_proxy_async_smem();
        issue(prev_st, c + nst - 1);
      }
      ok = __all_sync(0xffffffffu, mbar_wait_bounded(&wb[st], phase));
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
    // first tests four at a time while few of them pass (one window in 16
    // or fewer over the warp's last chunk), one at a time otherwise: where
    // many pass, the batch's later tests are wasted and its lanes diverge
    int tests = 0, hits = 0;
    int cnt;
    if (!batch_first)
      cnt = scan_segment<Q, STAGED, kCount, 1>(base, head, lo, hi, a, Fs, xv, sink);
    else if (STAGED && a.unchecked)
      cnt = scan_segment<Q, STAGED, kCount, kFirstTests, STAGED>(base, head, lo, hi, a, Fs, xv, sink, &tests, &hits);
    else
      cnt = scan_segment<Q, STAGED, kCount, kFirstTests>(base, head, lo, hi, a, Fs, xv, sink, &tests, &hits);
    if (batch_first) {
      const int wt = __reduce_add_sync(0xffffffffu, tests), wh = __reduce_add_sync(0xffffffffu, hits);
      if (wh * 16 > wt) { batch_first = false; probe_in = 32; }
    } else if (--probe_in == 0) {
      batch_first = true;  // look again now and then
    }

    if (__any_sync(0xffffffffu, cnt != 0)) {
      const uint32_t incl = warp_incl_scan_u32(static_cast<uint32_t>(cnt));
      const uint32_t excl = incl - static_cast<uint32_t>(cnt);
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      if (overflow == kNoOverflow) {
        if (T + total <= S) {
          const uint32_t rel = static_cast<uint32_t>(static_cast<unsigned long long>(i) * a.C);
          const unsigned long long ob = T + excl;
          if (cnt <= kSlots)
            for (int k = 0; k < cnt; ++k)
              if (HC_IN_BOUNDS(ob + k < S)) region[ob + k] = rel + sink.slot[k * kThreads];
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
        atomicOr(a.status, 1u);
        // let the copies still in flight land before the CTA's shared memory goes
        for (int j = i; j < nchunks && j < i + nst; ++j)
          (void)mbar_wait_bounded(&wb[j % nst], static_cast<uint32_t>(j / nst) & 1u);
      }
    }
  }
  if constexpr (STAGED) {
    __syncwarp();
    if (lane == 0 && ok)
      for (int k = 0; k < nst; ++k) mbar_inval(&wb[k]);
    __syncwarp();
  }
}

// The emit logic for record group g of a (copy part `part` of kEmitSplit);
// smem: at least F's words plus the slots (for re-scans).
template <int Q>
__device__ __forceinline__ void emit_group(const SearchArgs& a, unsigned long long g, unsigned part,
                                           uint8_t* smem) {
  __shared__ unsigned long long red[kWarps];
  __shared__ uint32_t warp_sum[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long r0 = g * a.emit_group;
  const unsigned long long r1 = min(r0 + a.emit_group, a.records);

  __shared__ unsigned long long s_tot[kMaxEmitGroup], s_ovf[kMaxEmitGroup];
  const int nrec = static_cast<int>(r1 - r0);
  // the group's own records first: independent of the prefix loads below,
  // so both rounds of loads are in flight together
  unsigned long long my_tot = 0, my_ovf = kNoOverflow;
  if (tid < nrec) {
    my_tot = a.cta_total[r0 + tid];
    my_ovf = a.cta_overflow[r0 + tid];
  }
  unsigned long long p = 0;
  if (a.blk_total != nullptr) {
    // sum of the earlier records' totals: the CTAs wholly before record r0
    // (one total each), then the records of r0's CTA before it
    const unsigned long long b0 = r0 / kWarps;
    for (unsigned long long k = tid; k < b0; k += kThreads) p += a.blk_total[k];
    for (unsigned long long k = b0 * kWarps + tid; k < r0; k += kThreads) p += a.cta_total[k];
  } else {
    // sum of the earlier records' totals: loads issued 8 at a time
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
  }
  p = warp_sum_u64(p);
  if (lane == 0) red[warp] = p;
  if (tid < nrec) {
    s_tot[tid] = my_tot;
    s_ovf[tid] = my_ovf;
  }
  __syncthreads();
  // per record of the group: output offset P, positions to copy, and the
  // prefix of 2-position units, so that the whole group is copied in one
  // pass (no per-record latency chain); warp 0, two records per lane, two
  // warp scans
  __shared__ unsigned long long s_P[kMaxEmitGroup + 1], s_U[kMaxEmitGroup + 1], s_N[kMaxEmitGroup];
  if (warp == 0) {
    unsigned long long P0 = 0;
    for (int w = 0; w < kWarps; ++w) P0 += red[w];
    const int k0 = 2 * lane, k1 = 2 * lane + 1;
    auto stored_of = [&](int k) -> unsigned long long {
      if (k >= nrec) return 0ull;
      const unsigned long long ovf = s_ovf[k];
      return ovf == kNoOverflow ? s_tot[k] : (ovf & ((1ull << 40) - 1));
    };
    const unsigned long long T0 = k0 < nrec ? s_tot[k0] : 0ull, T1 = k1 < nrec ? s_tot[k1] : 0ull;
    const unsigned long long Pk0 = P0 + warp_excl_scan_u64(T0 + T1), Pk1 = Pk0 + T0;
    const unsigned long long n0 = a.cap > Pk0 ? min(stored_of(k0), a.cap - Pk0) : 0ull;
    const unsigned long long n1 = a.cap > Pk1 ? min(stored_of(k1), a.cap - Pk1) : 0ull;
    const unsigned long long u0 = (n0 + 1) / 2, u1 = (n1 + 1) / 2;
    const unsigned long long Uk0 = warp_excl_scan_u64(u0 + u1), Uk1 = Uk0 + u0;
    if (k0 < nrec) {
      s_P[k0] = Pk0;
      s_U[k0] = Uk0;
      s_N[k0] = n0;
    }
    if (k1 < nrec) {
      s_P[k1] = Pk1;
      s_U[k1] = Uk1;
      s_N[k1] = n1;
    }
    const unsigned long long Ptot = P0 + warp_sum_u64(T0 + T1), Utot = warp_sum_u64(u0 + u1);
    if (lane == 0) {
      s_P[nrec] = Ptot;
      s_U[nrec] = Utot;
      if (part == 0 && r1 == a.records) *a.count_out = Ptot;
    }
  }
  __syncthreads();
  {
    // unit u of record k: region entries 2(u - U_k) and +1 (8-byte loads;
    // regions are 16-byte aligned); consecutive threads take consecutive
    // units, so a warp's 16-byte stores cover 512 contiguous bytes; 16-byte
    // stores where the output address is 16-byte aligned
    const unsigned long long U = s_U[nrec];
    const unsigned long long stride = static_cast<unsigned long long>(kThreads) * kEmitSplit;
    int rk = 0;  // record of this thread's current unit (units only increase)
    for (unsigned long long u0 = part * kThreads + tid; u0 < U; u0 += kEmitUnits * stride) {
      uint2 v[kEmitUnits];
      int rec[kEmitUnits];
#pragma unroll
      for (int uu = 0; uu < kEmitUnits; ++uu) {
        const unsigned long long u = u0 + static_cast<unsigned long long>(uu) * stride;
        rec[uu] = -1;
        if (u < U) {
          while (s_U[rk + 1] <= u) ++rk;
          rec[uu] = rk;
          const uint2* r2 = reinterpret_cast<const uint2*>(a.region + (r0 + rk) * a.region_entries);
          if (HC_IN_BOUNDS((u - s_U[rk]) * 2 + 2 <= a.region_entries)) v[uu] = __ldcs(r2 + (u - s_U[rk]));
          else rec[uu] = -1;
        }
      }
#pragma unroll
      for (int uu = 0; uu < kEmitUnits; ++uu) {
        if (rec[uu] < 0) continue;
        const int k = rec[uu];
        const unsigned long long u = u0 + static_cast<unsigned long long>(uu) * stride;
        const unsigned long long e = (u - s_U[k]) * 2;   // first entry of the unit
        const unsigned long long vbase = (r0 + k) * a.chunks_per_cta * a.C;
        if (!HC_IN_BOUNDS(s_P[k] + e < a.cap && e < s_N[k])) continue;
        if (a.pos32) {
          uint32_t* o = reinterpret_cast<uint32_t*>(a.pos) + s_P[k] + e;
          const uint32_t b32 = static_cast<uint32_t>(vbase);
          if (e + 2 <= s_N[k] && (reinterpret_cast<uintptr_t>(o) & 7u) == 0u) {
            *reinterpret_cast<uint2*>(o) = make_uint2(b32 + v[uu].x, b32 + v[uu].y);
          } else {
            o[0] = b32 + v[uu].x;
            if (e + 1 < s_N[k]) o[1] = b32 + v[uu].y;
          }
          continue;
        }
        unsigned long long* o = a.pos + s_P[k] + e;
        if (e + 2 <= s_N[k] && (reinterpret_cast<uintptr_t>(o) & 15u) == 0u) {
          *reinterpret_cast<ulonglong2*>(o) = make_ulonglong2(vbase + v[uu].x, vbase + v[uu].y);
        } else {
          o[0] = vbase + v[uu].x;
          if (e + 1 < s_N[k]) o[1] = vbase + v[uu].y;
        }
      }
    }
  }

  bool f_loaded = false;
  for (unsigned long long b = r0; b < r1; ++b) {
    const unsigned long long T = s_tot[b - r0];
    const unsigned long long ovf = s_ovf[b - r0];
    const unsigned long long P = s_P[b - r0];
    if (ovf == kNoOverflow || T == 0) continue;  // nothing to re-scan
    const unsigned long long stored = ovf & ((1ull << 40) - 1);
    const unsigned long long c0 = b * a.chunks_per_cta;
    if (part == 0) {
      if (P + stored < a.cap) {
        // re-scan the chunks from the first unstored one on
        uint32_t* Fs = reinterpret_cast<uint32_t*>(smem);
        uint32_t* slots = Fs + ((a.fwords + 3u) & ~3u);
        if (!f_loaded) {
          stage_words(Fs, a.F, a.fwords);
          __syncthreads();
          f_loaded = true;
        }
        const unsigned long long c1 = min(c0 + a.chunks_per_cta, a.num_chunks);
        unsigned long long out = P + stored;
        Sink cs_sink{};
        cs_sink.slot = slots + tid;
        // a chunk is C / L lane segments of L window starts (32 for the
        // per-warp chunks, kThreads for the dense ones): the CTA re-scans
        // kThreads * L / C consecutive chunks per round, thread order =
        // chunk-major, so the block scan keeps positions ascending
        const int lanes = static_cast<int>(a.C / static_cast<uint32_t>(a.L));
        const int per_round = max(1, kThreads / lanes);
        const int sub = tid / lanes;
        const int lo = (tid % lanes) * a.L;
        for (unsigned long long cb = c0 + (ovf >> 40); cb < c1 && out < a.cap; cb += per_round) {
          const unsigned long long c = cb + static_cast<unsigned long long>(sub);
          const bool mine = sub < per_round && c < c1;
          const unsigned long long cs = c * a.C;
          int hi = lo;
          if (mine) hi = max(lo, min(lo + a.L, static_cast<int>(min(static_cast<unsigned long long>(a.C), a.nwin - cs))));
          const uint8_t* base = a.y + (mine ? cs : 0ull);
          const int cnt = mine ? scan_segment<Q, false, kCount>(base, 0, lo, hi, a, Fs, a.x, cs_sink) : 0;
          uint32_t excl, total;
          block_scan(static_cast<uint32_t>(cnt), warp_sum, &excl, &total);
          if (mine) {  // warp-uniform: scan_segment is called by whole warps
            Sink w{};
            w.pos = a.pos;
            w.pos32 = a.pos32;
            w.obase = out + excl;
            w.vbase = cs;
            w.limit = a.cap;
            scan_segment<Q, false, kToPositions>(base, 0, lo, cnt > 0 ? hi : lo, a, Fs, a.x, w);
          }
          out += total;
          __syncthreads();
        }
      }
    }
  }
}

}  // namespace hc
