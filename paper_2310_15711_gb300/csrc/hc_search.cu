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
#include "hc_kernels.cuh"

namespace hc {

// bit 0: a bounded device-side wait gave up
__device__ unsigned int g_status;

// ---------------------------------------------------------------------------
// Kernel 1: per-lane HC.  Every warp is an independent stream: record
// w = blockIdx.x * 8 + warp owns a contiguous range of chunks of 32*L window
// starts; lane l scans starts [lL, lL + L) of each chunk.  Staged: the warp
// brings its chunks into its own ring of shared-memory buffers with bulk
// copies on its own mbarriers; direct: the lanes read the text from global
// memory.  Occurrences go, in text order, to the warp's spill region; the
// total to cta_total[w].  No CTA-wide barrier in the loop.
template <int Q, bool STAGED>
__global__ void __launch_bounds__(kThreads, 4) hc_scan_kernel(const SearchArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[kWarps][kMaxStages];
  pdl_launch_dependents();  // the emit kernel may be scheduled; it waits for this grid

  const int tid = threadIdx.x, warp = tid >> 5;
  uint32_t* Fs = reinterpret_cast<uint32_t*>(smem);
  const uint32_t f_bytes = (a.fwords * 4u + 15u) & ~15u;
  uint8_t* xs = smem + f_bytes;
  uint32_t* slots = reinterpret_cast<uint32_t*>(xs + a.x_smem);
  stage_words(Fs, a.F, a.fwords);
  stage_bytes(xs, a.x, min(a.x_smem, static_cast<uint32_t>(a.m)));
  const uint8_t* xv = a.x_smem ? xs : a.x;
  __syncthreads();
  // launched as a programmatic dependent of the previous search's emit
  // kernel: F and x (read above) are not written by it, but the text, the
  // workspace (which may reuse the previous one's memory) and the outputs
  // are touched only after that kernel has completed
  pdl_wait();
  uint8_t* stages = reinterpret_cast<uint8_t*>(slots + kSlots * kThreads) +
                    static_cast<size_t>(warp) * a.stages * a.stage_bytes;
  warp_stream<Q, STAGED>(a, static_cast<unsigned long long>(blockIdx.x) * kWarps + warp, Fs, xv,
                         slots, stages, bars[warp]);
  block_total(a);
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
// shared-memory buffers with bulk copies on its own mbarriers, queues the
// lanes that hold a candidate in a step, finishes them 32 at a time and
// appends the matches, in order, straight to its own spill region.  There is
// no CTA-wide barrier in the loop.
//
// Bitmap form (BM): instead, every lane turns its 16 windows of a step into
// a 16-bit mask, and the warp writes the masks as the text's window bitmap
// (bit j of group g: window 16g + j of the chunk; a lane's windows start
// `head` windows before a group boundary, so group g joins the upper bits of
// one lane's mask with the lower bits of the next lane's, the last lane's
// carried over to the next step).  The warp's total goes to its record; the
// emit kernel expands the bits.  No work per occurrence in the scan, and
// n / 8 bytes written and read back instead of 4 bytes per occurrence each
// way: the form for patterns with many occurrences.
template <int Q, bool BM>
__device__ __forceinline__ void dense_stream(const SearchArgs& a, uint8_t* smem, uint64_t* wb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lanes_below = (1u << lane) - 1u;
  const unsigned long long w_id = static_cast<unsigned long long>(blockIdx.x) * kWarps + warp;

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
  uint8_t* stages = smem + static_cast<size_t>(warp) * nst * a.stage_bytes;
  // spill form: the warp's queue of candidate lanes, after all warps' rings
  uint16_t* queue = reinterpret_cast<uint16_t*>(smem + static_cast<size_t>(kWarps) * nst * a.stage_bytes) +
                    static_cast<size_t>(warp) * kQueueCap;
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
  // HC's first test and H_v test, evaluated on x itself (see above); F
  // itself is read once from global memory (it is not staged: nothing else
  // of it is needed)
  const uint32_t hx = hash_bytes<Q>(xlo, xhi, a);
  const bool filter_passes = __ldg(a.F + hx) != 0u && hx == a.hv;
  int single_left = 0;  // chunks left in the one-stage byte test (q >= 5)

  const unsigned long long S = a.region_entries;
  uint32_t* region = BM ? nullptr : a.region + w_id * S;
  const int hd = a.head;
  const int gchunk = static_cast<int>(a.C / 16u);  // bitmap groups per chunk
  unsigned long long T = 0;                 // matches so far in this warp's range
  unsigned long long overflow = kNoOverflow;
  bool ok = true;
  int i = 0;
  // ring slot and mbarrier phase of chunk i, kept incrementally (no runtime
  // division by the ring size in the loop)
  int st = 0, prev_st = nst - 1;
  uint32_t phase = 0;
  for (; i < nchunks; ++i, prev_st = st, st = (st + 1 == nst) ? 0 : st + 1, phase ^= (st == 0) ? 1u : 0u) {
    const unsigned long long c = c0 + static_cast<unsigned long long>(i);
    if (lane == 0 && i > 0 && i + nst - 1 < nchunks) {
      // the buffer of chunk i-1 was released by the __syncwarp that ended it
      fence_proxy_async_smem();
      issue(prev_st, c + nst - 1);
    }
    ok = __all_sync(0xffffffffu, mbar_wait_bounded(&wb[st], phase));
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
    // q >= 5: a two-stage byte test (columns 0, 1, 4, 5 first; the others
    // only for the lanes with a candidate) while the first stage leaves few
    // candidates (the spill form: at most kTwoStageLanes lanes per step on
    // average; the bitmap form: candidates in at most half the steps), else
    // the one-stage test for the next 16 chunks
    const bool two = Q >= 5 && single_left == 0;
    int second = 0, steps = 0;
    // The first (or only) stage of the byte test for the step at `base`
    // (512 windows, 16 per lane): Tw and dg receive the lane's text words
    // and column differences; returns the lane's candidate flags.  Lanes
    // past the chunk's end read the buffer's last 32 bytes instead (no
    // branch; a 16-byte aligned offset, as every lane's is) and discard what
    // they find.
    auto test = [&](int base, uint32_t (&Tw)[6], uint32_t (&dg)[4]) -> uint32_t {
      const int w0 = base + 16 * lane;      // first window of this lane
      const bool live = w0 < wins;
      const uint32_t o = min(static_cast<uint32_t>(a.head + w0), a.stage_bytes - 32u);
      HC_IN_BOUNDS(static_cast<uint32_t>(a.head + w0) + 24u <= a.stage_bytes || !live);
      const uint4 A = *reinterpret_cast<const uint4*>(sb + o);
      const uint2 B = *reinterpret_cast<const uint2*>(sb + o + 16);
      Tw[0] = A.x; Tw[1] = A.y; Tw[2] = A.z; Tw[3] = A.w; Tw[4] = B.x; Tw[5] = B.y;  // bytes o .. o+23
      // byte k of dg[g] stays 0 while window w0+4g+k agrees with x
      dg[0] = dg[1] = dg[2] = dg[3] = 0u;
      if (two) or_columns<Q, 1, 0, 0>(Tw, xrep, dg);
      else or_columns<Q, 0, 0, 0>(Tw, xrep, dg);
      // nonzero iff some dg[g] has a zero byte (exact for the test; the flag
      // positions above a zero byte may be wrong, so they are not used)
      return (live && filter_passes) ? any_zero_byte4(dg) : 0u;
    };
    // The same for a step in which every lane's first window lies before
    // the chunk's end (no liveness test, no clamp), used only where
    // F[h(x)] != 0 and h(x) = H_v.
    auto test_full = [&](int base, uint32_t (&Tw)[6], uint32_t (&dg)[4]) -> uint32_t {
      const uint32_t o = static_cast<uint32_t>(a.head + base + 16 * lane);
      HC_IN_BOUNDS(o + 24u <= a.stage_bytes);
      const uint4 A = *reinterpret_cast<const uint4*>(sb + o);
      const uint2 B = *reinterpret_cast<const uint2*>(sb + o + 16);
      Tw[0] = A.x; Tw[1] = A.y; Tw[2] = A.z; Tw[3] = A.w; Tw[4] = B.x; Tw[5] = B.y;
      dg[0] = dg[1] = dg[2] = dg[3] = 0u;
      if (two) or_columns<Q, 1, 0, 0>(Tw, xrep, dg);
      else or_columns<Q, 0, 0, 0>(Tw, xrep, dg);
      return any_zero_byte4(dg);
    };
    // The steps' candidate lanes wait in the warp's queue (entry: step
    // index << 5 | lane, in step order, lanes in order within a step) and
    // are finished 32 at a time, one per lane: the lane tests its 16 windows
    // again with every column, takes the exact per-window flags, and the
    // warp writes the matches in window order to the spill region.  A step
    // with one or two candidates then costs a vote and a queue store
    // instead of a warp-wide finish.
    int qn = 0;   // entries in the queue
    auto flush = [&]() {
      for (int e0 = 0; e0 < qn; e0 += 32) {
        const int e = e0 + lane;
        uint32_t mbits = 0;
        int w0 = 0;
        if (e < qn) {
          const uint32_t ent = queue[e];
          w0 = -a.head + 512 * static_cast<int>(ent >> 5) + 16 * static_cast<int>(ent & 31u);
          const uint32_t o = static_cast<uint32_t>(a.head + w0);  // >= 0, 16-byte aligned: a live lane's
          HC_IN_BOUNDS(o + 24u <= a.stage_bytes);
          const uint4 A = *reinterpret_cast<const uint4*>(sb + o);
          const uint2 B = *reinterpret_cast<const uint2*>(sb + o + 16);
          const uint32_t Tw[6] = {A.x, A.y, A.z, A.w, B.x, B.y};
          uint32_t dg[4] = {0u, 0u, 0u, 0u};
          or_columns<Q, 0, 0, 0>(Tw, xrep, dg);
          // exact zero-byte test: bit 8k+7 of zg is set iff window w0+4g+k
          // equals x; packed to bit 4g+k of mbits
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const uint32_t zg = ~(((dg[g] & 0x7f7f7f7fu) + 0x7f7f7f7fu) | dg[g] | 0x7f7f7f7fu);
            mbits |= ((zg >> 7) * 0x01020408u >> 24) << (4 * g);
          }
          if (w0 < 0) mbits &= 0xffffu << min(-w0, 16);
          if (w0 + 16 > wins) mbits &= 0xffffu >> (16 - max(wins - w0, 0));
        }
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
      qn = 0;
    };
    // appends the candidate lanes `cl` of step sidx
    auto enqueue = [&](int sidx, uint32_t cl) {
      if ((cl >> lane) & 1u) queue[qn + __popc(cl & ((1u << lane) - 1u))] = static_cast<uint16_t>((sidx << 5) | lane);
      qn += __popc(cl);
    };
    // a step in which most lanes hold a candidate is finished at once, from
    // the column differences at hand (the queue, in window order before it,
    // is flushed first)
    auto finish_now = [&](int base, const uint32_t (&Tw)[6], uint32_t (&dg)[4], uint32_t cand) {
      if (qn != 0) flush();
      const int w0 = base + 16 * lane;
      uint32_t mbits = 0;
      if (cand != 0u) {
        if (two) or_columns<Q, 2, 0, 0>(Tw, xrep, dg);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const uint32_t zg = ~(((dg[g] & 0x7f7f7f7fu) + 0x7f7f7f7fu) | dg[g] | 0x7f7f7f7fu);
          mbits |= ((zg >> 7) * 0x01020408u >> 24) << (4 * g);
        }
        if (w0 < 0) mbits &= 0xffffu << min(-w0, 16);
        if (w0 + 16 > wins) mbits &= 0xffffu >> (16 - max(wins - w0, 0));
      }
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
    };
    if constexpr (BM) {
      // this lane's exact 16-bit mask (bit i: window w0 + i) from complete
      // column differences; windows outside [0, wins) cleared
      auto exact = [&](int base, const uint32_t (&dg)[4]) -> uint32_t {
        const int w0 = base + 16 * lane;
        uint32_t mb = 0;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const uint32_t zg = ~(((dg[g] & 0x7f7f7f7fu) + 0x7f7f7f7fu) | dg[g] | 0x7f7f7f7fu);
          mb |= ((zg >> 7) * 0x01020408u >> 24) << (4 * g);
        }
        if (w0 < 0) mb &= 0xffffu << min(-w0, 16);
        if (w0 + 16 > wins) mb &= 0xffffu >> (16 - max(wins - w0, 0));
        return mb;
      };
      uint16_t* bm = a.bitmap + c * static_cast<unsigned long long>(gchunk);
      uint32_t carry = 0;      // the last lane's mask of the previous step
      uint32_t chunk_cnt = 0;  // this lane's matches in the chunk
      int sidx = 0;            // step index in the chunk
      // group 32 * sidx + lane - 1 from the previous lane's mask (upper
      // 16 - hd bits) and this lane's (lower hd bits)
      auto put = [&](uint32_t mb) {
        const uint32_t up = __shfl_up_sync(0xffffffffu, mb, 1);
        const uint32_t prev = lane == 0 ? carry : up;
        carry = __shfl_sync(0xffffffffu, mb, 31);
        const int G = 32 * sidx + lane - 1;
        if (G >= 0 && G < gchunk) bm[G] = static_cast<uint16_t>(((prev >> hd) | (mb << (16 - hd))) & 0xffffu);
        chunk_cnt += static_cast<uint32_t>(__popc(mb));
        ++sidx;
      };
      for (int base = -a.head; base < wins; base += 1024) {
        uint32_t Tw0[6], dg0[4], Tw1[6], dg1[4];
        const uint32_t k0 = test(base, Tw0, dg0);
        const uint32_t k1 = test(base + 512, Tw1, dg1);
        steps += 2;
        uint32_t m0 = 0u, m1 = 0u;
        if (two) {
          // the other columns only where the first stage left a candidate
          if (__any_sync(0xffffffffu, (k0 | k1) != 0u)) {
            second += (__any_sync(0xffffffffu, k0 != 0u) ? 1 : 0) + (__any_sync(0xffffffffu, k1 != 0u) ? 1 : 0);
            if (k0 != 0u) {
              or_columns<Q, 2, 0, 0>(Tw0, xrep, dg0);
              m0 = exact(base, dg0);
            }
            if (k1 != 0u) {
              or_columns<Q, 2, 0, 0>(Tw1, xrep, dg1);
              m1 = exact(base + 512, dg1);
            }
          }
        } else if (__any_sync(0xffffffffu, (k0 | k1) != 0u)) {
          // one stage: dg is complete; a lane without a candidate (or past
          // the end, or with F[h(x)] = 0) has no match
          if (k0 != 0u) m0 = exact(base, dg0);
          if (k1 != 0u) m1 = exact(base + 512, dg1);
        }
        put(m0);
        put(m1);
      }
      // the last group, whose upper bits lie past the last step
      const int G = 32 * sidx - 1;
      if (lane == 0 && G < gchunk) bm[G] = static_cast<uint16_t>((carry >> hd) & 0xffffu);
      T += __reduce_add_sync(0xffffffffu, chunk_cnt);
      if (Q >= 5) {
        if (two && 2 * second > steps) single_left = 16;
        else if (!two) --single_left;
      }
      __syncwarp();  // staging buffer st is free again
      continue;
    }
    // hot loop: the first stage of two steps at once (independent loads,
    // one vote for both); a step in which some lane has a candidate is
    // finished apart.  A step past the chunk's end tests nothing (all its
    // lanes are past the end).
    // the candidates of the step pair at `base` (step indexes sidx, sidx + 1)
    auto handle = [&](int base, int sidx, uint32_t c0, uint32_t c1, const uint32_t (&Tw0)[6],
                      uint32_t (&dg0)[4], const uint32_t (&Tw1)[6], uint32_t (&dg1)[4]) {
      if (!__any_sync(0xffffffffu, (c0 | c1) != 0u)) return;
      const uint32_t cl0 = __ballot_sync(0xffffffffu, c0 != 0u);
      const uint32_t cl1 = __ballot_sync(0xffffffffu, c1 != 0u);
      const int n0 = __popc(cl0), n1 = __popc(cl1);
      second += n0 + n1;
      if (n0 < kDirectLanes && n1 < kDirectLanes) {
        // both steps into the queue
        if (qn > kQueueCap - 64) flush();
        if (c0 != 0u) queue[qn + __popc(cl0 & lanes_below)] = static_cast<uint16_t>((sidx << 5) | lane);
        if (c1 != 0u) queue[qn + n0 + __popc(cl1 & lanes_below)] = static_cast<uint16_t>(((sidx + 1) << 5) | lane);
        qn += n0 + n1;
        return;
      }
      if (n0 >= kDirectLanes) {
        finish_now(base, Tw0, dg0, c0);
      } else if (n0 != 0) {
        if (qn > kQueueCap - 32) flush();
        enqueue(sidx, cl0);
      }
      if (n1 >= kDirectLanes) {
        finish_now(base + 512, Tw1, dg1, c1);
      } else if (n1 != 0) {
        if (qn > kQueueCap - 32) flush();
        enqueue(sidx + 1, cl1);
      }
    };
    if (filter_passes) {
      int base = -a.head, sidx = 0;
      // step pairs whose windows all lie before the chunk's end
      for (; base + 1024 <= wins; base += 1024, sidx += 2) {
        uint32_t Tw0[6], dg0[4], Tw1[6], dg1[4];
        const uint32_t c0 = test_full(base, Tw0, dg0);
        const uint32_t c1 = test_full(base + 512, Tw1, dg1);
        steps += 2;
        handle(base, sidx, c0, c1, Tw0, dg0, Tw1, dg1);
      }
      // the last, partial pair (lanes past the end test nothing)
      if (base < wins) {
        uint32_t Tw0[6], dg0[4], Tw1[6], dg1[4];
        const uint32_t c0 = test(base, Tw0, dg0);
        const uint32_t c1 = test(base + 512, Tw1, dg1);
        steps += 2;
        handle(base, sidx, c0, c1, Tw0, dg0, Tw1, dg1);
      }
    }
    flush();  // before the staging buffer is released
    if (Q >= 5) {
      // the first stage pays while it leaves few candidate lanes per step
      if (two && second > kTwoStageLanes * steps) single_left = 16;
      else if (!two) --single_left;
    }
    if (store && t > S) overflow = (static_cast<unsigned long long>(i) << 40) | T;
    T = t;
    __syncwarp();  // staging buffer st is free again
  }

  if (lane == 0) {
    a.cta_total[w_id] = T;
    a.cta_overflow[w_id] = overflow;
    if (!ok) {
      atomicOr(a.status, 1u);
      // let the copies still in flight land before the CTA's shared memory goes
      for (int j = i; j < nchunks && j < i + nst; ++j)
        (void)mbar_wait_bounded(&wb[j % nst], static_cast<uint32_t>(j / nst) & 1u);
    }
  }
}

template <int Q, bool BM>
__global__ void __launch_bounds__(kThreads) hc_scan_dense_kernel(const SearchArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[kWarps][kMaxStages];
  pdl_launch_dependents();
  // launched as a programmatic dependent of the previous search's emit
  // kernel: nothing of memory is touched before that kernel has completed
  // (only the launch and the CTAs' start overlap its tail)
  pdl_wait();
  dense_stream<Q, BM>(a, smem, bars[threadIdx.x >> 5]);
  block_total(a);
}

// ---------------------------------------------------------------------------
// Kernel 2: record r's output offset is the sum of cta_total[0..r); copy its
// region to the output; re-scan (from global memory) the chunks whose
// occurrences did not fit in the region.  A CTA serves a group of
// emit_group consecutive records (so the sums over earlier records are made
// once per group), and kEmitSplit CTAs share each group's copying; the first
// of them writes the count (last record) and does the re-scans.
template <int Q>
__global__ void __launch_bounds__(kThreads, 4) hc_emit_kernel(const SearchArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  pdl_launch_dependents();  // the next search's scan may be scheduled; it waits for this grid
  pdl_wait();  // the scan grid has completed and its records are visible
  emit_group<Q>(a, blockIdx.x / kEmitSplit, blockIdx.x % kEmitSplit, smem);
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

template <bool BM>
KernelFn dense_kernel_for_q(int q) {
  switch (q) {
    case 1: return hc_scan_dense_kernel<1, BM>;
    case 2: return hc_scan_dense_kernel<2, BM>;
    case 3: return hc_scan_dense_kernel<3, BM>;
    case 4: return hc_scan_dense_kernel<4, BM>;
    case 5: return hc_scan_dense_kernel<5, BM>;
    case 6: return hc_scan_dense_kernel<6, BM>;
    case 7: return hc_scan_dense_kernel<7, BM>;
    default: return hc_scan_dense_kernel<8, BM>;
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
      L = 16;
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
  const int stages = o && o->stages ? o->stages : (kind == HC_MODE_DIRECT ? 3 : 2);
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
  // the loads that run past the copied bytes: the per-lane kernels read at
  // most 11 bytes past the last q-gram's first byte (three 32-bit words), the
  // dense kernel at most 20 past the chunk's last window start
  p.stage_bytes = stage_bytes_for(p.C, f->m, kind == HC_MODE_DENSE);
  const int sp_opt = o ? o->single_pass : 0;
  const int tile_steps_opt = o ? o->tile_steps : 0;
  if (sp_opt < -1 || sp_opt > 1) return set_error(HC_ERR_ARG, "hc_search: single_pass out of [-1, 1]");
  if (tile_steps_opt < 0 || tile_steps_opt > kSinglePassMaxSteps)
    return set_error(HC_ERR_ARG, "hc_search: tile_steps out of [0, 64]");
  if (kind == HC_MODE_DENSE && sp_opt == 1) {
    // single pass: chunks of a whole number of 512-window steps (L even),
    // tiles of whole chunks, at most kSinglePassMaxSteps steps per tile
    const int Ls = std::max(2, (L + 1) & ~1);
    const int spc = Ls / 2;  // steps per chunk
    const int want = tile_steps_opt ? tile_steps_opt : kSinglePassTileSteps;
    const int tc = std::max(1, (want + spc - 1) / spc);
    if (spc * tc <= kSinglePassMaxSteps) {
      p.single_pass = true;
      p.L = Ls;
      p.C = static_cast<uint32_t>(kThreads) * static_cast<uint32_t>(Ls);
      p.tile_chunks = tc;
      p.flag_steps = spc * tc;
      p.stage_bytes = stage_bytes_for(p.C, f->m, true);
      p.scan = dense_single_pass_kernel_for_q(f->q);
      p.init = single_pass_init_kernel();
      // per warp: its ring of staging buffers and two tiles' step masks (u16
      // per lane and step: the tile being scanned, the one being written)
      p.smem_scan = size_t(kWarps) * stages * p.stage_bytes + size_t(kWarps) * 2 * p.flag_steps * 64;
      if (p.smem_scan + static_smem(p.scan) > di.smem_optin) p.single_pass = false;
    } else if (sp_opt == 1) {
      return set_error(HC_ERR_ARG, "hc_search: single pass needs at most 64 steps of 512 windows per tile");
    }
    if (!p.single_pass) {
      if (sp_opt == 1) return set_error(HC_ERR_ARG, "hc_search: single-pass buffers exceed shared memory");
      p.L = L;
      p.C = static_cast<uint32_t>(kThreads) * static_cast<uint32_t>(L);
      p.stage_bytes = stage_bytes_for(p.C, f->m, true);
    }
  } else if (sp_opt == 1) {
    return set_error(HC_ERR_ARG, "hc_search: single_pass applies to the dense mode only");
  }
  const int bm_opt = o ? o->bitmap : 0;
  if (bm_opt < 0 || bm_opt > 1) return set_error(HC_ERR_ARG, "hc_search: bitmap must be 0 or 1");
  if (bm_opt == 1 && p.single_pass)
    return set_error(HC_ERR_ARG, "hc_search: the bitmap form and the single pass exclude each other");
  if (kind == HC_MODE_DENSE && !p.single_pass) {
    // one ring of `stages` buffers per warp
    p.bitmap = bm_opt == 1;
    p.scan = p.bitmap ? dense_kernel_for_q<true>(f->q) : dense_kernel_for_q<false>(f->q);
    // F is not staged; the spill form adds each warp's candidate queue
    p.smem_scan = size_t(kWarps) * stages * p.stage_bytes + (p.bitmap ? 0 : size_t(kWarps) * kQueueCap * 2);
    if (mode == HC_MODE_AUTO && p.smem_scan + static_smem(p.scan) > di.smem_optin) {
      kind = HC_MODE_STAGED;  // caller's lane_bytes too large for per-warp rings
      p.C = 32u * static_cast<uint32_t>(L);
      p.stage_bytes = stage_bytes_for(p.C, f->m, false);
      p.bitmap = false;
    }
  }
  if (bm_opt == 1 && !p.bitmap)
    return set_error(HC_ERR_ARG, "hc_search: the bitmap form applies to the dense mode only");
  p.kind = kind;
  const int sentinel = o ? o->sentinel : 0;
  if (sentinel < 0 || sentinel > 1) return set_error(HC_ERR_ARG, "hc_search: sentinel must be 0 or 1");
  if (sentinel == 1 && kind != HC_MODE_STAGED)
    return set_error(HC_ERR_ARG, "hc_search: the sentinel form applies to the staged mode only");
  if (kind == HC_MODE_STAGED && sentinel == 1) {
    // a lane's round of four first tests may reach three shifts past its
    // last window end (and the q-gram's three words 12 bytes further)
    p.stage_bytes += static_cast<uint32_t>((3 * shift + 16 + 15) & ~15);
    p.unchecked = true;
  }
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
  p.emit = p.bitmap ? emit_bitmap_kernel() : emit_kernel_for_q(f->q);
  p.smem_emit = p.bitmap ? 0 : (((f->F.size() + 3) & ~size_t(3)) * 4) + slot_bytes;
  // warp-speculative HC only on request: measured on GB300 it loses to the
  // per-lane form on every sweep cell (each first-test hit serialises the
  // warp), so the automatic choice is the per-lane form
  if (kind != HC_MODE_DENSE) p.spec = o != nullptr && o->speculate > 0;
  p.pos32 = o != nullptr && o->pos32 == 1;

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
  if (p.single_pass) {
    // chunk c holds window starts [cC - head, cC - head + C) (head = y mod
    // 16 < 16); a persistent grid of at most one wave of warps claims tiles
    const unsigned long long chunks = (nwin + 15 + p.C - 1) / p.C;
    p.max_tiles = (chunks + p.tile_chunks - 1) / p.tile_chunks;
    if (p.max_tiles >= (1ull << 30))
      return set_error(HC_ERR_ARG, "hc_search: text too long for the single-pass form (use single_pass = -1)");
    p.num_chunks = chunks;
    p.grid = std::min<unsigned long long>(static_cast<unsigned long long>(per_sm) * di.sm_count,
                                          (p.max_tiles + kWarps - 1) / kWarps);
    p.records = 0;
    p.emit = nullptr;
    p.emit_ctas = 0;
    // tile entries, group totals, group tree (nodes 0..G), tile counters
    const unsigned long long groups = (p.max_tiles + kSinglePassGroup - 1) / kSinglePassGroup;
    p.ws_bytes = (2 * groups + 1) * 8 + (p.max_tiles + kWarps) * 4;
    *out = p;
    return HC_OK;
  }
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
  if (p.bitmap) {
    // records' totals and overflow words, the CTAs' totals, then C / 8
    // bytes of window bits per chunk; the emit kernel has one warp per record
    p.region_entries = 0;
    p.emit_group = 0;
    p.emit_ctas = p.grid;
    p.bitmap_bytes = p.num_chunks * (p.C / 8);
    p.ws_bytes = ((p.records * 16 + p.grid * 8 + 15) & ~15ull) + p.bitmap_bytes;
    *out = p;
    return HC_OK;
  }
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
  p.ws_bytes = p.records * 16 + p.records * p.region_entries * 4 + p.grid * 8;
  *out = p;
  return HC_OK;
}

// Device address of g_status on the current device (looked up once per
// device; in host code the symbol's name is not a device address).
unsigned int* status_word() {
  static std::mutex mu;
  static std::map<int, unsigned int*> addr;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = addr.find(dev);
  if (it != addr.end()) return it->second;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  addr[dev] = static_cast<unsigned int*>(p);
  return static_cast<unsigned int*>(p);
}

void fill_args(const Filter* f, const SearchPlan& p, const uint8_t* y, size_t n, uint64_t* pos,
               size_t cap, uint64_t* count_dev, void* ws, void* args_out) {
  SearchArgs& a = *static_cast<SearchArgs*>(args_out);
  a = SearchArgs{};
  a.status = status_word();
  a.y = y;
  a.n = n;
  a.nwin = n - f->m + 1;
  a.F = f->dev_image ? f->dev_F() : nullptr;
  a.x = f->dev_image ? f->dev_x() : nullptr;
  a.fwords = static_cast<uint32_t>(f->F.size());
  a.m = static_cast<int>(f->m);
  a.q = f->q;
  a.s = f->s;
  a.mask = f->mask;
  a.hv = f->hv;
  a.pos = reinterpret_cast<unsigned long long*>(pos);
  a.cap = pos ? cap : 0;
  a.count_out = reinterpret_cast<unsigned long long*>(count_dev);
  if (p.single_pass) {
    const unsigned long long groups = (p.max_tiles + kSinglePassGroup - 1) / kSinglePassGroup;
    a.lb_gpack = static_cast<unsigned long long*>(ws);
    a.lb_gtree = a.lb_gpack + groups;
    a.lb_desc = reinterpret_cast<unsigned int*>(a.lb_gtree + groups + 1);
    a.lb_ticket = a.lb_desc + p.max_tiles;
    a.tile_chunks = p.tile_chunks;
    a.flag_steps = p.flag_steps;
  } else {
    a.cta_total = static_cast<unsigned long long*>(ws);
    a.cta_overflow = a.cta_total + p.records;
    a.region = reinterpret_cast<uint32_t*>(a.cta_overflow + p.records);
    // after the regions (R * S * 4 bytes, S a multiple of 4: 16-byte aligned)
    a.blk_total = reinterpret_cast<unsigned long long*>(a.region + p.records * p.region_entries);
    if (p.bitmap)
      a.bitmap = reinterpret_cast<uint16_t*>(static_cast<uint8_t*>(ws) + ((p.records * 16 + p.grid * 8 + 15) & ~15ull));
  }
  a.region_entries = p.region_entries;
  a.num_chunks = p.num_chunks;
  a.chunks_per_cta = p.chunks_per_cta;
  a.L = p.L;
  a.C = p.C;
  a.head = static_cast<int>(reinterpret_cast<uintptr_t>(y) & 15u);
  if (p.single_pass) {
    a.num_chunks = (a.nwin + static_cast<unsigned long long>(a.head) + p.C - 1) / p.C;
    a.num_tiles = (a.num_chunks + p.tile_chunks - 1) / p.tile_chunks;
    a.num_groups = (a.num_tiles + kSinglePassGroup - 1) / kSinglePassGroup;
  }
  a.stage_bytes = p.stage_bytes;
  a.x_smem = p.x_smem;
  a.stages = p.stages;
  a.records = p.records;
  a.spec = p.spec ? 1 : 0;
  a.unchecked = p.unchecked ? 1 : 0;
  a.pos32 = p.pos32 ? 1 : 0;
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

// Enqueues the kernels of one planned search: scan then emit (PDL), or for
// the single-pass form init then scan (PDL).
static int launch_args(const SearchPlan& p, const SearchArgs& a, cudaStream_t stream) {
  if (a.status == nullptr) return set_error(HC_ERR_CUDA, "device status word unavailable");
  const int kind = p.kind == HC_MODE_DENSE ? kKindScanDense
                   : (p.kind == HC_MODE_DIRECT ? kKindScanDirect : kKindScanStaged);
  cudaError_t e;
  if (p.single_pass) {
    const unsigned init_grid = static_cast<unsigned>(
        std::max<unsigned long long>(1, std::min<unsigned long long>((a.num_tiles + kThreads - 1) / kThreads, 1024)));
    TimingToken t0 = timing_begin(kKindInit, stream);
    p.init<<<init_grid, kThreads, 0, stream>>>(a);
    e = cudaGetLastError();
    timing_end(t0, stream);
    if (e != cudaSuccess) return cuda_error(e, "single-pass init launch");
    TimingToken t1 = timing_begin(kind, stream);
    e = launch_dependent(p.scan, static_cast<unsigned>(p.grid), kThreads, p.smem_scan, stream,
                         !t1.active(), a);
    if (e == cudaSuccess) e = cudaGetLastError();
    timing_end(t1, stream);
    g_launches.fetch_add(2);
    if (e != cudaSuccess) return cuda_error(e, "single-pass scan launch");
    return HC_OK;
  }
  TimingToken t0 = timing_begin(kind, stream);
  // a programmatic dependent of whatever kernel precedes it in the stream:
  // only this library's emit kernel lets a dependent start early, and the
  // scan waits for it before touching memory
  e = launch_dependent(p.scan, static_cast<unsigned>(p.grid), kThreads, p.smem_scan, stream,
                       !t0.active(), a);
  if (e == cudaSuccess) e = cudaGetLastError();
  timing_end(t0, stream);
  if (e != cudaSuccess) return cuda_error(e, "hc_scan_kernel launch");
  TimingToken t1 = timing_begin(kKindEmit, stream);
  e = launch_dependent(p.emit, static_cast<unsigned>(p.emit_ctas), kThreads, p.smem_emit, stream,
                       !t1.active(), a);
  if (e == cudaSuccess) e = cudaGetLastError();
  timing_end(t1, stream);
  g_launches.fetch_add(2);
  if (e != cudaSuccess) return cuda_error(e, "hc_emit_kernel launch");
  return HC_OK;
}

// Enqueues the kernels of one search with a caller-supplied workspace.
int launch_planned(const Filter* f, const SearchPlan& p, const uint8_t* y, size_t n, uint64_t* pos,
                   size_t cap, uint64_t* count_dev, void* ws, cudaStream_t stream) {
  SearchArgs a;
  fill_args(f, p, y, n, pos, cap, count_dev, ws, &a);
  return launch_args(p, a, stream);
}

// Enqueues the kernels of one search reading the filter words and the
// pattern from caller-supplied device copies instead of the filter's own.
int launch_planned_filter_ptrs(const Filter* f, const SearchPlan& p, const uint32_t* F_dev,
                               const uint8_t* x_dev, const uint8_t* y, size_t n, uint64_t* pos,
                               size_t cap, uint64_t* count_dev, void* ws, cudaStream_t stream) {
  SearchArgs a;
  fill_args(f, p, y, n, pos, cap, count_dev, ws, &a);
  a.F = F_dev;
  a.x = x_dev;
  return launch_args(p, a, stream);
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

int take_bound_violations_search(uint64_t* count) {
  *count = 0;
#ifdef HC_CHECKED
  unsigned long long v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_bound_violations, sizeof v);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bound_violations, &zero, sizeof zero);
  if (e != cudaSuccess) return cuda_error(e, "bound violation counter");
  *count = v;
  return HC_OK;
#else
  return HC_ERR_STATE;
#endif
}

}  // namespace hc

using namespace hc;

namespace {
int check_search_args(const char* who, Filter* f, const uint8_t* y_dev, size_t n,
                      const uint64_t* pos_dev, size_t cap, bool pos32 = false) {
  if (f == nullptr) return set_error(HC_ERR_ARG, std::string(who) + ": invalid filter");
  if (y_dev == nullptr && n > 0) return set_error(HC_ERR_ARG, std::string(who) + ": y_dev is NULL");
  if (pos_dev == nullptr && cap > 0)
    return set_error(HC_ERR_ARG, std::string(who) + ": pos_dev is NULL with cap > 0");
  if (pos32 ? (reinterpret_cast<uintptr_t>(pos_dev) & 3u) != 0 : !aligned8(pos_dev))
    return set_error(HC_ERR_ARG, std::string(who) + (pos32 ? ": pos_dev not 4-byte aligned" : ": pos_dev not 8-byte aligned"));
  if (pos32 && n >= f->m && n - f->m + 1 > (uint64_t(1) << 32))
    return set_error(HC_ERR_ARG, std::string(who) + ": uint32 positions need n - m + 1 <= 2^32");
  return HC_OK;
}
}  // namespace

extern "C" {

int hc_check_bounds(uint64_t* violations) {
  clear_error();
  if (violations == nullptr) return set_error(HC_ERR_ARG, "hc_check_bounds: violations is NULL");
  *violations = 0;
  uint64_t a = 0, b = 0, c = 0;
  int rc = take_bound_violations_search(&a);
  if (rc == HC_ERR_STATE) return set_error(HC_ERR_STATE, "hc_check_bounds: not a checked build");
  if (rc == HC_OK) rc = take_bound_violations_batch(&b);
  if (rc == HC_OK) rc = take_bound_violations_dense(&c);
  if (rc != HC_OK) return rc;
  *violations = a + b + c;
  return HC_OK;
}

int hc_search_ex(const hc_filter* fp, const uint8_t* y_dev, size_t n, uint64_t* pos_dev,
                 size_t cap, uint64_t* count_dev, const hc_search_opts* opts,
                 hc_stream_t stream) {
  clear_error();
  Filter* f = as_filter(fp);
  if (opts != nullptr && opts->struct_size != sizeof(hc_search_opts))
    return set_error(HC_ERR_ARG, "hc_search_ex: opts->struct_size mismatch");
  if (opts != nullptr && opts->pos32 != 0 && opts->pos32 != 1)
    return set_error(HC_ERR_ARG, "hc_search_ex: pos32 must be 0 or 1");
  int rc = check_search_args("hc_search_ex", f, y_dev, n, pos_dev, cap, opts != nullptr && opts->pos32 == 1);
  if (rc != HC_OK) return rc;
  if (count_dev == nullptr || !aligned8(count_dev))
    return set_error(HC_ERR_ARG, "hc_search_ex: count_dev is NULL or not 8-byte aligned");
  return launch_search(f, y_dev, n, pos_dev, cap, count_dev, opts,
                       reinterpret_cast<cudaStream_t>(stream));
}

int hc_search_async(const hc_filter* fp, const uint8_t* y_dev, size_t n, uint64_t* pos_dev,
                    size_t cap, uint64_t* count_dev, hc_stream_t stream) {
  clear_error();
  Filter* f = as_filter(fp);
  int rc = check_search_args("hc_search_async", f, y_dev, n, pos_dev, cap);
  if (rc != HC_OK) return rc;
  if (count_dev == nullptr || !aligned8(count_dev))
    return set_error(HC_ERR_ARG, "hc_search_async: count_dev is NULL or not 8-byte aligned");
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
