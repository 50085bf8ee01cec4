// hc_dense.cu -- single-pass HC search for m = q (Sec. 3.3, Fig. 5 left):
// the window is one q-gram, its back-walk is empty and every shift is one,
// so HC tests every window in turn and reports window w iff F[h(w)] != 0,
// h(w) = H_v and w = x.  Where w = x, h(w) = h(x), so the first two tests
// take the same value for every window that passes the third: the kernel
// evaluates F[h(x)] != 0 and h(x) = H_v once and compares the window bytes
// with x, 16 consecutive windows per lane with word-wide XOR/OR and an exact
// zero-byte test.
//
// Output in text order in one pass.  The window starts are cut into chunks
// of C starts (the bulk-copy unit) and tiles of tile_chunks consecutive
// chunks (the ordering unit).  A warp claims tiles from an atomic ticket, so
// tiles are claimed in text order by running warps; it streams each tile's
// chunks through its own ring of shared-memory buffers (1-D bulk copies on
// mbarriers) and keeps one 16-bit match mask per lane and 512-window step in
// shared memory.  At the end of a tile it publishes the tile's match count
// in the tile's descriptor, sums the counts of the tiles before it by a
// decoupled look-back (32 descriptors per read, stopping at the first tile
// whose inclusive count is known), publishes its own inclusive count and
// writes its positions straight to the output.  A tile only waits for tiles
// claimed before it, whose warps are running, so the waits always end; every
// wait is bounded all the same (a wait that gives up sets the status flag).
// The last tile writes the total count.  An init kernel, launched before the
// scan, zeroes the ticket and the descriptors; the scan is its programmatic
// dependent and waits for it before claiming a tile.
#include <cstdint>

#include "hc_device.cuh"
#include "hc_internal.h"
#include "hc_kernels.cuh"

namespace hc {

namespace {

// Tile descriptor: state in bits 62-63, count in bits 0-61.
constexpr unsigned long long kDescAggregate = 1ull << 62;  // the tile's own count
constexpr unsigned long long kDescInclusive = 2ull << 62;  // count of tiles 0..t
constexpr unsigned long long kDescCount = (1ull << 62) - 1;

// Zeroes the ticket and the tile descriptors of one single-pass search.
__global__ void __launch_bounds__(kThreads) hc_single_pass_init_kernel(const SearchArgs a) {
  pdl_launch_dependents();  // the scan may be scheduled; it waits for this grid
  const unsigned long long i0 = static_cast<unsigned long long>(blockIdx.x) * kThreads + threadIdx.x;
  const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * kThreads;
  if (i0 == 0) *a.lb_ticket = 0u;
  for (unsigned long long i = i0; i < a.num_tiles; i += stride) a.lb_desc[i] = 0ull;
}

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

// 16-bit mask, bit 4g + k set iff bit 8k + 7 of z[g] is set.
__device__ __forceinline__ uint32_t gather_mask(const uint32_t (&z)[4]) {
  uint32_t m = 0;
#pragma unroll
  for (int g = 0; g < 4; ++g) m |= (((z[g] >> 7) * 0x01020408u) >> 24) << (4 * g);
  return m;
}

}  // namespace

// ---------------------------------------------------------------------------
// The scan.  Warp-level worker: lane 0 claims tiles and drives the bulk
// copies; the warp tests 512 windows per step (16 per lane).  Shared
// memory per warp: `stages` staging buffers, then flag_steps * 32 masks.
template <int Q>
__global__ void __launch_bounds__(kThreads) hc_dense_single_pass_kernel(const SearchArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[kWarps][kMaxStages];
  __shared__ long long s_chunk[kWarps][kMaxStages];  // chunk in each buffer, -1: none

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nst = a.stages;
  const uint32_t C = a.C;
  const int steps_per_chunk = static_cast<int>(C >> 9);
  const int TC = a.tile_chunks;
  const int head = a.head;
  uint8_t* stages = smem + static_cast<size_t>(warp) * nst * a.stage_bytes;
  uint16_t* flags = reinterpret_cast<uint16_t*>(smem + static_cast<size_t>(kWarps) * nst * a.stage_bytes) +
                    static_cast<size_t>(warp) * a.flag_steps * 32;
  uint64_t* wb = bars[warp];
  long long* my_chunk = s_chunk[warp];

  // pattern byte c replicated into the 4 bytes of a word
  uint32_t xrep[Q];
  uint32_t xlo = 0, xhi = 0;
#pragma unroll
  for (int c = 0; c < Q; ++c) {
    const uint32_t xb = __ldg(a.x + c);
    xrep[c] = 0x01010101u * xb;
    if (c < 4) xlo |= xb << (8 * c); else xhi |= xb << (8 * (c - 4));
  }
  // HC's first test and H_v test, evaluated on x itself (see the file header)
  const uint32_t hx = hash_bytes<Q>(xlo, xhi, a);
  const bool filter_passes = __ldg(a.F + hx) != 0u && hx == a.hv;

  if (lane == 0) {
    for (int k = 0; k < nst; ++k) mbar_init(&wb[k], 1);
    fence_mbar_init();
  }
  __syncwarp();
  pdl_wait();  // the init kernel has zeroed the ticket and the descriptors

  // Lane 0's claim state: tile being staged (cur_t, chunk cur_k of cur_nk)
  // and the next tile, claimed one tile ahead so that the atomic's latency
  // is hidden.  A warp processes its tiles in the order it claims them.
  long long cur_t = -1, res_t = -1;
  int cur_k = 0, cur_nk = 0;
  const long long num_tiles = static_cast<long long>(a.num_tiles);
  const long long num_chunks = static_cast<long long>(a.num_chunks);
  auto tile_chunks = [&](long long t) { return static_cast<int>(min(static_cast<long long>(TC), num_chunks - t * TC)); };
  auto next_chunk = [&]() -> long long {
    if (cur_t < 0) return -1;
    if (cur_k == cur_nk) {
      cur_t = res_t;
      if (cur_t >= num_tiles) {
        cur_t = -1;
        return -1;
      }
      cur_k = 0;
      cur_nk = tile_chunks(cur_t);
      res_t = static_cast<long long>(atomicAdd(a.lb_ticket, 1u));
    }
    return cur_t * TC + cur_k++;
  };
  // stages chunk c (window starts [cC - head, cC - head + C)) in buffer st;
  // the copy starts at the 16-byte aligned text address y - head + cC
  auto issue = [&](int st, long long c) {
    my_chunk[st] = c;
    if (c < 0) return;
    const unsigned long long cs = static_cast<unsigned long long>(c) * C;
    const unsigned long long avail = a.n + static_cast<unsigned long long>(head) - cs;
    const unsigned long long len = min(static_cast<unsigned long long>(C) + a.m - 1, avail);
    const uint32_t bytes = static_cast<uint32_t>((len + 15) & ~15ull);
    mbar_arrive_expect_tx(&wb[st], bytes);
    bulk_copy_g2s(stages + static_cast<size_t>(st) * a.stage_bytes, a.y - head + cs, bytes, &wb[st]);
  };
  if (lane == 0) {
    cur_t = static_cast<long long>(atomicAdd(a.lb_ticket, 1u));
    res_t = static_cast<long long>(atomicAdd(a.lb_ticket, 1u));
    if (cur_t >= num_tiles) cur_t = -1;
    else cur_nk = tile_chunks(cur_t);
    for (int k = 0; k < nst; ++k) issue(k, next_chunk());
  }
  __syncwarp();

  uint32_t lane_cnt = 0;      // matches of this lane in the current tile
  unsigned long long stepbits = 0;  // steps of the current tile with a match
  int single_left = 0;        // chunks left in the one-stage byte test (Q >= 5)
  bool ok = true;
  bool refilled = false;  // a failed look-back left buffer st refilled
  int st = 0;
  uint32_t phase = 0;
  for (;; st = (st + 1 == nst) ? 0 : st + 1, phase ^= (st == 0) ? 1u : 0u) {
    const long long c = my_chunk[st];
    if (c < 0) break;
    ok = __all_sync(0xffffffffu, mbar_wait_bounded(&wb[st], phase));
    if (!ok) break;
    const long long t = c / TC;
    const int k = static_cast<int>(c - t * TC);
    if (k == 0) {
      lane_cnt = 0;
      stepbits = 0;
    }
    const uint8_t* sb = stages + static_cast<size_t>(st) * a.stage_bytes;
    // window starts of this chunk that exist: [vlo, vhi) relative to cC - head
    const long long cw0 = c * static_cast<long long>(C) - head;
    const int vlo = cw0 < 0 ? static_cast<int>(-cw0) : 0;
    const long long rem = static_cast<long long>(a.nwin) - cw0;
    const int vhi = rem < static_cast<long long>(C) ? static_cast<int>(rem) : static_cast<int>(C);
    const bool edge = vlo > 0 || vhi < static_cast<int>(C);
    const bool two = Q >= 5 && single_left == 0;
    int second = 0;  // steps that needed the second stage
    for (int j = 0; j < steps_per_chunk && (j << 9) < vhi; ++j) {
      const int w0 = (j << 9) + 16 * lane;  // buffer offset of the lane's first window
      uint32_t Tw[6];
      if (HC_IN_BOUNDS(static_cast<uint32_t>(w0) + 24u <= a.stage_bytes)) {
        const uint4 A = *reinterpret_cast<const uint4*>(sb + w0);
        const uint2 B = *reinterpret_cast<const uint2*>(sb + w0 + 16);
        Tw[0] = A.x; Tw[1] = A.y; Tw[2] = A.z; Tw[3] = A.w; Tw[4] = B.x; Tw[5] = B.y;
      } else {
#pragma unroll
        for (int u = 0; u < 6; ++u) Tw[u] = ~0u;
      }
      uint32_t d[4] = {0u, 0u, 0u, 0u};
      uint32_t z[4];
      bool any;
      if (two) {
        or_columns<Q, 1, 0, 0>(Tw, xrep, d);
        const uint32_t cand = has_zero_byte(d[0]) | has_zero_byte(d[1]) | has_zero_byte(d[2]) | has_zero_byte(d[3]);
        if (__ballot_sync(0xffffffffu, cand != 0u) == 0u) continue;
        ++second;
        or_columns<Q, 2, 0, 0>(Tw, xrep, d);
#pragma unroll
        for (int g = 0; g < 4; ++g) z[g] = zero_bytes(d[g]);
        any = true;
      } else {
        or_columns<Q, 0, 0, 0>(Tw, xrep, d);
#pragma unroll
        for (int g = 0; g < 4; ++g) z[g] = zero_bytes(d[g]);
        any = __ballot_sync(0xffffffffu, (z[0] | z[1] | z[2] | z[3]) != 0u) != 0u;
      }
      if (!any) continue;
      uint32_t m16 = gather_mask(z);
      if (edge) {
        const int lo = max(vlo - w0, 0), hi = min(vhi - w0, 16);
        m16 = hi > lo ? m16 & (0xffffu >> (16 - hi)) & (0xffffu << lo) : 0u;
      }
      if (!filter_passes) m16 = 0u;
      if (__ballot_sync(0xffffffffu, m16 != 0u) == 0u) continue;
      const int s = k * steps_per_chunk + j;  // step within the tile
      if (HC_IN_BOUNDS(s < a.flag_steps)) flags[s * 32 + lane] = static_cast<uint16_t>(m16);
      lane_cnt += static_cast<uint32_t>(__popc(m16));
      stepbits |= 1ull << s;
    }
    if (Q >= 5) {
      // the two-stage test pays off only while its first stage rejects most
      // steps; otherwise use the one-stage test for the next 16 chunks
      if (two && 2 * second > steps_per_chunk) single_left = 16;
      else if (!two) --single_left;
    }
    __syncwarp();  // buffer st is free again: stage the warp's next chunk in it
    if (lane == 0) {
      fence_proxy_async_smem();
      issue(st, next_chunk());
    }
    __syncwarp();
    if (k + 1 < tile_chunks(t)) continue;

    // ---- the tile is scanned: publish, look back, write ----
    const unsigned long long agg = warp_sum_u64(static_cast<unsigned long long>(lane_cnt));
    if (lane == 0)
      st_relaxed_u64(a.lb_desc + t, (t == 0 ? kDescInclusive : kDescAggregate) | agg);
    unsigned long long excl = 0;
    if (t > 0) {
      long long top = t - 1;  // lane l reads descriptor top - l
      uint64_t t0 = 0;        // start of the current wait
      uint32_t spins = 0;     // reads of the current wait
      for (;;) {
        const long long idx = top - lane;
        unsigned long long dsc = kDescInclusive;  // before tile 0: inclusive count 0
        if (idx >= 0) dsc = ld_relaxed_u64(a.lb_desc + idx);
        const unsigned incl_lanes = __ballot_sync(0xffffffffu, (dsc >> 62) == 2ull);
        const unsigned empty_lanes = __ballot_sync(0xffffffffu, (dsc >> 62) == 0ull);
        // lanes up to and including the nearest inclusive descriptor
        const unsigned need = incl_lanes ? ((incl_lanes & (0u - incl_lanes)) << 1) - 1u : 0xffffffffu;
        if ((empty_lanes & need) == 0u) {
          const unsigned long long v = ((need >> lane) & 1u) ? (dsc & kDescCount) : 0ull;
          excl += warp_sum_u64(v);
          if (incl_lanes) break;
          top -= 32;
          spins = 0;
          continue;
        }
        // a tile claimed earlier has not published its count yet: wait
        // (bounded; give up at once if another wait already gave up)
        if (spins++ == 0) t0 = global_timer_ns();
        bool give_up = false;
        if ((spins & 63u) == 0u) {
          give_up = global_timer_ns() - t0 > kWaitLimitNs || spins >= kMaxSpins ||
                    (ld_relaxed_u32(a.status) & 1u) != 0u;
        }
        if (__any_sync(0xffffffffu, give_up)) {
          if (lane == 0) atomicOr(a.status, 1u);
          ok = false;
          refilled = true;  // buffer st already holds the next chunk
          break;
        }
      }
      if (lane == 0) st_relaxed_u64(a.lb_desc + t, kDescInclusive | (excl + agg));
    }
    if (t == num_tiles - 1 && lane == 0) *a.count_out = excl + agg;

    // positions of the tile, in text order: steps, then lanes, then windows
    const long long tile_w0 = t * TC * static_cast<long long>(C) - head;
    unsigned long long run = excl;
    for (unsigned long long sbits = stepbits; sbits; sbits &= sbits - 1) {
      const int s = __ffsll(static_cast<long long>(sbits)) - 1;
      uint32_t m16 = HC_IN_BOUNDS(s < a.flag_steps) ? flags[s * 32 + lane] : 0u;
      const uint32_t mine = static_cast<uint32_t>(__popc(m16));
      const uint32_t incl = warp_incl_scan_u32(mine);
      unsigned long long o = run + (incl - mine);
      const unsigned long long pbase = static_cast<unsigned long long>(tile_w0 + (static_cast<long long>(s) << 9) + 16 * lane);
      for (; m16; m16 &= m16 - 1u, ++o) {
        if (o >= a.cap) break;
        const unsigned long long p = pbase + static_cast<unsigned>(__ffs(m16) - 1);
        if (a.pos32) reinterpret_cast<uint32_t*>(a.pos)[o] = static_cast<uint32_t>(p);
        else a.pos[o] = p;
      }
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (!ok) break;
    __syncwarp();  // the flag buffer is free for the next tile
  }

  if (!ok) {
    if (lane == 0) {
      atomicOr(a.status, 1u);
      // let the copies still in flight land before the CTA's shared memory
      // goes: the buffers from the oldest unconsumed one on
      int s0 = st;
      uint32_t p0 = phase;
      if (refilled) {
        s0 = (st + 1 == nst) ? 0 : st + 1;
        p0 ^= (s0 == 0) ? 1u : 0u;
      }
      for (int u = 0; u < nst; ++u) {
        const int sx = (s0 + u) % nst;
        const uint32_t px = p0 ^ ((s0 + u) >= nst ? 1u : 0u);
        if (my_chunk[sx] >= 0) (void)mbar_wait_bounded(&wb[sx], px);
      }
    }
  }
  __syncwarp();
  if (lane == 0 && ok)
    for (int k = 0; k < nst; ++k) mbar_inval(&wb[k]);
}

KernelFn dense_single_pass_kernel_for_q(int q) {
  switch (q) {
    case 1: return hc_dense_single_pass_kernel<1>;
    case 2: return hc_dense_single_pass_kernel<2>;
    case 3: return hc_dense_single_pass_kernel<3>;
    case 4: return hc_dense_single_pass_kernel<4>;
    case 5: return hc_dense_single_pass_kernel<5>;
    case 6: return hc_dense_single_pass_kernel<6>;
    case 7: return hc_dense_single_pass_kernel<7>;
    default: return hc_dense_single_pass_kernel<8>;
  }
}

KernelFn single_pass_init_kernel() { return hc_single_pass_init_kernel; }

}  // namespace hc
