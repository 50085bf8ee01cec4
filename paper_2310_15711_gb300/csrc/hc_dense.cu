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
// chunks (the ordering unit).  Warps claim tiles from atomic counters, in
// about text order, by running warps; a warp streams each tile's
// chunks through its own ring of shared-memory buffers (1-D bulk copies on
// mbarriers) and keeps one 16-bit match mask per lane and 512-window step in
// shared memory.  At the end of a tile it adds the tile's match count to the
// nodes of a Fenwick tree over the tiles (each node also counts the tiles
// added to it), reads the popcount(t) nodes that together cover tiles 0..t-1
// -- one round of loads, waiting only until those nodes are complete -- and
// writes its positions straight to the output.  A tile only waits for tiles
// claimed before it, whose warps are running, so the waits end; every wait
// is bounded all the same (a wait that gives up sets the status flag).  The
// last tile writes the total count.  An init kernel, launched before the
// scan, zeroes the ticket and the tree; the scan is its programmatic
// dependent and waits for it before claiming a tile.
//
// (A chain of per-tile descriptors -- the usual decoupled look-back -- was
// measured first: when thousands of warps finish their tiles at about the
// same time, the inclusive counts travel along the chain a few hundred
// tiles per read, which made the scan up to twice as slow; the tree needs
// one read of at most log2(T) nodes.)
#include <cstdint>

#include "hc_device.cuh"
#include "hc_internal.h"
#include "hc_kernels.cuh"

namespace hc {

namespace {

// Tile counters (see claim() in the scan): one per warp of a CTA.
constexpr int kTicketCounters = kWarps;
// Tiles per group (the group's total is one hot counter of this many adds).
constexpr unsigned int kGroupTiles = static_cast<unsigned int>(kSinglePassGroup);

// Counts of the tiles: tile t's entry holds its match count (bits 0-30,
// at most 32768 windows per tile) and a ready bit (31); a group's total and
// a node of the group tree hold the tiles (groups) added in bits 40-63 and
// their matches in bits 0-39.
constexpr unsigned int kTileReady = 1u << 31;
constexpr int kAddedShift = 40;
constexpr unsigned long long kOneAdded = 1ull << kAddedShift;
constexpr unsigned long long kCountBits = kOneAdded - 1;

// Zeroes the tile counters, the tile entries, the group totals and the
// group tree of one single-pass search.
__global__ void __launch_bounds__(kThreads) hc_single_pass_init_kernel(const SearchArgs a) {
  pdl_launch_dependents();  // the scan may be scheduled; it waits for this grid
  const unsigned long long i0 = static_cast<unsigned long long>(blockIdx.x) * kThreads + threadIdx.x;
  const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * kThreads;
  if (i0 < kTicketCounters) a.lb_ticket[i0] = 0u;
  for (unsigned long long i = i0; i < a.num_tiles; i += stride) a.lb_desc[i] = 0u;
  for (unsigned long long i = i0; i < a.num_groups; i += stride) a.lb_gpack[i] = 0ull;
  for (unsigned long long i = i0; i <= a.num_groups; i += stride) a.lb_gtree[i] = 0ull;
}

}  // namespace

// ---------------------------------------------------------------------------
// The scan.  Warp-level worker: lane 0 claims tiles and drives the bulk
// copies; the warp tests 512 windows per step (16 per lane).  Shared
// memory per warp: `stages` staging buffers, then 2 * flag_steps * 32 masks.
template <int Q>
__global__ void __launch_bounds__(kThreads, 4) hc_dense_single_pass_kernel(const SearchArgs a) {
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
                    static_cast<size_t>(warp) * 2 * a.flag_steps * 32;
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

  // Lane 0's claim state: the tile being staged (cur_t, its chunk cur_k of
  // cur_nk) and the next one, claimed when the last chunk of the current
  // tile is staged and first used at the next staging, so the atomic's
  // latency overlaps the scan of a chunk.  Every tile is thus claimed about
  // the same time (the ring's depth plus one chunk) before its scan begins,
  // and tiles are scanned in about the order they are claimed: a tile's
  // look-back seldom waits for a tile claimed long before it.
  int cur_t = -1, next_t = -1;
  int cur_k = 0, cur_nk = 0;
  const long long num_tiles = static_cast<long long>(a.num_tiles);
  const long long num_chunks = static_cast<long long>(a.num_chunks);
  auto tile_chunks = [&](long long t) { return static_cast<int>(min(static_cast<long long>(TC), num_chunks - t * TC)); };
  // Tiles are handed out by kTicketCounters counters, counter j (the warp's
  // index in its CTA) giving tiles j, j + kTicketCounters, ... in order:
  // each counter sees a few atomics per microsecond, where one counter for
  // the whole grid made the claims queue (the latency of an atomic on one
  // hot address grows with the rate).  A tile still waits only for lower
  // tiles, each of which is claimed, or will be claimed, by a warp that is
  // not waiting for a higher tile.
  auto claim = [&]() -> int {
    const unsigned int r = atomicAdd(a.lb_ticket + warp, 1u);
    return static_cast<int>(min(r * kTicketCounters + warp, 0x7fffffffu));
  };
  auto next_chunk = [&]() -> long long {
    if (cur_t < 0) return -1;
    if (cur_k == cur_nk) {
      cur_t = next_t;
      if (cur_t >= num_tiles) {
        cur_t = -1;
        return -1;
      }
      cur_k = 0;
      cur_nk = tile_chunks(cur_t);
    }
    const long long c = static_cast<long long>(cur_t) * TC + cur_k++;
    if (cur_k == cur_nk) next_t = claim();
    return c;
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
    cur_t = claim();
    if (cur_t >= num_tiles) cur_t = -1;
    else cur_nk = tile_chunks(cur_t);
    for (int k = 0; k < nst; ++k) issue(k, next_chunk());
  }
  __syncwarp();

  uint32_t lane_cnt = 0;            // matches of this lane in the current tile
  unsigned long long stepbits = 0;  // steps of the current tile with a match
  int single_left = 0;              // chunks left in the one-stage byte test (Q >= 5)
  bool ok = true;
  bool refilled = false;            // a wait gave up after buffer st was refilled
  int st = 0;
  uint32_t phase = 0;
  int fb = 0;                       // flag buffer of the current tile (two per warp)
  const int fstride = a.flag_steps * 32;
  // The pending tile: scanned, its count added to the tree, its positions
  // not yet written.  Its prefix is read without waiting while the next
  // tile is scanned, and its positions are written as soon as the prefix is
  // complete -- at the latest when the next tile is scanned, before that
  // tile's buffer is needed again.
  int p_t = -1;                     // its index (-1: none)
  int p_fb = 0;
  unsigned long long p_bits = 0, p_agg = 0;
  // this lane's part of the pending tile's prefix: the entries of tiles
  // base + lane and base + 32 + lane of its group (those below it), and one
  // node of the group tree
  unsigned int p_va = 0, p_vb = 0, p_node = 0;
  unsigned long long p_vc = 0;
  bool p_ha = false, p_hb = false, p_hc = false;
  // lane 0: the group total returned by the last tile's atomic add, to be
  // examined (its latency overlaps a chunk's scan): if that tile completed
  // its group, the group goes into the group tree
  bool g_pending = false;
  unsigned long long g_old = 0, g_agg = 0;
  unsigned int g_idx = 0, g_size = 0;

  // Writes the positions of tile pt (masks in flag buffer pfb, steps pbits),
  // after `excl` earlier occurrences, in text order: steps, lanes, windows.
  auto write_tile = [&](long long pt, int pfb, unsigned long long pbits, unsigned long long excl) {
    const uint16_t* fl = flags + pfb * fstride;
    const long long tile_w0 = pt * TC * static_cast<long long>(C) - head;
    unsigned long long run = excl;
    for (unsigned long long sbits = pbits; sbits; sbits &= sbits - 1) {
      const int s = __ffsll(static_cast<long long>(sbits)) - 1;
      uint32_t m16 = HC_IN_BOUNDS(s < a.flag_steps) ? fl[s * 32 + lane] : 0u;
      const uint32_t mine = static_cast<uint32_t>(__popc(m16));
      const uint32_t incl = warp_incl_scan_u32(mine);
      unsigned long long o = run + (incl - mine);
      const unsigned long long pbase =
          static_cast<unsigned long long>(tile_w0 + (static_cast<long long>(s) << 9) + 16 * lane);
      for (; m16; m16 &= m16 - 1u, ++o) {
        if (o >= a.cap) break;
        const unsigned long long pos = pbase + static_cast<unsigned>(__ffs(m16) - 1);
        if (a.pos32) reinterpret_cast<uint32_t*>(a.pos)[o] = static_cast<uint32_t>(pos);
        else a.pos[o] = pos;
      }
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
  };
  // The occurrences before tile t (group g = t / kGroupTiles) are those of
  // the groups before g -- the group-tree nodes g, g - lowbit(g), ..., one
  // per set bit of g, complete when all lowbit(node) groups have been added
  // -- plus those of the tiles of group g below t, each ready once its entry
  // is written.  All of them were claimed before t by running warps, so a
  // wait for them ends.  Lane k reads the k-th node and two tile entries:
  // one round of loads.
  auto start_prefix = [&](long long t) {
    const unsigned int ut = static_cast<unsigned int>(t);
    const unsigned int g = ut / kGroupTiles, base = g * kGroupTiles;
    const int nt = static_cast<int>(ut - base);
    const int nodes = __popc(g);
    unsigned int node = g;
    for (int k = 0; k < lane && k < nodes; ++k) node &= node - 1;
    p_ha = lane < nt;
    p_hb = lane + 32 < nt;
    p_hc = lane < nodes;
    p_node = node;
    p_va = p_ha ? ld_relaxed_u32(a.lb_desc + base + lane) : 0u;
    p_vb = p_hb ? ld_relaxed_u32(a.lb_desc + base + 32 + lane) : 0u;
    p_vc = p_hc ? ld_relaxed_u64(a.lb_gtree + node) : 0ull;
  };
  auto lane_complete = [&]() -> bool {
    return (!p_ha || (p_va & kTileReady)) && (!p_hb || (p_vb & kTileReady)) &&
           (!p_hc || (p_vc >> kAddedShift) == (p_node & (0u - p_node)));
  };
  auto reload = [&]() {
    const unsigned int base = static_cast<unsigned int>(p_t) / kGroupTiles * kGroupTiles;
    if (p_ha && !(p_va & kTileReady)) p_va = ld_relaxed_u32(a.lb_desc + base + lane);
    if (p_hb && !(p_vb & kTileReady)) p_vb = ld_relaxed_u32(a.lb_desc + base + 32 + lane);
    if (p_hc && (p_vc >> kAddedShift) != (p_node & (0u - p_node))) p_vc = ld_relaxed_u64(a.lb_gtree + p_node);
  };
  // true when the pending tile's prefix is complete; else the incomplete
  // parts are loaded again (no waiting)
  auto prefix_ready = [&]() -> bool {
    const bool complete = lane_complete();
    if (__all_sync(0xffffffffu, complete)) return true;
    if (!complete) reload();
    return false;
  };
  // lane 0: adds a group completed by this warp's last tile to the group
  // tree (nodes g+1, g+1+lowbit, ... <= number of groups)
  auto push_group = [&]() {
    if (lane == 0 && g_pending) {
      g_pending = false;
      if ((g_old >> kAddedShift) + 1 == g_size) {
        const unsigned long long add = kOneAdded | ((g_old & kCountBits) + g_agg);
        for (unsigned int i = g_idx + 1; i <= static_cast<unsigned int>(a.num_groups); i += i & (0u - i))
          atomicAdd(a.lb_gtree + i, add);
      }
    }
  };
  // waits until the pending tile's prefix is complete (bounded, a short
  // sleep between reads; given up at once if another wait already gave up);
  // false if the wait gave up
  auto wait_prefix = [&]() -> bool {
    push_group();  // a warp never waits while a group it completed is not in the tree
    bool complete = lane_complete();
    if (__all_sync(0xffffffffu, complete)) return true;
    const uint64_t t0 = global_timer_ns();
    bool give_up = false;
    for (uint32_t spins = 1; !complete && !give_up; ++spins) {
      __nanosleep(64);
      reload();
      complete = lane_complete();
      if (!complete && (spins & 15u) == 0u)
        give_up = global_timer_ns() - t0 > kWaitLimitNs || spins >= kMaxSpins ||
                  (ld_relaxed_u32(a.status) & 1u) != 0u;
    }
    if (__any_sync(0xffffffffu, give_up)) {
      if (lane == 0) atomicOr(a.status, 1u);
      return false;
    }
    return true;
  };
  // writes the pending tile (its prefix complete) and the total after the
  // last tile
  auto finish_pending = [&]() {
    const unsigned long long excl = warp_sum_u64(static_cast<unsigned long long>(p_va & ~kTileReady) +
                                                 (p_vb & ~kTileReady) + (p_vc & kCountBits));
    if (p_t == num_tiles - 1 && lane == 0) *a.count_out = excl + p_agg;
    write_tile(p_t, p_fb, p_bits, excl);
    p_t = -1;
  };

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
    uint16_t* cur_flags = flags + fb * fstride;
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
      if (HC_IN_BOUNDS(s < a.flag_steps)) cur_flags[s * 32 + lane] = static_cast<uint16_t>(m16);
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
    push_group();
    // the pending tile's positions, once its prefix is complete
    if (p_t >= 0 && prefix_ready()) finish_pending();
    if (k + 1 < tile_chunks(t)) continue;

    // ---- tile t is scanned: its count into its entry and its group ----
    const unsigned long long agg = warp_sum_u64(static_cast<unsigned long long>(lane_cnt));
    if (lane == 0) {
      st_relaxed_u32(a.lb_desc + t, kTileReady | static_cast<unsigned int>(agg));
      g_idx = static_cast<unsigned int>(t) / kGroupTiles;
      g_size = static_cast<unsigned int>(min(static_cast<unsigned long long>(kGroupTiles), a.num_tiles - static_cast<unsigned long long>(g_idx) * kGroupTiles));
      g_agg = agg;
      g_old = atomicAdd(a.lb_gpack + g_idx, kOneAdded | agg);
      g_pending = true;
    }
    // the next tile takes the pending tile's flag buffer: write that one first
    if (p_t >= 0) {
      if (!wait_prefix()) {
        ok = false;
        refilled = true;
        break;
      }
      finish_pending();
    }
    p_t = t;
    p_fb = fb;
    p_bits = stepbits;
    p_agg = agg;
    start_prefix(t);
    fb ^= 1;
    __syncwarp();
  }
  push_group();
  if (ok && p_t >= 0) {
    if (wait_prefix()) finish_pending();
    else ok = false;  // every chunk was consumed: no copy is in flight
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

// ---------------------------------------------------------------------------
// Emit of the dense scan's bitmap form: the scan's warp r (record r) has set
// bit j of group g for each occurrence at window 16g + j of its chunks and
// written its total; warp r of this grid writes record r's positions.  Its
// output offset is the sum of the totals before it: one total per earlier
// CTA of the scan (blk_total) plus the earlier warps of its own CTA.  It then
// walks the record's bits in text order, 1024 windows per round (one 32-bit
// word per lane; the words of kBitmapWords rounds are loaded at once, those
// of the next kBitmapWords rounds requested before these run, and a round
// without a set bit costs one vote): a warp scan of the words'
// popcounts gives each lane its first slot, the lane writes its window
// starts into the warp's shared-memory buffer in order, and the warp copies
// the buffer to the output with consecutive stores.  (Splitting a record's
// chunks over the 8 warps of a CTA, with per-chunk counts from the scan,
// measured slower on GB300 for the patterns this form serves: those with
// many occurrences, where every round has bits.)
namespace {
constexpr int kBitmapWords = 4;
constexpr int kBitmapRound = 1024;  // windows per round (32 lanes x 32 bits)
}  // namespace

__global__ void __launch_bounds__(kThreads, 4) hc_emit_bitmap_kernel(const SearchArgs a) {
  // per warp: a round's window starts, from slot `ph` on (ph < 4: the
  // output's misalignment, so that buffer slot i pairs with an output
  // element of the same 16-byte alignment)
  __shared__ __align__(16) uint32_t s_buf[kWarps][kBitmapRound + 4];
  __shared__ unsigned long long s_red[kWarps];
  pdl_launch_dependents();  // the next search's scan may be scheduled; it waits for this grid
  pdl_wait();               // the scan grid has completed: its bits and totals are visible
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long p = 0;
  for (unsigned long long k = tid; k < blockIdx.x; k += kThreads) p += a.blk_total[k];
  p = warp_sum_u64(p);
  if (lane == 0) s_red[warp] = p;
  __syncthreads();
  const unsigned long long rb = static_cast<unsigned long long>(blockIdx.x) * kWarps;
  unsigned long long P = 0;
  for (int w = 0; w < kWarps; ++w) P += s_red[w];
  for (int w = 0; w < warp; ++w) P += a.cta_total[rb + w];
  const unsigned long long r = rb + warp;
  const unsigned long long T = a.cta_total[r];
  if (r + 1 == a.records && lane == 0) *a.count_out = P + T;
  const unsigned long long c0 = r * a.chunks_per_cta;
  const unsigned long long c1 = min(c0 + a.chunks_per_cta, a.num_chunks);
  if (T == 0 || c0 >= c1 || P >= a.cap) return;
  const unsigned long long W0 = c0 * a.C;              // a multiple of 256
  const unsigned long long W1 = min(c1 * a.C, a.nwin);
  const unsigned long long end = min(P + T, a.cap);    // output slots of this record
  const uint32_t* bits = reinterpret_cast<const uint32_t*>(a.bitmap);
  uint32_t* buf = s_buf[warp];
  const unsigned long long step = static_cast<unsigned long long>(kBitmapRound) * kBitmapWords;
  // the lane's words of the kBitmapWords rounds from window w on (0 past W1)
  auto load_block = [&](unsigned long long w, uint32_t (&dst)[kBitmapWords]) {
#pragma unroll
    for (int u = 0; u < kBitmapWords; ++u) {
      const unsigned long long wl = w + static_cast<unsigned long long>(u * 32 + lane) * 32;
      dst[u] = 0u;
      if (wl < W1 && HC_IN_BOUNDS(wl / 32 < a.num_chunks * (a.C / 32))) dst[u] = __ldcs(bits + wl / 32);
    }
  };
  uint32_t nv[kBitmapWords];
  load_block(W0, nv);
  for (unsigned long long w = W0; w < W1 && P < end; w += step) {
    uint32_t v[kBitmapWords];
#pragma unroll
    for (int u = 0; u < kBitmapWords; ++u) v[u] = nv[u];
    // the next block's words are requested before this block's rounds run
    if (w + step < W1) load_block(w + step, nv);
#pragma unroll
    for (int u = 0; u < kBitmapWords; ++u) {
      // bits of windows at or past W1 are cleared: the scan leaves the groups
      // past the last window of the text unwritten
      const unsigned long long wl = w + static_cast<unsigned long long>(u * 32 + lane) * 32;
      if (wl < W1 && W1 - wl < 32) v[u] &= (1u << (W1 - wl)) - 1u;
    }
#pragma unroll
    for (int u = 0; u < kBitmapWords; ++u) {
      if (!__any_sync(0xffffffffu, v[u] != 0u)) continue;
      const uint32_t cnt = static_cast<uint32_t>(__popc(v[u]));
      const uint32_t incl = warp_incl_scan_u32(cnt);
      const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      // window of this lane's bit 0, counted from W0 (< 2^32: a record's
      // windows are fewer than 2^32)
      const uint32_t rel = static_cast<uint32_t>(w - W0) + static_cast<uint32_t>(u * 32 + lane) * 32u;
      // output element P + j goes to buffer slot ph + j, where ph aligns
      // the slots with the output's 16-byte blocks (4 u32 or 2 u64 each)
      const uintptr_t oaddr = reinterpret_cast<uintptr_t>(a.pos);
      const uint32_t ph = a.pos32 ? static_cast<uint32_t>(((oaddr >> 2) + P) & 3u)
                                  : static_cast<uint32_t>(((oaddr >> 3) + P) & 1u);
      uint32_t o = ph + incl - cnt, b = v[u];
      while (b) {
        if (HC_IN_BOUNDS(o < static_cast<uint32_t>(kBitmapRound + 4))) buf[o] = rel + static_cast<uint32_t>(__ffs(b) - 1);
        ++o;
        b &= b - 1u;
      }
      __syncwarp();
      const uint32_t lim = static_cast<uint32_t>(min(static_cast<unsigned long long>(tot), end - P));
      const uint32_t last = ph + lim;  // slots [ph, last) are written out
      if (a.pos32) {
        // 16-byte stores of four positions where a block lies inside
        // [ph, last), 4-byte stores at the two ends
        uint32_t* out = reinterpret_cast<uint32_t*>(a.pos);
        const uint32_t b32 = static_cast<uint32_t>(W0);
        for (uint32_t k = lane; 4 * k < last; k += 32) {
          const uint32_t i0 = 4 * k;
          if (i0 >= ph && i0 + 4 <= last) {
            uint4 w = *reinterpret_cast<const uint4*>(buf + i0);
            w.x += b32; w.y += b32; w.z += b32; w.w += b32;
            *reinterpret_cast<uint4*>(out + (P + i0 - ph)) = w;
          } else {
            for (uint32_t i = max(i0, ph); i < min(i0 + 4, last); ++i) out[P + i - ph] = b32 + buf[i];
          }
        }
      } else {
        unsigned long long* out = a.pos;
        for (uint32_t k = lane; 2 * k < last; k += 32) {
          const uint32_t i0 = 2 * k;
          if (i0 >= ph && i0 + 2 <= last) {
            const uint2 w = *reinterpret_cast<const uint2*>(buf + i0);
            *reinterpret_cast<ulonglong2*>(out + (P + i0 - ph)) = make_ulonglong2(W0 + w.x, W0 + w.y);
          } else {
            for (uint32_t i = max(i0, ph); i < min(i0 + 2, last); ++i) out[P + i - ph] = W0 + buf[i];
          }
        }
      }
      __syncwarp();  // the buffer is free again
      P += tot;
      if (P >= end) break;
    }
  }
}

KernelFn emit_bitmap_kernel() { return hc_emit_bitmap_kernel; }

// This translation unit's bound-violation counter (checked build).
int take_bound_violations_dense(uint64_t* count) {
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
