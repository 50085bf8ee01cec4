// hc_search.cu -- the HC searching phase (Sec. 3.3, Fig. 5 left, with the H_v
// early reject of Sec. 3.4) on sm_103a.
//
// Decomposition.  The window starts [0, n-m] are cut into chunks of C = 256*L
// consecutive starts; chunk k reads text bytes [kC, kC + C + m - 1).  A
// persistent grid of CTAs claims chunks in increasing order from an atomic
// counter.  Each CTA keeps F (2^alpha words) and x in shared memory and
// double-buffers its chunks: while it scans one chunk, the next one is
// already in flight from HBM into shared memory as a 1-D bulk copy (TMA,
// cp.async.bulk, 16-byte aligned) completing on an mbarrier.
//
// Inside a chunk, thread t runs the sequential HC loop over its own L window
// starts [tL, tL + L).  This is exact: HC started at any window reports every
// occurrence that starts at or after it (its shifts never pass over one), so
// it reports exactly the occurrences that start in [tL, tL+L) if it stops at
// the first window starting at or beyond tL + L.  L is 4 times an odd number,
// so the 32 lanes of a warp, whose windows advance in step while they miss,
// read 32 different shared-memory banks.
//
// Output in text order.  Each thread counts its occurrences (keeping the
// first four in shared memory); a block scan gives each thread's offset in
// the chunk and the chunk total; a single-pass decoupled look-back over the
// per-chunk states (aggregate / inclusive prefix) gives the chunk's offset
// in the output; threads then write their positions (threads with more than
// four re-scan their segment from shared memory to write the rest).  Chunk
// 0's inclusive prefix needs no look-back, so the chain always resolves.
//
// Every wait (bulk-copy completion, a predecessor chunk's state) is bounded;
// a wait that gives up sets the status flag and the kernel returns.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>

#include "hc_device.cuh"
#include "hc_internal.h"

namespace hc {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kStages = 2;
constexpr int kSlots = 4;
constexpr int kMaxSmemX = 4096;             // larger patterns verify from global memory
constexpr size_t kMaxStagedM = 16384;       // larger patterns use the unstaged kernel
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

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
  unsigned long long* state; // per-chunk look-back state, zeroed
  unsigned long long* claim; // chunk claim counter, zeroed
  unsigned long long num_chunks;
  int L;                     // window starts per thread
  uint32_t C;                // window starts per chunk (kThreads * L)
  int head;                  // y mod 16: offset of y[kC] in its staged buffer
  uint32_t stage_bytes;      // bytes per staging buffer (16-byte multiple)
  uint32_t x_smem;           // bytes of shared memory for x (0: verify from global)
};

// ---------------------------------------------------------------------------
// q-gram hash h (Eq. 3, Eq. 4): the q bytes starting at byte offset o of
// `base`, weight 2^(s*k) for the k-th byte, mod 2^alpha.  Evaluated by
// Horner's rule from the last byte down, as in the paper's Hash routine.
// Staged: `base` is a 16-byte aligned shared-memory buffer with at least 12
// readable bytes past the q-gram; the bytes come from two or three aligned
// 32-bit loads and funnel shifts.  Unstaged: byte loads from global memory.
template <int Q, bool STAGED>
__device__ __forceinline__ uint32_t qgram_hash(const uint8_t* base, int o, int s,
                                               uint32_t mask) {
  uint32_t v = 0;
  if constexpr (STAGED) {
    const uint32_t* W = reinterpret_cast<const uint32_t*>(base);
    const int wi = o >> 2;
    const uint32_t r = static_cast<uint32_t>(o & 3) * 8u;
    const uint32_t w0 = W[wi], w1 = W[wi + 1];
    const uint32_t lo = __funnelshift_r(w0, w1, r);
    uint32_t hi = 0;
    if constexpr (Q > 4) hi = __funnelshift_r(w1, W[wi + 2], r);
#pragma unroll
    for (int k = Q - 1; k >= 0; --k) {
      const uint32_t b = (k < 4) ? ((lo >> (8 * k)) & 0xffu) : ((hi >> (8 * (k - 4))) & 0xffu);
      v = (v << s) + b;
    }
  } else {
#pragma unroll
    for (int k = Q - 1; k >= 0; --k) v = (v << s) + static_cast<uint32_t>(__ldg(base + o + k));
  }
  return v & mask;
}

__device__ __forceinline__ bool verify_window(const uint8_t* w, const uint8_t* x, int m) {
  for (int k = 0; k < m; ++k)
    if (w[k] != x[k]) return false;
  return true;
}

// Sequential HC (Fig. 5 left) over the window starts [lo, hi) of a chunk.
// Chunk-relative text byte k is base[head + k].  Counts the occurrences;
// without WRITE the first kSlots starts go to slot[0], slot[kThreads], ...;
// with WRITE every occurrence is written to pos[obase + i] (if below cap).
template <int Q, bool STAGED, bool WRITE>
__device__ __forceinline__ int scan_segment(const uint8_t* base, int head, int lo, int hi,
                                            const SearchArgs& a, const uint32_t* Fs,
                                            const uint8_t* xv, uint32_t* slot,
                                            unsigned long long obase,
                                            unsigned long long chunk_start) {
  const int m = a.m, s = a.s;
  const uint32_t mask = a.mask, hv = a.hv;
  const int shift = m - Q + 1;
  int cnt = 0;
  int e = lo + m - 1;              // window end (chunk-relative)
  const int e_end = hi + m - 1;    // first window end past the segment
  while (e < e_end) {
    // first test: the q-gram ending at the window end
    uint32_t v = qgram_hash<Q, STAGED>(base, head + e - Q + 1, s, mask);
    uint32_t z = Fs[v];
    if (z == 0) {
      e += shift;
      continue;
    }
    // back-walk over the q-grams to the left, each linked to its right one
    int j = e;
    const int i = e - m + 2 * Q;
    bool full = true;
    while (j >= i) {
      j -= Q;
      v = qgram_hash<Q, STAGED>(base, head + j - Q + 1, s, mask);
      if ((z & (1u << (v & 31u))) == 0) {
        full = false;
        break;
      }
      z = Fs[v];
    }
    if (!full) {
      e = j + shift;               // shift past the unlinked q-gram
      continue;
    }
    const int start = e - m + 1;
    if (v == hv && verify_window(base + head + start, xv, m)) {
      if constexpr (WRITE) {
        const unsigned long long idx = obase + static_cast<unsigned long long>(cnt);
        if (idx < a.cap) a.pos[idx] = chunk_start + static_cast<unsigned long long>(start);
      } else {
        if (cnt < kSlots) slot[cnt * kThreads] = static_cast<uint32_t>(start);
      }
      ++cnt;
    }
    e += 1;                        // full read: advance by one
  }
  return cnt;
}

// Decoupled look-back by one warp: publishes chunk c's aggregate, sums the
// predecessors' values back to the nearest inclusive prefix, publishes c's
// inclusive prefix.  Returns false if a wait gave up.
__device__ bool chunk_lookback(const SearchArgs& a, long long c, unsigned long long total,
                               unsigned long long* excl_out) {
  const int lane = threadIdx.x & 31;
  if (c == 0) {
    if (lane == 0) st_relaxed_u64(&a.state[0], kFlagInc | total);
    *excl_out = 0;
    return true;
  }
  if (lane == 0) st_relaxed_u64(&a.state[c], kFlagAgg | total);
  unsigned long long excl = 0;
  long long base = c - 1;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    const long long idx = base - lane;
    unsigned long long v = kFlagInc;  // before chunk 0: inclusive prefix 0
    if (idx >= 0) {
      v = ld_relaxed_u64(&a.state[idx]);
      for (uint32_t spins = 0; (v >> 62) == 0 && spins < kMaxSpins; ++spins) {
        if ((spins & 63u) == 63u && global_timer_ns() - t0 > kWaitLimitNs) break;
        __nanosleep(64);
        v = ld_relaxed_u64(&a.state[idx]);
      }
    }
    if (__any_sync(0xffffffffu, (v >> 62) == 0)) return false;
    const unsigned inc = __ballot_sync(0xffffffffu, (v >> 62) == 2);
    const int stop = inc ? (__ffs(inc) - 1) : 31;
    excl += warp_sum_u64(lane <= stop ? (v & kValMask) : 0ull);
    if (inc) break;
    base -= 32;
  }
  if (lane == 0) st_relaxed_u64(&a.state[c], kFlagInc | (excl + total));
  *excl_out = excl;
  return true;
}

// Starts the bulk copy of chunk c's text into staging buffer `st`.
__device__ __forceinline__ void issue_chunk(const SearchArgs& a, uint8_t* stages, uint64_t* bars,
                                            int st, long long c) {
  const unsigned long long cs = static_cast<unsigned long long>(c) * a.C;
  const unsigned long long len = min(static_cast<unsigned long long>(a.C) + a.m - 1, a.n - cs);
  const uint32_t bytes = static_cast<uint32_t>((a.head + len + 15) & ~15ull);
  const uint8_t* src = a.y + cs - a.head;  // 16-byte aligned: C is a multiple of 16
  mbar_arrive_expect_tx(&bars[st], bytes);
  bulk_copy_g2s(stages + static_cast<size_t>(st) * a.stage_bytes, src, bytes, &bars[st]);
}

template <int Q, bool STAGED>
__global__ void __launch_bounds__(kThreads) hc_search_kernel(const SearchArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ long long chunk_id[kStages];
  __shared__ uint32_t warp_sum[kWarps];
  __shared__ unsigned long long s_excl;
  __shared__ int s_abort;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* Fs = reinterpret_cast<uint32_t*>(smem);
  const uint32_t f_bytes = (a.fwords * 4u + 15u) & ~15u;
  uint8_t* xs = smem + f_bytes;
  uint8_t* stages = xs + a.x_smem;
  uint32_t* slots = reinterpret_cast<uint32_t*>(stages + (STAGED ? kStages * a.stage_bytes : 0u));

  for (uint32_t i = tid; i < a.fwords; i += kThreads) Fs[i] = a.F[i];
  for (uint32_t i = tid; i < a.x_smem && i < static_cast<uint32_t>(a.m); i += kThreads)
    xs[i] = a.x[i];
  const uint8_t* xv = a.x_smem ? xs : a.x;

  uint32_t inflight = 0;  // thread 0: bit st set while stage st has a copy in flight
  if (tid == 0) {
    s_abort = 0;
    const long long c = static_cast<long long>(atomicAdd(a.claim, 1ull));
    chunk_id[0] = c;
    if constexpr (STAGED) {
      for (int st = 0; st < kStages; ++st) mbar_init(&bars[st], 1);
      fence_mbar_init();
      if (c < static_cast<long long>(a.num_chunks)) {
        issue_chunk(a, stages, bars, 0, c);
        inflight |= 1u;
      }
    }
  }
  __syncthreads();

  uint32_t parity = 0;  // bit st: parity of the next completion of stage st
  int st = 0;
  for (;; st ^= 1) {
    const long long c = chunk_id[st];
    if (c >= static_cast<long long>(a.num_chunks)) break;
    if (tid == 0) {  // claim (and prefetch) the next chunk
      const long long cn = static_cast<long long>(atomicAdd(a.claim, 1ull));
      chunk_id[st ^ 1] = cn;
      if constexpr (STAGED) {
        if (cn < static_cast<long long>(a.num_chunks)) {
          fence_proxy_async_smem();
          issue_chunk(a, stages, bars, st ^ 1, cn);
          inflight |= 2u >> st;
        }
      }
    }
    if constexpr (STAGED) {
      if (mbar_wait_bounded(&bars[st], (parity >> st) & 1u)) {
        parity ^= 1u << st;
        inflight &= ~(1u << st);
      } else {
        s_abort = 1;
      }
      __syncthreads();
      if (s_abort) break;
    }

    const unsigned long long cs = static_cast<unsigned long long>(c) * a.C;
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
    const int lo = tid * a.L;
    const int hi = min(lo + a.L, wins);
    uint32_t* my_slot = slots + tid;
    int cnt = 0;
    if (lo < hi)
      cnt = scan_segment<Q, STAGED, false>(base, head, lo, hi, a, Fs, xv, my_slot, 0, 0);

    // block-wide exclusive scan of the per-thread counts
    const uint32_t incl = warp_incl_scan_u32(static_cast<uint32_t>(cnt));
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < kWarps ? warp_sum[lane] : 0u;
      w = warp_incl_scan_u32(w);
      if (lane < kWarps) warp_sum[lane] = w;
    }
    __syncthreads();
    const uint32_t thread_excl = (warp ? warp_sum[warp - 1] : 0u) + incl - static_cast<uint32_t>(cnt);
    const uint32_t total = warp_sum[kWarps - 1];
    if (warp == 0) {
      unsigned long long ex = 0;
      const bool ok = chunk_lookback(a, c, total, &ex);
      if (lane == 0) {
        s_excl = ex;
        if (!ok) s_abort = 1;
        else if (c == static_cast<long long>(a.num_chunks) - 1) *a.count_out = ex + total;
      }
    }
    __syncthreads();
    if (s_abort) break;
    if (cnt > 0) {
      const unsigned long long ob = s_excl + thread_excl;
      if (cnt <= kSlots) {
        for (int k = 0; k < cnt; ++k) {
          const unsigned long long idx = ob + static_cast<unsigned long long>(k);
          if (idx < a.cap) a.pos[idx] = cs + my_slot[k * kThreads];
        }
      } else {
        scan_segment<Q, STAGED, true>(base, head, lo, hi, a, Fs, xv, nullptr, ob, cs);
      }
    }
    __syncthreads();  // staging buffer st and the scan scratch are free again
  }

  if (s_abort && tid == 0) {
    atomicOr(&g_status, 1u);
    if constexpr (STAGED) {
      // let copies still in flight land before the CTA's shared memory goes
      for (int k = 0; k < kStages; ++k)
        if (inflight & (1u << k)) (void)mbar_wait_bounded(&bars[k], (parity >> k) & 1u);
    }
  }
}

// ---------------------------------------------------------------------------
// host side
namespace {

using KernelFn = void (*)(const SearchArgs);

template <bool STAGED>
KernelFn kernel_for_q(int q) {
  switch (q) {
    case 1: return hc_search_kernel<1, STAGED>;
    case 2: return hc_search_kernel<2, STAGED>;
    case 3: return hc_search_kernel<3, STAGED>;
    case 4: return hc_search_kernel<4, STAGED>;
    case 5: return hc_search_kernel<5, STAGED>;
    case 6: return hc_search_kernel<6, STAGED>;
    case 7: return hc_search_kernel<7, STAGED>;
    default: return hc_search_kernel<8, STAGED>;
  }
}

std::mutex g_attr_mu;
std::set<std::pair<int, const void*>> g_attr_done;

int ensure_smem_attr(int dev, KernelFn fn, size_t smem) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  auto key = std::make_pair(dev, reinterpret_cast<const void*>(fn));
  if (g_attr_done.count(key)) return HC_OK;
  const DeviceInfo& di = device_info(dev);
  cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(fn),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(di.smem_optin));
  if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
  g_attr_done.insert(key);
  (void)smem;
  return HC_OK;
}

struct Plan {
  bool staged;
  int L;
  uint32_t C, stage_bytes, x_smem;
  size_t smem;
  unsigned long long num_chunks;
};

Plan make_plan(const Filter* f, size_t n, size_t smem_limit, bool staged) {
  Plan p{};
  const int m = static_cast<int>(std::min<size_t>(f->m, 1u << 30));
  const int shift = m - f->q + 1;
  p.staged = staged;
  // L = 4 * (odd number of words) >= max(64, 4 * shift), at most 188 bytes
  int lw = std::max(16, shift) | 1;
  lw = std::min(lw, 47);
  p.L = 4 * lw;
  p.C = static_cast<uint32_t>(kThreads * p.L);
  p.stage_bytes = static_cast<uint32_t>(((16 + p.C + f->m - 1 + 15) & ~size_t(15)) + 16);
  p.x_smem = f->m <= static_cast<size_t>(kMaxSmemX) ? static_cast<uint32_t>((f->m + 15) & ~size_t(15)) : 0u;
  const size_t fbytes = (f->F.size() * 4 + 15) & ~size_t(15);
  p.smem = fbytes + p.x_smem + (p.staged ? size_t(kStages) * p.stage_bytes : 0) +
           size_t(kSlots) * kThreads * 4;
  const unsigned long long nwin = n - f->m + 1;
  p.num_chunks = (nwin + p.C - 1) / p.C;
  (void)smem_limit;
  return p;
}

}  // namespace

// Enqueues the search; count_dev receives the total.  Internal entry shared
// by the C ABI functions.
int launch_search(Filter* f, const uint8_t* y, size_t n, uint64_t* pos, size_t cap,
                  uint64_t* count_dev, cudaStream_t stream) {
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
  const DeviceInfo& di = device_info(dev);
  Plan p = make_plan(f, n, di.smem_optin, f->m <= kMaxStagedM);
  if (p.staged && p.smem > di.smem_optin) p = make_plan(f, n, di.smem_optin, false);
  if (p.smem > di.smem_optin)
    return set_error(HC_ERR_ARG, "hc_search: filter exceeds shared memory");
  KernelFn fn = p.staged ? kernel_for_q<true>(f->q) : kernel_for_q<false>(f->q);
  rc = ensure_smem_attr(dev, fn, p.smem);
  if (rc != HC_OK) return rc;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, p.smem);
  if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  per_sm = std::max(per_sm, 1);
  const unsigned long long grid =
      std::min<unsigned long long>(p.num_chunks, static_cast<unsigned long long>(per_sm) * di.sm_count);

  const size_t ws_bytes = (p.num_chunks + 1) * sizeof(unsigned long long);
  void* ws = nullptr;
  e = cudaMallocAsync(&ws, ws_bytes, stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(workspace)");
  e = cudaMemsetAsync(ws, 0, ws_bytes, stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(ws, stream);
    return cuda_error(e, "cudaMemsetAsync(workspace)");
  }

  SearchArgs a{};
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
  a.claim = static_cast<unsigned long long*>(ws);
  a.state = static_cast<unsigned long long*>(ws) + 1;
  a.num_chunks = p.num_chunks;
  a.L = p.L;
  a.C = p.C;
  a.head = static_cast<int>(reinterpret_cast<uintptr_t>(y) & 15u);
  a.stage_bytes = p.stage_bytes;
  a.x_smem = p.x_smem;

  fn<<<static_cast<unsigned>(grid), kThreads, p.smem, stream>>>(a);
  e = cudaGetLastError();
  g_launches.fetch_add(1);
  cudaFreeAsync(ws, stream);
  if (e != cudaSuccess) return cuda_error(e, "hc_search kernel launch");
  return HC_OK;
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

extern "C" {

int hc_search_async(const hc_filter* fp, const uint8_t* y_dev, size_t n, uint64_t* pos_dev,
                    size_t cap, uint64_t* count_dev, hc_stream_t stream) {
  clear_error();
  Filter* f = as_filter(fp);
  if (f == nullptr) return set_error(HC_ERR_ARG, "hc_search_async: invalid filter");
  if (count_dev == nullptr) return set_error(HC_ERR_ARG, "hc_search_async: count_dev is NULL");
  if (y_dev == nullptr && n > 0) return set_error(HC_ERR_ARG, "hc_search_async: y_dev is NULL");
  if (pos_dev == nullptr && cap > 0)
    return set_error(HC_ERR_ARG, "hc_search_async: pos_dev is NULL with cap > 0");
  return launch_search(f, y_dev, n, pos_dev, cap, count_dev, reinterpret_cast<cudaStream_t>(stream));
}

int hc_search(const hc_filter* fp, const uint8_t* x, const uint8_t* y_dev, size_t n,
              uint64_t* pos_dev, size_t cap, size_t* count, hc_stream_t stream_) {
  clear_error();
  Filter* f = as_filter(fp);
  if (f == nullptr) return set_error(HC_ERR_ARG, "hc_search: invalid filter");
  if (x == nullptr || count == nullptr) return set_error(HC_ERR_ARG, "hc_search: x or count is NULL");
  if (std::memcmp(x, f->x.data(), f->m) != 0)
    return set_error(HC_ERR_ARG, "hc_search: x is not the pattern the filter was built from");
  if (y_dev == nullptr && n > 0) return set_error(HC_ERR_ARG, "hc_search: y_dev is NULL");
  if (pos_dev == nullptr && cap > 0) return set_error(HC_ERR_ARG, "hc_search: pos_dev is NULL with cap > 0");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  void* cnt_dev = nullptr;
  cudaError_t e = cudaMallocAsync(&cnt_dev, sizeof(uint64_t), stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(count)");
  int rc = launch_search(f, y_dev, n, pos_dev, cap, static_cast<uint64_t*>(cnt_dev), stream);
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
