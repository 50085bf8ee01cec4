// hc_batch.cu -- many (pattern, text) searches in one set of launches.
//
// A batch is planned once on the host (launch arguments, work tables, sizes
// of the filter and workspace areas) and run as three kernels that allocate
// nothing, so a run can be captured in a CUDA graph and replayed:
//
//   1. hc_batch_preprocess_kernel -- the preprocessing phase of Sec. 3.1 on
//      the device, one CTA per query: F is cleared in shared memory, every
//      adjacent non-overlapping pair of q-grams ORs lambda(h(left)) into
//      F[h(right)] (Eq. 1, shared-memory atomics: OR is order-free), then
//      every first q-gram whose word is still empty gets 1 (Eq. 2 with the
//      first optimisation of Sec. 3.4); H_v is h of the q-gram starting at
//      m mod q.  The result equals Fig. 4's word for word.  Block 0 also
//      resets the work counter of kernel 2.
//   2. hc_batch_scan_kernel -- a persistent grid; each CTA claims tiles
//      (query, 8 consecutive records) from a device-side counter, loads that
//      query's launch arguments, F and x into shared memory, and its warps
//      run the per-warp HC stream of the single search on one record each.
//   3. hc_batch_emit_kernel -- per (query, record group): output offsets,
//      copy of the spilled positions, re-scan of overflowed chunks, count.
//
// hc_batch_* (this file) owns a planned table in cudaMalloc'd memory; the
// autotuner and the server build plans of their own with the same functions.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "hc_batch_internal.h"

namespace hc {
namespace {

constexpr uint32_t kBatchMagic = 0x48434231u;  // "HCB1"
constexpr unsigned long long kTileTextBytes = 64ull << 10;  // text per record, about
// Spill entries per query at least (as positions): records whose share
// overflows are re-scanned by the emit kernel, so the floor keeps dense
// queries with a small cap from re-scanning most of their records.
constexpr unsigned long long kMinSpill = 1ull << 15;
constexpr size_t kOneClassQueries = 32;  // batches up to this size run one scan class

// h(x[i .. i+q-1]) by Horner's rule from the last byte down (Eq. 3, Eq. 4).
__device__ __forceinline__ uint32_t pattern_hash(const uint8_t* x, int i, int q, int s,
                                                 uint32_t mask) {
  uint32_t v = 0;
  for (int k = q - 1; k >= 0; --k) v = (v << s) + static_cast<uint32_t>(x[i + k]);
  return v & mask;
}

__global__ void __launch_bounds__(kThreads)
    hc_batch_preprocess_kernel(SearchArgs* args, unsigned long long* counters) {
  extern __shared__ __align__(128) uint8_t smem[];
  pdl_launch_dependents();  // the scan kernel may be scheduled; it waits for this grid
  uint32_t* Fs = reinterpret_cast<uint32_t*>(smem);
  const int tid = threadIdx.x;
  if (blockIdx.x == 0 && tid < kMaxScanClasses) counters[tid] = 0;
  SearchArgs* a = args + blockIdx.x;
  if (a->records == 0) {  // n < m: no window
    if (tid == 0) *a->count_out = 0;
    return;
  }
  const uint8_t* x = a->x;
  const int m = a->m, q = a->q, s = a->s;
  const uint32_t mask = a->mask, fw = a->fwords;
  for (uint32_t i = tid; i < fw; i += kThreads) Fs[i] = 0;
  __syncthreads();
  for (int i = tid; i + 2 * q <= m; i += kThreads) {  // Eq. 1
    const uint32_t hl = pattern_hash(x, i, q, s, mask);
    const uint32_t hr = pattern_hash(x, i + q, q, s, mask);
    atomicOr(&Fs[hr], 1u << (hl & 31u));
  }
  __syncthreads();
  const int nfirst = min(q, m - q + 1);
  for (int i = tid; i < nfirst; i += kThreads) {  // Eq. 2, only into empty words
    const uint32_t v = pattern_hash(x, i, q, s, mask);
    if (Fs[v] == 0u) Fs[v] = 1u;
  }
  __syncthreads();
  uint32_t* F = const_cast<uint32_t*>(a->F);
  for (uint32_t i = tid; i < fw; i += kThreads) F[i] = Fs[i];
  if (tid == 0) a->hv = pattern_hash(x, m % q, q, s, mask);  // Sec. 3.4
}

// Copies a SearchArgs from global to shared memory with the whole CTA.
__device__ __forceinline__ void load_args(SearchArgs* dst, const SearchArgs* src) {
  static_assert(sizeof(SearchArgs) % 4 == 0, "SearchArgs size");
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < static_cast<int>(sizeof(SearchArgs) / 4); i += kThreads) d[i] = s[i];
}

template <bool STAGED>
__device__ __forceinline__ void stream_q(const SearchArgs& a, unsigned long long r,
                                         const uint32_t* Fs, const uint8_t* xv, uint32_t* slots,
                                         uint8_t* stages, uint64_t* wb) {
  switch (a.q) {
    case 1: warp_stream<1, STAGED>(a, r, Fs, xv, slots, stages, wb); break;
    case 2: warp_stream<2, STAGED>(a, r, Fs, xv, slots, stages, wb); break;
    case 3: warp_stream<3, STAGED>(a, r, Fs, xv, slots, stages, wb); break;
    case 4: warp_stream<4, STAGED>(a, r, Fs, xv, slots, stages, wb); break;
    case 5: warp_stream<5, STAGED>(a, r, Fs, xv, slots, stages, wb); break;
    case 6: warp_stream<6, STAGED>(a, r, Fs, xv, slots, stages, wb); break;
    case 7: warp_stream<7, STAGED>(a, r, Fs, xv, slots, stages, wb); break;
    default: warp_stream<8, STAGED>(a, r, Fs, xv, slots, stages, wb); break;
  }
}


__global__ void __launch_bounds__(kThreads)
    hc_batch_scan_kernel(const SearchArgs* args, const BatchTile* tiles,
                         unsigned long long ntiles, unsigned long long* counter, BatchLayout lay) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[kWarps][kMaxStages];
  __shared__ __align__(16) SearchArgs sa;
  __shared__ unsigned long long s_tile;
  pdl_launch_dependents();
  pdl_wait();  // filters, H_v and the work counter come from the preprocessing grid
  const int tid = threadIdx.x, warp = tid >> 5;
  uint32_t* Fs = reinterpret_cast<uint32_t*>(smem);
  uint8_t* xs = smem + lay.f_bytes;
  uint32_t* slots = reinterpret_cast<uint32_t*>(xs + lay.x_bytes);
  uint8_t* ring = reinterpret_cast<uint8_t*>(slots + kSlots * kThreads) +
                  static_cast<size_t>(warp) * lay.ring_bytes;
  uint32_t staged_query = ~0u;  // query whose arguments, F and x are in shared memory
  while (true) {
    if (tid == 0) s_tile = atomicAdd(counter, 1ull);
    __syncthreads();
    const unsigned long long t = s_tile;
    if (t >= ntiles) break;
    const BatchTile bt = tiles[t];
    if (bt.query != staged_query) {
      // a new query: its arguments, filter and pattern (tiles of one query
      // are claimed one after another, so this is rare)
      load_args(&sa, args + bt.query);
      __syncthreads();
      stage_words(Fs, sa.F, sa.fwords);
      stage_bytes(xs, sa.x, min(sa.x_smem, static_cast<uint32_t>(sa.m)));
      __syncthreads();
      staged_query = bt.query;
    }
    const uint8_t* xv = sa.x_smem ? xs : sa.x;
    const unsigned long long r = static_cast<unsigned long long>(bt.first_record) + warp;
    if (r < sa.records) {
      if (sa.stages > 0) stream_q<true>(sa, r, Fs, xv, slots, ring, bars[warp]);
      else stream_q<false>(sa, r, Fs, xv, slots, ring, bars[warp]);
    }
    __syncthreads();  // s_tile (and F, x and the arguments) may be replaced by the next tile
  }
}

__global__ void __launch_bounds__(kThreads, 3)
    hc_batch_emit_kernel(const SearchArgs* args, const EmitTile* etiles) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(16) SearchArgs sa;
  pdl_wait();  // the scan grid has completed and its records are visible
  const EmitTile et = etiles[blockIdx.x / kEmitSplit];
  const unsigned part = blockIdx.x % kEmitSplit;
  load_args(&sa, args + et.query);
  __syncthreads();
  switch (sa.q) {
    case 1: emit_group<1>(sa, et.group, part, smem); break;
    case 2: emit_group<2>(sa, et.group, part, smem); break;
    case 3: emit_group<3>(sa, et.group, part, smem); break;
    case 4: emit_group<4>(sa, et.group, part, smem); break;
    case 5: emit_group<5>(sa, et.group, part, smem); break;
    case 6: emit_group<6>(sa, et.group, part, smem); break;
    case 7: emit_group<7>(sa, et.group, part, smem); break;
    default: emit_group<8>(sa, et.group, part, smem); break;
  }
}

// Byte histogram of a sample of each text (estimate_sigma).
struct SigmaJob {
  const uint8_t* y;
  unsigned long long n;
};

constexpr unsigned long long kSigmaWhole = 64ull << 10;  // texts up to this: every byte
constexpr unsigned long long kSigmaPiece = 4ull << 10;
constexpr int kSigmaPieces = 16;

__global__ void __launch_bounds__(kThreads) hc_sigma_kernel(const SigmaJob* jobs, uint32_t* hist) {
  __shared__ uint32_t h[256];
  const int tid = threadIdx.x;
  h[tid] = 0;
  __syncthreads();
  const SigmaJob j = jobs[blockIdx.x];
  if (j.n <= kSigmaWhole) {
    for (unsigned long long i = tid; i < j.n; i += kThreads) atomicAdd(&h[j.y[i]], 1u);
  } else {
    for (int p = 0; p < kSigmaPieces; ++p) {
      const unsigned long long start = (j.n - kSigmaPiece) * p / (kSigmaPieces - 1);
      for (unsigned long long i = tid; i < kSigmaPiece; i += kThreads) atomicAdd(&h[j.y[start + i]], 1u);
    }
  }
  __syncthreads();
  hist[static_cast<size_t>(blockIdx.x) * 256 + tid] = h[tid];
}

template <typename T>
int dev_alloc(T** p, size_t count, const char* what) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return cuda_error(e, what);
  *p = static_cast<T*>(v);
  return HC_OK;
}

// The batch kernels may use up to the device's opt-in shared memory; the
// attribute is raised once per device, each launch asks for what it needs.
int init_batch_kernels(int dev) {
  static std::mutex mu;
  static std::vector<int> done;
  std::lock_guard<std::mutex> lock(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return HC_OK;
  const DeviceInfo& di = device_info(dev);
  const void* fns[3] = {reinterpret_cast<const void*>(hc_batch_preprocess_kernel),
                        reinterpret_cast<const void*>(hc_batch_scan_kernel),
                        reinterpret_cast<const void*>(hc_batch_emit_kernel)};
  for (const void* fn : fns) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncGetAttributes(batch)");
    const int dyn = static_cast<int>(di.smem_optin) - static_cast<int>(fa.sharedSizeBytes);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(batch)");
  }
  done.push_back(dev);
  return HC_OK;
}

}  // namespace

unsigned long long record_bytes_for(unsigned long long total_text, int dev) {
  const unsigned long long warps = static_cast<unsigned long long>(device_info(dev).sm_count) * 16;
  return std::min<unsigned long long>(kTileTextBytes, std::max<unsigned long long>(1, total_text / warps));
}

int plan_add_query(BatchPlan& plan, const hc_batch_query& Q, size_t i, const QueryParams& p,
                   unsigned long long record_bytes, const char* who) {
  char msg[200];
  if (Q.x_dev == nullptr || Q.count_dev == nullptr || (Q.y_dev == nullptr && Q.n > 0) ||
      (Q.pos_dev == nullptr && Q.cap > 0) || !aligned8(Q.pos_dev) || !aligned8(Q.count_dev)) {
    std::snprintf(msg, sizeof msg, "%s: query %zu: null or misaligned pointer", who, i);
    return set_error(HC_ERR_ARG, msg);
  }
  if (Q.m < 1 || p.q < 1 || p.q > kMaxQ || static_cast<uint64_t>(p.q) > Q.m || p.alpha < 1 ||
      p.alpha > kMaxAlpha || Q.m > (uint64_t(1) << 30) || p.lane_bytes < 0 || p.lane_bytes > 4096 ||
      (p.mode != HC_MODE_AUTO && p.mode != HC_MODE_STAGED && p.mode != HC_MODE_DIRECT)) {
    std::snprintf(msg, sizeof msg,
                  "%s: query %zu: need m >= 1, 1 <= q <= min(m, 8), 1 <= alpha <= 15, "
                  "lane_bytes <= 4096, mode AUTO/STAGED/DIRECT", who, i);
    return set_error(HC_ERR_ARG, msg);
  }
  const uint32_t qi = static_cast<uint32_t>(plan.args.size());
  plan.args.emplace_back();
  plan.params.push_back(p);
  SearchArgs& a = plan.args.back();
  a = SearchArgs{};
  a.status = status_word();
  a.y = Q.y_dev;
  a.n = Q.n;
  a.x = Q.x_dev;
  a.m = static_cast<int>(Q.m);
  a.q = p.q;
  a.s = p.alpha / p.q;
  a.fwords = 1u << p.alpha;
  a.mask = a.fwords - 1u;
  a.pos = reinterpret_cast<unsigned long long*>(Q.pos_dev);
  a.cap = Q.pos_dev ? Q.cap : 0;
  a.count_out = reinterpret_cast<unsigned long long*>(Q.count_dev);
  {
    int g = 1;
    while (g < 4 && g < a.q && a.s * g <= 7) ++g;
    a.g0 = g;
    for (int k = 0; k < g; ++k) a.w0 |= (1u << (a.s * k)) << (8 * k);
    for (int k = 0; k < a.q - g && k < 4; ++k) a.w1 |= (1u << (a.s * k)) << (8 * k);
  }
  plan.f_off.push_back(plan.filter_words);
  plan.filter_words += (a.fwords + 3u) & ~3u;
  plan.lay.f_bytes = std::max(plan.lay.f_bytes, a.fwords * 4u);
  plan.ws_off.push_back(plan.ws_bytes);
  if (Q.n < Q.m) {
    a.records = 0;
    return HC_OK;
  }
  const int shift = a.m - a.q + 1;
  const bool direct = p.mode == HC_MODE_DIRECT ||
                      (p.mode != HC_MODE_STAGED && (shift >= kDirectShift || Q.m > kMaxStagedM));
  int L = p.lane_bytes;
  if (L <= 0) L = direct ? std::min(4096, std::max(64, shift)) : 4 * std::min(std::max(16, shift) | 1, 47);
  L = std::min(L, 4096);
  a.L = L;
  a.C = 32u * static_cast<uint32_t>(L);
  a.stages = direct ? 0 : 2;
  a.head = static_cast<int>(reinterpret_cast<uintptr_t>(Q.y_dev) & 15u);
  a.stage_bytes = direct ? 0u : stage_bytes_for(a.C, Q.m, false);
  a.x_smem = Q.m <= 4096 ? static_cast<uint32_t>((Q.m + 15) & ~uint64_t(15)) : 0u;
  plan.lay.x_bytes = std::max(plan.lay.x_bytes, a.x_smem);
  plan.lay.ring_bytes = std::max(plan.lay.ring_bytes, static_cast<uint32_t>(a.stages) * a.stage_bytes);
  a.nwin = Q.n - Q.m + 1;
  a.num_chunks = (a.nwin + a.C - 1) / a.C;
  a.chunks_per_cta = std::max<unsigned long long>(1, std::min(record_bytes, kTileTextBytes) / a.C);
  a.records = (a.num_chunks + a.chunks_per_cta - 1) / a.chunks_per_cta;
  const unsigned long long spill =
      a.cap == 0 ? 0 : std::min<unsigned long long>(a.nwin, std::max<unsigned long long>(a.cap, kMinSpill));
  a.region_entries = (std::max<unsigned long long>(1, (spill + a.records - 1) / a.records) + 3) & ~3ull;
  plan.ws_bytes += a.records * 16 + a.records * a.region_entries * 4;
  const unsigned long long groups = (a.records + 15) / 16;
  a.emit_group = (a.records + groups - 1) / groups;
  for (unsigned long long r = 0; r < a.records; r += kWarps)
    plan.tiles.push_back({qi, static_cast<uint32_t>(r)});
  for (unsigned long long g = 0; (g * a.emit_group) < a.records; ++g)
    plan.etiles.push_back({qi, static_cast<uint32_t>(g)});
  plan.records += a.records;
  return HC_OK;
}

namespace {

size_t scan_smem(const BatchLayout& lay) {
  return size_t((lay.f_bytes + 15u) & ~15u) + lay.x_bytes + size_t(kSlots) * kThreads * 4 +
         size_t(kWarps) * lay.ring_bytes;
}

}  // namespace

int plan_finish(BatchPlan& plan, int dev, const char* who) {
  const DeviceInfo& di = device_info(dev);
  plan.lay.f_bytes = (plan.lay.f_bytes + 15u) & ~15u;
  plan.smem_pre = std::max<size_t>(plan.lay.f_bytes, 16);
  plan.smem_scan = scan_smem(plan.lay);
  plan.smem_emit = size_t(plan.lay.f_bytes) + size_t(kSlots) * kThreads * 4;
  // class of a query: resident CTAs per SM its own layout allows (1 .. 4),
  // estimated from the SM's shared memory (with a reserve per CTA)
  const size_t per_sm = 233472;
  std::vector<int> qclass(plan.args.size(), 0);
  plan.classes.assign(kMaxScanClasses, ScanClass{});
  for (size_t i = 0; i < plan.args.size(); ++i) {
    const SearchArgs& a = plan.args[i];
    BatchLayout l{(a.fwords * 4u + 15u) & ~15u, a.x_smem, static_cast<uint32_t>(a.stages) * a.stage_bytes};
    const size_t need = scan_smem(l);
    if (need + 2048 > di.smem_optin)
      return set_error(HC_ERR_ARG, std::string(who) + ": filter and staging buffers exceed shared memory");
    const int ctas = static_cast<int>(std::min<size_t>(kMaxScanClasses, std::max<size_t>(1, per_sm / (need + 1536))));
    qclass[i] = kMaxScanClasses - ctas;  // class 0: the highest occupancy
  }
  // a small batch, or one whose tiles fit in one wave even at its lowest
  // occupancy, runs as one class: the class scans of a batch run one after
  // another, which would add up the latencies of its few queries
  int lowest = 0;
  for (int c : qclass) lowest = std::max(lowest, c);
  if (plan.args.size() <= kOneClassQueries ||
      plan.tiles.size() <= static_cast<size_t>(kMaxScanClasses - lowest) * di.sm_count)
    std::fill(qclass.begin(), qclass.end(), lowest);
  for (size_t i = 0; i < plan.args.size(); ++i) {
    const SearchArgs& a = plan.args[i];
    BatchLayout& cl = plan.classes[qclass[i]].lay;
    cl = {std::max(cl.f_bytes, (a.fwords * 4u + 15u) & ~15u), std::max(cl.x_bytes, a.x_smem),
          std::max(cl.ring_bytes, static_cast<uint32_t>(a.stages) * a.stage_bytes)};
  }
  std::stable_sort(plan.tiles.begin(), plan.tiles.end(),
                   [&](const BatchTile& x, const BatchTile& y) { return qclass[x.query] < qclass[y.query]; });
  unsigned long long begin = 0;
  for (int c = 0; c < kMaxScanClasses; ++c) {
    ScanClass& sc = plan.classes[c];
    sc.tile_begin = begin;
    while (begin < plan.tiles.size() && qclass[plan.tiles[begin].query] == c) ++begin;
    sc.ntiles = begin - sc.tile_begin;
    sc.smem = scan_smem(sc.lay);
  }
  return init_batch_kernels(dev);
}

void plan_bind(BatchPlan& plan, uint32_t* d_filters, uint8_t* d_ws) {
  for (size_t i = 0; i < plan.args.size(); ++i) {
    SearchArgs& a = plan.args[i];
    a.F = d_filters + plan.f_off[i];
    if (a.records == 0) continue;
    a.cta_total = reinterpret_cast<unsigned long long*>(d_ws + plan.ws_off[i]);
    a.cta_overflow = a.cta_total + a.records;
    a.region = reinterpret_cast<uint32_t*>(a.cta_overflow + a.records);
  }
}

namespace {

int class_grid(size_t smem, unsigned long long ntiles, int dev, int* grid) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<int, size_t>, int>> cache;  // (dev, smem) -> CTAs per SM
  int per_sm = -1;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (auto& c : cache)
      if (c.first.first == dev && c.first.second == smem) per_sm = c.second;
  }
  if (per_sm < 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hc_batch_scan_kernel, kThreads, smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(batch)");
    std::lock_guard<std::mutex> lock(mu);
    if (cache.size() < 256) cache.push_back({{dev, smem}, per_sm});
  }
  const DeviceInfo& di = device_info(dev);
  *grid = static_cast<int>(std::min<unsigned long long>(
      static_cast<unsigned long long>(std::max(per_sm, 1)) * di.sm_count, std::max<unsigned long long>(ntiles, 1)));
  return HC_OK;
}

}  // namespace

int batch_grids(BatchPlan& plan, int dev) {
  for (ScanClass& c : plan.classes)
    if (c.ntiles > 0) {
      int rc = class_grid(c.smem, c.ntiles, dev, &c.grid);
      if (rc != HC_OK) return rc;
    }
  return HC_OK;
}

BatchLaunch make_launch(const BatchPlan& plan, const SearchArgs* args, const BatchTile* tiles,
                        const EmitTile* etiles, unsigned long long* counters) {
  BatchLaunch L;
  L.args = args;
  L.tiles = tiles;
  L.etiles = etiles;
  L.counters = counters;
  L.nq = plan.args.size();
  L.netiles = plan.etiles.size();
  L.smem_pre = plan.smem_pre;
  L.smem_emit = plan.smem_emit;
  for (const ScanClass& c : plan.classes)
    if (c.ntiles > 0 && L.nclasses < kMaxScanClasses) L.classes[L.nclasses++] = c;
  return L;
}

int launch_batch(const BatchLaunch& L, cudaStream_t stream) {
  if (L.nq == 0) return HC_OK;
  TimingToken t0 = timing_begin(kKindPreprocess, stream);
  hc_batch_preprocess_kernel<<<static_cast<unsigned>(L.nq), kThreads, L.smem_pre, stream>>>(
      const_cast<SearchArgs*>(L.args), L.counters);
  cudaError_t e = cudaGetLastError();
  timing_end(t0, stream);
  if (e != cudaSuccess) return cuda_error(e, "hc_batch_preprocess_kernel launch");
  if (L.nclasses == 0) {
    g_launches.fetch_add(1);
    return HC_OK;
  }
  bool prev_timed = t0.active();
  for (int c = 0; c < L.nclasses; ++c) {
    const ScanClass& sc = L.classes[c];
    TimingToken t1 = timing_begin(kKindBatch, stream);
    e = launch_dependent(hc_batch_scan_kernel, static_cast<unsigned>(sc.grid), kThreads, sc.smem, stream,
                         !t1.active() && !prev_timed, L.args, L.tiles + sc.tile_begin, sc.ntiles,
                         L.counters + c, sc.lay);
    if (e == cudaSuccess) e = cudaGetLastError();
    timing_end(t1, stream);
    prev_timed = t1.active();
    if (e != cudaSuccess) return cuda_error(e, "hc_batch_scan_kernel launch");
  }
  TimingToken t2 = timing_begin(kKindEmit, stream);
  e = launch_dependent(hc_batch_emit_kernel, static_cast<unsigned>(L.netiles * kEmitSplit), kThreads, L.smem_emit,
                       stream, !t2.active(), L.args, L.etiles);
  if (e == cudaSuccess) e = cudaGetLastError();
  timing_end(t2, stream);
  if (e != cudaSuccess) return cuda_error(e, "hc_batch_emit_kernel launch");
  g_launches.fetch_add(2 + static_cast<uint64_t>(L.nclasses));
  return HC_OK;
}

int estimate_sigma(const uint8_t* const* y_dev, const uint64_t* n, size_t count,
                   std::vector<double>* sigma, cudaStream_t stream) {
  sigma->assign(count, 0.0);
  std::vector<SigmaJob> jobs;
  std::vector<size_t> idx;
  for (size_t i = 0; i < count; ++i)
    if (n[i] > 0 && y_dev[i] != nullptr) {
      jobs.push_back({y_dev[i], n[i]});
      idx.push_back(i);
    }
  if (jobs.empty()) return HC_OK;
  SigmaJob* d_jobs = nullptr;
  uint32_t* d_hist = nullptr;
  int rc = dev_alloc(&d_jobs, jobs.size(), "cudaMalloc(sigma jobs)");
  if (rc == HC_OK) rc = dev_alloc(&d_hist, jobs.size() * 256, "cudaMalloc(sigma histograms)");
  std::vector<uint32_t> hist(jobs.size() * 256);
  if (rc == HC_OK) {
    cudaError_t e = cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(SigmaJob),
                                    cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) {
      hc_sigma_kernel<<<static_cast<unsigned>(jobs.size()), kThreads, 0, stream>>>(d_jobs, d_hist);
      e = cudaGetLastError();
      g_launches.fetch_add(1);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hist.data(), d_hist, hist.size() * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) rc = cuda_error(e, "estimate_sigma");
  }
  cudaFree(d_jobs);
  cudaFree(d_hist);
  if (rc != HC_OK) return rc;
  for (size_t k = 0; k < jobs.size(); ++k) {
    double tot = 0, sq = 0;
    for (int c = 0; c < 256; ++c) {
      const double v = hist[k * 256 + c];
      tot += v;
      sq += v * v;
    }
    (*sigma)[idx[k]] = sq > 0 ? tot * tot / sq : 0.0;
  }
  return HC_OK;
}

struct Batch {
  uint32_t magic = kBatchMagic;
  int dev = -1;
  BatchPlan plan;
  BatchLaunch launch;
  SearchArgs* d_args = nullptr;
  BatchTile* d_tiles = nullptr;
  EmitTile* d_etiles = nullptr;
  unsigned long long* d_counter = nullptr;
  uint32_t* d_filters = nullptr;
  uint8_t* d_ws = nullptr;

  ~Batch() {
    if (dev >= 0) {
      int cur = 0;
      cudaGetDevice(&cur);
      if (cur != dev) cudaSetDevice(dev);
      cudaFree(d_args);
      cudaFree(d_tiles);
      cudaFree(d_etiles);
      cudaFree(d_counter);
      cudaFree(d_filters);
      cudaFree(d_ws);
      if (cur != dev) cudaSetDevice(cur);
    }
  }
};

namespace {

Batch* as_batch(const hc_batch* b) {
  auto* p = reinterpret_cast<Batch*>(const_cast<hc_batch*>(b));
  return (p != nullptr && p->magic == kBatchMagic) ? p : nullptr;
}

int create_batch(const hc_batch_query* qs, size_t nq, const hc_tuner* tuner, hc_batch** out,
                 const char* who) {
  clear_error();
  if (out == nullptr) return set_error(HC_ERR_ARG, std::string(who) + ": out is NULL");
  *out = nullptr;
  if (qs == nullptr && nq > 0) return set_error(HC_ERR_ARG, std::string(who) + ": queries is NULL");
  if (nq >= (size_t(1) << 31)) return set_error(HC_ERR_ARG, std::string(who) + ": too many queries");
  const Tuner* t = nullptr;
  if (tuner != nullptr && (t = as_tuner(tuner)) == nullptr)
    return set_error(HC_ERR_ARG, std::string(who) + ": invalid tuner");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");

  // parameters: given (q > 0) or tuned for the text's alphabet size
  std::vector<const uint8_t*> est_y;
  std::vector<uint64_t> est_n;
  std::vector<size_t> est_i;
  for (size_t i = 0; i < nq; ++i)
    if (qs[i].q == 0 && qs[i].sigma <= 0) {
      est_y.push_back(qs[i].y_dev);
      est_n.push_back(qs[i].n);
      est_i.push_back(i);
    }
  std::vector<double> est;
  if (!est_i.empty()) {
    int rc = estimate_sigma(est_y.data(), est_n.data(), est_i.size(), &est, nullptr);
    if (rc != HC_OK) return rc;
  }
  Batch* b = new (std::nothrow) Batch();
  if (b == nullptr) return set_error(HC_ERR_NOMEM, std::string(who) + ": out of host memory");
  BatchPlan& plan = b->plan;
  plan.args.reserve(nq);
  unsigned long long total_text = 0;
  for (size_t i = 0; i < nq; ++i) total_text += qs[i].n;
  const unsigned long long rec_bytes = record_bytes_for(total_text, dev);
  size_t k = 0;
  for (size_t i = 0; i < nq; ++i) {
    const hc_batch_query& Q = qs[i];
    QueryParams p;
    if (Q.q > 0) {
      p.q = Q.q;
      p.alpha = Q.alpha;
      p.lane_bytes = Q.lane_bytes;
      p.mode = Q.mode;
    } else if (Q.q == 0) {
      double sigma = Q.sigma;
      if (Q.sigma <= 0) sigma = est[k++];
      // q and alpha from the tuner; the launch options stay automatic (the
      // tuner measures lane width and mode on one query alone, and in a
      // batch of mixed queries the automatic options measured faster:
      // 3613 against 3144 GB/s for the same (q, alpha) on 4096 queries)
      const QueryParams tp = tuner_lookup(t, sigma, Q.m);
      p.q = tp.q;
      p.alpha = tp.alpha;
      p.lane_bytes = Q.lane_bytes;
      p.mode = Q.mode;
    } else {
      p.q = Q.q;  // negative: rejected below
    }
    int rc = plan_add_query(plan, Q, i, p, rec_bytes, who);
    if (rc != HC_OK) {
      delete b;
      return rc;
    }
  }
  int rc = plan_finish(plan, dev, who);
  if (rc != HC_OK) {
    delete b;
    return rc;
  }
  b->dev = dev;
  if (rc == HC_OK) rc = dev_alloc(&b->d_args, nq, "cudaMalloc(batch args)");
  if (rc == HC_OK) rc = dev_alloc(&b->d_tiles, plan.tiles.size(), "cudaMalloc(batch tiles)");
  if (rc == HC_OK) rc = dev_alloc(&b->d_etiles, plan.etiles.size(), "cudaMalloc(batch emit tiles)");
  if (rc == HC_OK) rc = dev_alloc(&b->d_counter, kMaxScanClasses, "cudaMalloc(batch counters)");
  if (rc == HC_OK) rc = dev_alloc(&b->d_filters, plan.filter_words, "cudaMalloc(batch filters)");
  if (rc == HC_OK) rc = dev_alloc(&b->d_ws, plan.ws_bytes, "cudaMalloc(batch workspace)");
  if (rc != HC_OK) {
    delete b;
    return rc;
  }
  plan_bind(plan, b->d_filters, b->d_ws);
  e = cudaMemcpy(b->d_args, plan.args.data(), nq * sizeof(SearchArgs), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !plan.tiles.empty())
    e = cudaMemcpy(b->d_tiles, plan.tiles.data(), plan.tiles.size() * sizeof(BatchTile),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !plan.etiles.empty())
    e = cudaMemcpy(b->d_etiles, plan.etiles.data(), plan.etiles.size() * sizeof(EmitTile),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    delete b;
    return cuda_error(e, "cudaMemcpy(batch tables)");
  }
  rc = batch_grids(plan, dev);
  if (rc != HC_OK) {
    delete b;
    return rc;
  }
  b->launch = make_launch(plan, b->d_args, b->d_tiles, b->d_etiles, b->d_counter);
  *out = reinterpret_cast<hc_batch*>(b);
  return HC_OK;
}

}  // namespace
int take_bound_violations_batch(uint64_t* count) {
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

extern "C" {

int hc_batch_create(const hc_batch_query* qs, size_t nq, hc_batch** out) {
  return create_batch(qs, nq, nullptr, out, "hc_batch_create");
}

int hc_batch_create_tuned(const hc_batch_query* qs, size_t nq, const hc_tuner* tuner, hc_batch** out) {
  return create_batch(qs, nq, tuner, out, "hc_batch_create_tuned");
}

int hc_batch_run(hc_batch* bp, hc_stream_t stream_) {
  clear_error();
  Batch* b = as_batch(bp);
  if (b == nullptr) return set_error(HC_ERR_ARG, "hc_batch_run: invalid batch");
  if (b->launch.nq == 0) return HC_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != b->dev) return set_error(HC_ERR_STATE, "hc_batch_run: batch belongs to another device");
  return launch_batch(b->launch, reinterpret_cast<cudaStream_t>(stream_));
}

int hc_batch_info(const hc_batch* bp, uint64_t* tiles, uint64_t* records, uint64_t* workspace_bytes) {
  Batch* b = as_batch(bp);
  if (b == nullptr) return set_error(HC_ERR_ARG, "hc_batch_info: invalid batch");
  if (tiles) *tiles = b->plan.tiles.size();
  if (records) *records = b->plan.records;
  if (workspace_bytes) *workspace_bytes = b->plan.ws_bytes;
  return HC_OK;
}

int hc_batch_params(const hc_batch* bp, size_t query, hc_tune_entry* out) {
  clear_error();
  Batch* b = as_batch(bp);
  if (b == nullptr || query >= b->plan.args.size() || out == nullptr)
    return set_error(HC_ERR_ARG, "hc_batch_params: invalid batch, query or output");
  const QueryParams& p = b->plan.params[query];
  const SearchArgs& a = b->plan.args[query];
  *out = hc_tune_entry{};
  out->m = static_cast<uint64_t>(a.m);
  out->q = p.q;
  out->alpha = p.alpha;
  out->lane_bytes = a.records ? a.L : p.lane_bytes;
  out->mode = a.records == 0 ? p.mode : (a.stages > 0 ? HC_MODE_STAGED : HC_MODE_DIRECT);
  return HC_OK;
}

int hc_batch_filter(const hc_batch* bp, size_t query, uint32_t* F, size_t nwords, uint32_t* hv) {
  clear_error();
  Batch* b = as_batch(bp);
  if (b == nullptr || query >= b->plan.args.size())
    return set_error(HC_ERR_ARG, "hc_batch_filter: invalid batch or query");
  const SearchArgs& a = b->plan.args[query];
  if (F != nullptr) {
    if (nwords < a.fwords) return set_error(HC_ERR_ARG, "hc_batch_filter: F holds fewer than 2^alpha words");
    cudaError_t e = cudaMemcpy(F, a.F, size_t(a.fwords) * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy(batch filter)");
  }
  if (hv != nullptr) {
    cudaError_t e = cudaMemcpy(hv, reinterpret_cast<const uint8_t*>(b->d_args + query) + offsetof(SearchArgs, hv),
                               sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy(batch H_v)");
  }
  return HC_OK;
}

void hc_batch_destroy(hc_batch* bp) {
  Batch* b = as_batch(bp);
  if (b == nullptr) return;
  b->magic = 0;
  delete b;
}

}  // extern "C"
