// hc_batch.cu -- many (pattern, text) searches in one set of launches.
//
// hc_batch_create plans a table of queries once (and allocates everything
// the runs need); hc_batch_run then enqueues three kernels and allocates
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
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "hc_kernels.cuh"

namespace hc {
namespace {

constexpr uint32_t kBatchMagic = 0x48434231u;  // "HCB1"
constexpr unsigned long long kTileTextBytes = 64ull << 10;  // text per record, about

struct BatchTile {
  uint32_t query;
  uint32_t first_record;
};

struct EmitTile {
  uint32_t query;
  uint32_t group;
};

// h(x[i .. i+q-1]) by Horner's rule from the last byte down (Eq. 3, Eq. 4).
__device__ __forceinline__ uint32_t pattern_hash(const uint8_t* x, int i, int q, int s,
                                                 uint32_t mask) {
  uint32_t v = 0;
  for (int k = q - 1; k >= 0; --k) v = (v << s) + static_cast<uint32_t>(x[i + k]);
  return v & mask;
}

__global__ void __launch_bounds__(kThreads)
    hc_batch_preprocess_kernel(SearchArgs* args, unsigned long long* counter) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t* Fs = reinterpret_cast<uint32_t*>(smem);
  const int tid = threadIdx.x;
  if (blockIdx.x == 0 && tid == 0) *counter = 0;
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

struct BatchLayout {
  uint32_t f_bytes;        // shared memory for F (largest query)
  uint32_t x_bytes;        // shared memory for x (largest staged pattern)
  uint32_t ring_bytes;     // per-warp staging ring (largest query)
};

__global__ void __launch_bounds__(kThreads)
    hc_batch_scan_kernel(const SearchArgs* args, const BatchTile* tiles,
                         unsigned long long ntiles, unsigned long long* counter, BatchLayout lay) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[kWarps][kMaxStages];
  __shared__ __align__(16) SearchArgs sa;
  __shared__ unsigned long long s_tile;
  const int tid = threadIdx.x, warp = tid >> 5;
  uint32_t* Fs = reinterpret_cast<uint32_t*>(smem);
  uint8_t* xs = smem + lay.f_bytes;
  uint32_t* slots = reinterpret_cast<uint32_t*>(xs + lay.x_bytes);
  uint8_t* ring = reinterpret_cast<uint8_t*>(slots + kSlots * kThreads) +
                  static_cast<size_t>(warp) * lay.ring_bytes;
  while (true) {
    if (tid == 0) s_tile = atomicAdd(counter, 1ull);
    __syncthreads();
    const unsigned long long t = s_tile;
    if (t >= ntiles) break;
    const BatchTile bt = tiles[t];
    load_args(&sa, args + bt.query);
    __syncthreads();
    for (uint32_t i = tid; i < sa.fwords; i += kThreads) Fs[i] = sa.F[i];
    for (uint32_t i = tid; i < sa.x_smem && i < static_cast<uint32_t>(sa.m); i += kThreads)
      xs[i] = sa.x[i];
    __syncthreads();
    const uint8_t* xv = sa.x_smem ? xs : sa.x;
    const unsigned long long r = static_cast<unsigned long long>(bt.first_record) + warp;
    if (r < sa.records) {
      if (sa.stages > 0) stream_q<true>(sa, r, Fs, xv, slots, ring, bars[warp]);
      else stream_q<false>(sa, r, Fs, xv, slots, ring, bars[warp]);
    }
    __syncthreads();  // F, x and the arguments are replaced by the next tile
  }
}

__global__ void __launch_bounds__(kThreads)
    hc_batch_emit_kernel(const SearchArgs* args, const EmitTile* etiles) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(16) SearchArgs sa;
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

template <typename T>
int dev_alloc(T** p, size_t count, const char* what) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return cuda_error(e, what);
  *p = static_cast<T*>(v);
  return HC_OK;
}

}  // namespace

struct Batch {
  uint32_t magic = kBatchMagic;
  int dev = -1;
  size_t nq = 0;
  std::vector<SearchArgs> host_args;
  SearchArgs* d_args = nullptr;
  BatchTile* d_tiles = nullptr;
  EmitTile* d_etiles = nullptr;
  unsigned long long* d_counter = nullptr;
  uint32_t* d_filters = nullptr;
  uint8_t* d_ws = nullptr;
  unsigned long long ntiles = 0, netiles = 0, records = 0;
  size_t ws_bytes = 0;
  BatchLayout lay{};
  size_t smem_pre = 0, smem_scan = 0, smem_emit = 0;
  int grid_scan = 0;

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

int set_kernel_smem(const void* fn, size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(bytes));
  return e == cudaSuccess ? HC_OK : cuda_error(e, "cudaFuncSetAttribute(batch)");
}

}  // namespace
}  // namespace hc

using namespace hc;

extern "C" {

int hc_batch_create(const hc_batch_query* qs, size_t nq, hc_batch** out) {
  clear_error();
  if (out == nullptr) return set_error(HC_ERR_ARG, "hc_batch_create: out is NULL");
  *out = nullptr;
  if (qs == nullptr && nq > 0) return set_error(HC_ERR_ARG, "hc_batch_create: queries is NULL");
  if (nq >= (size_t(1) << 31)) return set_error(HC_ERR_ARG, "hc_batch_create: too many queries");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  const DeviceInfo& di = device_info(dev);
  Batch* b = new (std::nothrow) Batch();
  if (b == nullptr) return set_error(HC_ERR_NOMEM, "hc_batch_create: out of host memory");
  b->nq = nq;
  b->host_args.resize(nq);
  std::vector<BatchTile> tiles;
  std::vector<EmitTile> etiles;
  size_t filter_words = 0, ws_bytes = 0;
  std::vector<size_t> f_off(nq), ws_off(nq);
  uint32_t f_max = 0, x_max = 0, ring_max = 0;
  const int stages = 2;

  for (size_t i = 0; i < nq; ++i) {
    const hc_batch_query& Q = qs[i];
    char msg[160];
    if (Q.x_dev == nullptr || Q.count_dev == nullptr || (Q.y_dev == nullptr && Q.n > 0) ||
        (Q.pos_dev == nullptr && Q.cap > 0) || !aligned8(Q.pos_dev) || !aligned8(Q.count_dev)) {
      std::snprintf(msg, sizeof msg, "hc_batch_create: query %zu: null or misaligned pointer", i);
      delete b;
      return set_error(HC_ERR_ARG, msg);
    }
    if (Q.m < 1 || Q.q < 1 || Q.q > kMaxQ || static_cast<uint64_t>(Q.q) > Q.m || Q.alpha < 1 ||
        Q.alpha > kMaxAlpha || Q.m > (uint64_t(1) << 30)) {
      std::snprintf(msg, sizeof msg,
                    "hc_batch_create: query %zu: need m >= 1, 1 <= q <= min(m, 8), 1 <= alpha <= 15", i);
      delete b;
      return set_error(HC_ERR_ARG, msg);
    }
    SearchArgs& a = b->host_args[i];
    a = SearchArgs{};
    a.status = status_word();
    a.y = Q.y_dev;
    a.n = Q.n;
    a.x = Q.x_dev;
    a.m = static_cast<int>(Q.m);
    a.q = Q.q;
    a.s = Q.alpha / Q.q;
    a.fwords = 1u << Q.alpha;
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
    f_off[i] = filter_words;
    filter_words += (a.fwords + 3u) & ~3u;
    f_max = std::max(f_max, a.fwords * 4u);
    if (Q.n < Q.m) {
      a.records = 0;
      continue;
    }
    const int shift = a.m - a.q + 1;
    const bool direct = Q.mode == HC_MODE_DIRECT ||
                        (Q.mode != HC_MODE_STAGED && (shift >= 200 || Q.m > 16384));
    int L = Q.lane_bytes;
    if (L <= 0) L = direct ? std::min(4096, std::max(64, shift)) : 4 * std::min(std::max(16, shift) | 1, 47);
    L = std::min(L, 4096);
    a.L = L;
    a.C = 32u * static_cast<uint32_t>(L);
    a.stages = direct ? 0 : stages;
    a.head = static_cast<int>(reinterpret_cast<uintptr_t>(Q.y_dev) & 15u);
    a.stage_bytes = direct ? 0u : static_cast<uint32_t>(((16 + a.C + Q.m - 1 + 15) & ~uint64_t(15)) + 64);
    a.x_smem = Q.m <= 4096 ? static_cast<uint32_t>((Q.m + 15) & ~uint64_t(15)) : 0u;
    x_max = std::max(x_max, a.x_smem);
    ring_max = std::max(ring_max, static_cast<uint32_t>(a.stages) * a.stage_bytes);
    a.nwin = Q.n - Q.m + 1;
    a.num_chunks = (a.nwin + a.C - 1) / a.C;
    a.chunks_per_cta = std::max<unsigned long long>(1, (kTileTextBytes + a.C - 1) / a.C);
    a.records = (a.num_chunks + a.chunks_per_cta - 1) / a.chunks_per_cta;
    const unsigned long long spill =
        a.cap == 0 ? 0 : std::min<unsigned long long>(a.nwin, std::max<unsigned long long>(a.cap, 4096));
    a.region_entries = (std::max<unsigned long long>(1, (spill + a.records - 1) / a.records) + 3) & ~3ull;
    ws_off[i] = ws_bytes;
    ws_bytes += a.records * 16 + a.records * a.region_entries * 4;
    const unsigned long long groups = (a.records + 15) / 16;
    a.emit_group = (a.records + groups - 1) / groups;
    for (unsigned long long r = 0; r < a.records; r += kWarps)
      tiles.push_back({static_cast<uint32_t>(i), static_cast<uint32_t>(r)});
    for (unsigned long long g = 0; (g * a.emit_group) < a.records; ++g)
      etiles.push_back({static_cast<uint32_t>(i), static_cast<uint32_t>(g)});
    b->records += a.records;
  }

  b->dev = dev;
  int rc = HC_OK;
  if (rc == HC_OK) rc = dev_alloc(&b->d_args, nq, "cudaMalloc(batch args)");
  if (rc == HC_OK) rc = dev_alloc(&b->d_tiles, tiles.size(), "cudaMalloc(batch tiles)");
  if (rc == HC_OK) rc = dev_alloc(&b->d_etiles, etiles.size(), "cudaMalloc(batch emit tiles)");
  if (rc == HC_OK) rc = dev_alloc(&b->d_counter, 1, "cudaMalloc(batch counter)");
  if (rc == HC_OK) rc = dev_alloc(&b->d_filters, filter_words, "cudaMalloc(batch filters)");
  if (rc == HC_OK) rc = dev_alloc(&b->d_ws, ws_bytes, "cudaMalloc(batch workspace)");
  if (rc != HC_OK) {
    delete b;
    return rc;
  }
  for (size_t i = 0; i < nq; ++i) {
    SearchArgs& a = b->host_args[i];
    a.F = b->d_filters + f_off[i];
    if (a.records == 0) continue;
    a.cta_total = reinterpret_cast<unsigned long long*>(b->d_ws + ws_off[i]);
    a.cta_overflow = a.cta_total + a.records;
    a.region = reinterpret_cast<uint32_t*>(a.cta_overflow + a.records);
  }
  b->ntiles = tiles.size();
  b->netiles = etiles.size();
  b->ws_bytes = ws_bytes;
  e = cudaMemcpy(b->d_args, b->host_args.data(), nq * sizeof(SearchArgs), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tiles.empty())
    e = cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !etiles.empty())
    e = cudaMemcpy(b->d_etiles, etiles.data(), etiles.size() * sizeof(EmitTile), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    delete b;
    return cuda_error(e, "cudaMemcpy(batch tables)");
  }

  b->lay.f_bytes = (f_max + 15u) & ~15u;
  b->lay.x_bytes = x_max;
  b->lay.ring_bytes = ring_max;
  b->smem_pre = f_max;
  b->smem_scan = size_t(b->lay.f_bytes) + b->lay.x_bytes + size_t(kSlots) * kThreads * 4 +
                 size_t(kWarps) * b->lay.ring_bytes;
  b->smem_emit = size_t(b->lay.f_bytes) + size_t(kSlots) * kThreads * 4;
  if (b->smem_scan + 2048 > di.smem_optin) {
    delete b;
    return set_error(HC_ERR_ARG, "hc_batch_create: filter and staging buffers exceed shared memory");
  }
  rc = set_kernel_smem(reinterpret_cast<const void*>(hc_batch_preprocess_kernel), std::max<size_t>(b->smem_pre, 1));
  if (rc == HC_OK) rc = set_kernel_smem(reinterpret_cast<const void*>(hc_batch_scan_kernel), b->smem_scan);
  if (rc == HC_OK) rc = set_kernel_smem(reinterpret_cast<const void*>(hc_batch_emit_kernel), b->smem_emit);
  int per_sm = 0;
  if (rc == HC_OK) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hc_batch_scan_kernel, kThreads, b->smem_scan);
    if (e != cudaSuccess) rc = cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(batch)");
  }
  if (rc != HC_OK) {
    delete b;
    return rc;
  }
  b->grid_scan = static_cast<int>(std::min<unsigned long long>(
      std::max(per_sm, 1) * static_cast<unsigned long long>(di.sm_count), std::max<unsigned long long>(b->ntiles, 1)));
  *out = reinterpret_cast<hc_batch*>(b);
  return HC_OK;
}

int hc_batch_run(hc_batch* bp, hc_stream_t stream_) {
  clear_error();
  Batch* b = as_batch(bp);
  if (b == nullptr) return set_error(HC_ERR_ARG, "hc_batch_run: invalid batch");
  if (b->nq == 0) return HC_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != b->dev) return set_error(HC_ERR_STATE, "hc_batch_run: batch belongs to another device");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  TimingToken t0 = timing_begin(kKindPreprocess, stream);
  hc_batch_preprocess_kernel<<<static_cast<unsigned>(b->nq), kThreads, b->smem_pre, stream>>>(
      b->d_args, b->d_counter);
  cudaError_t e = cudaGetLastError();
  timing_end(t0, stream);
  if (e != cudaSuccess) return cuda_error(e, "hc_batch_preprocess_kernel launch");
  if (b->ntiles > 0) {
    TimingToken t1 = timing_begin(kKindBatch, stream);
    hc_batch_scan_kernel<<<b->grid_scan, kThreads, b->smem_scan, stream>>>(
        b->d_args, b->d_tiles, b->ntiles, b->d_counter, b->lay);
    e = cudaGetLastError();
    timing_end(t1, stream);
    if (e != cudaSuccess) return cuda_error(e, "hc_batch_scan_kernel launch");
    TimingToken t2 = timing_begin(kKindEmit, stream);
    hc_batch_emit_kernel<<<static_cast<unsigned>(b->netiles * kEmitSplit), kThreads, b->smem_emit, stream>>>(
        b->d_args, b->d_etiles);
    e = cudaGetLastError();
    timing_end(t2, stream);
    if (e != cudaSuccess) return cuda_error(e, "hc_batch_emit_kernel launch");
    g_launches.fetch_add(3);
  } else {
    g_launches.fetch_add(1);
  }
  return HC_OK;
}

int hc_batch_info(const hc_batch* bp, uint64_t* tiles, uint64_t* records, uint64_t* workspace_bytes) {
  Batch* b = as_batch(bp);
  if (b == nullptr) return set_error(HC_ERR_ARG, "hc_batch_info: invalid batch");
  if (tiles) *tiles = b->ntiles;
  if (records) *records = b->records;
  if (workspace_bytes) *workspace_bytes = b->ws_bytes;
  return HC_OK;
}

int hc_batch_filter(const hc_batch* bp, size_t query, uint32_t* F, size_t nwords, uint32_t* hv) {
  clear_error();
  Batch* b = as_batch(bp);
  if (b == nullptr || query >= b->nq) return set_error(HC_ERR_ARG, "hc_batch_filter: invalid batch or query");
  const SearchArgs& a = b->host_args[query];
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
