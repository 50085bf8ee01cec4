// hc_host.cu -- host side of the library: the preprocessing phase (Sec. 3.1,
// Eq. 1-5), the filter object, its device copy, error reporting.
//
// The filter is built pair by pair rather than chain by chain: every q-gram
// hash is computed once (Eq. 3, Eq. 4), then every adjacent non-overlapping
// pair (x[i..i+q-1], x[i+q..i+2q-1]), 0 <= i <= m-2q, ORs lambda(h(left))
// into F[h(right)] (Eq. 1), then every first q-gram (start < min(q, m-q+1))
// whose word is still empty gets 1 (Eq. 2, first optimisation of Sec. 3.4).
// Both steps are order-independent (OR is commutative; the marking step only
// writes into words that the linking step left empty), so F equals the
// chain-ordered construction of the paper's Fig. 4 word for word.  H_v is the
// hash of the first q-gram of the chain ending at m-1, which starts at
// m mod q (Sec. 3.4).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <unordered_map>

#include "hc_internal.h"

namespace hc {

namespace {
thread_local std::string t_last_error;
std::mutex g_dev_mu;
std::unordered_map<int, DeviceInfo> g_dev_info;
}  // namespace

std::atomic<uint64_t> g_launches{0};

const char* const kKindNames[kNumKinds] = {"scan_staged", "scan_direct", "scan_dense",
                                           "emit", "preprocess", "batch", "lb_init"};

namespace {
std::atomic<bool> g_timing_on{false};
std::mutex g_timing_mu;
struct TimedLaunch {
  int kind;
  cudaEvent_t ev0, ev1;
};
std::vector<TimedLaunch> g_timed;       // recorded, not yet summed
std::vector<cudaEvent_t> g_event_pool;  // free events

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

bool timing_enabled() { return g_timing_on.load(std::memory_order_relaxed); }

TimingToken timing_begin(int kind, cudaStream_t stream) {
  TimingToken t;
  if (!timing_enabled()) return t;
  std::lock_guard<std::mutex> lk(g_timing_mu);
  t.ev0 = take_event();
  if (t.ev0 == nullptr) return t;
  if (cudaEventRecord(t.ev0, stream) != cudaSuccess) {
    cudaGetLastError();
    g_event_pool.push_back(t.ev0);
    t.ev0 = nullptr;
    return t;
  }
  t.kind = kind;
  return t;
}

void timing_end(const TimingToken& t, cudaStream_t stream) {
  if (t.ev0 == nullptr) return;
  std::lock_guard<std::mutex> lk(g_timing_mu);
  cudaEvent_t ev1 = take_event();
  if (ev1 == nullptr || cudaEventRecord(ev1, stream) != cudaSuccess) {
    cudaGetLastError();
    g_event_pool.push_back(t.ev0);
    if (ev1) g_event_pool.push_back(ev1);
    return;
  }
  g_timed.push_back({t.kind, t.ev0, ev1});
}

int set_error(int code, const std::string& msg) {
  t_last_error = msg;
  return code;
}

int cuda_error(cudaError_t e, const char* where) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s: %s (%s)", where, cudaGetErrorString(e),
                cudaGetErrorName(e));
  t_last_error = buf;
  return e == cudaErrorMemoryAllocation ? HC_ERR_NOMEM : HC_ERR_CUDA;
}

void clear_error() { t_last_error.clear(); }

const DeviceInfo& device_info(int dev) {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  auto it = g_dev_info.find(dev);
  if (it != g_dev_info.end()) return it->second;
  DeviceInfo di;
  cudaDeviceGetAttribute(&di.sm_count, cudaDevAttrMultiProcessorCount, dev);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  di.smem_optin = static_cast<size_t>(optin);
  return g_dev_info.emplace(dev, di).first->second;
}

cudaMemPool_t device_pool(int dev) {
  static std::mutex mu;
  static std::unordered_map<int, cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lk(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    cudaDeviceGetDefaultMemPool(&pool, dev);
  }
  uint64_t keep = ~0ull;  // never hand freed memory back to the driver
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  pools.emplace(dev, pool);
  return pool;
}

int filter_to_device(Filter* f) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(f->mu);
  if (f->dev_image != nullptr) {
    if (f->dev == dev) return HC_OK;
    return set_error(HC_ERR_STATE,
                     "filter already resides on another device; build one filter per device");
  }
  std::vector<uint8_t> img(f->image_bytes(), 0);
  std::memcpy(img.data(), f->F.data(), f->F.size() * 4);
  std::memcpy(img.data() + f->F.size() * 4, f->x.data(), f->m);
  void* p = nullptr;
  e = cudaMalloc(&p, img.size());
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(filter image)");
  e = cudaMemcpy(p, img.data(), img.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p);
    return cuda_error(e, "cudaMemcpy(filter image)");
  }
  f->dev_image = static_cast<uint8_t*>(p);
  f->dev = dev;
  return HC_OK;
}

}  // namespace hc

using namespace hc;

extern "C" {

int hc_version(void) { return 100; }

const char* hc_last_error(void) { return t_last_error.c_str(); }

uint64_t hc_kernel_launches(void) { return g_launches.load(); }

int hc_timing_enable(int on) {
  g_timing_on.store(on != 0);
  return HC_OK;
}

int hc_timing_report(double* ms, uint64_t* launches, int nkinds, int reset) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_timing_mu);
  std::vector<double> acc(kNumKinds, 0.0);
  std::vector<uint64_t> cnt(kNumKinds, 0);
  for (const TimedLaunch& t : g_timed) {
    cudaError_t e = cudaEventSynchronize(t.ev1);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventSynchronize(timing)");
    float v = 0.f;
    e = cudaEventElapsedTime(&v, t.ev0, t.ev1);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventElapsedTime(timing)");
    acc[t.kind] += v;
    cnt[t.kind] += 1;
  }
  for (int k = 0; k < nkinds && k < kNumKinds; ++k) {
    if (ms) ms[k] = acc[k];
    if (launches) launches[k] = cnt[k];
  }
  if (reset) {
    for (const TimedLaunch& t : g_timed) {
      g_event_pool.push_back(t.ev0);
      g_event_pool.push_back(t.ev1);
    }
    g_timed.clear();
  }
  return HC_OK;
}

const char* hc_timing_kind_name(int kind) {
  return (kind >= 0 && kind < kNumKinds) ? kKindNames[kind] : "";
}

int hc_preprocess(const uint8_t* x, size_t m, int q, int alpha, hc_filter** out) {
  clear_error();
  if (out == nullptr) return set_error(HC_ERR_ARG, "hc_preprocess: out is NULL");
  *out = nullptr;
  if (x == nullptr) return set_error(HC_ERR_ARG, "hc_preprocess: x is NULL");
  if (m == 0) return set_error(HC_ERR_ARG, "hc_preprocess: m must be >= 1");
  if (q < 1 || q > kMaxQ || static_cast<size_t>(q) > m)
    return set_error(HC_ERR_ARG, "hc_preprocess: need 1 <= q <= min(m, 8)");
  if (alpha < 1 || alpha > kMaxAlpha)
    return set_error(HC_ERR_ARG, "hc_preprocess: need 1 <= alpha <= 15");
  if (m > (size_t(1) << 30)) return set_error(HC_ERR_ARG, "hc_preprocess: m above 2^30");

  Filter* f = new (std::nothrow) Filter();
  if (f == nullptr) return set_error(HC_ERR_NOMEM, "hc_preprocess: out of host memory");
  try {
    f->m = m;
    f->q = q;
    f->alpha = alpha;
    f->s = alpha / q;                              // Eq. 4
    f->mask = (uint32_t(1) << alpha) - 1u;         // mod 2^alpha as an AND
    f->F.assign(size_t(1) << alpha, 0u);
    f->x.assign(x, x + m);

    // h of every q-gram, indexed by its start: h(u) = sum_k u[k] * 2^(s*k)
    // mod 2^alpha (Eq. 3), evaluated from the last character down.
    const size_t nq = m - static_cast<size_t>(q) + 1;
    std::vector<uint32_t> h(nq);
    for (size_t i = 0; i < nq; ++i) {
      uint32_t v = 0;
      for (int k = q - 1; k >= 0; --k) v = (v << f->s) + x[i + static_cast<size_t>(k)];
      h[i] = v & f->mask;
    }
    // Eq. 1 for every adjacent non-overlapping pair.
    for (size_t i = 0; i + 2 * static_cast<size_t>(q) <= m; ++i)
      f->F[h[i + q]] |= 1u << (h[i] & 31u);
    // Eq. 2, only into words still empty.
    const size_t nfirst = std::min(static_cast<size_t>(q), nq);
    for (size_t i = 0; i < nfirst; ++i)
      if (f->F[h[i]] == 0) f->F[h[i]] = 1u;
    f->hv = h[m % static_cast<size_t>(q)];
  } catch (const std::bad_alloc&) {
    delete f;
    return set_error(HC_ERR_NOMEM, "hc_preprocess: out of host memory");
  }
  *out = reinterpret_cast<hc_filter*>(f);
  return HC_OK;
}

void hc_filter_free(hc_filter* fp) {
  Filter* f = as_filter(fp);
  if (f == nullptr) return;
  if (f->dev_image != nullptr) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != f->dev) cudaSetDevice(f->dev);
    cudaFree(f->dev_image);
    if (cur != f->dev) cudaSetDevice(cur);
  }
  f->magic = 0;
  delete f;
}

int hc_filter_words(const hc_filter* fp, const uint32_t** F, size_t* nwords, uint32_t* hv) {
  Filter* f = as_filter(fp);
  if (f == nullptr) return set_error(HC_ERR_ARG, "hc_filter_words: invalid filter");
  if (F) *F = f->F.data();
  if (nwords) *nwords = f->F.size();
  if (hv) *hv = f->hv;
  return HC_OK;
}

int hc_filter_params(const hc_filter* fp, size_t* m, int* q, int* alpha, int* s) {
  Filter* f = as_filter(fp);
  if (f == nullptr) return set_error(HC_ERR_ARG, "hc_filter_params: invalid filter");
  if (m) *m = f->m;
  if (q) *q = f->q;
  if (alpha) *alpha = f->alpha;
  if (s) *s = f->s;
  return HC_OK;
}

int hc_filter_to_device(hc_filter* fp) {
  clear_error();
  Filter* f = as_filter(fp);
  if (f == nullptr) return set_error(HC_ERR_ARG, "hc_filter_to_device: invalid filter");
  return filter_to_device(f);
}

int hc_mapped_alloc(size_t bytes, void** host_ptr, void** dev_ptr) {
  clear_error();
  if (host_ptr == nullptr || dev_ptr == nullptr || bytes == 0)
    return set_error(HC_ERR_ARG, "hc_mapped_alloc: NULL output or zero size");
  *host_ptr = nullptr;
  *dev_ptr = nullptr;
  void* h = nullptr;
  cudaError_t e = cudaHostAlloc(&h, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
  if (e != cudaSuccess) return cuda_error(e, "cudaHostAlloc(mapped)");
  void* d = nullptr;
  e = cudaHostGetDevicePointer(&d, h, 0);
  if (e != cudaSuccess) {
    cudaFreeHost(h);
    return cuda_error(e, "cudaHostGetDevicePointer");
  }
  *host_ptr = h;
  *dev_ptr = d;
  return HC_OK;
}

void hc_mapped_free(void* host_ptr) {
  if (host_ptr != nullptr) cudaFreeHost(host_ptr);
}

}  // extern "C"
