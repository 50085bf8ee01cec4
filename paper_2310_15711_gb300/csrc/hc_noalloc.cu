// hc_noalloc.cu -- hc_search_noalloc: the search for callers that must not
// allocate device memory.
//
// Some callers cannot let a library allocate: applications whose device
// memory is planned in full by their own allocator or arena (a hidden
// cudaMalloc can exceed the plan, and cudaFree synchronises the device), and
// latency-critical paths where an allocator round trip is not allowed.  This
// entry point gives them the same search
// with every buffer provided: the caller passes the filter words and the
// pattern in device memory, the text, the output positions and the count;
// the scratch that holds each CTA's occurrences until their output offsets
// are known lives in one fixed array of this file, allocated when the
// library is loaded and held by every GPU that loads it until the process
// exits.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "hc_internal.h"

namespace hc {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr unsigned long long kNoAllocMaxPositions = 2000000ull;
// The spill form's scratch is at most 33 bytes per record (16 of totals, up
// to 16 of rounding of its region, 1 of its CTA's total) plus 4 per held
// position; records are capped so that any request within
// kNoAllocMaxPositions fits.
constexpr unsigned long long kNoAllocMaxRecords =
    (kNoAllocScratchBytes - 4 * kNoAllocMaxPositions) / 40;

// Scratch of hc_search_noalloc: per-CTA totals and overflow marks, then the
// per-CTA spill regions.  Every entry the kernels read is written by the
// same call first, so it needs no clearing between calls.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
std::unordered_map<int, void*> g_scratch_addr;  // device -> device address of the scratch

// Looks up (once per device, with that device current) the device address of
// the scratch array; in host code the array's name is not a device address.
int scratch_for_device(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  auto it = g_scratch_addr.find(dev);
  if (it != g_scratch_addr.end()) {
    *out = it->second;
    return HC_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-alloc scratch)");
  g_scratch_addr.emplace(dev, p);
  *out = p;
  return HC_OK;
}

}  // namespace
}  // namespace hc

using namespace hc;

extern "C" int hc_search_noalloc(const hc_filter* fp, const uint32_t* F_dev, const uint8_t* x_dev,
                                 const uint8_t* y_dev, size_t n, uint64_t* pos_dev, size_t cap,
                                 uint64_t* count_dev, hc_stream_t stream_) {
  clear_error();
  Filter* f = as_filter(fp);
  if (f == nullptr) return set_error(HC_ERR_ARG, "hc_search_noalloc: invalid filter");
  if (F_dev == nullptr || x_dev == nullptr)
    return set_error(HC_ERR_ARG, "hc_search_noalloc: F_dev and x_dev are required");
  if (count_dev == nullptr || !aligned8(count_dev) || !aligned8(pos_dev))
    return set_error(HC_ERR_ARG, "hc_search_noalloc: count_dev NULL, or pos/count not 8-byte aligned");
  if (y_dev == nullptr && n > 0) return set_error(HC_ERR_ARG, "hc_search_noalloc: y_dev is NULL");
  if (pos_dev == nullptr && cap > 0)
    return set_error(HC_ERR_ARG, "hc_search_noalloc: pos_dev is NULL with cap > 0");
  if (pos_dev == nullptr) cap = 0;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (n < f->m) {
    cudaError_t e = cudaMemsetAsync(count_dev, 0, sizeof(uint64_t), stream);
    return e == cudaSuccess ? HC_OK : cuda_error(e, "cudaMemsetAsync(count)");
  }
  // positions held in the scratch until their output offsets are known
  const unsigned long long nwin = n - f->m + 1;
  const unsigned long long held = std::min<unsigned long long>(cap, nwin);
  if (held > kNoAllocMaxPositions) {
    char buf[200];
    std::snprintf(buf, sizeof buf,
                  "hc_search_noalloc: min(cap, n-m+1) = %llu exceeds the %llu positions its "
                  "fixed scratch holds; use a smaller cap or hc_search_async",
                  held, kNoAllocMaxPositions);
    return set_error(HC_ERR_ARG, buf);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  void* scratch = nullptr;
  int rc = scratch_for_device(dev, &scratch);
  if (rc != HC_OK) return rc;
  hc_search_opts o{};
  o.struct_size = sizeof o;
  o.spill_entries = std::max<unsigned long long>(held, 1);
  // one record per warp: at most kNoAllocMaxRecords of them on this device
  const unsigned long long sms = static_cast<unsigned long long>(device_info(dev).sm_count);
  o.ctas_per_sm = static_cast<int>(std::max<unsigned long long>(1, kNoAllocMaxRecords / (8 * std::max(sms, 1ull))));
  SearchPlan p;
  rc = plan_search(f, n, cap, &o, dev, &p);
  if (rc != HC_OK) return rc;
  if (p.single_pass && p.ws_bytes > kNoAllocScratchBytes) {
    // too many tiles for the scratch (a text of tens of GB): the spill form
    o.single_pass = -1;
    rc = plan_search(f, n, cap, &o, dev, &p);
    if (rc != HC_OK) return rc;
  }
  if (p.ws_bytes > kNoAllocScratchBytes) {
    char buf[200];
    std::snprintf(buf, sizeof buf,
                  "hc_search_noalloc: this search needs %zu bytes of scratch, above the fixed %zu",
                  p.ws_bytes, kNoAllocScratchBytes);
    return set_error(HC_ERR_ARG, buf);
  }
  return launch_planned_filter_ptrs(f, p, F_dev, x_dev, y_dev, n, pos_dev, cap, count_dev,
                                    scratch, stream);
}
