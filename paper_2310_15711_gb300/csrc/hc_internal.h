// hc_internal.h -- private declarations shared by the library's translation
// units (host filter object, error reporting, launch bookkeeping).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "hc.h"

namespace hc {

constexpr uint32_t kFilterMagic = 0x48433331u;  // "HC31"
constexpr int kMaxQ = 8;
constexpr int kMaxAlpha = 15;

// Host-side filter (Sec. 3.1): F, s, F' (mask), H_v and a copy of x, plus a
// lazily made device image laid out as [F: 2^alpha uint32][x: m bytes],
// 16-byte aligned.
struct Filter {
  uint32_t magic = kFilterMagic;
  size_t m = 0;
  int q = 0, alpha = 0, s = 0;
  uint32_t mask = 0, hv = 0;
  std::vector<uint32_t> F;
  std::vector<uint8_t> x;
  std::mutex mu;
  int dev = -1;
  uint8_t* dev_image = nullptr;  // owned, cudaMalloc'd
  size_t image_bytes() const { return (F.size() * 4 + m + 15) & ~size_t(15); }
  const uint32_t* dev_F() const { return reinterpret_cast<const uint32_t*>(dev_image); }
  const uint8_t* dev_x() const { return dev_image + F.size() * 4; }
};

inline Filter* as_filter(const hc_filter* f) {
  auto* p = reinterpret_cast<Filter*>(const_cast<hc_filter*>(f));
  return (p != nullptr && p->magic == kFilterMagic) ? p : nullptr;
}

// uint64 outputs (positions, counts) need their natural alignment; NULL passes.
inline bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0u; }

// Error reporting: per-thread last message.
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* where);
void clear_error();

// Counts launches of this library's kernels.
extern std::atomic<uint64_t> g_launches;

// Kernel families for hc_timing_report.
enum KernelKind {
  kKindScanStaged = 0,
  kKindScanDirect = 1,
  kKindScanDense = 2,
  kKindEmit = 3,
  kKindPreprocess = 4,
  kKindBatch = 5,
  kKindInit = 6,
  kNumKinds = 7
};
extern const char* const kKindNames[kNumKinds];

// Kernel timing (profiling aid).  When enabled, timing_begin/timing_end
// record a CUDA event pair around a launch; hc_timing_report sums them.
bool timing_enabled();
struct TimingToken {
  cudaEvent_t ev0 = nullptr;
  int kind = -1;
  bool active() const { return ev0 != nullptr; }
};

// Launches kernel fn on `stream`; with pdl, as a programmatic dependent of
// the kernel before it in the stream (which must call pdl_launch_dependents
// and fn must call pdl_wait before reading that kernel's results): the launch
// and the kernel's prologue overlap the previous kernel's tail.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*fn)(KArgs...), unsigned grid, unsigned block, size_t smem,
                             cudaStream_t stream, bool pdl, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, fn, std::forward<Args>(args)...);
}
TimingToken timing_begin(int kind, cudaStream_t stream);
void timing_end(const TimingToken& t, cudaStream_t stream);

// Checked builds: the bounds violations counted by the kernels of
// hc_search.cu and hc_batch.cu since the last call (then reset).
int take_bound_violations_search(uint64_t* count);
int take_bound_violations_batch(uint64_t* count);
int take_bound_violations_dense(uint64_t* count);

// Copies the filter to the current device (once).  Returns an HC_* code.
int filter_to_device(Filter* f);

// Device properties cached per device.
struct DeviceInfo {
  int sm_count = 0;
  size_t smem_optin = 0;
};
const DeviceInfo& device_info(int dev);

// The library's stream-ordered memory pool of a device (workspaces); it keeps
// freed memory for reuse instead of returning it to the driver.
cudaMemPool_t device_pool(int dev);

// Launch shape of one search (two kernels: scan, emit) and its workspace.
struct SearchArgs;
using KernelFn = void (*)(const SearchArgs);
struct SearchPlan {
  int kind = HC_MODE_STAGED;      // HC_MODE_STAGED, HC_MODE_DIRECT or HC_MODE_DENSE
  int L = 0;                      // window starts per thread
  uint32_t C = 0;                 // window starts per chunk
  int stages = 0;                 // staging buffers per CTA
  uint32_t stage_bytes = 0, x_smem = 0;
  size_t smem_scan = 0, smem_emit = 0;
  KernelFn scan = nullptr, emit = nullptr;
  unsigned long long num_chunks = 0, chunks_per_cta = 0, grid = 0, region_entries = 0;
  unsigned long long records = 0;  // spill records: one per CTA (one per warp when dense)
  unsigned long long emit_group = 0, emit_ctas = 0;  // emit kernel: records per CTA group, CTAs
  bool spec = false;              // warp-speculative HC (staged/direct kinds)
  bool unchecked = false;         // staged: padded buffers, no position test per first test
  bool pos32 = false;             // positions written as uint32
  size_t ws_bytes = 0;            // workspace bytes (device), no zeroing needed
  // single-pass dense form: an init kernel zeroes the tile ticket and the
  // tile descriptors, then the scan writes positions and the count itself
  // (no spill regions, no emit kernel)
  bool single_pass = false;
  KernelFn init = nullptr;
  int tile_chunks = 0, flag_steps = 0;
  unsigned long long max_tiles = 0;  // descriptors in the workspace
  // bitmap form of the dense scan: one bit per window start in the
  // workspace instead of spill regions; the emit kernel expands the bits
  bool bitmap = false;
  unsigned long long bitmap_bytes = 0;
};

int plan_search(const Filter* f, size_t n, size_t cap, const hc_search_opts* o, int dev,
                SearchPlan* out);
// The single-pass dense scan for a given q and its init kernel (hc_dense.cu).
KernelFn dense_single_pass_kernel_for_q(int q);
KernelFn single_pass_init_kernel();
// The emit kernel of the dense scan's bitmap form (hc_dense.cu).
KernelFn emit_bitmap_kernel();
// Device address of the library's status word on the current device.
unsigned int* status_word();
int launch_planned(const Filter* f, const SearchPlan& p, const uint8_t* y, size_t n,
                   uint64_t* pos, size_t cap, uint64_t* count_dev, void* ws,
                   cudaStream_t stream);
int launch_planned_filter_ptrs(const Filter* f, const SearchPlan& p, const uint32_t* F_dev,
                               const uint8_t* x_dev, const uint8_t* y, size_t n, uint64_t* pos,
                               size_t cap, uint64_t* count_dev, void* ws, cudaStream_t stream);

}  // namespace hc
