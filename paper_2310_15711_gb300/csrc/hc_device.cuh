// hc_device.cuh -- inline-PTX helpers for sm_103a: mbarriers, 1-D bulk
// copies (TMA, cp.async.bulk) global -> shared, relaxed gpu-scope loads and
// stores for the chunk look-back, and a bounded-wait clock.
#pragma once

#include <cstdint>

namespace hc {

// Checked builds (compiled with HC_CHECKED, the library's test variant):
// HC_IN_BOUNDS(cond) tests an index condition and counts a failure in this
// translation unit's violation counter (read by hc_check_bounds); callers
// then skip or clamp the access instead of making it.  In the regular build
// it is `true` and the condition is not evaluated.
#ifdef HC_CHECKED
static __device__ unsigned long long g_bound_violations;
__device__ __forceinline__ bool checked_bound(bool ok) {
  if (!ok) atomicAdd(&g_bound_violations, 1ull);
  return ok;
}
#define HC_IN_BOUNDS(cond) (::hc::checked_bound(cond))
#else
#define HC_IN_BOUNDS(cond) (true)
#endif

// Upper bounds for every device-side wait.  A wait that exceeds them sets the
// library's status flag and makes the kernel return instead of spinning on.
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s of %globaltimer
constexpr uint32_t kMaxSpins = 1u << 26;          // hard iteration cap

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// 1-D bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned)
// from global to this CTA's shared memory; completion is signalled on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Programmatic dependent launch (sm_90 and later): a kernel that calls
// pdl_launch_dependents lets the next kernel of its stream, when that one was
// launched with programmatic stream serialization, start before it ends; the
// dependent kernel's pdl_wait returns once this grid has completed and its
// memory operations are visible.  Without the launch attribute both are
// no-ops and the kernels run one after the other as usual.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Waits for phase `parity` of `bar` to complete; false if the wait gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t spins = 0; spins < kMaxSpins; ++spins) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spins & 63u) == 63u && global_timer_ns() - t0 > kWaitLimitNs) return false;
  }
  return false;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

// Exclusive prefix sum over the lanes of a warp (all 32 lanes call it).
__device__ __forceinline__ unsigned long long warp_excl_scan_u64(unsigned long long v) {
  const int lane = threadIdx.x & 31;
  unsigned long long x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long o = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += o;
  }
  return x - v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

}  // namespace hc

namespace hc {
// Invalidates an mbarrier whose phases are all complete, so that its memory
// can be initialised again.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
}  // namespace hc
