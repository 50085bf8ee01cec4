// hc_selftest.cu -- a check of the failure path every bulk-copy wait of the
// library takes: one thread waits on an mbarrier that nothing completes,
// with the same bounded wait the scan kernels use (mbar_wait_bounded: at
// most 2 s of %globaltimer and 2^26 polls).  The wait gives up, the thread
// sets the status flag as a stalled copy would, and the kernel returns:
// nothing hangs, and hc_check_status then reports HC_ERR_TIMEOUT.
#include "hc_device.cuh"
#include "hc_internal.h"

namespace hc {
namespace {

__global__ void hc_selftest_wait_kernel(unsigned int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);   // one arrival expected; none is made
  fence_mbar_init();
  if (!mbar_wait_bounded(&bar, 0u)) atomicOr(status, 1u);
}

}  // namespace
}  // namespace hc

using namespace hc;

extern "C" int hc_selftest_wait_timeout(hc_stream_t stream_) {
  clear_error();
  unsigned int* status = status_word();
  if (status == nullptr) return set_error(HC_ERR_CUDA, "device status word unavailable");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  hc_selftest_wait_kernel<<<1, 32, 0, stream>>>(status);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "hc_selftest_wait_kernel launch");
  g_launches.fetch_add(1);
  return HC_OK;
}
