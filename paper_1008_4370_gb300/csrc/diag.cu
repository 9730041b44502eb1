// Diagnostic: the expiry path of the kernels' bounded mbarrier waits, exercised on purpose.
//
// One thread arms an mbarrier for 16 bytes of bulk-copy data that no copy will ever deliver and
// waits on it with the same bounded wait the decoding kernels use, but with a budget given by
// the caller. Nothing is in flight, nothing faults: the wait runs out, the kernel writes
// NBFD_ETIMEDOUT into a status word and returns, and the host reports it the way nbfd_decode does.
#include <cuda_runtime.h>

#include <cstdint>

#include "bulk_copy.cuh"
#include "nbfd_internal.h"

using namespace nbfd;

namespace {

__global__ void k_wait_expiry(long long budget_cycles, int32_t *status) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  mbar_expect_tx(&bar, 16u);  // the arrival happens; the 16 bytes never come
  const bool ok = mbar_wait_bounded(&bar, 0u, budget_cycles);
  *status = ok ? NBFD_OK : NBFD_ETIMEDOUT;
}

}  // namespace

extern "C" int nbfd_diag_wait_expiry(long long budget_cycles, void *stream_) {
  if (budget_cycles < 0 || budget_cycles > kWaitBudgetCycles)
    return set_error(NBFD_EINVAL, "budget must be in [0, %lld] cycles", kWaitBudgetCycles);
  cudaStream_t s = static_cast<cudaStream_t>(stream_);
  int32_t *d = nullptr;
  if (int st = check_cuda(cudaMallocAsync(reinterpret_cast<void **>(&d), 4, s), "cudaMallocAsync"))
    return st;
  int32_t h = -1;
  int st = check_cuda(cudaMemsetAsync(d, 0xff, 4, s), "cudaMemsetAsync");
  if (!st) {
    k_wait_expiry<<<1, 32, 0, s>>>(budget_cycles, d);
    st = check_cuda(cudaGetLastError(), "diagnostic kernel");
  }
  if (!st) st = check_cuda(cudaMemcpyAsync(&h, d, 4, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
  cudaFreeAsync(d, s);
  if (!st) st = check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (st) return st;
  if (h == NBFD_ETIMEDOUT) return set_error(NBFD_ETIMEDOUT, "bounded wait expired (as arranged)");
  return h;
}
