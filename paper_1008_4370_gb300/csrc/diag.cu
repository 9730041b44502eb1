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

// ---- FP32 FMA rate ---------------------------------------------------------------------------
// Peak of the FP32 pipe (no tensor cores): every thread runs 8 independent FMA chains
// a = a * x + y (x slightly below 1, so the values converge and never overflow or go subnormal),
// scalar fmaf or packed __ffma2_rn (two lanes per instruction). The chains' sum is stored only if
// it equals a value it cannot reach, which keeps them live without a store per thread.
namespace {

constexpr int kFmaThreads = 256;
constexpr int kFmaChains = 8;

template <bool kPacked>
__global__ void __launch_bounds__(kFmaThreads) k_fma_rate(long long iters, float x, float y,
                                                          float *sink) {
  float s = 0.0f;
  if constexpr (kPacked) {
    float2 a[kFmaChains];
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i)
      a[i] = make_float2(1e-3f * (threadIdx.x & 7) + i, 0.5f * i);
    const float2 xx = make_float2(x, x), yy = make_float2(y, y);
    for (long long n = 0; n < iters; ++n) {
#pragma unroll
      for (int i = 0; i < kFmaChains; ++i) a[i] = __ffma2_rn(a[i], xx, yy);
    }
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i) s += a[i].x + a[i].y;
  } else {
    float a[kFmaChains];
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i) a[i] = 1e-3f * (threadIdx.x & 7) + i;
    for (long long n = 0; n < iters; ++n) {
#pragma unroll
      for (int i = 0; i < kFmaChains; ++i) a[i] = fmaf(a[i], x, y);
    }
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i) s += a[i];
  }
  if (s == -1.0f) *sink = s;  // the chains stay positive: never taken
}

}  // namespace

extern "C" int nbfd_diag_fp32_rate(int packed, int blocks_per_sm, long long iters, double *tflops,
                                   double *ms, void *stream_) {
  if (blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || iters > (1LL << 30) || !tflops)
    return set_error(NBFD_EINVAL, "blocks_per_sm in [1, 8], iters in [1, 2^30], tflops != NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream_);
  float *sink = nullptr;
  if (int st = check_cuda(cudaMallocAsync(reinterpret_cast<void **>(&sink), 4, s), "cudaMallocAsync"))
    return st;
  cudaEvent_t a = nullptr, b = nullptr;
  int st = check_cuda(cudaEventCreate(&a), "cudaEventCreate");
  if (!st) st = check_cuda(cudaEventCreate(&b), "cudaEventCreate");
  const int grid = sm_count() * blocks_per_sm;
  if (!st) {
    // one launch to warm up the clocks and the instruction cache, then the timed one
    for (int rep = 0; rep < 2 && !st; ++rep) {
      if (rep == 1) cudaEventRecord(a, s);
      if (packed)
        k_fma_rate<true><<<grid, kFmaThreads, 0, s>>>(iters, 0.9999999f, 1e-7f, sink);
      else
        k_fma_rate<false><<<grid, kFmaThreads, 0, s>>>(iters, 0.9999999f, 1e-7f, sink);
      st = check_cuda(cudaGetLastError(), "FMA-rate kernel");
    }
    if (!st) cudaEventRecord(b, s);
  }
  float t = 0.0f;
  if (!st) st = check_cuda(cudaEventSynchronize(b), "cudaEventSynchronize");
  if (!st) st = check_cuda(cudaEventElapsedTime(&t, a, b), "cudaEventElapsedTime");
  cudaFreeAsync(sink, s);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) return st;
  const double fma = (double)grid * kFmaThreads * kFmaChains * (packed ? 2.0 : 1.0) * (double)iters;
  *tflops = 2.0 * fma / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return NBFD_OK;
}
