// nbfd_decode_noalloc: the decoding loop of nbfd_decode with its scratch (messages in both
// directions, per-edge syndrome words, active-frame lists and counters) in a fixed device array
// that belongs to the library, so that the call allocates nothing.
//
// Who needs it: programs that may not allocate device memory while they decode -- for example a
// receiver whose device memory is reserved up front by another runtime (a framework's caching
// allocator or a signal-processing pipeline that claims the whole GPU at start-up), or a real-time
// loop that forbids cudaMalloc/cudaFree because they can synchronise the device and take
// unbounded time. The array costs NBFD_NOALLOC_SCRATCH_BYTES on every device that loads the
// library, until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "nbfd_internal.h"

using namespace nbfd;

// The scratch itself. In host code this name is only a host-side stand-in for the device
// variable: the device address must come from cudaGetSymbolAddress (below), never from &name.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NBFD_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_addr_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch on device `dev` (which must be current). Looked up once per
// device, on the first call made on that device.
int scratch_address(int dev, void **out) {
  if (dev < 0 || dev >= kMaxDevices) return set_error(NBFD_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (g_addr[dev] == nullptr) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return check_cuda(e, "cudaGetSymbolAddress(no-allocation scratch)");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return NBFD_OK;
}

}  // namespace

extern "C" int nbfd_decode_noalloc(const nbfd_code *c, int F, const float *llr, int max_iter,
                                   int form, uint16_t *symbols, uint8_t *ok, int32_t *iters,
                                   void *stream_) {
  if (!c) return set_error(NBFD_EINVAL, "code is NULL");
  if (F < 0) return set_error(NBFD_EINVAL, "n_frames < 0");
  if (max_iter < 1) return set_error(NBFD_EINVAL, "max_iter must be >= 1");
  if (!form_supported(form, c->m)) return set_error(NBFD_ENOTSUP, "form %d not supported", form);
  if (F == 0) return NBFD_OK;
  if (!llr || !symbols || !ok || !iters) return set_error(NBFD_EINVAL, "NULL buffer");
  int dev = -1;
  if (int st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return st;
  if (dev != c->device)
    return set_error(NBFD_EINVAL, "current device %d differs from the code's device %d", dev,
                     c->device);
  // the very layout nbfd_decode uses (message words of 2 or 4 bytes by the form), checked whole
  // against the array before any of it is touched
  const DecodeScratch probe = carve_decode_scratch(c, F, max_iter, form, nullptr);
  if (probe.bytes > (size_t)NBFD_NOALLOC_SCRATCH_BYTES)
    return set_error(NBFD_ENOMEM,
                     "%d frames need %zu bytes of scratch, above the %zu-byte fixed array of "
                     "nbfd_decode_noalloc; decode fewer frames per call or use nbfd_decode",
                     F, probe.bytes, (size_t)NBFD_NOALLOC_SCRATCH_BYTES);
  void *base = nullptr;
  if (int st = scratch_address(dev, &base)) return st;
  const DecodeScratch w = carve_decode_scratch(c, F, max_iter, form, static_cast<char *>(base));
  // Pageable host words: a device-to-host copy into pageable memory has completed when
  // cudaMemcpyAsync returns, and they cost no pinned allocation. The kernel timers are left off
  // (they create CUDA events).
  int32_t host_words[2] = {0, 0};
  return decode_loop(c, F, llr, max_iter, form, symbols, ok, iters, w, host_words, false,
                     static_cast<cudaStream_t>(stream_));
}
