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

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Scratch {
  float *v2c, *c2v;
  uint8_t *fsyn;
  int32_t *list[2];
  int32_t *count;
  int32_t *stats;
};

// Same partition as nbfd_decode's workspace (its size is nbfd_decode_workspace_size()).
Scratch carve(const nbfd_code *c, int F, int max_iter, char *base) {
  Scratch w{};
  const size_t msg = align256((size_t)F * c->E * c->q * sizeof(float));
  size_t off = 0;
  w.v2c = reinterpret_cast<float *>(base + off);
  off += msg;
  w.c2v = reinterpret_cast<float *>(base + off);
  off += msg;
  w.fsyn = reinterpret_cast<uint8_t *>(base + off);
  off += align256((size_t)F * c->E);
  w.list[0] = reinterpret_cast<int32_t *>(base + off);
  off += align256((size_t)F * 4);
  w.list[1] = reinterpret_cast<int32_t *>(base + off);
  off += align256((size_t)F * 4);
  w.count = reinterpret_cast<int32_t *>(base + off);
  off += align256((size_t)(max_iter + 2) * 4);
  w.stats = reinterpret_cast<int32_t *>(base + off);
  return w;
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
  const size_t need = nbfd_decode_workspace_size(c, F, max_iter, form);
  if (need > (size_t)NBFD_NOALLOC_SCRATCH_BYTES)
    return set_error(NBFD_ENOMEM,
                     "%d frames need %zu bytes of scratch, above the %zu-byte fixed array of "
                     "nbfd_decode_noalloc; decode fewer frames per call or use nbfd_decode",
                     F, need, (size_t)NBFD_NOALLOC_SCRATCH_BYTES);
  void *base = nullptr;
  if (int st = scratch_address(dev, &base)) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream_);
  Scratch w = carve(c, F, max_iter, static_cast<char *>(base));
  // The array keeps whatever the previous call left: clear every counter this call relies on.
  if (int st = check_cuda(cudaMemsetAsync(w.count, 0, (size_t)(max_iter + 2) * 4, s), "cudaMemsetAsync"))
    return st;
  if (int st = check_cuda(cudaMemsetAsync(w.stats, 0, 64, s), "cudaMemsetAsync")) return st;
  if (int st = check_cuda(cudaMemsetAsync(ok, 0, (size_t)F, s), "cudaMemsetAsync")) return st;
  if (int st = check_cuda(launch_init(c, F, llr, nullptr, w.v2c, w.list[1], w.count + 1, s,
                                      stores_f16(form)),
                          "init kernel"))
    return st;
  int32_t active = F;  // pageable host word: the copy below completes before it returns
  // the last few GF(256) frames: one launch for all their remaining iterations (as nbfd_decode)
  const bool symbol = (form & NBFD_DECIDE_SYMBOL) != 0;
  int tail_ctas = 0;
  const int tail_max = (form & 0xff) == NBFD_FORM_FP32_FWHT && !stores_f16(form)
                           ? tail_clusters(c, symbol, &tail_ctas)
                           : 0;
  for (int it = 1; it <= max_iter && active > 0; ++it) {
    if (active <= tail_max) {
      FrameSet fs;
      fs.list = w.list[it & 1];
      fs.count = w.count + it;
      fs.n_static = active;
      if (int st = check_cuda(launch_tail_x2(c, fs, llr, w.v2c, w.c2v, symbols, w.fsyn, it,
                                             max_iter, ok, iters, w.stats, s, symbol),
                              "tail kernel"))
        return st;
      return check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    }
    FrameSet fs;
    fs.list = w.list[it & 1];
    fs.count = w.count + it;
    fs.n_static = F;
    if (int st = check_cuda(launch_check(c, fs, w.v2c, w.c2v, s, nullptr, {}, {}, stores_f16(form)),
                            "check kernel"))
      return st;
    if (int st = check_cuda(launch_var(c, fs, form, llr, w.c2v, w.v2c, symbols, w.fsyn, s),
                            "variable kernel"))
      return st;
    if (int st = check_cuda(launch_stop(c, fs, symbols, w.fsyn, it, max_iter,
                                        w.list[(it + 1) & 1], w.count + it + 1, ok, iters,
                                        w.stats, s),
                            "stop kernel"))
      return st;
    if (int st = check_cuda(cudaMemcpyAsync(&active, w.count + it + 1, sizeof(int32_t),
                                            cudaMemcpyDeviceToHost, s),
                            "cudaMemcpyAsync(count)"))
      return st;
    if (int st = check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize")) return st;
  }
  return NBFD_OK;
}
