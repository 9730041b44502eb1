// C ABI entry points that run kernels: the decoding loop (Section 2's four steps with the
// Log-Fourier rules of Section 3.2), the step-level calls and the kernel timers.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "nbfd_internal.h"

using namespace nbfd;

namespace {

// ---- kernel timers ------------------------------------------------------------------------
struct ProfTotals {
  double ms[NBFD_KERNEL_COUNT] = {};
  long long launches[NBFD_KERNEL_COUNT] = {};
  long long units[NBFD_KERNEL_COUNT] = {};
};
std::mutex g_prof_mu;
int g_prof_mask = 0;  // bit k: time kernel k
ProfTotals g_prof;

struct PendingTimer {
  int kernel;
  int iter;  // decoding iteration of the launch (0 = INITIALIZATION)
  cudaEvent_t a, b;
};

// CUDA events around every launch; the frames each launch processed are taken from the
// per-iteration active-frame counts once the decode is over.
std::vector<cudaEvent_t> g_event_pool;  // reused across decodes (guarded by g_prof_mu)

class Timers {
 public:
  explicit Timers(int mask) : on_(mask != 0), mask_(mask) {}
  ~Timers() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &p : pending_) {
      g_event_pool.push_back(p.a);
      g_event_pool.push_back(p.b);
    }
  }
  bool on() const { return on_; }
  void begin(int kernel, int iter, cudaStream_t s) {
    cur_on_ = on_ && ((mask_ >> kernel) & 1);
    if (!cur_on_) return;
    cur_ = {kernel, iter, get(), get()};
    cudaEventRecord(cur_.a, s);
  }
  void end(cudaStream_t s) {
    if (!cur_on_) return;
    cudaEventRecord(cur_.b, s);
    pending_.push_back(cur_);
  }
  // counts[i] = frames active in iteration i (counts[0] unused: INITIALIZATION covers F frames).
  void flush(const std::vector<int32_t> &counts, int F) {
    if (!on_) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &p : pending_) {
      float ms = 0.0f;
      if (cudaEventSynchronize(p.b) == cudaSuccess &&
          cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        g_prof.ms[p.kernel] += ms;
        g_prof.launches[p.kernel] += 1;
        g_prof.units[p.kernel] +=
            p.iter == 0 ? F : (p.iter < (int)counts.size() ? counts[p.iter] : 0);
      }
      g_event_pool.push_back(p.a);
      g_event_pool.push_back(p.b);
    }
    pending_.clear();
  }

 private:
  static cudaEvent_t get() {
    {
      std::lock_guard<std::mutex> lk(g_prof_mu);
      if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
      }
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  bool on_;
  int mask_;
  bool cur_on_ = false;
  PendingTimer cur_{};
  std::vector<PendingTimer> pending_;
};

int check_device(const nbfd_code *c) {
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != c->device)
    return set_error(NBFD_EINVAL, "current device %d differs from the code's device %d", dev,
                     c->device);
  return NBFD_OK;
}

}  // namespace

// ---- workspace layout (shared by nbfd_decode and nbfd_decode_noalloc) -----------------------
namespace nbfd {

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

DecodeScratch carve_decode_scratch(const nbfd_code *c, int F, int max_iter, int form, char *base) {
  DecodeScratch w{};
  const size_t msg = align256((size_t)F * c->E * c->q * (stores_f16(form) ? 2 : 4));
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
  off += align256(16 * 4);
  w.bytes = off;
  return w;
}

}  // namespace nbfd

extern "C" int nbfd_prof_enable(int kernel_mask) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_mask = kernel_mask & ((1 << NBFD_KERNEL_COUNT) - 1);
  g_prof = ProfTotals{};
  return NBFD_OK;
}

extern "C" int nbfd_prof_get(int kernel, double *ms, long long *launches, long long *units) {
  if (kernel < 0 || kernel >= NBFD_KERNEL_COUNT) return set_error(NBFD_EINVAL, "bad kernel id");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (ms) *ms = g_prof.ms[kernel];
  if (launches) *launches = g_prof.launches[kernel];
  if (units) *units = g_prof.units[kernel];
  return NBFD_OK;
}

extern "C" size_t nbfd_decode_workspace_size(const nbfd_code *c, int n_frames, int max_iter,
                                             int form) {
  if (!c || n_frames < 0 || max_iter < 0) return 0;
  return carve_decode_scratch(c, n_frames, max_iter, form, nullptr).bytes;
}

// the disagreement count of the calling thread's last nbfd_decode or nbfd_decode_noalloc
// (nbfd_last_decode_stats)
static thread_local long long g_last_fourier_only = -1;

// A pinned host word per host thread for the active-frame count, allocated on first use and kept
// for the thread's lifetime (a per-call cudaMallocHost / cudaFreeHost pair would synchronise the
// device).
static int32_t *pinned_word() {
  struct Holder {
    int32_t *p = nullptr;
    ~Holder() {
      if (p) cudaFreeHost(p);
    }
  };
  thread_local Holder h;
  if (!h.p) {
    void *p = nullptr;
    if (cudaHostAlloc(&p, 2 * sizeof(int32_t), cudaHostAllocPortable) != cudaSuccess) return nullptr;
    h.p = static_cast<int32_t *>(p);
  }
  return h.p;
}

extern "C" int nbfd_last_decode_stats(long long *fourier_only_clears) {
  if (!fourier_only_clears) return set_error(NBFD_EINVAL, "NULL pointer");
  if (g_last_fourier_only < 0) return set_error(NBFD_EINVAL, "no nbfd_decode in this thread yet");
  *fourier_only_clears = g_last_fourier_only;
  return NBFD_OK;
}

namespace {
// nbfd_diag_preset_status: the value the next decode of this thread starts its status word with
thread_local int32_t g_preset_status = 0;
}  // namespace

extern "C" int nbfd_diag_preset_status(int32_t value) {
  g_preset_status = value;
  return NBFD_OK;
}

namespace nbfd {

int decode_loop(const nbfd_code *c, int F, const float *llr, int max_iter, int form,
                uint16_t *symbols, uint8_t *ok, int32_t *iters, const DecodeScratch &w,
                int32_t *host_words, bool timers, cudaStream_t s) {
  const bool f16 = stores_f16(form);
  int st = NBFD_OK;
  g_last_fourier_only = -1;
  int prof_mask = 0;
  if (timers) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_mask = g_prof_mask;
  }
  Timers tm(prof_mask);
  CheckTune check_tune;
  VarTune var_tune;
  tune_lookup(c, F, form, &check_tune, &var_tune);  // shapes from nbfd_autotune, if any
  const int32_t preset = g_preset_status;
  g_preset_status = 0;
  do {
    // the scratch may hold anything (a caller's workspace, or the previous no-allocation call's
    // leftovers): clear every counter and status word the loop relies on
    if ((st = check_cuda(cudaMemsetAsync(w.count, 0, (size_t)(max_iter + 2) * 4, s),
                         "cudaMemsetAsync")))
      break;
    if ((st = check_cuda(cudaMemsetAsync(w.stats, 0, 64, s), "cudaMemsetAsync"))) break;
    if (preset != 0) {
      host_words[0] = preset;
      if ((st = check_cuda(cudaMemcpyAsync(w.stats + 1, host_words, sizeof(int32_t),
                                           cudaMemcpyHostToDevice, s),
                           "cudaMemcpyAsync(preset status)")))
        break;
      // the copy reads host_words before host_words is written again below
      if ((st = check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize"))) break;
    }
    if ((st = check_cuda(cudaMemsetAsync(ok, 0, (size_t)F, s), "cudaMemsetAsync"))) break;
    // Once the frames left fit the tail kernel's resident clusters, one launch runs all their
    // remaining iterations (one thread-block cluster per frame).
    const bool symbol = (form & NBFD_DECIDE_SYMBOL) != 0;
    int tail_ctas = 0;
    const long long tail_max =
        (form & 0xff) == NBFD_FORM_FP32_FWHT && !f16 ? tail_clusters(c, symbol, &tail_ctas) : 0;
    // INITIALIZATION (+ list of iteration 1 = all frames, count[1] = F). V->C of both edges of a
    // variable is its Lambda0: with float storage, unless the tail kernel runs from the first
    // iteration, Lambda0 is written once per variable ([frame][variable][z], in the V->C buffer,
    // which the first variable-node launch overwrites) and the first check launch gathers it
    // per edge -- half the INITIALIZATION's writes (for q >= 64, where a vector is one bulk copy
    // of at least 256 bytes).
    const float *lambda0 = !f16 && F > tail_max && c->q >= 64 ? w.v2c : nullptr;
    // Small GF(16) codes: every frame decoded start to finish in one launch, its messages kept
    // in shared memory (bit-identical to the per-iteration path below)
    const bool fused = fused_small_applies(c, form);
    if (fused) {
      tm.begin(NBFD_KERNEL_FUSED, 0, s);
      if ((st = check_cuda(launch_fused_small(c, F, llr, symbols, ok, iters, w.stats, max_iter,
                                              symbol, s),
                           "fused small-code kernel")))
        break;
      tm.end(s);
    } else {
      tm.begin(NBFD_KERNEL_INIT, 0, s);
      if ((st = check_cuda(launch_init(c, F, llr, lambda0 ? w.v2c : nullptr,
                                       lambda0 ? nullptr : w.v2c, w.list[1], w.count + 1, s, f16),
                           "init kernel")))
        break;
      tm.end(s);
    }
    // The host reads the active-frame count every few iterations; in between it queues
    // iterations blindly (a launch with no active frame returns at once) and sizes each grid by
    // the last count it read, an upper bound since counts only shrink. With the tail kernel the
    // count is read every 4 iterations, so that the switch to it comes early; without it, every
    // 16 once few frames are left (a host round trip then costs as much as several iterations).
    long long active = fused ? 0 : F;
    int it = 1;
    while (st == NBFD_OK && it <= max_iter && active > 0) {
      if (active <= tail_max) {
        FrameSet fs;
        fs.list = w.list[it & 1];
        fs.count = w.count + it;
        fs.n_static = static_cast<int>(active);
        tm.begin(NBFD_KERNEL_TAIL, it, s);
        if ((st = check_cuda(launch_tail_x2(c, fs, llr, w.v2c, w.c2v, symbols, w.fsyn, it,
                                            max_iter, ok, iters, w.stats, s, symbol),
                             "tail kernel")))
          break;
        tm.end(s);
        if ((st = check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize"))) break;
        active = 0;
        break;
      }
      const int sync_every = active * 16 <= F && tail_max == 0 ? 16 : 4;
      const int last = it + sync_every - 1 < max_iter ? it + sync_every - 1 : max_iter;
      for (; it <= last; ++it) {
        FrameSet fs;
        fs.list = w.list[it & 1];
        fs.count = w.count + it;
        fs.n_static = static_cast<int>(active);
        tm.begin(NBFD_KERNEL_CHECK, it, s);
        if ((st = check_cuda(launch_check(c, fs, w.v2c, w.c2v, s, w.stats + 1, {}, check_tune, f16,
                                          it == 1 ? lambda0 : nullptr),
                             "check kernel")))
          break;
        tm.end(s);
        tm.begin(NBFD_KERNEL_VAR, it, s);
        if ((st = check_cuda(launch_var(c, fs, form, llr, w.c2v, w.v2c, symbols, w.fsyn, s,
                                        w.stats + 1, var_tune),
                             "variable kernel")))
          break;
        tm.end(s);
        tm.begin(NBFD_KERNEL_SYNDROME, it, s);
        if ((st = check_cuda(launch_stop(c, fs, symbols, w.fsyn, it, max_iter,
                                         w.list[(it + 1) & 1], w.count + it + 1, ok, iters,
                                         w.stats, s),
                             "stop kernel")))
          break;
        tm.end(s);
      }
      if (st) break;
      if ((st = check_cuda(cudaMemcpyAsync(host_words, w.count + it, sizeof(int32_t),
                                           cudaMemcpyDeviceToHost, s),
                           "cudaMemcpyAsync(count)")))
        break;
      if ((st = check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize"))) break;
      active = host_words[0];
    }
    if (st == NBFD_OK) {
      // stats[0] counts iterations where a frame's Fourier-domain syndrome cleared while its
      // GF(2^m) syndrome did not; stats[1] holds NBFD_ETIMEDOUT if a bounded wait expired
      if ((st = check_cuda(cudaMemcpyAsync(host_words, w.stats, 2 * sizeof(int32_t),
                                           cudaMemcpyDeviceToHost, s),
                           "cudaMemcpyAsync(status)")))
        break;
      if ((st = check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize"))) break;
      g_last_fourier_only = host_words[0];
      if (host_words[1] != 0)
        st = set_error(NBFD_ETIMEDOUT, "a bounded device-side wait expired (status %d)",
                       host_words[1]);
    }
    if (st == NBFD_OK && tm.on()) {
      std::vector<int32_t> counts((size_t)max_iter + 2, 0);
      if ((st = check_cuda(cudaMemcpy(counts.data(), w.count, counts.size() * 4,
                                      cudaMemcpyDeviceToHost),
                           "cudaMemcpy(counts)")))
        break;
      tm.flush(counts, F);
    }
  } while (false);
  return st;
}

}  // namespace nbfd

extern "C" int nbfd_decode(const nbfd_code *c, int F, const float *llr, int max_iter, int form,
                           uint16_t *symbols, uint8_t *ok, int32_t *iters, void *workspace,
                           size_t workspace_bytes, void *stream_) {
  if (!c) return set_error(NBFD_EINVAL, "code is NULL");
  if (F < 0) return set_error(NBFD_EINVAL, "n_frames < 0");
  if (max_iter < 1) return set_error(NBFD_EINVAL, "max_iter must be >= 1");
  if (!form_supported(form, c->m)) return set_error(NBFD_ENOTSUP, "form %d not supported", form);
  if (F == 0) return NBFD_OK;
  if (!llr || !symbols || !ok || !iters) return set_error(NBFD_EINVAL, "NULL buffer");
  if (int st = check_device(c)) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream_);
  const size_t need = nbfd_decode_workspace_size(c, F, max_iter, form);
  int32_t *host_words = pinned_word();
  if (!host_words) return set_error(NBFD_ECUDA, "cudaHostAlloc of the count word failed");
  bool owned = false;
  if (workspace == nullptr) {
    if (int st = check_cuda(cudaMallocAsync(&workspace, need, s), "cudaMallocAsync(workspace)"))
      return st;
    owned = true;
  } else if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)) {
    return set_error(NBFD_ENOMEM, "workspace of %zu bytes (need %zu, 256-byte aligned)",
                     workspace_bytes, need);
  }
  const DecodeScratch w = carve_decode_scratch(c, F, max_iter, form, static_cast<char *>(workspace));
  const int st = decode_loop(c, F, llr, max_iter, form, symbols, ok, iters, w, host_words, true, s);
  if (owned) cudaFreeAsync(workspace, s);
  return st;
}

// ---- step-level entry points ----------------------------------------------------------------

extern "C" int nbfd_init_messages(const nbfd_code *c, int F, const float *llr, float *lambda0,
                                  float *v2c, void *stream) {
  if (!c || F < 0) return set_error(NBFD_EINVAL, "bad argument");
  if (F == 0) return NBFD_OK;
  if (!llr) return set_error(NBFD_EINVAL, "llr is NULL");
  if (int st = check_device(c)) return st;
  return check_cuda(launch_init(c, F, llr, lambda0, v2c, nullptr, nullptr,
                                static_cast<cudaStream_t>(stream)),
                    "init kernel");
}

extern "C" int nbfd_init_messages_f16(const nbfd_code *c, int F, const float *llr, uint16_t *v2c,
                                      void *stream) {
  if (!c || F < 0) return set_error(NBFD_EINVAL, "bad argument");
  if (c->m != 8) return set_error(NBFD_ENOTSUP, "half message storage needs m = 8");
  if (F == 0) return NBFD_OK;
  if (!llr || !v2c) return set_error(NBFD_EINVAL, "NULL buffer");
  if (int st = check_device(c)) return st;
  return check_cuda(launch_init(c, F, llr, nullptr, reinterpret_cast<float *>(v2c), nullptr,
                                nullptr, static_cast<cudaStream_t>(stream), true),
                    "init kernel");
}

extern "C" int nbfd_check_update_f16(const nbfd_code *c, int F, const uint16_t *v2c, uint16_t *c2v,
                                     void *stream) {
  if (!c || F < 0) return set_error(NBFD_EINVAL, "bad argument");
  if (c->m != 8) return set_error(NBFD_ENOTSUP, "half message storage needs m = 8");
  if (F == 0) return NBFD_OK;
  if (!v2c || !c2v || v2c == c2v) return set_error(NBFD_EINVAL, "bad message buffers");
  if (int st = check_device(c)) return st;
  FrameSet fs;
  fs.n_static = F;
  return check_cuda(launch_check(c, fs, reinterpret_cast<const float *>(v2c),
                                 reinterpret_cast<float *>(c2v), static_cast<cudaStream_t>(stream),
                                 nullptr, {}, {}, true),
                    "check kernel");
}

extern "C" int nbfd_check_update(const nbfd_code *c, int F, const float *v2c, float *c2v,
                                 void *stream) {
  if (!c || F < 0) return set_error(NBFD_EINVAL, "bad argument");
  if (F == 0) return NBFD_OK;
  if (!v2c || !c2v || v2c == c2v) return set_error(NBFD_EINVAL, "bad message buffers");
  if (int st = check_device(c)) return st;
  FrameSet fs;
  fs.n_static = F;
  return check_cuda(launch_check(c, fs, v2c, c2v, static_cast<cudaStream_t>(stream)),
                    "check kernel");
}

extern "C" int nbfd_var_update(const nbfd_code *c, int F, int form, const float *llr,
                               const float *c2v, float *v2c, uint16_t *symbols, uint8_t *fsyn,
                               void *stream) {
  if (!c || F < 0) return set_error(NBFD_EINVAL, "bad argument");
  if (!form_supported(form, c->m)) return set_error(NBFD_ENOTSUP, "form %d not supported", form);
  if (F == 0) return NBFD_OK;
  if (!llr || !c2v || !v2c || v2c == c2v) return set_error(NBFD_EINVAL, "bad buffers");
  if (int st = check_device(c)) return st;
  FrameSet fs;
  fs.n_static = F;
  return check_cuda(launch_var(c, fs, form, llr, c2v, v2c, symbols, fsyn,
                               static_cast<cudaStream_t>(stream)),
                    "variable kernel");
}

extern "C" int nbfd_syndrome(const nbfd_code *c, int F, const uint16_t *symbols,
                             const uint8_t *fsyn, uint16_t *fourier, uint16_t *exact,
                             void *stream) {
  if (!c || F < 0) return set_error(NBFD_EINVAL, "bad argument");
  if (F == 0) return NBFD_OK;
  if (!symbols) return set_error(NBFD_EINVAL, "symbols is NULL");
  if (fourier && !fsyn) return set_error(NBFD_EINVAL, "fourier output needs fsyn");
  if (int st = check_device(c)) return st;
  return check_cuda(launch_syndrome(c, F, symbols, fsyn, fourier, exact,
                                    static_cast<cudaStream_t>(stream)),
                    "syndrome kernel");
}

// ---- conventional Log-SP (Section 2.2), step by step --------------------------------------

extern "C" int nbfd_logsp_init(const nbfd_code *c, int F, const float *llr, float *v2c,
                               void *stream) {
  if (!c || F < 0) return set_error(NBFD_EINVAL, "bad argument");
  if (!logsp_supported(c->m)) return set_error(NBFD_ENOTSUP, "Log-SP needs m in [3, 8]");
  if (F == 0) return NBFD_OK;
  if (!llr || !v2c) return set_error(NBFD_EINVAL, "NULL buffer");
  if (int st = check_device(c)) return st;
  return check_cuda(launch_logsp_var(c, F, llr, nullptr, v2c, nullptr, true,
                                     static_cast<cudaStream_t>(stream)),
                    "Log-SP initialization kernel");
}

extern "C" int nbfd_logsp_check_update(const nbfd_code *c, int F, const float *v2c, float *c2v,
                                       void *stream) {
  if (!c || F < 0) return set_error(NBFD_EINVAL, "bad argument");
  if (!logsp_supported(c->m) || c->k < 3)
    return set_error(NBFD_ENOTSUP, "Log-SP check node needs m in [3, 8] and k >= 3");
  if (F == 0) return NBFD_OK;
  if (!v2c || !c2v || v2c == c2v) return set_error(NBFD_EINVAL, "bad message buffers");
  if (int st = check_device(c)) return st;
  return check_cuda(launch_logsp_check(c, F, v2c, c2v, static_cast<cudaStream_t>(stream)),
                    "Log-SP check kernel");
}

extern "C" int nbfd_logsp_var_update(const nbfd_code *c, int F, const float *llr,
                                     const float *c2v, float *v2c, uint16_t *symbols,
                                     void *stream) {
  if (!c || F < 0) return set_error(NBFD_EINVAL, "bad argument");
  if (!logsp_supported(c->m)) return set_error(NBFD_ENOTSUP, "Log-SP needs m in [3, 8]");
  if (F == 0) return NBFD_OK;
  if (!llr || !c2v || !v2c || v2c == c2v) return set_error(NBFD_EINVAL, "bad buffers");
  if (int st = check_device(c)) return st;
  return check_cuda(launch_logsp_var(c, F, llr, c2v, v2c, symbols, false,
                                     static_cast<cudaStream_t>(stream)),
                    "Log-SP variable kernel");
}
