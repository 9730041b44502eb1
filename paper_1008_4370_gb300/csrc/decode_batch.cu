// Uneven batches: frames of several codes (different N, k and q) decoded by one call, with the
// iteration loop replayed from a CUDA graph, and the autotuner that picks the launch shapes of
// the check and variable-node kernels.
//
// Graph. Each code gets its own workspace, with the loop state kept in device words: a ring of
// two active-frame lists and counts, and an iteration counter. Iteration t reads list/count
// t & 1 and its stop kernel appends the survivors to list/count (t + 1) & 1; the check kernel of
// the iteration increments the counter and clears the count the stop kernel will append to
// (LoopTick). Two consecutive iterations therefore have fixed arguments, and one graph holds
// two iterations of every code, each code a separate branch (forked streams during capture), so
// that the codes' kernels overlap once their active sets are small. The host replays the graph
// and reads the codes' active counts every few replays; an iteration past max_iter finds no
// active frame and does nothing.
//
// Autotuner. For a (device, code shape, frame count, form) it times candidate launch shapes on
// the real buffers (check kernel: warps per block x pipeline depth x blocks per SM;
// variable-node kernel: blocks per SM) with CUDA events and keeps the fastest. nbfd_decode and
// nbfd_decode_batch use a cached result when there is one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "nbfd_internal.h"

using namespace nbfd;

namespace {

// ---- tune cache ----------------------------------------------------------------------------
using TuneKey = std::tuple<int, int, int, int, int, int>;  // device, m, k, N, F, form & 0xff
struct TuneVal {
  CheckTune check;
  VarTune var;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

TuneKey key_of(const nbfd_code *c, int F, int form) {
  return TuneKey(c->device, c->m, c->k, c->N, F, form & 0xff);
}

float time_launches(cudaStream_t s, int reps, const std::function<cudaError_t()> &fn) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float ms = -1.0f;
  if (fn() == cudaSuccess) {  // warm
    cudaEventRecord(a, s);
    bool ok = true;
    for (int r = 0; r < reps && ok; ++r) ok = fn() == cudaSuccess;
    cudaEventRecord(b, s);
    if (ok && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  }
  cudaGetLastError();  // a rejected shape is not an error of the caller
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms < 0.0f ? -1.0f : ms / reps;
}

// Times the candidates on buffers whose v2c holds INITIALIZATION messages; leaves v2c
// overwritten (the caller runs INITIALIZATION again).
int tune_code(const nbfd_code *c, int F, int form, const float *llr, float *v2c, float *c2v,
              uint16_t *sym, uint8_t *fsyn, cudaStream_t s, TuneVal *out) {
  FrameSet fs;
  fs.n_static = F;
  const int epl = c->q < 8 ? c->q : 8;
  const int cpw = 32 * epl / c->q;
  const int sms = sm_count();
  const long long tiles = ((long long)F * c->M + cpw - 1) / cpw;
  TuneVal best{};
  float best_ms = -1.0f;
  for (int warps : {1, 2, 4, 8}) {
    for (int stages : {3, 4, 6}) {
      const size_t smem = 128 * 8 + (size_t)warps * stages * cpw * c->k * c->q * 4;
      if (smem > kMaxSmemPerBlock) continue;
      const int fit = static_cast<int>((228 * 1024) / (smem + 1024));
      // one wave (bps <= fit) and oversubscribed grids of 2, 4 and 8 waves
      for (int bps : {1, 2, 3, 4, 6, 2 * fit, 4 * fit, 8 * fit}) {
        const bool over = bps > 6;
        if (!over && bps > fit) continue;
        // shapes that cannot give every warp a tile (or, oversubscribed, four tiles) are not
        // worth timing
        if ((long long)bps * sms * warps * (over ? 4 : 1) > tiles * (over ? 1 : 2) && bps > 1)
          continue;
        CheckTune ct{warps, stages, bps};
        const float ms = time_launches(s, 3, [&] {
          return launch_check(c, fs, v2c, c2v, s, nullptr, {}, ct, stores_f16(form));
        });
        if (ms > 0.0f && (best_ms < 0.0f || ms < best_ms)) {
          best_ms = ms;
          best.check = ct;
        }
      }
    }
  }
  if (c->q >= 128) {  // the team variant: a block's warps share one pipeline of whole checks
    const long long checks = (long long)F * c->M;
    for (int stages : {3, 4, 6}) {
      const size_t smem = 128 + (size_t)stages * c->k * c->q * (stores_f16(form) ? 2 : 4);
      if (smem > kMaxSmemPerBlock) continue;
      const int fit = static_cast<int>((228 * 1024) / (smem + 1024));
      for (int bps : {1, 2, 3, 4, 6, 8, 2 * fit, 4 * fit, 8 * fit}) {
        const bool over = bps > fit;
        if (bps > 16 && !over) continue;
        if ((long long)bps * sms * (over ? 4 : 1) > checks * (over ? 1 : 2) && bps > 1) continue;
        CheckTune ct{0, stages, bps, 1};
        const float ms = time_launches(s, 3, [&] {
          return launch_check(c, fs, v2c, c2v, s, nullptr, {}, ct, stores_f16(form));
        });
        if (ms > 0.0f && (best_ms < 0.0f || ms < best_ms)) {
          best_ms = ms;
          best.check = ct;
        }
      }
    }
  }
  if (best_ms < 0.0f) return set_error(NBFD_ECUDA, "autotune: no check-kernel shape ran");
  best_ms = -1.0f;
  const bool x8 = (form & 0xff) == NBFD_FORM_FP32_FWHT && var_fwht6x8_applies(c);
  const std::vector<int> var_bps =
      (form & 0xff) == NBFD_FORM_FP32_FWHT && (c->m == 8 || x8)
          ? std::vector<int>{1, 2, 3, 4, 8, 16, 32}
          : std::vector<int>{1, 2, 4, 8, 16, 32};
  // the GF(64) kernel's block shapes: 4 warps (3 blocks per SM), 7 (2), 15 (1)
  const std::vector<int> var_warps = x8 ? std::vector<int>{4, 7, 15} : std::vector<int>{0};
  for (int w : var_warps) {
    for (int bps : var_bps) {
      VarTune vt{bps, w};
      const float ms = time_launches(s, 3, [&] {
        return launch_var(c, fs, form, llr, c2v, v2c, sym, fsyn, s, nullptr, vt);
      });
      if (ms > 0.0f && (best_ms < 0.0f || ms < best_ms)) {
        best_ms = ms;
        best.var = vt;
      }
    }
  }
  if (best_ms < 0.0f) return set_error(NBFD_ECUDA, "autotune: no variable-node shape ran");
  *out = best;
  return NBFD_OK;
}

// ---- per-code workspace of the graph-driven loop -----------------------------------------
struct CodeWs {
  float *v2c, *c2v;
  uint8_t *fsyn;
  int32_t *list[2];
  int32_t *state;  // [0..1] counts of the two lists, [2] iteration, [16..31] status words
  size_t bytes;
};

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

CodeWs carve_code(const nbfd_code *c, int F, int form, char *base) {
  CodeWs w{};
  size_t off = 0;
  const size_t msg = a256((size_t)F * c->E * c->q * (stores_f16(form) ? 2 : 4));
  w.v2c = reinterpret_cast<float *>(base + off);
  off += msg;
  w.c2v = reinterpret_cast<float *>(base + off);
  off += msg;
  w.fsyn = reinterpret_cast<uint8_t *>(base + off);
  off += a256((size_t)F * c->E);
  w.list[0] = reinterpret_cast<int32_t *>(base + off);
  off += a256((size_t)F * 4);
  w.list[1] = reinterpret_cast<int32_t *>(base + off);
  off += a256((size_t)F * 4);
  w.state = reinterpret_cast<int32_t *>(base + off);
  off += 256;
  w.bytes = off;
  return w;
}

constexpr int kMaxCodes = 64;

// streams for the graph branches, per host thread and device
std::vector<cudaStream_t> &branch_streams(int n) {
  thread_local std::map<int, std::vector<cudaStream_t>> pool;
  int dev = 0;
  cudaGetDevice(&dev);
  auto &v = pool[dev];
  while ((int)v.size() < n) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) break;
    v.push_back(s);
  }
  return v;
}

int32_t *pinned_counts() {
  struct Holder {
    int32_t *p = nullptr;
    ~Holder() {
      if (p) cudaFreeHost(p);
    }
  };
  thread_local Holder h;
  if (!h.p) {
    void *p = nullptr;
    if (cudaHostAlloc(&p, 2 * kMaxCodes * sizeof(int32_t), cudaHostAllocPortable) != cudaSuccess)
      return nullptr;
    h.p = static_cast<int32_t *>(p);
  }
  return h.p;
}

int code_device_ok(const nbfd_code *c) {
  int dev = -1;
  cudaGetDevice(&dev);
  return dev == c->device;
}

}  // namespace

namespace nbfd {
bool tune_lookup(const nbfd_code *c, int F, int form, CheckTune *ct, VarTune *vt) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key_of(c, F, form));
  if (it == g_tune.end()) return false;
  *ct = it->second.check;
  *vt = it->second.var;
  return true;
}
}  // namespace nbfd

extern "C" int nbfd_autotune(const nbfd_code *c, int F, int form, void *stream_) {
  if (!c || F <= 0) return set_error(NBFD_EINVAL, "bad argument");
  if (!form_supported(form, c->m)) return set_error(NBFD_ENOTSUP, "form %d not supported", form);
  if (!code_device_ok(c)) return set_error(NBFD_EINVAL, "current device differs from the code's");
  cudaStream_t s = static_cast<cudaStream_t>(stream_);
  const size_t msg = a256((size_t)F * c->E * c->q * (stores_f16(form) ? 2 : 4));
  const size_t bytes = 2 * msg + a256((size_t)F * c->N * c->m * 4) + a256((size_t)F * c->N * 2) +
                       a256((size_t)F * c->E);
  char *buf = nullptr;
  if (int st = check_cuda(cudaMallocAsync(reinterpret_cast<void **>(&buf), bytes, s),
                          "cudaMallocAsync(autotune)"))
    return st;
  float *v2c = reinterpret_cast<float *>(buf), *c2v = reinterpret_cast<float *>(buf + msg);
  float *llr = reinterpret_cast<float *>(buf + 2 * msg);
  uint16_t *sym = reinterpret_cast<uint16_t *>(buf + 2 * msg + a256((size_t)F * c->N * c->m * 4));
  uint8_t *fsyn = reinterpret_cast<uint8_t *>(reinterpret_cast<char *>(sym) + a256((size_t)F * c->N * 2));
  int st = check_cuda(cudaMemsetAsync(llr, 0, (size_t)F * c->N * c->m * 4, s), "cudaMemsetAsync");
  if (!st)
    st = check_cuda(launch_init(c, F, llr, nullptr, v2c, nullptr, nullptr, s, stores_f16(form)),
                    "init kernel");
  TuneVal tv{};
  if (!st) st = tune_code(c, F, form, llr, v2c, c2v, sym, fsyn, s, &tv);
  cudaFreeAsync(buf, s);
  if (!st) st = check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (st) return st;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key_of(c, F, form)] = tv;
  return NBFD_OK;
}

extern "C" int nbfd_autotune_result(const nbfd_code *c, int F, int form, int *check_warps,
                                    int *check_stages, int *check_blocks_per_sm,
                                    int *var_blocks_per_sm, int *var_warps) {
  if (!c) return set_error(NBFD_EINVAL, "code is NULL");
  CheckTune ct;
  VarTune vt;
  if (!tune_lookup(c, F, form, &ct, &vt)) return set_error(NBFD_EINVAL, "shape not tuned");
  if (check_warps) *check_warps = ct.team > 0 ? -kCheckTeamWarps : ct.warps;
  if (check_stages) *check_stages = ct.stages;
  if (check_blocks_per_sm) *check_blocks_per_sm = ct.blocks_per_sm;
  if (var_blocks_per_sm) *var_blocks_per_sm = vt.blocks_per_sm;
  if (var_warps) *var_warps = vt.warps;
  return NBFD_OK;
}

extern "C" size_t nbfd_decode_batch_workspace_size(int n, const nbfd_code *const *codes,
                                                   const int *n_frames, int max_iter, int form) {
  (void)max_iter;
  if (n <= 0 || n > kMaxCodes || !codes || !n_frames) return 0;
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    if (!codes[i] || n_frames[i] < 0) return 0;
    total += carve_code(codes[i], n_frames[i], form, nullptr).bytes;
  }
  return total;
}

extern "C" int nbfd_decode_batch(int n, const nbfd_code *const *codes, const int *n_frames,
                                 const float *const *llr, int max_iter, int form, int flags,
                                 uint16_t *const *symbols, uint8_t *const *ok,
                                 int32_t *const *iters, void *workspace, size_t workspace_bytes,
                                 void *stream_) {
  if (n <= 0 || n > kMaxCodes) return set_error(NBFD_EINVAL, "n_codes must be in [1, %d]", kMaxCodes);
  if (!codes || !n_frames || !llr || !symbols || !ok || !iters)
    return set_error(NBFD_EINVAL, "NULL array");
  if (max_iter < 1) return set_error(NBFD_EINVAL, "max_iter must be >= 1");
  if (flags & ~NBFD_BATCH_AUTOTUNE) return set_error(NBFD_EINVAL, "unknown flags 0x%x", flags);
  long long total_frames = 0;
  for (int i = 0; i < n; ++i) {
    if (!codes[i] || n_frames[i] < 0) return set_error(NBFD_EINVAL, "code %d: bad argument", i);
    if (!form_supported(form, codes[i]->m))
      return set_error(NBFD_ENOTSUP, "form %d not supported for m = %d", form, codes[i]->m);
    if (!code_device_ok(codes[i]))
      return set_error(NBFD_EINVAL, "code %d lives on another device", i);
    if (n_frames[i] > 0 && (!llr[i] || !symbols[i] || !ok[i] || !iters[i]))
      return set_error(NBFD_EINVAL, "code %d: NULL buffer", i);
    total_frames += n_frames[i];
  }
  if (total_frames == 0) return NBFD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream_);
  const size_t need = nbfd_decode_batch_workspace_size(n, codes, n_frames, max_iter, form);
  bool owned = false;
  if (!workspace) {
    if (int st = check_cuda(cudaMallocAsync(&workspace, need, s), "cudaMallocAsync(workspace)"))
      return st;
    owned = true;
  } else if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)) {
    return set_error(NBFD_ENOMEM, "workspace of %zu bytes (need %zu, 256-byte aligned)",
                     workspace_bytes, need);
  }
  std::vector<CodeWs> ws(n);
  {
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
      ws[i] = carve_code(codes[i], n_frames[i], form, static_cast<char *>(workspace) + off);
      off += ws[i].bytes;
    }
  }
  std::vector<TuneVal> tune(n);
  // groups of small GF(16) codes decode start to finish in one fused launch each, on their own
  // branch stream beside the graph replays of the other groups
  std::vector<char> fused(n, 0);
  for (int i = 0; i < n; ++i) fused[i] = n_frames[i] > 0 && fused_small_applies(codes[i], form);
  int32_t *host = pinned_counts();
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> events;
  int st = host ? NBFD_OK : set_error(NBFD_ECUDA, "cudaHostAlloc of the count words failed");
  auto init_code = [&](int i) {
    const nbfd_code *c = codes[i];
    int r = check_cuda(cudaMemsetAsync(ws[i].state, 0, 256, s), "cudaMemsetAsync");
    if (!r) r = check_cuda(cudaMemsetAsync(ok[i], 0, (size_t)n_frames[i], s), "cudaMemsetAsync");
    if (!r)
      r = check_cuda(launch_init(c, n_frames[i], llr[i], nullptr, ws[i].v2c, ws[i].list[1],
                                 ws[i].state + 1, s, stores_f16(form)),
                     "init kernel");
    return r;
  };
  do {
    if (st) break;
    // INITIALIZATION (list 1 = all frames, count 1 = F), launch shapes
    for (int i = 0; i < n && !st; ++i) {
      if (n_frames[i] == 0) continue;
      if (fused[i]) {  // its launch writes every output; only the state words start at 0
        st = check_cuda(cudaMemsetAsync(ws[i].state, 0, 256, s), "cudaMemsetAsync");
        continue;
      }
      if ((st = init_code(i))) break;
      if (!tune_lookup(codes[i], n_frames[i], form, &tune[i].check, &tune[i].var) &&
          (flags & NBFD_BATCH_AUTOTUNE)) {
        TuneVal tv{};
        if ((st = tune_code(codes[i], n_frames[i], form, llr[i], ws[i].v2c, ws[i].c2v, symbols[i],
                            ws[i].fsyn, s, &tv)))
          break;
        {
          std::lock_guard<std::mutex> lk(g_tune_mu);
          g_tune[key_of(codes[i], n_frames[i], form)] = tv;
        }
        tune[i] = tv;
        if ((st = init_code(i))) break;  // the timing runs overwrote the messages
      }
    }
    if (st) break;
    // capture two iterations of every code, one branch per code, on the library's own origin
    // stream (the caller's stream may be the legacy default stream, which cannot be captured)
    std::vector<cudaStream_t> &br = branch_streams(n + 1);
    if ((int)br.size() < n + 1) {
      st = set_error(NBFD_ECUDA, "cudaStreamCreate failed");
      break;
    }
    cudaStream_t cs = br[n];
    events.assign(n + 2, nullptr);
    for (auto &e : events)
      if ((st = check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate")))
        break;
    if (st) break;
    if ((st = check_cuda(cudaEventRecord(events[n + 1], s), "cudaEventRecord")) ||
        (st = check_cuda(cudaStreamWaitEvent(cs, events[n + 1], 0), "cudaStreamWaitEvent")))
      break;
    for (int i = 0; i < n && !st; ++i) {
      if (!fused[i]) continue;
      if ((st = check_cuda(cudaStreamWaitEvent(br[i], events[n + 1], 0), "cudaStreamWaitEvent")))
        break;
      st = check_cuda(launch_fused_small(codes[i], n_frames[i], llr[i], symbols[i], ok[i], iters[i],
                                         ws[i].state + 16, max_iter,
                                         (form & NBFD_DECIDE_SYMBOL) != 0, br[i]),
                      "fused small-code kernel");
      if (!st) st = check_cuda(cudaEventRecord(events[i], br[i]), "cudaEventRecord");
    }
    if (st) break;
    if ((st = check_cuda(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed),
                         "cudaStreamBeginCapture")))
      break;
    cudaError_t ce = cudaEventRecord(events[n], cs);
    for (int i = 0; i < n && ce == cudaSuccess; ++i) {
      const nbfd_code *c = codes[i];
      const int F = n_frames[i];
      cudaStream_t b = br[i];
      if (fused[i]) continue;
      ce = cudaStreamWaitEvent(b, events[n], 0);
      for (int p = 1; p >= 0 && ce == cudaSuccess && F > 0; --p) {
        FrameSet fs;
        fs.list = ws[i].list[p];
        fs.count = ws[i].state + p;
        fs.n_static = F;
        LoopTick tick;
        tick.iter = ws[i].state + 2;
        tick.zero = ws[i].state + (1 - p);
        ce = launch_check(c, fs, ws[i].v2c, ws[i].c2v, b, ws[i].state + 17, tick, tune[i].check,
                          stores_f16(form));
        if (ce == cudaSuccess)
          ce = launch_var(c, fs, form, llr[i], ws[i].c2v, ws[i].v2c, symbols[i], ws[i].fsyn, b,
                          ws[i].state + 17, tune[i].var);
        if (ce == cudaSuccess)
          ce = launch_stop(c, fs, symbols[i], ws[i].fsyn, 0, max_iter, ws[i].list[1 - p],
                           ws[i].state + (1 - p), ok[i], iters[i], ws[i].state + 16, b,
                           ws[i].state + 2);
      }
      if (ce == cudaSuccess) ce = cudaEventRecord(events[i], b);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs, events[i], 0);
    }
    const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    if ((st = check_cuda(ce, "graph capture")) || (st = check_cuda(ee, "cudaStreamEndCapture")))
      break;
    if ((st = check_cuda(cudaGraphInstantiate(&exec, graph, 0), "cudaGraphInstantiate"))) break;
    // replay; read the active counts every few replays (after an even iteration the survivors
    // are in list/count 1)
    long long active = total_frames;
    int it = 0;
    while (it < max_iter && active > 0) {
      const int reps = active * 16 <= total_frames ? 8 : 2;
      for (int r = 0; r < reps && it < max_iter; ++r, it += 2)
        if ((st = check_cuda(cudaGraphLaunch(exec, cs), "cudaGraphLaunch"))) break;
      if (st) break;
      for (int i = 0; i < n && !st; ++i)
        st = check_cuda(cudaMemcpyAsync(host + i, ws[i].state + 1, 4, cudaMemcpyDeviceToHost, cs),
                        "cudaMemcpyAsync(count)");
      if (st) break;
      if ((st = check_cuda(cudaStreamSynchronize(cs), "cudaStreamSynchronize"))) break;
      active = 0;
      for (int i = 0; i < n; ++i) active += n_frames[i] > 0 && !fused[i] ? host[i] : 0;
    }
    if (st) break;
    // the fused groups' launches
    for (int i = 0; i < n && !st; ++i)
      if (fused[i]) st = check_cuda(cudaStreamWaitEvent(cs, events[i], 0), "cudaStreamWaitEvent");
    if (st) break;
    for (int i = 0; i < n && !st; ++i)
      st = check_cuda(cudaMemcpyAsync(host + kMaxCodes + i, ws[i].state + 17, 4,
                                      cudaMemcpyDeviceToHost, cs),
                      "cudaMemcpyAsync(status)");
    if (!st) st = check_cuda(cudaStreamSynchronize(cs), "cudaStreamSynchronize");
    for (int i = 0; i < n && !st; ++i)
      if (n_frames[i] > 0 && host[kMaxCodes + i] != 0)
        st = set_error(NBFD_ETIMEDOUT, "code %d: a bounded device-side wait expired", i);
  } while (false);
  // work left on the library's streams after an error must finish before the workspace is freed
  if (st != NBFD_OK) {
    std::vector<cudaStream_t> &br = branch_streams(0);
    for (cudaStream_t b : br) cudaStreamSynchronize(b);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  for (auto e : events)
    if (e) cudaEventDestroy(e);
  if (owned) cudaFreeAsync(workspace, s);
  return st;
}
