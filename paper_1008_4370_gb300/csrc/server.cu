// Serving: continuous batching of single-frame decode requests over resident slot pools.
//
// A worker thread owns one pool per code (fixed number of slots, sized from the memory budget when
// the code is first seen, on a stream of its own so that the pools' work overlaps on the device).
// Each round it
//   1. admits queued requests into free slots (LLRs copied in, INITIALIZATION of Section 3.2 run
//      for exactly those slots, the slots appended to the pool's active list);
//   2. runs one decoding iteration (check update, variable update + tentative decision) over each
//      pool's active list with the same kernels as nbfd_decode;
//   3. runs the serving stop test: every active slot counts its own iterations, and a slot whose
//      Fourier-domain and GF(2^m) syndromes are zero, or that reached its own max_iter, leaves
//      the active list for a done list;
//   4. copies the done slots' decisions back, completes their tickets and frees the slots.
// Rounds are pipelined two deep: the host issues round r, then retires round r-1 and admits
// and stages round r+1 while round r runs, so its work stays off the device's critical path.
// The active list is extended on the device, and slots freed by round r-1 are reused from
// round r+1 on.
// A frame's arithmetic never involves another frame, so its result is identical alone and in
// any mix of requests.
#include <cuda_runtime.h>

#include <chrono>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "device_common.cuh"
#include "nbfd_internal.h"

namespace nbfd {

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum Phase { kAdmit = 0, kIssue = 1, kWait = 2, kRetire = 3, kIdle = 4 };

// INITIALIZATION for the slots list[0..*count): V->C on both edges of every variable = Lambda0.
template <int MB>
__global__ void __launch_bounds__(256)
    k_init_slots(const float *__restrict__ llr, float *__restrict__ v2c,
                 const int32_t *__restrict__ var_edges, int N, int E,
                 const int32_t *__restrict__ list, const int32_t *__restrict__ count) {
  using CL = ChannelLayout<MB>;
  constexpr int Q = CL::Q, VPT = CL::VPT;
  const int lane = threadIdx.x & 31, sub = lane / CL::LPV, l = lane % CL::LPV;
  const long long total = (long long)__ldg(count) * N;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  for (long long base = (gtid >> 5) * CL::VPW; base < total; base += (nthr >> 5) * CL::VPW) {
    const long long item = base + sub;
    const bool valid = item < total;
    const long long ic = valid ? item : total - 1;
    const int f = __ldg(list + ic / N);
    const int v = static_cast<int>(ic % N);
    float g[VPT];
    channel_gamma<MB>(llr + ((size_t)f * N + v) * MB, l, g);
    if (valid) {
      const int e1 = __ldg(var_edges + 2 * v), e2 = __ldg(var_edges + 2 * v + 1);
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        v2c[((size_t)f * E + e1) * Q + l * VPT + j] = g[j];
        v2c[((size_t)f * E + e2) * Q + l * VPT + j] = g[j];
      }
    }
  }
}

// Serving stop test, one block per active slot: the slot's own iteration counter advances; a
// slot whose syndromes clear (or that reached its own max_iter) goes to the done list with its
// flag and iteration count, the others to the next active list.
__global__ void __launch_bounds__(128)
    k_stop_serve(const int32_t *__restrict__ list, const int32_t *__restrict__ count,
                 const uint16_t *__restrict__ sym, const uint8_t *__restrict__ fsyn,
                 const int32_t *__restrict__ edge_var, const uint8_t *__restrict__ edge_h,
                 const uint8_t *__restrict__ gexp_g, const uint8_t *__restrict__ glog_g, int q,
                 int N, int M, int k, int E, int32_t *__restrict__ iter, const int32_t *__restrict__ maxit,
                 uint8_t *__restrict__ ok, int32_t *__restrict__ next_list,
                 int32_t *__restrict__ next_count, int32_t *__restrict__ done_list,
                 int32_t *__restrict__ done_count) {
  __shared__ uint8_t gexp[512];
  __shared__ uint8_t glog[256];
  for (int i = threadIdx.x; i < 2 * q; i += blockDim.x) gexp[i] = gexp_g[i];
  for (int i = threadIdx.x; i < q; i += blockDim.x) glog[i] = glog_g[i];
  __syncthreads();
  const int nf = __ldg(count);
  for (int s = blockIdx.x; s < nf; s += gridDim.x) {
    const int f = __ldg(list + s);
    int ffail = 0, efail = 0;
    for (int c = threadIdx.x; c < M; c += blockDim.x) {
      int fsv = 0, esv = 0;
      for (int j = 0; j < k; ++j) {
        const int e = c * k + j;
        fsv ^= fsyn[(size_t)f * E + e];
        const int x = sym[(size_t)f * N + __ldg(edge_var + e)];
        esv ^= x == 0 ? 0 : gexp[glog[__ldg(edge_h + e)] + glog[x]];
      }
      ffail |= fsv != 0;
      efail |= esv != 0;
    }
    ffail = __syncthreads_or(ffail);
    efail = __syncthreads_or(efail);
    if (threadIdx.x == 0) {
      const int it = iter[f] + 1;
      iter[f] = it;
      if ((!ffail && !efail) || it >= maxit[f]) {
        ok[f] = efail ? 0 : 1;
        done_list[atomicAdd(done_count, 1)] = f;
      } else {
        next_list[atomicAdd(next_count, 1)] = f;
      }
    }
  }
}

// Admission: scatter n staged LLR frames to their slots, set each slot's max_iter, clear its
// iteration counter.
__global__ void k_admit(const float *__restrict__ staged, const int32_t *__restrict__ slots,
                        const int32_t *__restrict__ maxits, int n, int per_frame,
                        float *__restrict__ llr, int32_t *__restrict__ iter,
                        int32_t *__restrict__ maxit) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int slot = slots[i];
    if ((per_frame & 3) == 0) {  // rows start on 16-byte boundaries: vector copies
      const float4 *src = reinterpret_cast<const float4 *>(staged + (size_t)i * per_frame);
      float4 *dst = reinterpret_cast<float4 *>(llr + (size_t)slot * per_frame);
      for (int j = threadIdx.x; j < per_frame / 4; j += blockDim.x) dst[j] = src[j];
    } else {
      for (int j = threadIdx.x; j < per_frame; j += blockDim.x)
        llr[(size_t)slot * per_frame + j] = staged[(size_t)i * per_frame + j];
    }
    if (threadIdx.x == 0) {
      iter[slot] = 0;
      maxit[slot] = maxits[i];
    }
  }
}

// Appends the n admitted slots to the active list at its current length on the device (the
// host does not wait for the previous round's stop test to learn it).
__global__ void __launch_bounds__(256)
    k_append(const int32_t *__restrict__ slots, int n, int32_t *__restrict__ list,
             int32_t *__restrict__ count) {
  const int base = *count;
  for (int i = threadIdx.x; i < n; i += blockDim.x) list[base + i] = slots[i];
  __syncthreads();
  if (threadIdx.x == 0) *count = base + n;
}

// Retirement: pack the decisions, flags and iteration counts of the done slots contiguously.
__global__ void k_gather_done(const int32_t *__restrict__ done_list,
                              const int32_t *__restrict__ done_count,
                              const uint16_t *__restrict__ sym, const uint8_t *__restrict__ ok,
                              const int32_t *__restrict__ iter, int N,
                              uint16_t *__restrict__ out_sym, uint8_t *__restrict__ out_ok,
                              int32_t *__restrict__ out_iter) {
  const int n = __ldg(done_count);
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int slot = done_list[i];
    for (int j = threadIdx.x; j < N; j += blockDim.x) out_sym[(size_t)i * N + j] = sym[(size_t)slot * N + j];
    if (threadIdx.x == 0) {
      out_ok[i] = ok[slot];
      out_iter[i] = iter[slot];
    }
  }
}

struct Request {
  uint64_t ticket;
  std::vector<float> llr;
  int max_iter;
  double t_submit;  // arrival time (server clock) latency is measured from
};

struct Result {
  std::vector<uint16_t> sym;
  uint8_t ok = 0;
  int32_t iters = 0;
  double latency = 0.0;
};

// Words of Pool::cnt.
constexpr int kCntActive = 0;  // [0], [1]: lengths of active lists 0 and 1
constexpr int kCntDone = 2;    // [2], [3]: done-list lengths of the rounds of parity 0 and 1
constexpr int kCntErr = 4;     // set to NBFD_ETIMEDOUT by a kernel whose bounded wait expired
constexpr int kCntNew = 5;     // frames admitted by the current round

// Rounds alternate between two parities. Everything a round reads from or writes to the host
// (staged admissions, counts, packed results) exists once per parity, so the host can stage
// round r+1 and retire round r-1 while round r runs on the device.
struct Pool {
  const nbfd_code *code = nullptr;
  int S = 0;  // slots
  size_t bytes = 0;
  void *block = nullptr;
  float *v2c = nullptr, *c2v = nullptr, *llr = nullptr;
  uint16_t *sym = nullptr;
  uint8_t *fsyn = nullptr, *ok = nullptr;
  int32_t *iter = nullptr, *maxit = nullptr, *lists[2] = {nullptr, nullptr};
  float *stage_llr = nullptr;                             // [S][N][m] admitted frames, packed
  int32_t *stage_slot = nullptr, *stage_maxit = nullptr;  // [S]
  int32_t *done_list[2] = {nullptr, nullptr};             // [S] per parity
  uint16_t *pack_sym[2] = {nullptr, nullptr};             // [S][N] retired frames, packed
  uint8_t *pack_ok[2] = {nullptr, nullptr};               // [S]
  int32_t *pack_iter[2] = {nullptr, nullptr};             // [S]
  int32_t *cnt = nullptr;                                 // kCnt* words
  int cur = 0;  // active list the next round reads
  int par = 0;  // parity of the next round
  std::deque<int> issued;  // parities of rounds issued and not yet retired, oldest first
  std::vector<int> free_slots;
  std::unordered_map<int, Request> in_flight;  // changed only under the server lock
  std::deque<Request> queue;
  size_t reserved = 0;  // frames a running nbfd_srv_submit_many has counted but not queued yet
  cudaStream_t stream = nullptr;       // rounds
  cudaStream_t copy_stream = nullptr;  // result copies, overlapping the next round
  cudaEvent_t round_done[2] = {nullptr, nullptr};
  // pinned host buffers
  float *h_llr[2] = {nullptr, nullptr};       // [S][N][m] staged admissions
  int32_t *h_slot[2] = {nullptr, nullptr};    // [S] their slots
  int32_t *h_maxit[2] = {nullptr, nullptr};   // [S] their max_iter
  int32_t *h_cnt[2] = {nullptr, nullptr};     // [4]: in: [0] admitted; out: [1] next active,
                                              // [2] done, [3] error word
  int32_t *h_done = nullptr;                  // [S] done slots of the round being retired
  uint16_t *h_sym = nullptr;                  // [S][N]
  uint8_t *h_ok = nullptr;                    // [S]
  int32_t *h_iters = nullptr;                 // [S]
};

}  // namespace
}  // namespace nbfd

struct nbfd_server {
  size_t budget = 0, used = 0;
  int form = NBFD_FORM_FP32_FWHT;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::map<const nbfd_code *, std::unique_ptr<nbfd::Pool>> pools;
  std::unordered_map<uint64_t, nbfd::Result> done;
  std::deque<uint64_t> done_order;  // retirement order, for nbfd_srv_collect
  std::unordered_map<uint64_t, int> pending;  // tickets queued or in flight
  size_t queue_limit = 1 << 16;
  int error = NBFD_OK;
  std::thread worker;
  long long rounds = 0;
  // worker time per phase, nanoseconds: admission, issue, wait, retire, idle
  std::atomic<long long> phase_ns[5] = {};
};

namespace nbfd {
namespace {

size_t slot_bytes(const nbfd_code *c) {
  return (size_t)2 * c->E * c->q * 4 + (size_t)2 * c->N * c->m * 4 + (size_t)3 * c->N * 2 + c->E +
         3 + 10 * 4 + 64;
}

void free_pool(Pool *p) {
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->copy_stream) cudaStreamSynchronize(p->copy_stream);
  if (p->block) cudaFree(p->block);
  if (p->stream) cudaStreamDestroy(p->stream);
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  for (int b = 0; b < 2; ++b) {
    if (p->round_done[b]) cudaEventDestroy(p->round_done[b]);
    cudaFreeHost(p->h_llr[b]);
    cudaFreeHost(p->h_slot[b]);
    cudaFreeHost(p->h_maxit[b]);
    cudaFreeHost(p->h_cnt[b]);
  }
  cudaFreeHost(p->h_done);
  cudaFreeHost(p->h_sym);
  cudaFreeHost(p->h_ok);
  cudaFreeHost(p->h_iters);
  p->block = nullptr;
  p->stream = p->copy_stream = nullptr;
}

int make_pool(nbfd_server *srv, const nbfd_code *c, Pool **out) {
  auto it = srv->pools.find(c);
  if (it != srv->pools.end()) {
    *out = it->second.get();
    return NBFD_OK;
  }
  const size_t per = slot_bytes(c);
  const size_t left = srv->budget > srv->used ? srv->budget - srv->used : 0;
  // a pool takes at most a quarter of the budget, so that several codes can be served
  const size_t share = srv->budget / 4 < left ? srv->budget / 4 : left;
  long long S = (long long)(share / per);
  if (S > 4096) S = 4096;
  if (S < 1 && left >= per) S = 1;
  if (S < 1) return set_error(NBFD_EBUSY, "memory budget exhausted: no pool for this code");
  auto p = std::make_unique<Pool>();
  p->code = c;
  p->S = static_cast<int>(S);
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t msg = al((size_t)S * c->E * c->q * 4);
  const size_t frames_f = al((size_t)S * c->N * c->m * 4), frames_u16 = al((size_t)S * c->N * 2);
  const size_t ints = al((size_t)S * 4), bytes = al((size_t)S);
  size_t o = 0;
  auto take = [&](size_t n) {
    const size_t at = o;
    o += n;
    return at;
  };
  const size_t o_v2c = take(msg), o_c2v = take(msg), o_llr = take(frames_f);
  const size_t o_sym = take(frames_u16), o_fsyn = take(al((size_t)S * c->E)), o_ok = take(bytes);
  const size_t o_iter = take(ints), o_maxit = take(ints), o_list0 = take(ints),
               o_list1 = take(ints), o_cnt = take(al(8 * 4));
  const size_t o_stage = take(frames_f), o_stage_slot = take(ints), o_stage_maxit = take(ints);
  size_t o_done[2], o_psym[2], o_pok[2], o_piter[2];
  for (int b = 0; b < 2; ++b) {
    o_done[b] = take(ints);
    o_psym[b] = take(frames_u16);
    o_pok[b] = take(bytes);
    o_piter[b] = take(ints);
  }
  p->bytes = o;
  if (int st = check_cuda(cudaMalloc(&p->block, o), "cudaMalloc(server pool)")) return st;
  char *base = static_cast<char *>(p->block);
  p->v2c = reinterpret_cast<float *>(base + o_v2c);
  p->c2v = reinterpret_cast<float *>(base + o_c2v);
  p->llr = reinterpret_cast<float *>(base + o_llr);
  p->sym = reinterpret_cast<uint16_t *>(base + o_sym);
  p->fsyn = reinterpret_cast<uint8_t *>(base + o_fsyn);
  p->ok = reinterpret_cast<uint8_t *>(base + o_ok);
  p->iter = reinterpret_cast<int32_t *>(base + o_iter);
  p->maxit = reinterpret_cast<int32_t *>(base + o_maxit);
  p->lists[0] = reinterpret_cast<int32_t *>(base + o_list0);
  p->lists[1] = reinterpret_cast<int32_t *>(base + o_list1);
  p->cnt = reinterpret_cast<int32_t *>(base + o_cnt);
  p->stage_llr = reinterpret_cast<float *>(base + o_stage);
  p->stage_slot = reinterpret_cast<int32_t *>(base + o_stage_slot);
  p->stage_maxit = reinterpret_cast<int32_t *>(base + o_stage_maxit);
  for (int b = 0; b < 2; ++b) {
    p->done_list[b] = reinterpret_cast<int32_t *>(base + o_done[b]);
    p->pack_sym[b] = reinterpret_cast<uint16_t *>(base + o_psym[b]);
    p->pack_ok[b] = reinterpret_cast<uint8_t *>(base + o_pok[b]);
    p->pack_iter[b] = reinterpret_cast<int32_t *>(base + o_piter[b]);
  }
  // the pool owns its memory from here on: free_pool releases whatever was made
  Pool *raw = p.get();
  srv->used += p->bytes;
  srv->pools[c] = std::move(p);
  const size_t llr_bytes = (size_t)S * c->N * c->m * 4;
  int st = check_cuda(cudaMemset(raw->cnt, 0, 32), "cudaMemset");
  if (!st) st = check_cuda(cudaStreamCreateWithFlags(&raw->stream, cudaStreamNonBlocking), "stream");
  if (!st)
    st = check_cuda(cudaStreamCreateWithFlags(&raw->copy_stream, cudaStreamNonBlocking), "stream");
  for (int b = 0; b < 2 && !st; ++b) {
    st = check_cuda(cudaEventCreateWithFlags(&raw->round_done[b], cudaEventDisableTiming), "event");
    if (!st) st = check_cuda(cudaMallocHost(&raw->h_llr[b], llr_bytes), "pinned");
    if (!st) st = check_cuda(cudaMallocHost(&raw->h_slot[b], (size_t)S * 4), "pinned");
    if (!st) st = check_cuda(cudaMallocHost(&raw->h_maxit[b], (size_t)S * 4), "pinned");
    if (!st) st = check_cuda(cudaMallocHost(&raw->h_cnt[b], 16), "pinned");
  }
  if (!st) st = check_cuda(cudaMallocHost(&raw->h_done, (size_t)S * 4), "pinned");
  if (!st) st = check_cuda(cudaMallocHost(&raw->h_sym, (size_t)S * c->N * 2), "pinned");
  if (!st) st = check_cuda(cudaMallocHost(&raw->h_ok, (size_t)S), "pinned");
  if (!st) st = check_cuda(cudaMallocHost(&raw->h_iters, (size_t)S * 4), "pinned");
  if (st) {
    free_pool(raw);
    srv->used -= raw->bytes;
    srv->pools.erase(c);
    return st;
  }
  for (int s = raw->S - 1; s >= 0; --s) raw->free_slots.push_back(s);
  *out = raw;
  return NBFD_OK;
}

cudaError_t launch_init_slots(const nbfd_code *c, const float *llr, float *v2c,
                              const int32_t *list, const int32_t *count, int n, cudaStream_t s) {
  const long long total = (long long)n * c->N;
  const long long cap = (long long)sm_count() * 8;
#define NBFD_INIT_SLOTS(MB)                                                              \
  {                                                                                      \
    constexpr int VPW = ChannelLayout<MB>::VPW;                                          \
    long long g = (total + 8 * VPW - 1) / (8 * VPW);                                     \
    if (g > cap) g = cap;                                                                \
    if (g < 1) g = 1;                                                                    \
    k_init_slots<MB><<<(int)g, 256, 0, s>>>(llr, v2c, c->d_var_edges, c->N, c->E, list,  \
                                            count);                                      \
  }
  switch (c->m) {
    case 2: NBFD_INIT_SLOTS(2) break;
    case 3: NBFD_INIT_SLOTS(3) break;
    case 4: NBFD_INIT_SLOTS(4) break;
    case 5: NBFD_INIT_SLOTS(5) break;
    case 6: NBFD_INIT_SLOTS(6) break;
    case 7: NBFD_INIT_SLOTS(7) break;
    case 8: NBFD_INIT_SLOTS(8) break;
    default: return cudaErrorInvalidValue;
  }
#undef NBFD_INIT_SLOTS
  return cudaGetLastError();
}

// Charges the time since the previous lap to one worker phase.
struct PhaseClock {
  nbfd_server *srv;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  void lap(Phase ph) {
    const auto n = std::chrono::steady_clock::now();
    srv->phase_ns[ph].fetch_add(std::chrono::duration_cast<std::chrono::nanoseconds>(n - t).count(),
                                std::memory_order_relaxed);
    t = n;
  }
};

// Issues one round of pool p on its stream: the n_new admissions staged in the host buffers of
// parity p->par, one decoding iteration over the active list, the serving stop test and the
// packing of the done slots. n_bound >= the active list's length after admission (it sizes grids
// only: every kernel reads the length on the device).
void round_issue(nbfd_server *srv, Pool *p, int n_new, int n_bound) {
  const nbfd_code *c = p->code;
  cudaStream_t s = p->stream;
  const int b = p->par;
  int32_t *cur = p->lists[p->cur], *cur_n = p->cnt + kCntActive + p->cur;
  int32_t *next = p->lists[p->cur ^ 1], *next_n = p->cnt + kCntActive + (p->cur ^ 1);
  int32_t *done_n = p->cnt + kCntDone + b;
  cudaError_t e = cudaSuccess;
  if (n_new > 0) {
    const size_t per = (size_t)c->N * c->m;
    p->h_cnt[b][0] = n_new;
    cudaMemcpyAsync(p->stage_llr, p->h_llr[b], (size_t)n_new * per * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->stage_slot, p->h_slot[b], (size_t)n_new * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->stage_maxit, p->h_maxit[b], (size_t)n_new * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->cnt + kCntNew, p->h_cnt[b], 4, cudaMemcpyHostToDevice, s);
    const int g = n_new < sm_count() * 8 ? n_new : sm_count() * 8;
    k_admit<<<g, 128, 0, s>>>(p->stage_llr, p->stage_slot, p->stage_maxit, n_new,
                              static_cast<int>(per), p->llr, p->iter, p->maxit);
    k_append<<<1, 256, 0, s>>>(p->stage_slot, n_new, cur, cur_n);
    e = launch_init_slots(c, p->llr, p->v2c, p->stage_slot, p->cnt + kCntNew, n_new, s);
  }
  cudaMemsetAsync(next_n, 0, 4, s);
  cudaMemsetAsync(done_n, 0, 4, s);
  FrameSet fs;
  fs.list = cur;
  fs.count = cur_n;
  fs.n_static = n_bound;
  if (e == cudaSuccess) e = launch_check(c, fs, p->v2c, p->c2v, s, p->cnt + kCntErr);
  if (e == cudaSuccess)
    e = launch_var(c, fs, srv->form, p->llr, p->c2v, p->v2c, p->sym, p->fsyn, s, p->cnt + kCntErr);
  if (e == cudaSuccess) {
    const int grid = n_bound < sm_count() * 16 ? n_bound : sm_count() * 16;
    k_stop_serve<<<grid, 128, 0, s>>>(cur, cur_n, p->sym, p->fsyn, c->d_edge_var, c->d_edge_h,
                                      c->d_gf_exp, c->d_gf_log, c->q, c->N, c->M, c->k, c->E,
                                      p->iter, p->maxit, p->ok, next, next_n, p->done_list[b],
                                      done_n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const int g = n_bound < sm_count() * 8 ? n_bound : sm_count() * 8;
    k_gather_done<<<g, 128, 0, s>>>(p->done_list[b], done_n, p->sym, p->ok, p->iter, c->N,
                                    p->pack_sym[b], p->pack_ok[b], p->pack_iter[b]);
    e = cudaGetLastError();
  }
  cudaMemcpyAsync(&p->h_cnt[b][1], next_n, 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&p->h_cnt[b][2], done_n, 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&p->h_cnt[b][3], p->cnt + kCntErr, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventRecord(p->round_done[b], s);
  if (e != cudaSuccess) {  // the server stops; this round is never retired
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->error = check_cuda(e, "serving kernels");
    return;
  }
  p->issued.push_back(b);
  p->cur ^= 1;
  p->par ^= 1;
}

// Waits for the oldest issued round of pool p, copies its done slots' results back on the copy
// stream (the round after it keeps the device busy meanwhile) and completes their tickets.
void round_retire(nbfd_server *srv, Pool *p, PhaseClock &clk) {
  const int b = p->issued.front();
  p->issued.pop_front();
  const nbfd_code *c = p->code;
  cudaError_t e = cudaEventSynchronize(p->round_done[b]);
  clk.lap(kWait);
  const int n_done = p->h_cnt[b][2];
  int st = check_cuda(e, "serving round");
  if (!st && p->h_cnt[b][3] != 0)
    st = set_error(NBFD_ETIMEDOUT, "a bounded wait in a serving kernel expired");
  if (!st && (n_done < 0 || n_done > p->S))
    st = set_error(NBFD_ECUDA, "serving round reported %d done slots", n_done);
  if (!st && n_done > 0) {
    cudaStream_t cs = p->copy_stream;
    e = cudaStreamWaitEvent(cs, p->round_done[b], 0);
    if (e == cudaSuccess) {
      cudaMemcpyAsync(p->h_done, p->done_list[b], (size_t)n_done * 4, cudaMemcpyDeviceToHost, cs);
      cudaMemcpyAsync(p->h_sym, p->pack_sym[b], (size_t)n_done * c->N * 2, cudaMemcpyDeviceToHost,
                      cs);
      cudaMemcpyAsync(p->h_ok, p->pack_ok[b], (size_t)n_done, cudaMemcpyDeviceToHost, cs);
      cudaMemcpyAsync(p->h_iters, p->pack_iter[b], (size_t)n_done * 4, cudaMemcpyDeviceToHost, cs);
      e = cudaStreamSynchronize(cs);
    }
    st = check_cuda(e, "serving result copy");
  }
  if (st) {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (!srv->error) srv->error = st;
    clk.lap(kRetire);
    return;
  }
  // results are built outside the lock; only this thread changes in_flight
  const double t = now_s();
  struct Done {
    int slot;
    uint64_t ticket;
    Result r;
  };
  std::vector<Done> out;
  out.reserve(n_done);
  for (int i = 0; i < n_done; ++i) {
    const int slot = p->h_done[i];
    auto it = p->in_flight.find(slot);
    if (it == p->in_flight.end()) continue;
    Done d;
    d.slot = slot;
    d.ticket = it->second.ticket;
    d.r.sym.assign(p->h_sym + (size_t)i * c->N, p->h_sym + (size_t)(i + 1) * c->N);
    d.r.ok = p->h_ok[i];
    d.r.iters = p->h_iters[i];
    d.r.latency = t - it->second.t_submit;
    out.push_back(std::move(d));
  }
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    for (Done &d : out) {
      srv->done[d.ticket] = std::move(d.r);
      srv->done_order.push_back(d.ticket);
      srv->pending.erase(d.ticket);
      p->in_flight.erase(d.slot);
      p->free_slots.push_back(d.slot);
    }
    ++srv->rounds;
  }
  srv->cv.notify_all();
  clk.lap(kRetire);
}

// The worker keeps up to two rounds per pool on the device: after issuing round r it retires
// round r-1, then admits and stages round r+1 while round r runs.
void worker_main(nbfd_server *srv) {
  cudaSetDevice(srv->device);
  struct Work {
    Pool *p;
    std::vector<int> slots;  // admitted this round
    int bound;               // frames in flight after admission
  };
  PhaseClock clk{srv};
  while (true) {
    std::vector<Work> work;
    std::vector<Pool *> live;  // pools with rounds issued or about to be
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      auto has = [&](bool want_issued) {
        for (auto &kv : srv->pools) {
          const Pool *p = kv.second.get();
          if (want_issued ? !p->issued.empty()
                          : !p->in_flight.empty() || (!p->queue.empty() && !p->free_slots.empty()))
            return true;
        }
        return false;
      };
      if (!has(true))
        srv->cv.wait_for(lk, std::chrono::milliseconds(20),
                         [&] { return srv->stop || srv->error || has(false); });
      clk.lap(kIdle);
      if (srv->stop) break;
      if (srv->error) {  // no new rounds after a failure; callers see the error
        srv->cv.wait_for(lk, std::chrono::milliseconds(20), [&] { return srv->stop; });
        continue;
      }
      for (auto &kv : srv->pools) {
        Pool *p = kv.second.get();
        Work w{p, {}, 0};
        while (!p->queue.empty() && !p->free_slots.empty()) {
          const int slot = p->free_slots.back();
          p->free_slots.pop_back();
          p->in_flight.emplace(slot, std::move(p->queue.front()));
          p->queue.pop_front();
          w.slots.push_back(slot);
        }
        w.bound = static_cast<int>(p->in_flight.size());
        if (w.bound > 0 || !p->issued.empty()) live.push_back(p);
        if (w.bound > 0) work.push_back(std::move(w));
      }
    }
    // stage and issue: this host work overlaps the rounds already on the device
    for (Work &w : work) {
      Pool *p = w.p;
      const int b = p->par;
      const size_t per = (size_t)p->code->N * p->code->m;
      const int n_new = static_cast<int>(w.slots.size());
      for (int i = 0; i < n_new; ++i) {
        const Request &r = p->in_flight.at(w.slots[i]);
        memcpy(p->h_llr[b] + (size_t)i * per, r.llr.data(), per * 4);
        p->h_slot[b][i] = w.slots[i];
        p->h_maxit[b][i] = r.max_iter;
      }
      clk.lap(kAdmit);
      round_issue(srv, p, n_new, w.bound);
      clk.lap(kIssue);
    }
    // retire all but the round just issued
    for (Pool *p : live) {
      bool issued_now = false;
      for (const Work &w : work) issued_now |= w.p == p;
      while (p->issued.size() > (issued_now ? 1u : 0u)) round_retire(srv, p, clk);
    }
  }
}

}  // namespace
}  // namespace nbfd

using namespace nbfd;

extern "C" int nbfd_srv_create(size_t mem_budget_bytes, int form, nbfd_server **out) {
  if (!out) return set_error(NBFD_EINVAL, "out is NULL");
  *out = nullptr;
  if ((form & 0xff) > NBFD_FORM_FP32_TC || (form & ~(0xff | NBFD_DECIDE_SYMBOL)))
    return set_error(NBFD_EINVAL, "bad form %d", form);
  auto *srv = new (std::nothrow) nbfd_server();
  if (!srv) return set_error(NBFD_ENOMEM, "host allocation failed");
  srv->budget = mem_budget_bytes;
  srv->form = form;
  cudaGetDevice(&srv->device);
  srv->worker = std::thread(worker_main, srv);
  *out = srv;
  return NBFD_OK;
}

extern "C" void nbfd_srv_destroy(nbfd_server *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv.notify_all();
  if (srv->worker.joinable()) srv->worker.join();
  for (auto &kv : srv->pools) free_pool(kv.second.get());
  delete srv;
}

extern "C" int nbfd_srv_submit(nbfd_server *srv, const nbfd_code *code, const float *llr_host,
                               int max_iter, uint64_t *ticket) {
  if (!srv || !code || !llr_host || !ticket) return set_error(NBFD_EINVAL, "NULL argument");
  if (max_iter < 1) return set_error(NBFD_EINVAL, "max_iter must be >= 1");
  if (!form_supported(srv->form, code->m))
    return set_error(NBFD_ENOTSUP, "the server's form does not support m = %d", code->m);
  Request r;  // copied before the lock is taken: the worker shares it
  r.t_submit = now_s();
  r.llr.assign(llr_host, llr_host + (size_t)code->N * code->m);
  r.max_iter = max_iter;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->error) return set_error(srv->error, "the server stopped after an error");
  Pool *p = nullptr;
  if (int st = make_pool(srv, code, &p)) return st;
  if (p->queue.size() + p->reserved >= srv->queue_limit)
    return set_error(NBFD_EBUSY, "request queue full");
  r.ticket = srv->next_ticket++;
  *ticket = r.ticket;
  srv->pending[r.ticket] = 1;
  p->queue.push_back(std::move(r));
  srv->cv.notify_all();
  return NBFD_OK;
}

extern "C" int nbfd_srv_poll(nbfd_server *srv, uint64_t ticket, uint16_t *symbols_host,
                             uint8_t *ok, int32_t *iters, double *latency_s) {
  if (!srv) return set_error(NBFD_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->done.find(ticket);
  if (it == srv->done.end()) {
    if (srv->error) return set_error(srv->error, "the server stopped after an error");
    if (srv->pending.count(ticket)) return 0;
    return set_error(NBFD_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  }
  const Result &r = it->second;
  if (symbols_host) memcpy(symbols_host, r.sym.data(), r.sym.size() * 2);
  if (ok) *ok = r.ok;
  if (iters) *iters = r.iters;
  if (latency_s) *latency_s = r.latency;
  srv->done.erase(it);
  return 1;
}

extern "C" double nbfd_srv_clock(void) { return now_s(); }

extern "C" int nbfd_srv_submit_many(nbfd_server *srv, const nbfd_code *code, int n,
                                    const float *llr_host, int max_iter, const double *arrival,
                                    uint64_t *tickets) {
  if (!srv || !code || n < 0 || (n > 0 && (!llr_host || !tickets)))
    return set_error(NBFD_EINVAL, "bad argument");
  if (max_iter < 1) return set_error(NBFD_EINVAL, "max_iter must be >= 1");
  if (!form_supported(srv->form, code->m))
    return set_error(NBFD_ENOTSUP, "the server's form does not support m = %d", code->m);
  const size_t per = (size_t)code->N * code->m;
  const double t = now_s();
  Pool *p = nullptr;
  {
    // tickets and queue room are taken for all n frames at once, in arrival order
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->error) return set_error(srv->error, "the server stopped after an error");
    if (int st = make_pool(srv, code, &p)) return st;
    if (p->queue.size() + p->reserved + (size_t)n > srv->queue_limit)
      return set_error(NBFD_EBUSY, "request queue full");
    p->reserved += (size_t)n;
    for (int i = 0; i < n; ++i) {
      tickets[i] = srv->next_ticket++;
      srv->pending[tickets[i]] = 1;
    }
  }
  // the frames are copied and queued in chunks, outside the lock, so that the worker starts
  // on the first chunk while the rest is copied
  constexpr int kChunk = 256;
  std::vector<Request> reqs;
  for (int i0 = 0; i0 < n; i0 += kChunk) {
    const int i1 = n - i0 < kChunk ? n : i0 + kChunk;
    reqs.clear();
    reqs.resize(i1 - i0);
    for (int i = i0; i < i1; ++i) {
      Request &r = reqs[i - i0];
      r.ticket = tickets[i];
      r.llr.assign(llr_host + per * i, llr_host + per * (i + 1));
      r.max_iter = max_iter;
      r.t_submit = arrival ? arrival[i] : t;
    }
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      for (Request &r : reqs) p->queue.push_back(std::move(r));
      p->reserved -= reqs.size();
    }
    srv->cv.notify_all();
  }
  return NBFD_OK;
}

extern "C" int nbfd_srv_collect(nbfd_server *srv, int max_n, uint64_t *tickets, uint8_t *ok,
                                int32_t *iters, double *latency_s) {
  if (!srv || max_n < 0) return set_error(NBFD_EINVAL, "bad argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  int n = 0;
  while (n < max_n && !srv->done_order.empty()) {
    const uint64_t t = srv->done_order.front();
    srv->done_order.pop_front();
    auto it = srv->done.find(t);
    if (it == srv->done.end()) continue;  // already taken by nbfd_srv_poll
    if (tickets) tickets[n] = t;
    if (ok) ok[n] = it->second.ok;
    if (iters) iters[n] = it->second.iters;
    if (latency_s) latency_s[n] = it->second.latency;
    srv->done.erase(it);
    ++n;
  }
  if (n == 0 && srv->error) return set_error(srv->error, "the server stopped after an error");
  return n;
}

extern "C" int nbfd_srv_stats(nbfd_server *srv, long long *rounds, long long *queued,
                              long long *in_flight, size_t *device_bytes) {
  if (!srv) return set_error(NBFD_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(srv->mu);
  long long q = 0, f = 0;
  for (auto &kv : srv->pools) {
    q += (long long)(kv.second->queue.size() + kv.second->reserved);
    f += (long long)kv.second->in_flight.size();
  }
  if (rounds) *rounds = srv->rounds;
  if (queued) *queued = q;
  if (in_flight) *in_flight = f;
  if (device_bytes) *device_bytes = srv->used;
  return NBFD_OK;
}

extern "C" int nbfd_srv_register(nbfd_server *srv, const nbfd_code *code) {
  if (!srv || !code) return set_error(NBFD_EINVAL, "NULL argument");
  if (!form_supported(srv->form, code->m))
    return set_error(NBFD_ENOTSUP, "the server's form does not support m = %d", code->m);
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->error) return set_error(srv->error, "the server stopped after an error");
  Pool *p = nullptr;
  return make_pool(srv, code, &p);
}

extern "C" int nbfd_srv_worker_times(nbfd_server *srv, double *seconds) {
  if (!srv || !seconds) return set_error(NBFD_EINVAL, "NULL argument");
  for (int i = 0; i < 5; ++i)
    seconds[i] = 1e-9 * (double)srv->phase_ns[i].load(std::memory_order_relaxed);
  return NBFD_OK;
}
