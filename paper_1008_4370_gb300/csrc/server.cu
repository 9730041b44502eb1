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
// A frame's arithmetic never involves another frame, so its result is identical alone and in
// any mix of requests.
#include <cuda_runtime.h>

#include <chrono>
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

struct Pool {
  const nbfd_code *code = nullptr;
  int S = 0;  // slots
  size_t bytes = 0;
  void *block = nullptr;
  float *v2c = nullptr, *c2v = nullptr, *llr = nullptr;
  uint16_t *sym = nullptr;
  uint8_t *fsyn = nullptr, *ok = nullptr;
  int32_t *iter = nullptr, *maxit = nullptr, *lists[2] = {nullptr, nullptr};
  float *stage_llr = nullptr;                    // [S][N][m] admitted frames, packed
  int32_t *stage_slot = nullptr, *stage_maxit = nullptr;  // [S]
  uint16_t *pack_sym = nullptr;                  // [S][N] retired frames, packed
  uint8_t *pack_ok = nullptr;                    // [S]
  int32_t *pack_iter = nullptr;                  // [S]
  int32_t *done_list = nullptr, *cnt = nullptr;  // cnt: [0] active(list 0), [1] active(list 1),
                                                 // [2] done, [3] new-slot count, [4] error word
  int cur = 0;
  int active = 0;  // frames in lists[cur] (known on the host after each round)
  std::vector<int> free_slots;
  std::unordered_map<int, Request> in_flight;
  std::deque<Request> queue;
  cudaStream_t stream = nullptr;
  // pinned host buffers
  float *h_llr = nullptr;      // [S][N][m]
  uint16_t *h_sym = nullptr;   // [S][N]
  int32_t *h_io = nullptr;     // [S] slot ids in / done list out
  int32_t *h_small = nullptr;  // [8]: counts, per-slot max_iter staging
  int32_t *h_maxit = nullptr;  // [S]
  int32_t *h_iters = nullptr;  // [S]
  uint8_t *h_ok = nullptr;     // [S]
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
};

namespace nbfd {
namespace {

size_t slot_bytes(const nbfd_code *c) {
  return (size_t)2 * c->E * c->q * 4 + (size_t)2 * c->N * c->m * 4 + (size_t)2 * c->N * 2 + c->E +
         2 + 8 * 4 + 64;
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
  size_t off[19], o = 0;
  off[0] = o; o += msg;                                   // v2c
  off[1] = o; o += msg;                                   // c2v
  off[2] = o; o += al((size_t)S * c->N * c->m * 4);       // llr
  off[3] = o; o += al((size_t)S * c->N * 2);              // sym
  off[4] = o; o += al((size_t)S * c->E);                  // fsyn
  off[5] = o; o += al((size_t)S);                         // ok
  off[6] = o; o += al((size_t)S * 4);                     // iter
  off[7] = o; o += al((size_t)S * 4);                     // maxit
  off[8] = o; o += al((size_t)S * 4);                     // list 0
  off[9] = o; o += al((size_t)S * 4);                     // list 1
  off[10] = o; o += al((size_t)S * 4);                    // done list
  off[11] = o; o += al(8 * 4);                            // counters
  off[12] = o; o += al((size_t)S * c->N * c->m * 4);      // staged LLRs
  off[13] = o; o += al((size_t)S * 4);                    // staged slots
  off[14] = o; o += al((size_t)S * 4);                    // staged max_iter
  off[15] = o; o += al((size_t)S * c->N * 2);             // packed decisions
  off[16] = o; o += al((size_t)S);                        // packed flags
  off[17] = o; o += al((size_t)S * 4);                    // packed iterations
  p->bytes = o;
  if (int st = check_cuda(cudaMalloc(&p->block, o), "cudaMalloc(server pool)")) return st;
  char *b = static_cast<char *>(p->block);
  p->v2c = reinterpret_cast<float *>(b + off[0]);
  p->c2v = reinterpret_cast<float *>(b + off[1]);
  p->llr = reinterpret_cast<float *>(b + off[2]);
  p->sym = reinterpret_cast<uint16_t *>(b + off[3]);
  p->fsyn = reinterpret_cast<uint8_t *>(b + off[4]);
  p->ok = reinterpret_cast<uint8_t *>(b + off[5]);
  p->iter = reinterpret_cast<int32_t *>(b + off[6]);
  p->maxit = reinterpret_cast<int32_t *>(b + off[7]);
  p->lists[0] = reinterpret_cast<int32_t *>(b + off[8]);
  p->lists[1] = reinterpret_cast<int32_t *>(b + off[9]);
  p->done_list = reinterpret_cast<int32_t *>(b + off[10]);
  p->cnt = reinterpret_cast<int32_t *>(b + off[11]);
  p->stage_llr = reinterpret_cast<float *>(b + off[12]);
  p->stage_slot = reinterpret_cast<int32_t *>(b + off[13]);
  p->stage_maxit = reinterpret_cast<int32_t *>(b + off[14]);
  p->pack_sym = reinterpret_cast<uint16_t *>(b + off[15]);
  p->pack_ok = reinterpret_cast<uint8_t *>(b + off[16]);
  p->pack_iter = reinterpret_cast<int32_t *>(b + off[17]);
  int st = check_cuda(cudaMemset(p->cnt, 0, 32), "cudaMemset");
  if (!st) st = check_cuda(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking), "stream");
  if (!st) st = check_cuda(cudaMallocHost(&p->h_llr, (size_t)S * c->N * c->m * 4), "pinned");
  if (!st) st = check_cuda(cudaMallocHost(&p->h_sym, (size_t)S * c->N * 2), "pinned");
  if (!st) st = check_cuda(cudaMallocHost(&p->h_io, (size_t)S * 4), "pinned");
  if (!st) st = check_cuda(cudaMallocHost(&p->h_small, 64), "pinned");
  if (!st) st = check_cuda(cudaMallocHost(&p->h_maxit, (size_t)S * 4), "pinned");
  if (!st) st = check_cuda(cudaMallocHost(&p->h_iters, (size_t)S * 4), "pinned");
  if (!st) st = check_cuda(cudaMallocHost(&p->h_ok, (size_t)S), "pinned");
  if (st) return st;
  for (int s = p->S - 1; s >= 0; --s) p->free_slots.push_back(s);
  srv->used += p->bytes;
  *out = p.get();
  srv->pools[c] = std::move(p);
  return NBFD_OK;
}

void free_pool(Pool *p) {
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->block) cudaFree(p->block);
  if (p->stream) cudaStreamDestroy(p->stream);
  cudaFreeHost(p->h_llr);
  cudaFreeHost(p->h_sym);
  cudaFreeHost(p->h_io);
  cudaFreeHost(p->h_small);
  cudaFreeHost(p->h_maxit);
  cudaFreeHost(p->h_iters);
  cudaFreeHost(p->h_ok);
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

// One round for one pool: admit from its queue, iterate, stop test; enqueued on the pool stream.
// Returns the number of newly admitted frames (their tickets move to in_flight).
int round_issue(nbfd_server *srv, Pool *p, std::deque<Request> &admit) {
  const nbfd_code *c = p->code;
  cudaStream_t s = p->stream;
  const int n_new = static_cast<int>(admit.size());
  int32_t *cur = p->lists[p->cur];
  if (n_new > 0) {
    const size_t per = (size_t)c->N * c->m;
    for (int i = 0; i < n_new; ++i) {
      const int slot = p->free_slots.back();
      p->free_slots.pop_back();
      Request &r = admit[i];
      memcpy(p->h_llr + (size_t)i * per, r.llr.data(), per * 4);
      p->h_io[i] = slot;
      p->h_maxit[i] = r.max_iter;
      p->in_flight[slot] = std::move(r);
    }
    cudaMemcpyAsync(p->stage_llr, p->h_llr, (size_t)n_new * per * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->stage_slot, p->h_io, (size_t)n_new * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->stage_maxit, p->h_maxit, (size_t)n_new * 4, cudaMemcpyHostToDevice, s);
    const int g = n_new < sm_count() * 8 ? n_new : sm_count() * 8;
    k_admit<<<g, 128, 0, s>>>(p->stage_llr, p->stage_slot, p->stage_maxit, n_new,
                              static_cast<int>(per), p->llr, p->iter, p->maxit);
    // new slots appended to the active list
    cudaMemcpyAsync(cur + p->active, p->stage_slot, (size_t)n_new * 4, cudaMemcpyDeviceToDevice, s);
    p->h_small[0] = p->active + n_new;
    p->h_small[1] = n_new;
    cudaMemcpyAsync(p->cnt + p->cur, &p->h_small[0], 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->cnt + 3, &p->h_small[1], 4, cudaMemcpyHostToDevice, s);
    launch_init_slots(c, p->llr, p->v2c, cur + p->active, p->cnt + 3, n_new, s);
  }
  const int total = p->active + n_new;
  if (total == 0) return n_new;
  cudaMemsetAsync(p->cnt + (p->cur ^ 1), 0, 4, s);
  cudaMemsetAsync(p->cnt + 2, 0, 4, s);
  FrameSet fs;
  fs.list = cur;
  fs.count = p->cnt + p->cur;
  fs.n_static = total;
  cudaError_t e = launch_check(c, fs, p->v2c, p->c2v, s, p->cnt + 4);
  if (e == cudaSuccess) e = launch_var(c, fs, srv->form, p->llr, p->c2v, p->v2c, p->sym, p->fsyn, s, p->cnt + 4);
  if (e == cudaSuccess) {
    int grid = total < sm_count() * 16 ? total : sm_count() * 16;
    k_stop_serve<<<grid, 128, 0, s>>>(cur, p->cnt + p->cur, p->sym, p->fsyn, c->d_edge_var,
                                      c->d_edge_h, c->d_gf_exp, c->d_gf_log, c->q, c->N, c->M,
                                      c->k, c->E, p->iter, p->maxit, p->ok, p->lists[p->cur ^ 1],
                                      p->cnt + (p->cur ^ 1), p->done_list, p->cnt + 2);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->error = check_cuda(e, "serving kernels");
  }
  {
    const int g = total < sm_count() * 8 ? total : sm_count() * 8;
    k_gather_done<<<g, 128, 0, s>>>(p->done_list, p->cnt + 2, p->sym, p->ok, p->iter, c->N,
                                    p->pack_sym, p->pack_ok, p->pack_iter);
  }
  // counts back: [active next, done]
  cudaMemcpyAsync(&p->h_small[2], p->cnt + (p->cur ^ 1), 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&p->h_small[3], p->cnt + 2, 4, cudaMemcpyDeviceToHost, s);
  return n_new;
}

void worker_main(nbfd_server *srv) {
  cudaSetDevice(srv->device);
  while (true) {
    // 1. take admissions (under the lock)
    std::vector<std::pair<Pool *, std::deque<Request>>> work;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      auto busy = [&]() {
        for (auto &kv : srv->pools)
          if (kv.second->active > 0 || !kv.second->queue.empty()) return true;
        return false;
      };
      srv->cv.wait_for(lk, std::chrono::milliseconds(20), [&] { return srv->stop || busy(); });
      if (srv->stop) break;
      for (auto &kv : srv->pools) {
        Pool *p = kv.second.get();
        std::deque<Request> admit;
        while (!p->queue.empty() && !p->free_slots.empty() &&
               admit.size() < p->free_slots.size()) {
          admit.push_back(std::move(p->queue.front()));
          p->queue.pop_front();
        }
        if (p->active > 0 || !admit.empty()) work.emplace_back(p, std::move(admit));
      }
    }
    if (work.empty()) continue;
    // 2. issue one round per pool (pools overlap on their own streams)
    for (auto &w : work) round_issue(srv, w.first, w.second);
    // 3. retire
    for (auto &w : work) {
      Pool *p = w.first;
      cudaStreamSynchronize(p->stream);
      const int n_next = p->h_small[2], n_done = p->h_small[3];
      const nbfd_code *c = p->code;
      if (n_done) {
        cudaMemcpyAsync(p->h_io, p->done_list, (size_t)n_done * 4, cudaMemcpyDeviceToHost, p->stream);
        cudaMemcpyAsync(p->h_sym, p->pack_sym, (size_t)n_done * c->N * 2, cudaMemcpyDeviceToHost, p->stream);
        cudaMemcpyAsync(p->h_ok, p->pack_ok, (size_t)n_done, cudaMemcpyDeviceToHost, p->stream);
        cudaMemcpyAsync(p->h_iters, p->pack_iter, (size_t)n_done * 4, cudaMemcpyDeviceToHost, p->stream);
        cudaStreamSynchronize(p->stream);
      }
      const double t = now_s();
      std::lock_guard<std::mutex> lk(srv->mu);
      for (int i = 0; i < n_done; ++i) {
        const int slot = p->h_io[i];
        auto it = p->in_flight.find(slot);
        if (it == p->in_flight.end()) continue;
        Result r;
        r.sym.assign(p->h_sym + (size_t)i * c->N, p->h_sym + (size_t)i * c->N + c->N);
        r.ok = p->h_ok[i];
        r.iters = p->h_iters[i];
        r.latency = t - it->second.t_submit;
        srv->done[it->second.ticket] = std::move(r);
        srv->done_order.push_back(it->second.ticket);
        srv->pending.erase(it->second.ticket);
        p->in_flight.erase(it);
        p->free_slots.push_back(slot);
      }
      p->active = n_next;
      p->cur ^= 1;
      ++srv->rounds;
    }
    srv->cv.notify_all();
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
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->error) return set_error(srv->error, "the server stopped after an error");
  Pool *p = nullptr;
  if (int st = make_pool(srv, code, &p)) return st;
  if (p->queue.size() >= srv->queue_limit) return set_error(NBFD_EBUSY, "request queue full");
  Request r;
  r.ticket = srv->next_ticket++;
  r.llr.assign(llr_host, llr_host + (size_t)code->N * code->m);
  r.max_iter = max_iter;
  r.t_submit = now_s();
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
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->error) return set_error(srv->error, "the server stopped after an error");
  Pool *p = nullptr;
  if (int st = make_pool(srv, code, &p)) return st;
  if (p->queue.size() + (size_t)n > srv->queue_limit) return set_error(NBFD_EBUSY, "request queue full");
  const size_t per = (size_t)code->N * code->m;
  const double t = now_s();
  for (int i = 0; i < n; ++i) {
    Request r;
    r.ticket = srv->next_ticket++;
    r.llr.assign(llr_host + per * i, llr_host + per * (i + 1));
    r.max_iter = max_iter;
    r.t_submit = arrival ? arrival[i] : t;
    tickets[i] = r.ticket;
    srv->pending[r.ticket] = 1;
    p->queue.push_back(std::move(r));
  }
  srv->cv.notify_all();
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
    q += (long long)kv.second->queue.size();
    f += (long long)kv.second->in_flight.size();
  }
  if (rounds) *rounds = srv->rounds;
  if (queued) *queued = q;
  if (in_flight) *in_flight = f;
  if (device_bytes) *device_bytes = srv->used;
  return NBFD_OK;
}
