// CHECK TO VARIABLE (Section 3.2) as a per-warp bulk-copy pipeline.
//
// A check's k slots are one contiguous block of k*q floats ([slot][z], slots check-major), and
// consecutive checks of a frame are contiguous too. Each warp owns a sequence of tiles of CPW
// checks; lane 0 streams the next S-2 tiles into the warp's shared memory with cp.async.bulk
// (the bulk copy engine, completion counted on one mbarrier per stage) while the warp works on
// the current tile in place: a lane gathers entries H_e z of every slot e of its check, forms the
// leave-one-out Gamma sums (prefix and suffix passes: no subtraction, so +inf magnitudes stay
// exact; signs XOR), and writes output H_e z of slot e back to the same word (z -> H_e z is a
// bijection, so each word has one reader and one writer). Lane 0 then writes the tile back with
// one bulk shared->global copy per run of checks of one frame.
//
// Every mbarrier wait is bounded by a clock budget: on expiry the kernel records
// NBFD_ETIMEDOUT in *err, waits (bounded) for its own copies and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "bulk_copy.cuh"
#include "check_math.cuh"
#include "device_common.cuh"
#include "nbfd_internal.h"

namespace nbfd {

namespace {

// item / M and item % M; 32-bit when the item count fits (the usual case: F * M < 2^32)
__device__ __forceinline__ long long div_m(long long item, int M, bool narrow) {
  return narrow ? static_cast<long long>(static_cast<uint32_t>(item) / static_cast<uint32_t>(M))
                : item / M;
}

__device__ __forceinline__ int n_frames_of(const FrameSet &fs) {
  return fs.list ? __ldg(fs.count) : fs.n_static;
}
__device__ __forceinline__ int frame_id(const FrameSet &fs, long long slot) {
  return fs.list ? __ldg(fs.list + slot) : static_cast<int>(slot);
}

// Issue one bulk copy per run of consecutive checks of one frame in stage `st` (items
// st*T .. st*T+T-1 of the flattened (frame slot, check) list). Returns the bytes moved.
template <bool kLoad, typename W>
__device__ uint32_t stage_copies(const FrameSet &fs, long long st, int T, long long total, int M,
                                 int k, int E, int Q, const W *gsrc, W *gdst, W *sbuf,
                                 uint64_t *bar) {
  const bool narrow = total < (1ll << 32);
  const uint32_t check_bytes = static_cast<uint32_t>(k * Q * sizeof(W));
  uint32_t bytes = 0;
  long long item = st * T;
  const long long end = (st * T + T < total) ? st * T + T : total;
  while (item < end) {
    const long long slot = div_m(item, M, narrow);
    const int c0 = static_cast<int>(item - slot * M);
    long long run = M - c0;
    if (item + run > end) run = end - item;
    const int f = frame_id(fs, slot);
    const size_t goff = ((size_t)f * E + (size_t)c0 * k) * Q;
    W *s = sbuf + (size_t)(item - st * T) * k * Q;
    const uint32_t nb = static_cast<uint32_t>(run) * check_bytes;
    if constexpr (kLoad) {
      bulk_load(s, gsrc + goff, nb, bar);
    } else {
      bulk_store(gdst + goff, s, nb);
    }
    bytes += nb;
    item += run;
  }
  return bytes;
}

// The first iteration's loads (lambda0 given): V->C of every edge of a variable is still its
// INITIALIZATION message Lambda0 (Section 3.2), stored once per variable as [frame][variable][z];
// slot e of check c gets a copy of Lambda0 of its variable. Returns the bytes moved.
template <typename W>
__device__ uint32_t stage_copies_l0(const FrameSet &fs, long long st, int T, long long total,
                                    int M, int k, int N, int Q, const W *l0,
                                    const int32_t *__restrict__ edge_var, W *sbuf, uint64_t *bar) {
  const bool narrow = total < (1ll << 32);
  const uint32_t vb = static_cast<uint32_t>(Q * sizeof(W));
  uint32_t bytes = 0;
  const long long end = (st * T + T < total) ? st * T + T : total;
  for (long long item = st * T; item < end; ++item) {
    const long long slot = div_m(item, M, narrow);
    const int c = static_cast<int>(item - slot * M);
    const int f = frame_id(fs, slot);
    W *s = sbuf + (size_t)(item - st * T) * k * Q;
    for (int j = 0; j < k; ++j) {
      const int v = __ldg(edge_var + (size_t)c * k + j);
      bulk_load(s + (size_t)j * Q, l0 + ((size_t)f * N + v) * Q, vb, bar);
      bytes += vb;
    }
  }
  return bytes;
}

}  // namespace

// Per-warp variant: each warp runs its own S-stage pipeline of tiles of CPW checks (no block
// barriers); lane l works on entries t = l*EPL .. l*EPL+EPL-1 of the tile (check t / Q, z = t % Q,
// EPL consecutive z of one check), so the index map of an edge is read as EPL consecutive bytes.
template <int MB, int KMAX>
struct WarpCheck {
  static constexpr int Q = 1 << MB;
  static constexpr int EPL = Q < 8 ? Q : 8;  // entries per lane
  static constexpr int CPW = 32 * EPL / Q;   // checks per warp tile
};

template <int MB, int KMAX, typename W, bool L0>
__global__ void __launch_bounds__(256)
    k_check_warp(const W *__restrict__ v2c, W *__restrict__ c2v,
                 const uint8_t *__restrict__ edge_h, const uint8_t *__restrict__ perm, int M, int k,
                 int E, int S, FrameSet fs, int32_t *err, LoopTick tick,
                 const int32_t *__restrict__ edge_var, int N) {
  using WC = WarpCheck<MB, KMAX>;
  constexpr int Q = WC::Q, EPL = WC::EPL, CPW = WC::CPW;
  griddep_wait();
  griddep_release();
  if (tick.iter && blockIdx.x == 0 && threadIdx.x == 0) {
    *tick.iter += 1;   // iteration number of this launch, read by the stop kernel
    *tick.zero = 0;    // the stop kernel's output count (its previous readers are done)
  }
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw) + wib * 8;
  const size_t tile_floats = (size_t)CPW * k * Q;
  W *stages = reinterpret_cast<W *>(smem_raw + 128 * 8) + (size_t)wib * S * tile_floats;
  const long long total = (long long)n_frames_of(fs) * M;
  const bool narrow = total < (1ll << 32);
  const long long n_tiles = (total + CPW - 1) / CPW;
  const long long gw = (long long)blockIdx.x * nwarps + wib;
  const long long nw = (long long)gridDim.x * nwarps;
  const long long my_count = gw < n_tiles ? (n_tiles - gw + nw - 1) / nw : 0;
  if (my_count == 0) return;
  if (lane == 0) {
    for (int b = 0; b < S; ++b) mbar_init(&bars[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  long long issued = 0;
  auto issue = [&](long long j) {
    const long long tj = gw + j * nw;
    const int bj = static_cast<int>(j % S);
    const long long first = tj * CPW;
    const long long n = (first + CPW < total ? CPW : total - first);
    mbar_expect_tx(&bars[bj], static_cast<uint32_t>(n * k * Q * sizeof(W)));
    if constexpr (L0)
      stage_copies_l0<W>(fs, tj, CPW, total, M, k, N, Q, v2c, edge_var,
                         stages + (size_t)bj * tile_floats, &bars[bj]);
    else
      stage_copies<true, W>(fs, tj, CPW, total, M, k, E, Q, v2c, nullptr,
                            stages + (size_t)bj * tile_floats, &bars[bj]);
  };
  if (lane == 0)
    for (; issued < S - 2 && issued < my_count; ++issued) issue(issued);
  const int ci = lane * EPL / Q;       // this lane's check within the tile
  const int z0 = (lane * EPL) % Q;     // first of its EPL entries
  long long i = 0;
  bool failed = false;
  for (; i < my_count; ++i) {
    const int b = static_cast<int>(i % S);
    const long long tile = gw + i * nw;
    if (lane == 0 && issued < my_count) {
      bulk_wait_read_all_but_one();  // the buffer of tile i-2 was written back
      issue(issued);
      ++issued;
    }
    const bool ok = mbar_wait_bounded(&bars[b], static_cast<uint32_t>((i / S) & 1));
    if (__any_sync(0xffffffffu, !ok)) {
      failed = true;
      break;
    }
    const long long item = tile * CPW + ci;
    if (item < total) {
      const int c = static_cast<int>(item - div_m(item, M, narrow) * M);
      W *s = stages + (size_t)b * tile_floats + (size_t)ci * k * Q;
      check_lane_inplace<Q, EPL, KMAX, W>(s, c, k, z0, edge_h, perm);
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      stage_copies<false, W>(fs, tile, CPW, total, M, k, E, Q, nullptr, c2v,
                          stages + (size_t)b * tile_floats, nullptr);
      bulk_commit();
    }
  }
  if (lane == 0) {
    if (failed) {
      if (err) atomicExch(err, NBFD_ETIMEDOUT);
      for (long long j = i; j < issued; ++j)
        mbar_wait_bounded(&bars[j % S], static_cast<uint32_t>((j / S) & 1));
    }
    bulk_wait_read_all();  // the CTA's shared memory must outlive the bulk stores' reads
  }
}

// Team variant for tiles of one whole check (q >= 128): the kTeam warps of a block share one
// S-stage pipeline, so an SM holds a block's S tiles per kTeam warps instead of S per warp. At
// q = 256 and k = 16 a check is 16 KiB: three stages per warp left 4 warps on an SM, the team
// variant keeps 16. Thread t works on entries t*EPL .. t*EPL+EPL-1 of the check; thread 0 drives
// the bulk copies; block barriers separate the in-place work from the write-back.
constexpr int kTeam = kCheckTeamWarps;

template <int MB, int KMAX, typename W, bool L0>
__global__ void __launch_bounds__(32 * kTeam, KMAX <= 16 ? 4 : 2)
    k_check_team(const W *__restrict__ v2c, W *__restrict__ c2v,
                 const uint8_t *__restrict__ edge_h, const uint8_t *__restrict__ perm, int M, int k,
                 int E, int S, FrameSet fs, int32_t *err, LoopTick tick,
                 const int32_t *__restrict__ edge_var, int N) {
  constexpr int Q = 1 << MB, EPL = Q / (32 * kTeam);
  static_assert(EPL >= 1 && EPL * 32 * kTeam == Q, "one check per tile");
  griddep_wait();
  griddep_release();
  if (tick.iter && blockIdx.x == 0 && threadIdx.x == 0) {
    *tick.iter += 1;
    *tick.zero = 0;
  }
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
  const size_t tile = (size_t)k * Q;
  W *stages = reinterpret_cast<W *>(smem_raw + 128);
  const int tid = threadIdx.x;
  const long long total = (long long)n_frames_of(fs) * M;
  const bool narrow = total < (1ll << 32);
  const long long gb = blockIdx.x, nb = gridDim.x;
  const long long my_count = gb < total ? (total - gb + nb - 1) / nb : 0;
  if (my_count == 0) return;  // block-uniform
  if (tid == 0) {
    for (int b = 0; b < S; ++b) mbar_init(&bars[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  long long issued = 0;  // thread 0's count of tiles whose loads it issued
  auto issue = [&](long long j) {
    const long long tj = gb + j * nb;
    const int bj = static_cast<int>(j % S);
    mbar_expect_tx(&bars[bj], static_cast<uint32_t>(tile * sizeof(W)));
    if constexpr (L0)
      stage_copies_l0<W>(fs, tj, 1, total, M, k, N, Q, v2c, edge_var, stages + bj * tile,
                         &bars[bj]);
    else
      stage_copies<true, W>(fs, tj, 1, total, M, k, E, Q, v2c, nullptr, stages + bj * tile,
                            &bars[bj]);
  };
  if (tid == 0)
    for (; issued < S - 2 && issued < my_count; ++issued) issue(issued);
  auto check_of = [&](long long item) {
    return static_cast<int>(item - div_m(item, M, narrow) * M);
  };
  // index words of the current check; those of the next one load while it is worked on (0.754
  // -> 0.764 of HBM at 256 GF(256) N=2048 k=16 frames; the per-warp kernel measured slower with
  // it, its registers costing more than the latency it hides)
  CheckIndex<Q, EPL, KMAX> ix;
  check_index_load<Q, EPL, KMAX>(ix, check_of(gb), k, tid * EPL, edge_h, perm);
  long long i = 0;
  bool failed = false;
  for (; i < my_count; ++i) {
    const int b = static_cast<int>(i % S);
    const long long item = gb + i * nb;
    if (tid == 0 && issued < my_count) {
      bulk_wait_read_all_but_one();  // the buffer of tile i-2 was written back
      issue(issued);
      ++issued;
    }
    CheckIndex<Q, EPL, KMAX> ix_next;
    if (i + 1 < my_count)
      check_index_load<Q, EPL, KMAX>(ix_next, check_of(item + nb), k, tid * EPL, edge_h, perm);
    const bool ok = mbar_wait_bounded(&bars[b], static_cast<uint32_t>((i / S) & 1));
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    check_lane_apply<Q, EPL, KMAX, W>(stages + b * tile, k, ix);
    ix = ix_next;
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      stage_copies<false, W>(fs, item, 1, total, M, k, E, Q, nullptr, c2v, stages + b * tile,
                             nullptr);
      bulk_commit();
    }
  }
  if (tid == 0) {
    if (failed) {
      if (err) atomicExch(err, NBFD_ETIMEDOUT);
      for (long long j = i; j < issued; ++j)
        mbar_wait_bounded(&bars[j % S], static_cast<uint32_t>((j / S) & 1));
    }
    bulk_wait_read_all();  // the CTA's shared memory must outlive the bulk stores' reads
  }
}

// The team variant's launch (q = 128 or 256).
static cudaError_t launch_check_team(const nbfd_code *c, FrameSet fs, const float *v2c, float *c2v,
                                     cudaStream_t s, int32_t *err, LoopTick tick, CheckTune tune,
                                     bool f16, const float *lambda0) {
  const int Q = c->q, k = c->k;
  const size_t wb = f16 ? 2 : 4;
  const int S = tune.stages > 0 ? tune.stages : 3;
  const size_t smem = 128 + (size_t)S * k * Q * wb;
  if (S < 3 || S > 8 || smem > kMaxSmemPerBlock || (c->m != 7 && c->m != 8))
    return cudaErrorInvalidValue;
  const long long total = (long long)fs.n_static * c->M;
  int fill = static_cast<int>((228 * 1024) / (smem + 1024));
  fill = fill < 1 ? 1 : (fill > 16 ? 16 : fill);
  const int per_sm = tune.blocks_per_sm > 0
                         ? tune.blocks_per_sm
                         : fill * oversubscribed_waves(total, (long long)sm_count() * fill);
  long long grid = (long long)sm_count() * per_sm;
  if (grid > total) grid = total;
  if (grid < 1) grid = 1;
#define NBFD_TEAM_T(MB, KM, W, L0)                                                             \
  {                                                                                             \
    const cudaError_t ae = ensure_smem((const void *)k_check_team<MB, KM, W, L0>, smem);        \
    if (ae != cudaSuccess) return ae;                                                           \
    const cudaError_t le = launch_dependent(                                                    \
        k_check_team<MB, KM, W, L0>, dim3((int)grid), dim3(32 * kTeam), smem, s,               \
        reinterpret_cast<const W *>(L0 ? lambda0 : v2c), reinterpret_cast<W *>(c2v),            \
        c->d_edge_h, c->d_perm, c->M, k, c->E, S, fs, err, tick, c->d_edge_var, c->N);          \
    if (le != cudaSuccess) return le;                                                           \
    return cudaGetLastError();                                                                  \
  }
#define NBFD_TEAM_K(MB, W, L0)                     \
  {                                                \
    if (k <= 4) NBFD_TEAM_T(MB, 4, W, L0)          \
    else if (k <= 8) NBFD_TEAM_T(MB, 8, W, L0)     \
    else if (k <= 16) NBFD_TEAM_T(MB, 16, W, L0)   \
    else NBFD_TEAM_T(MB, 32, W, L0)                \
  }
  if (f16) {
    if (c->m != 8) return cudaErrorNotSupported;
    NBFD_TEAM_K(8, __half, false)
  }
  if (c->m == 8) {
    if (lambda0) NBFD_TEAM_K(8, float, true)
    NBFD_TEAM_K(8, float, false)
  }
  if (lambda0) NBFD_TEAM_K(7, float, true)
  NBFD_TEAM_K(7, float, false)
#undef NBFD_TEAM_K
#undef NBFD_TEAM_T
}

// Built-in choice of the team variant: one-check tiles of 8 KiB or more, where per-warp stages
// would leave an SM few warps.
static bool team_default(const nbfd_code *c) { return c->q >= 128 && c->k > 8; }

cudaError_t launch_check(const nbfd_code *c, FrameSet fs, const float *v2c, float *c2v,
                         cudaStream_t s, int32_t *err, LoopTick tick, CheckTune tune, bool f16,
                         const float *lambda0) {
  if (lambda0 && f16) return cudaErrorNotSupported;
  const bool team = tune.team > 0 || (tune.team < 0 && tune.warps == 0 && team_default(c));
  if (team) return launch_check_team(c, fs, v2c, c2v, s, err, tick, tune, f16, lambda0);
  const int Q = c->q, k = c->k;
  const size_t wb = f16 ? 2 : 4;  // bytes per stored message entry
  const int epl = Q < 8 ? Q : 8;
  const int cpw = 32 * epl / Q;
  const int S = tune.stages > 0 ? tune.stages : 3;
  const int warps =
      tune.warps > 0 ? tune.warps : (k <= 4 ? 8 : (k <= 8 ? 4 : (k <= 16 ? 2 : 1)));
  const size_t smem = 128 * 8 + (size_t)warps * S * cpw * k * Q * wb;
  if (warps > 8 || S < 3 || S > 8 || smem > kMaxSmemPerBlock) return cudaErrorInvalidValue;
  const long long total = (long long)fs.n_static * c->M;
  const long long n_tiles = (total + cpw - 1) / cpw;
  // default: waves of as many blocks per SM as shared memory holds (at least 2, at most 8)
  int fill = static_cast<int>((228 * 1024) / (smem + 1024));
  fill = fill < 2 ? 2 : (fill > 8 ? 8 : fill);
  const int per_sm = tune.blocks_per_sm > 0
                         ? tune.blocks_per_sm
                         : fill * oversubscribed_waves(n_tiles, (long long)sm_count() * fill * warps);
  long long grid = (long long)sm_count() * per_sm;
  const long long need = (n_tiles + warps - 1) / warps;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
#define NBFD_CHK_T(MB, KM, W, L0)                                                              \
  {                                                                                             \
    const cudaError_t ae = ensure_smem((const void *)k_check_warp<MB, KM, W, L0>, smem);        \
    if (ae != cudaSuccess) return ae;                                                           \
    const cudaError_t le = launch_dependent(                                                    \
        k_check_warp<MB, KM, W, L0>, dim3((int)grid), dim3(warps * 32), smem, s,                \
        reinterpret_cast<const W *>(L0 ? lambda0 : v2c), reinterpret_cast<W *>(c2v),            \
        c->d_edge_h, c->d_perm, c->M, k, c->E, S, fs, err, tick, c->d_edge_var, c->N);          \
    if (le != cudaSuccess) return le;                                                           \
  }
#define NBFD_CHK(MB, KM)                       \
  {                                            \
    if (lambda0) NBFD_CHK_T(MB, KM, float, true) \
    else NBFD_CHK_T(MB, KM, float, false)        \
  }
#define NBFD_CHK_M(MB)                     \
  {                                        \
    if (k <= 4) NBFD_CHK(MB, 4)            \
    else if (k <= 6) NBFD_CHK(MB, 6)       \
    else if (k <= 8) NBFD_CHK(MB, 8)       \
    else if (k <= 16) NBFD_CHK(MB, 16)     \
    else NBFD_CHK(MB, 32)                  \
  }
  if (f16) {  // half storage: GF(256) only
    if (c->m != 8) return cudaErrorNotSupported;
    if (k <= 4) NBFD_CHK_T(8, 4, __half, false)
    else if (k <= 8) NBFD_CHK_T(8, 8, __half, false)
    else if (k <= 16) NBFD_CHK_T(8, 16, __half, false)
    else NBFD_CHK_T(8, 32, __half, false)
    return cudaGetLastError();
  }
  switch (c->m) {
    case 2: NBFD_CHK_M(2) break;
    case 3: NBFD_CHK_M(3) break;
    case 4: NBFD_CHK_M(4) break;
    case 5: NBFD_CHK_M(5) break;
    case 6: NBFD_CHK_M(6) break;
    case 7: NBFD_CHK_M(7) break;
    case 8: NBFD_CHK_M(8) break;
    default: return cudaErrorInvalidValue;
  }
#undef NBFD_CHK_M
#undef NBFD_CHK
#undef NBFD_CHK_T
  return cudaGetLastError();
}

}  // namespace nbfd
