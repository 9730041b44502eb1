// Internal declarations shared by the translation units of libnbfd.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "nbfd.h"

struct nbfd_code {
  int N = 0, M = 0, k = 0, m = 0, q = 0, E = 0;
  uint32_t poly = 0;
  int device = 0;
  std::vector<int32_t> caller_edge_of_slot;  // [E]
  std::vector<uint8_t> index_map;            // [q][q]: H z for h = row (Appendix A)
  // device tables, carved from one allocation
  void *d_block = nullptr;
  int32_t *d_edge_var = nullptr;   // [E] variable of each slot (check-major)
  uint8_t *d_edge_h = nullptr;     // [E] h of each slot
  int32_t *d_var_edges = nullptr;  // [N][2] the two slots of each variable
  uint8_t *d_perm = nullptr;       // [q][q] index map, row h
  uint8_t *d_gf_exp = nullptr;     // [2q] alpha^i, i in [0, 2q)
  uint8_t *d_gf_log = nullptr;     // [q]  log_alpha(x), x != 0
  uint8_t *d_edge_z = nullptr;     // [E][8] H alpha^i (i < m) of each slot, 0 past m
};

namespace nbfd {

// Frames a launch works on: either frames 0..n_static-1, or the first *count entries of list.
struct FrameSet {
  const int32_t *list = nullptr;
  const int32_t *count = nullptr;
  int n_static = 0;
};

// Device words a check-kernel launch updates once (thread 0 of block 0, after the dependent-launch
// wait), so that a replayed graph of iterations needs no per-iteration arguments: the iteration
// number *iter is incremented and the next active-frame count *zero is cleared.
struct LoopTick {
  int32_t *iter = nullptr;
  int32_t *zero = nullptr;
};

// Launch shapes picked by the autotuner (0 = the built-in default).
struct CheckTune {
  int warps = 0;          // warps per block, 1..8
  int stages = 0;         // bulk-copy pipeline depth per warp (per block with `team`), 3..8
  int blocks_per_sm = 0;  // grid cap in blocks per SM
  int team = -1;          // 1: the block's warps share one pipeline of whole checks (q >= 128),
                          // 0: one pipeline per warp, -1: the built-in choice
};
struct VarTune {
  int blocks_per_sm = 0;  // grid cap in blocks per SM
  int warps = 0;          // warps per block where the kernel has several shapes (GF(64): 4, 7, 15)
};
constexpr size_t kMaxSmemPerBlock = 227 * 1024;
constexpr int kCheckTeamWarps = 4;  // warps of a block of the check kernel's team variant
// Waves of resident blocks for a grid-stride kernel with `work` items over `warps_per_wave`
// warps: one wave leaves the warps' finishing times uneven (memory bandwidth is not shared
// evenly), so the grid is oversubscribed -- up to 8 waves, the block scheduler then evening out
// the load -- as long as every warp still gets about a dozen items to amortise its pipeline fill.
inline int oversubscribed_waves(long long work, long long warps_per_wave) {
  constexpr long long kItemsPerWarp = 12, kMaxWaves = 8;
  if (warps_per_wave < 1) return 1;
  const long long w = work / (warps_per_wave * kItemsPerWarp);
  return static_cast<int>(w < 1 ? 1 : (w > kMaxWaves ? kMaxWaves : w));
}
// Launch shapes cached by the autotuner for (device, code shape, n_frames, form), if any.
bool tune_lookup(const nbfd_code *c, int F, int form, CheckTune *ct, VarTune *vt);

// Scratch of one decoding loop, carved from one 256-byte aligned block (nbfd_decode's workspace
// or nbfd_decode_noalloc's fixed array); bytes is the block size it needs (base may be NULL).
struct DecodeScratch {
  float *v2c, *c2v;  // messages [F][E][q], float or (NBFD_STORE_F16) half words
  uint8_t *fsyn;     // [F][E] per-edge Fourier syndrome words
  int32_t *list[2];  // active-frame lists, ping-pong
  int32_t *count;    // [max_iter + 2] active count per iteration
  int32_t *stats;    // [16]: [0] Fourier-only clears, [1] NBFD_ETIMEDOUT if a bounded wait expired
  size_t bytes;
};
DecodeScratch carve_decode_scratch(const nbfd_code *c, int F, int max_iter, int form, char *base);
// The decoding loop of nbfd_decode on the scratch w (arguments already validated). host_words:
// two int32 host words for the count and status read-backs (pinned or pageable). timers: honour
// nbfd_prof_enable. Sets the calling thread's nbfd_last_decode_stats; returns NBFD_ETIMEDOUT if
// a kernel's bounded wait expired.
int decode_loop(const nbfd_code *c, int F, const float *llr, int max_iter, int form,
                uint16_t *symbols, uint8_t *ok, int32_t *iters, const DecodeScratch &w,
                int32_t *host_words, bool timers, cudaStream_t s);

int set_error(int status, const char *fmt, ...);
int check_cuda(cudaError_t e, const char *what);
int sm_count();
cudaError_t ensure_smem(const void *kernel, size_t bytes);

// Launch with programmatic stream serialization: the kernel may be scheduled while the previous
// kernel of the stream still runs, and must call griddep_wait() before reading its outputs.
template <typename... Exp, typename... Act>
cudaError_t launch_dependent(void (*kernel)(Exp...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t s, Act &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Exp>(args)...);
}

// kernel launchers (return cudaGetLastError() after the launch)
cudaError_t launch_init(const nbfd_code *c, int F, const float *llr, float *lambda0, float *v2c,
                        int32_t *list_out, int32_t *count_out, cudaStream_t s, bool f16 = false);
inline bool stores_f16(int form) { return (form & NBFD_STORE_F16) != 0; }
// err (device word, may be NULL) receives NBFD_ETIMEDOUT if a bounded wait of the kernel expired.
// f16: messages stored as IEEE half (NBFD_STORE_F16); the float pointers then address halves.
// lambda0 (float storage only): the first iteration's V->C given as Lambda0 once per variable,
// [frame][variable][z] (the INITIALIZATION's message on both edges); v2c is then unused.
cudaError_t launch_check(const nbfd_code *c, FrameSet fs, const float *v2c, float *c2v,
                         cudaStream_t s, int32_t *err = nullptr, LoopTick tick = {},
                         CheckTune tune = {}, bool f16 = false, const float *lambda0 = nullptr);
cudaError_t launch_var(const nbfd_code *c, FrameSet fs, int form, const float *llr,
                       const float *c2v, float *v2c, uint16_t *sym, uint8_t *fsyn, cudaStream_t s,
                       int32_t *err = nullptr, VarTune tune = {});
cudaError_t launch_syndrome(const nbfd_code *c, int F, const uint16_t *sym, const uint8_t *fsyn,
                            uint16_t *fourier, uint16_t *exact, cudaStream_t s);
// Stop test + compaction of one decoding iteration (see decode.cu). With iter_dev the iteration
// number is read from that device word instead of `iter`.
cudaError_t launch_stop(const nbfd_code *c, FrameSet fs, const uint16_t *sym, const uint8_t *fsyn,
                        int iter, int max_iter, int32_t *next_list, int32_t *next_count,
                        uint8_t *ok, int32_t *iters, int32_t *stats, cudaStream_t s,
                        const int32_t *iter_dev = nullptr);
bool form_supported(int form, int m);
cudaError_t launch_var_tc(const nbfd_code *c, FrameSet fs, int form, const float *llr,
                          const float *c2v, float *v2c, uint16_t *sym, uint8_t *fsyn, int32_t *err,
                          cudaStream_t s, bool symbol, VarTune tune = {});
// The same forms on the 5th-generation tensor cores (tcgen05 MMA, accumulators in tensor memory;
// kernels_var_tc5.cu), on sm_103 devices.
bool var_tc5_available();
bool tc_uses_tcgen05(int form);  // the path a tensor-core form runs on (NBFD_TCGEN05 / NBFD_MMA_SYNC)
cudaError_t launch_var_tc5(const nbfd_code *c, FrameSet fs, int form, const float *llr,
                           const float *c2v, float *v2c, uint16_t *sym, uint8_t *fsyn,
                           int32_t *err, cudaStream_t s, bool symbol, VarTune tune = {});
cudaError_t launch_var_fwht(const nbfd_code *c, FrameSet fs, const float *llr, const float *c2v,
                            float *v2c, uint16_t *sym, uint8_t *fsyn, int32_t *err,
                            cudaStream_t s, bool symbol, VarTune tune = {});
// GF(16): one lane per variable, every stage in registers
cudaError_t launch_var_fwht4(const nbfd_code *c, FrameSet fs, const float *llr, const float *c2v,
                             float *v2c, uint16_t *sym, uint8_t *fsyn, cudaStream_t s,
                             bool symbol, VarTune tune = {});
// GF(64) with N % 8 == 0: eight variables per warp, 16 entries per lane, one transpose per
// transform
bool var_fwht6x8_applies(const nbfd_code *c);
cudaError_t launch_var_fwht6x8(const nbfd_code *c, FrameSet fs, const float *llr, const float *c2v,
                               float *v2c, uint16_t *sym, uint8_t *fsyn, int32_t *err,
                               cudaStream_t s, bool symbol, VarTune tune = {});
// GF(256), float storage, k <= 8: all iterations it0 .. max_iter of the frames in fs, one
// thread-block cluster per frame (see kernels_var_fwht8x2.cu). tail_clusters gives how many
// clusters can be resident at once (0: not available) and their size in CTAs.
int tail_clusters(const nbfd_code *c, bool symbol, int *ctas);
cudaError_t launch_tail_x2(const nbfd_code *c, FrameSet fs, const float *llr, float *v2c,
                           float *c2v, uint16_t *sym, uint8_t *fsyn, int it0, int max_iter,
                           uint8_t *ok, int32_t *iters, int32_t *stats, cudaStream_t s,
                           bool symbol);
// Small GF(16) codes (FWHT form, float storage, per-frame messages within 96 KiB of shared
// memory): the INITIALIZATION and every iteration of each frame in one launch, the frame's
// messages kept in shared memory (kernels_fused_small.cu). ok[f], iters[f] and sym[f] as
// nbfd_decode writes them; stats[0] counts the Fourier-only clears, stats[2] is the launch's
// frame counter: stats[0] and stats[2] must be 0 when it starts.
bool fused_small_applies(const nbfd_code *c, int form);
size_t fused_small_smem(const nbfd_code *c);
cudaError_t launch_fused_small(const nbfd_code *c, int F, const float *llr, uint16_t *sym,
                               uint8_t *ok, int32_t *iters, int32_t *stats, int max_iter,
                               bool symbol, cudaStream_t s);
// Conventional Log-SP of Section 2.2 (kernels_logsp.cu), m = 3..8: the check node's log-
// convolutions and the variable node's additions, x-domain log-probability messages.
bool logsp_supported(int m);
cudaError_t launch_logsp_check(const nbfd_code *c, int F, const float *v2c, float *c2v,
                               cudaStream_t s);
cudaError_t launch_logsp_var(const nbfd_code *c, int F, const float *llr, const float *c2v,
                             float *v2c, uint16_t *sym, bool init, cudaStream_t s);
// GF(256) only: the same computation with two variables per warp, 16 entries per lane, one
// shared-memory transpose per transform and packed f32x2 butterflies
cudaError_t launch_var_fwht8x2(const nbfd_code *c, FrameSet fs, const float *llr, const float *c2v,
                               float *v2c, uint16_t *sym, uint8_t *fsyn, int32_t *err,
                               cudaStream_t s, bool symbol, VarTune tune = {}, bool f16 = false);

}  // namespace nbfd
