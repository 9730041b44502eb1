// VARIABLE TO CHECK + TENTATIVE DECISION, FWHT form (FP32).
//
// The boxplus of Section 3.2 is an XOR convolution of Fourier-domain vectors, so by the
// convolution theorem of Section 2.1 it is a pointwise product in the x-domain:
//   Lambda0 [+] Lambda_c'v  =  Gamma( WHT( p0 . WHT(Gamma^{-1}(Lambda_c'v)) ) ) up to a positive scale,
// which the normalisation to P(0) = 1 removes. Per variable: two transforms take the two
// check messages to the x-domain (c1x, c2x), the channel term p0 is rebuilt from the LLRs directly
// in the x-domain, and three transforms return U1 = p0.c2x, U2 = p0.c1x and M = p0.c1x.c2x to the
// Fourier domain. O(q log q) adds instead of O(q^2) FMAs, exact +-1 arithmetic in the butterflies.
//
// Layout: a group of LPV lanes holds one vector, index l*VPT + j in register j of lane l
// (ChannelLayout); butterflies run on register bits then across lanes with shuffles.
#include <cuda_runtime.h>

#include <cstdint>

#include "bulk_copy.cuh"
#include "device_common.cuh"
#include "nbfd_internal.h"

namespace nbfd {

namespace {

template <int N>
__device__ __forceinline__ void ld_global(float (&v)[N], const float *__restrict__ src) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int j = 0; j < N; j += 4) {
      const float4 x = __ldg(reinterpret_cast<const float4 *>(src + j));
      v[j] = x.x;
      v[j + 1] = x.y;
      v[j + 2] = x.z;
      v[j + 3] = x.w;
    }
  } else if constexpr (N == 2) {
    const float2 x = __ldg(reinterpret_cast<const float2 *>(src));
    v[0] = x.x;
    v[1] = x.y;
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = __ldg(src + j);
  }
}

template <int N>
__device__ __forceinline__ void st_global(float *dst, const float (&v)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int j = 0; j < N; j += 4)
      *reinterpret_cast<float4 *>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
  } else if constexpr (N == 2) {
    *reinterpret_cast<float2 *>(dst) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) dst[j] = v[j];
  }
}

__device__ __forceinline__ int frames_in(const FrameSet &fs) {
  return fs.list ? __ldg(fs.count) : fs.n_static;
}
__device__ __forceinline__ int frame_of(const FrameSet &fs, long long slot) {
  return fs.list ? __ldg(fs.list + slot) : static_cast<int>(slot);
}

}  // namespace

// Per warp, two stages of shared memory hold the two check messages of the warp's VPW
// variables; lane 0 resolves the next variables' frame and edge indices and brings their
// messages in with cp.async.bulk (one mbarrier per stage, bounded waits) while the warp
// transforms the current ones.
template <int MB>
struct VarStage {
  static constexpr int Q = 1 << MB;
  static constexpr int VPW = ChannelLayout<MB>::VPW;
  float msg[2][VPW][2][Q];  // [stage][variable][edge 1, edge 2][z]
  int4 idx[2][VPW];         // [stage][variable] = (frame, variable, slot e1, slot e2)
  float m[VPW][Q];          // M of each variable, for the read-out
  uint64_t bar[2];
};

template <int MB>
__device__ __forceinline__ void var_issue(VarStage<MB> &ws, int st, long long base, long long total,
                                          int N, int E, const FrameSet &fs,
                                          const int32_t *__restrict__ var_edges,
                                          const float *__restrict__ c2v) {
  constexpr int Q = VarStage<MB>::Q, VPW = VarStage<MB>::VPW;
  uint32_t bytes = 0;
  for (int g = 0; g < VPW; ++g) {
    const long long item = base + g;
    // past the end: a valid stand-in so that every index the warp uses stays in bounds
    const long long it = item < total ? item : 0;
    const long long slot = it / N;
    const int v = static_cast<int>(it - slot * N);
    const int f = frame_of(fs, slot);
    ws.idx[st][g] = make_int4(f, v, __ldg(var_edges + 2 * v), __ldg(var_edges + 2 * v + 1));
    if (item < total) bytes += 2u * Q * 4u;
  }
  mbar_expect_tx(&ws.bar[st], bytes);
  for (int g = 0; g < VPW; ++g) {
    if (base + g >= total) break;
    const int4 ix = ws.idx[st][g];
    bulk_load(ws.msg[st][g][0], c2v + ((size_t)ix.x * E + ix.z) * Q, Q * 4u, &ws.bar[st]);
    bulk_load(ws.msg[st][g][1], c2v + ((size_t)ix.x * E + ix.w) * Q, Q * 4u, &ws.bar[st]);
  }
}

// warps per block: 8 unless the per-warp stages would pass the 48 KiB static shared-memory limit
template <int MB>
constexpr int fwht_wpb() {
  return sizeof(VarStage<MB>) * 8 <= 46 * 1024 ? 8 : 4;
}

template <int MB, bool SYMBOL>
__global__ void __launch_bounds__(256, 3)
    k_var_fwht(const float *__restrict__ llr, const float *__restrict__ c2v,
               float *__restrict__ v2c, uint16_t *__restrict__ sym, uint8_t *__restrict__ fsyn,
               const int32_t *__restrict__ var_edges, const uint8_t *__restrict__ edge_h,
               const uint8_t *__restrict__ perm, int N, int E, FrameSet fs, int32_t *err) {
  using CL = ChannelLayout<MB>;
  constexpr int Q = CL::Q, VPT = CL::VPT, LPV = CL::LPV, VPW = CL::VPW;
  __shared__ VarStage<MB> stage_mem[fwht_wpb<MB>()];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  VarStage<MB> &ws = stage_mem[wib];
  const int sub = lane / LPV, l = lane % LPV;
  const long long total = (long long)frames_in(fs) * N;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  if (gw * VPW >= total) return;
  if (lane == 0) {
    mbar_init(&ws.bar[0], 1);
    mbar_init(&ws.bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    var_issue<MB>(ws, 0, gw * VPW, total, N, E, fs, var_edges, c2v);
  }
  __syncwarp();
  long long t = 0;
  bool failed = false, next_issued = false;
  for (long long base = gw * VPW; base < total; base += nw * VPW, ++t) {
    const int b = static_cast<int>(t & 1);
    const long long next = base + nw * VPW;
    next_issued = next < total;
    if (lane == 0 && next_issued) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      var_issue<MB>(ws, b ^ 1, next, total, N, E, fs, var_edges, c2v);
    }
    const bool ok = mbar_wait_bounded(&ws.bar[b], static_cast<uint32_t>((t >> 1) & 1));
    if (__any_sync(kFull, !ok)) {
      failed = true;
      break;
    }
    const long long item = base + sub;
    const bool valid = item < total;
    const int4 ix = ws.idx[b][sub];
    const int f = ix.x, v = ix.y, e1 = ix.z, e2 = ix.w;
    float c1[VPT], c2[VPT];
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      c1[j] = gamma_decode_fast(ws.msg[b][sub][0][l * VPT + j]);
      c2[j] = gamma_decode_fast(ws.msg[b][sub][1][l * VPT + j]);
    }
    wht_inplace<MB>(c1, l);  // q * (x-domain check message of e1)
    wht_inplace<MB>(c2, l);
    // x-domain messages are probability vectors (non-negative in exact arithmetic): drop the
    // negative rounding noise of the transform
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      c1[j] = fmaxf(c1[j], 0.0f);
      c2[j] = fmaxf(c2[j], 0.0f);
    }
    float p[VPT];
    channel_probs_shared<MB>(llr + ((size_t)f * N + v) * MB, l, p);  // x-domain channel message
    // M_v = p0 . c1x . c2x (all checks), read out below from shared memory
    float *m_sh = ws.m[sub];
    float nm = 0.0f;
    int best_x = 0;
    if constexpr (SYMBOL) {
      // symbol decision: argmax over x of the x-domain marginal p0 . c1x . c2x (ties: lowest x)
      float best = -1.0f;
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        const float mv = p[j] * c1[j] * c2[j];
        if (mv > best) {
          best = mv;
          best_x = l * VPT + j;
        }
      }
#pragma unroll
      for (int o = 1; o < LPV; o <<= 1) {
        const float ob = __shfl_xor_sync(kFull, best, o);
        const int oi = __shfl_xor_sync(kFull, best_x, o);
        if (ob > best || (ob == best && oi < best_x)) {
          best = ob;
          best_x = oi;
        }
      }
    } else {
      float mm[VPT];
#pragma unroll
      for (int j = 0; j < VPT; ++j) mm[j] = p[j] * c1[j] * c2[j];
      wht_inplace<MB>(mm, l);
      nm = __shfl_sync(kFull, mm[0], sub * LPV);
#pragma unroll
      for (int j = 0; j < VPT; ++j) m_sh[l * VPT + j] = mm[j];
    }
    // V->C on e1 excludes the check of e1: U1 = WHT(p0 . c2x); likewise U2 = WHT(p0 . c1x)
#pragma unroll
    for (int j = 0; j < VPT; ++j) c2[j] *= p[j];
    wht_inplace<MB>(c2, l);
    const float n1 = __shfl_sync(kFull, c2[0], sub * LPV);
    const float r1 = n1 > 0.0f ? 1.0f / n1 : 0.0f;  // U(0) <= 0 only by underflow: send delta_0
    if (valid) {
#pragma unroll
      for (int j = 0; j < VPT; ++j) c2[j] = gamma_encode_fast((l == 0 && j == 0) ? 1.0f : c2[j] * r1);
      st_global<VPT>(v2c + ((size_t)f * E + e1) * Q + l * VPT, c2);
    }
#pragma unroll
    for (int j = 0; j < VPT; ++j) c1[j] *= p[j];
    wht_inplace<MB>(c1, l);
    const float n2 = __shfl_sync(kFull, c1[0], sub * LPV);
    const float r2 = n2 > 0.0f ? 1.0f / n2 : 0.0f;
    if (valid) {
#pragma unroll
      for (int j = 0; j < VPT; ++j) c1[j] = gamma_encode_fast((l == 0 && j == 0) ? 1.0f : c1[j] * r2);
      st_global<VPT>(v2c + ((size_t)f * E + e2) * Q + l * VPT, c1);
    }
    if constexpr (SYMBOL) {
      // the Fourier-domain syndrome words describe bitwise decisions: with symbol decisions they
      // are written as 0, so that the stop test rests on the GF(2^m) syndrome alone
      if (valid && l == 0) {
        if (sym) sym[(size_t)f * N + v] = static_cast<uint16_t>(best_x);
        if (fsyn) {
          fsyn[(size_t)f * E + e1] = 0;
          fsyn[(size_t)f * E + e2] = 0;
        }
      }
      __syncwarp();
      continue;
    }
    // TENTATIVE: signs of M at alpha^{i-1} (t < MB), H_e1 alpha^{i-1} (t < 2MB) and
    // H_e2 alpha^{i-1} (t < 3MB), one read-out point per lane, gathered with ballots.
    __syncwarp();
    const int h1 = __ldg(edge_h + e1), h2 = __ldg(edge_h + e2);
    uint32_t word = 0;
#pragma unroll
    for (int r = 0; r < (3 * MB + LPV - 1) / LPV; ++r) {
      const int tt = r * LPV + l;
      bool neg_pt = false;
      if (tt < 3 * MB) {
        const int kind = tt / MB, i = tt - kind * MB;
        const int z = kind == 0 ? (1 << i) : __ldg(perm + (kind == 1 ? h1 : h2) * Q + (1 << i));
        neg_pt = m_sh[z] < 0.0f;
      }
      const uint32_t bal = __ballot_sync(kFull, neg_pt);
      const uint32_t mine = LPV == 32 ? bal : (bal >> (sub * LPV)) & ((1u << LPV) - 1u);
      word |= mine << (r * LPV);
    }
    if (nm < 0.0f) word = ~word;
    if (valid && l == 0) {
      const uint32_t mask = (1u << MB) - 1u;
      if (sym) sym[(size_t)f * N + v] = static_cast<uint16_t>(word & mask);
      if (fsyn) {
        fsyn[(size_t)f * E + e1] = static_cast<uint8_t>((word >> MB) & mask);
        fsyn[(size_t)f * E + e2] = static_cast<uint8_t>((word >> (2 * MB)) & mask);
      }
    }
    __syncwarp();
  }
  if (failed && lane == 0) {
    if (err) atomicExch(err, NBFD_ETIMEDOUT);
    // the prefetch of the next stage may still be landing in this warp's shared memory
    if (next_issued)
      mbar_wait_bounded(&ws.bar[(t + 1) & 1], static_cast<uint32_t>(((t + 1) >> 1) & 1));
  }
}

cudaError_t launch_var_fwht(const nbfd_code *c, FrameSet fs, const float *llr, const float *c2v,
                            float *v2c, uint16_t *sym, uint8_t *fsyn, int32_t *err,
                            cudaStream_t s, bool symbol, VarTune tune) {
  const long long total = (long long)fs.n_static * c->N;
  const long long cap = (long long)sm_count() * (tune.blocks_per_sm > 0 ? tune.blocks_per_sm : 8);
#define NBFD_VAR_FWHT(MB)                                                                   \
  {                                                                                         \
    constexpr int VPW = ChannelLayout<MB>::VPW, WPB = fwht_wpb<MB>();                       \
    long long g = (total + WPB * VPW - 1) / (WPB * VPW);                                    \
    if (g > cap * 8 / WPB) g = cap * 8 / WPB;                                               \
    if (g < 1) g = 1;                                                                       \
    if (symbol)                                                                             \
      k_var_fwht<MB, true><<<(int)g, 32 * WPB, 0, s>>>(llr, c2v, v2c, sym, fsyn,            \
                                                       c->d_var_edges, c->d_edge_h,         \
                                                       c->d_perm, c->N, c->E, fs, err);     \
    else                                                                                    \
      k_var_fwht<MB, false><<<(int)g, 32 * WPB, 0, s>>>(llr, c2v, v2c, sym, fsyn,           \
                                                        c->d_var_edges, c->d_edge_h,        \
                                                        c->d_perm, c->N, c->E, fs, err);    \
  }
  switch (c->m) {
    case 2: NBFD_VAR_FWHT(2) break;
    case 3: NBFD_VAR_FWHT(3) break;
    case 4: return launch_var_fwht4(c, fs, llr, c2v, v2c, sym, fsyn, s, symbol, tune);
    case 5: NBFD_VAR_FWHT(5) break;
    case 6:
      if (var_fwht6x8_applies(c))
        return launch_var_fwht6x8(c, fs, llr, c2v, v2c, sym, fsyn, err, s, symbol, tune);
      NBFD_VAR_FWHT(6) break;
    case 7: NBFD_VAR_FWHT(7) break;
    case 8: return launch_var_fwht8x2(c, fs, llr, c2v, v2c, sym, fsyn, err, s, symbol, tune, false);
    default: return cudaErrorInvalidValue;
  }
#undef NBFD_VAR_FWHT
  return cudaGetLastError();
}

}  // namespace nbfd
