// VARIABLE TO CHECK + TENTATIVE DECISION, FWHT form (FP32), GF(64): eight variables per warp.
//
// The algebra is that of kernels_var_fwht.cu (Section 3.2 boxplus = XOR convolution = pointwise
// product in the x-domain, reached with the Section 2.1 transform). Four lanes own one variable
// and each lane 16 entries of a 64-entry vector: 4 index bits in registers, 2 across the 4
// lanes. A transform is 4 butterfly stages in registers, one transpose through shared memory
// that swaps two register bits with the two lane bits, and 2 more stages.
//
// Index layouts (x = index of the 64-entry vector, bit i written x_i; j = register, l = lane
// within the variable's group of 4):
//   P0: registers j0..j3 hold x0, x1, x4, x5; lanes l0, l1 hold x2, x3
//       (x = (j & 3) + 4 l + 16 (j >> 2): 16-byte chunks for shared and global memory)
//   P1: registers hold x2, x3, x4, x5; lanes hold x0, x1
// Forward transform (natural input): stages on j0..j3 in P0, transpose, stages on j0, j1 (x2,
// x3) in P1. Inverse direction: stages on j0..j3 in P1, transpose, stages on j0, j1 (x0, x1) in
// P0, which is natural order. Stages on different bits commute.
//
// Transpose buffers: entry x of variable g sits at 76 g + sum_i x_i w_i, w = (1, 2, 5, 10, 19, 38)
// (float2 pairs, and single floats for M); every access of both layouts is free of bank
// conflicts, and the position splits into a per-lane offset plus a compile-time offset per
// register. A unit of work is 8 consecutive variables of one frame (N % 8 == 0), so its LLR rows
// are one contiguous 192-byte block that the bulk copy engine brings in with the messages.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "bulk_copy.cuh"
#include "device_common.cuh"
#include "nbfd_internal.h"

namespace nbfd {

namespace {

constexpr int kQ6 = 64;
constexpr int kMsgStride = 2 * kQ6 + 16;  // floats per variable in a stage: 2 messages + 64 B pad
constexpr int kVar = 76;                  // buffer entries per variable (max position 75)
constexpr int kNat = 80;                  // floats per variable of M in natural order

__host__ __device__ constexpr int w6(int b) {
  return b == 0 ? 1 : b == 1 ? 2 : b == 2 ? 5 : b == 3 ? 10 : b == 4 ? 19 : 38;
}
__host__ __device__ constexpr int roff0(int j) {  // P0: registers hold x0, x1, x4, x5
  return ((j & 1) ? w6(0) : 0) + ((j & 2) ? w6(1) : 0) + ((j & 4) ? w6(4) : 0) + ((j & 8) ? w6(5) : 0);
}
__host__ __device__ constexpr int roff1(int j) {  // P1: registers hold x2, x3, x4, x5
  return ((j & 1) ? w6(2) : 0) + ((j & 2) ? w6(3) : 0) + ((j & 4) ? w6(4) : 0) + ((j & 8) ? w6(5) : 0);
}
static_assert(roff0(15) + w6(2) + w6(3) < kVar && roff1(15) + w6(0) + w6(1) < kVar, "buffer");

// buf[stage] first holds the unit's check messages ([variable][edge 1 | edge 2 | pad], bulk-copy
// targets), then -- once they are decoded into registers -- the transposes, M in single floats
// and M in natural order. Sharing the space keeps a warp at 10.5 KB (5 blocks of 4 warps per SM).
constexpr int kStageFloats = 2 * 8 * kVar;  // the transpose buffers, >= 8 variables' messages
static_assert(8 * kMsgStride <= kStageFloats && 8 * kNat <= kStageFloats, "stage buffer");
template <int S>
struct X8Stage {
  float buf[S][kStageFloats];   // [stage]
  float llr[S][8 * 6];          // [stage] LLR rows of the unit's 8 variables
  int4 idx[S][8];               // [stage][variable] = (frame, variable, slot e1, slot e2)
  float2 pbt[8][6];             // [variable][bit] = (Pr(b = 0), Pr(b = 1))
  uint64_t bar[S];
  __device__ float *msg(int st, int g) { return &buf[st][g * kMsgStride]; }
};

__device__ __forceinline__ void bfly(float2 &a, float2 &b) {
  const float2 s = __fadd2_rn(a, b);
  b = __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
  a = s;
}
template <int R>
__device__ __forceinline__ void stage(float2 (&v)[16]) {
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (!(j & (1 << R))) bfly(v[j], v[j | (1 << R)]);
}
// one vector as 8 pairs u[i] = (entry i, entry i + 8): register bits 0..2 across the pairs,
// register bit 3 inside each pair
template <int R>
__device__ __forceinline__ void stage_one(float2 (&u)[8]) {
  if constexpr (R < 3) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (!(i & (1 << R))) bfly(u[i], u[i | (1 << R)]);
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float a = u[i].x, b = u[i].y;
      u[i] = make_float2(a + b, a - b);
    }
  }
}

}  // namespace

template <bool SYMBOL, int WARPS, int S, int MINB>
__global__ void __launch_bounds__(32 * WARPS, MINB)
    k_var_fwht6x8(const float *__restrict__ llr, const float *__restrict__ c2v,
                  float *__restrict__ v2c, uint16_t *__restrict__ sym,
                  uint8_t *__restrict__ fsyn, const int32_t *__restrict__ var_edges,
                  const uint8_t *__restrict__ edge_z, int N, int E, FrameSet fs, int32_t *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, l = lane & 3;  // variable of the unit, lane within its group
  X8Stage<S> &ws = reinterpret_cast<X8Stage<S> *>(smem_raw)[wib];
  griddep_wait();
  griddep_release();
  const int F = fs.list ? __ldg(fs.count) : fs.n_static;
  const long long units = (long long)F * N / 8;  // N % 8 == 0
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  if (gw >= units) return;
  const long long n_units = (units - gw + nw - 1) / nw;
  // the warp's units gw, gw + nw, ... as (slot, first variable), without a division per unit
  long long cur_slot = (8 * gw) / N;
  int cur_v = static_cast<int>(8 * gw - cur_slot * N);
  const long long step_s = (8 * nw) / N;
  const int step_v = static_cast<int>(8 * nw - step_s * N);
  int pf_f = 0, pf_v = 0;
  int2 pf_e = make_int2(0, 0);  // lanes 0..7: the edges of variable pf_v + lane, loaded a unit early
  auto load_next = [&]() {  // lane 0 steps, then lanes 0..7 start loading the edges
    if (lane == 0) {
      pf_f = fs.list ? __ldg(fs.list + cur_slot) : static_cast<int>(cur_slot);
      pf_v = cur_v;
      cur_slot += step_s;
      cur_v += step_v;
      if (cur_v >= N) {
        cur_v -= N;
        ++cur_slot;
      }
    }
    const int v = __shfl_sync(kFull, pf_v, 0);
    if (lane < 8) pf_e = __ldg(reinterpret_cast<const int2 *>(var_edges) + v + lane);
  };
  // all lanes: lane 0 arms the barrier, lanes 0..7 issue their variable's two message copies,
  // lane 8 the LLR block (one SIMT instruction each)
  auto issue = [&](int st, int f, int v0) {
    if (lane == 0) mbar_expect_tx(&ws.bar[st], 8u * 2u * kQ6 * 4u + 8u * 6u * 4u);
    __syncwarp();
    if (lane < 8) {
      const int2 e = pf_e;
      ws.idx[st][lane] = make_int4(f, v0 + lane, e.x, e.y);
      bulk_load(ws.msg(st, lane), c2v + ((size_t)f * E + e.x) * kQ6, kQ6 * 4u, &ws.bar[st]);
      bulk_load(ws.msg(st, lane) + kQ6, c2v + ((size_t)f * E + e.y) * kQ6, kQ6 * 4u, &ws.bar[st]);
    } else if (lane == 8) {
      bulk_load(ws.llr[st], llr + ((size_t)f * N + v0) * 6, 8u * 6u * 4u, &ws.bar[st]);
    }
  };
  if (lane == 0) {
#pragma unroll
    for (int st = 0; st < S; ++st) mbar_init(&ws.bar[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  for (int k = 0; k < S - 1 && k < n_units; ++k) {
    load_next();
    issue(k, __shfl_sync(kFull, pf_f, 0), __shfl_sync(kFull, pf_v, 0));
  }
  if (S - 1 < n_units) load_next();
  __syncwarp();
  // per-lane transpose offsets: P0 lanes hold x2, x3; P1 lanes hold x0, x1
  const int o0 = g * kVar + ((l & 1) ? w6(2) : 0) + ((l & 2) ? w6(3) : 0);
  const int o1 = g * kVar + ((l & 1) ? w6(0) : 0) + ((l & 2) ? w6(1) : 0);
  long long t = 0;
  bool failed = false;
  for (; t < n_units; ++t) {
    const int b = static_cast<int>(t % S);
    if (t + S - 1 < n_units) {
      // every issuing lane orders the warp's earlier generic accesses of the stage it refills
      // (made visible to it by the loop-end __syncwarp) before its bulk copies
      fence_proxy_async_smem();
      __syncwarp();
      issue(static_cast<int>((t + S - 1) % S), __shfl_sync(kFull, pf_f, 0),
            __shfl_sync(kFull, pf_v, 0));
      if (t + S < n_units) load_next();
    }
    const bool ok = mbar_wait_bounded(&ws.bar[b], static_cast<uint32_t>((t / S) & 1));
    if (__any_sync(kFull, !ok)) {
      failed = true;
      break;
    }
    float2 *sb2 = reinterpret_cast<float2 *>(ws.buf[b]);
    float *sb1 = ws.buf[b];
    const int4 ix = ws.idx[b][g];
    const int f = ix.x, v = ix.y, e1 = ix.z, e2 = ix.w;
    // TENTATIVE read-out points of this lane, loaded now and used at the end: 18 per variable,
    // 4 per round (point p = 4 round + l): p < 6 alpha^p, p < 12 H_e1 alpha^(p-6), p < 18 H_e2
    // alpha^(p-12)
    int zr[5];
    if constexpr (!SYMBOL) {
#pragma unroll
      for (int round = 0; round < 5; ++round) {
        const int p = 4 * round + l;
        const int kind = p / 6, i = p - 6 * kind;
        zr[round] = p >= 18 ? 0
                    : kind == 0 ? (1 << i)
                                : __ldg(edge_z + (size_t)(kind == 1 ? e1 : e2) * 8 + i);
      }
    }
    // channel bit probabilities: lanes 0, 1 of a group compute bits l and l + 4, lanes 2, 3 bit l
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int bit = l + 4 * r;
      if (bit < 6) {
        const float Li = ws.llr[b][6 * g + bit];
        const float e = expf(-fabsf(Li));
        const float big = rcp_ftz(1.0f + e), small = e * big;
        ws.pbt[g][bit] = Li >= 0.0f ? make_float2(big, small) : make_float2(small, big);
      }
    }
    // both check messages in layout P0, decoded from the Gamma form
    float2 c[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 a = *reinterpret_cast<const float4 *>(ws.msg(b, g) + 4 * l + 16 * q);
      const float4 d = *reinterpret_cast<const float4 *>(ws.msg(b, g) + kQ6 + 4 * l + 16 * q);
      // packed pairs along the 16-byte loads (aligned register pairs)
      const float2 ax = gamma_decode2_ftz(a.x, a.y), az = gamma_decode2_ftz(a.z, a.w);
      const float2 dx = gamma_decode2_ftz(d.x, d.y), dz = gamma_decode2_ftz(d.z, d.w);
      c[4 * q + 0] = make_float2(ax.x, dx.x);
      c[4 * q + 1] = make_float2(ax.y, dx.y);
      c[4 * q + 2] = make_float2(az.x, dz.x);
      c[4 * q + 3] = make_float2(az.y, dz.y);
    }
    __syncwarp();  // every lane has read its messages before the transposes reuse their space
    // forward transforms of the pair, P0 -> P1
    stage<0>(c);
    stage<1>(c);
    stage<2>(c);
    stage<3>(c);
#pragma unroll
    for (int j = 0; j < 16; ++j) sb2[o0 + roff0(j)] = c[j];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 16; ++j) c[j] = sb2[o1 + roff1(j)];
    __syncwarp();
    stage<0>(c);
    stage<1>(c);
    // x-domain messages are probability vectors: drop the negative rounding noise
#pragma unroll
    for (int j = 0; j < 16; ++j) c[j] = make_float2(fmaxf(c[j].x, 0.0f), fmaxf(c[j].y, 0.0f));
    // channel term p0(x) in P1 (lane bits x0 x1, register bits x2..x5), then
    // M_v = p0 . c1x . c2x and w = (p0 . c1x, p0 . c2x) = (U of e2, U of e1) in place of c
    float mu[16];
    {
      const float2 q0 = ws.pbt[g][0], q1 = ws.pbt[g][1];
      const float lf = ((l & 1) ? q0.y : q0.x) * ((l & 2) ? q1.y : q1.x);
      const float2 q2 = ws.pbt[g][2], q3 = ws.pbt[g][3], q4 = ws.pbt[g][4], q5 = ws.pbt[g][5];
      const float a0 = lf * q2.x, a1 = lf * q2.y;
      const float bq[4] = {a0 * q3.x, a1 * q3.x, a0 * q3.y, a1 * q3.y};
      const float c45[4] = {q4.x * q5.x, q4.y * q5.x, q4.x * q5.y, q4.y * q5.y};
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float pj = bq[j & 3] * c45[j >> 2];
        mu[j] = pj * c[j].x * c[j].y;
        c[j] = __fmul2_rn(make_float2(pj, pj), c[j]);
      }
    }
    int best_x = 0;
    if constexpr (SYMBOL) {
      // symbol decision: argmax over x of the x-domain marginal (ties: lowest x); x = l + 4 j
      float best = -1.0f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int x = l + 4 * j;
        if (mu[j] > best || (mu[j] == best && x < best_x)) {
          best = mu[j];
          best_x = x;
        }
      }
#pragma unroll
      for (int o = 1; o < 4; o <<= 1) {
        const float ob = __shfl_xor_sync(kFull, best, o);
        const int oi = __shfl_xor_sync(kFull, best_x, o);
        if (ob > best || (ob == best && oi < best_x)) {
          best = ob;
          best_x = oi;
        }
      }
    }
    // inverse-direction transforms of the pair, P1 -> P0 (natural order)
    stage<0>(c);
    stage<1>(c);
    stage<2>(c);
    stage<3>(c);
#pragma unroll
    for (int j = 0; j < 16; ++j) sb2[o1 + roff1(j)] = c[j];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 16; ++j) c[j] = sb2[o0 + roff0(j)];
    __syncwarp();
    stage<0>(c);
    stage<1>(c);
    // normalise to U(0) = 1 (x = 0: register 0 of the group's lane 0); U(0) <= 0 only by
    // underflow: then the message is delta_0
    const float n2 = __shfl_sync(kFull, c[0].x, lane & 28), n1 = __shfl_sync(kFull, c[0].y, lane & 28);
    const float2 r = make_float2(n2 > 0.0f ? rcp_ftz(n2) : 0.0f, n1 > 0.0f ? rcp_ftz(n1) : 0.0f);
    {
      float *d2 = v2c + ((size_t)f * E + e2) * kQ6, *d1 = v2c + ((size_t)f * E + e1) * kQ6;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float o2[4], o1[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 sc = __ffma2_rn(c[4 * q + i], r, make_float2(0.0f, 0.0f));  // -0 -> +0
          const float2 o = gamma_encode2_ftz(sc);
          o2[i] = o.x;
          o1[i] = o.y;
        }
        if (q == 0 && l == 0) {
          o2[0] = 0.0f;  // Gamma(1)
          o1[0] = 0.0f;
        }
        *reinterpret_cast<float4 *>(d2 + 4 * l + 16 * q) = make_float4(o2[0], o2[1], o2[2], o2[3]);
        *reinterpret_cast<float4 *>(d1 + 4 * l + 16 * q) = make_float4(o1[0], o1[1], o1[2], o1[3]);
      }
    }
    if constexpr (SYMBOL) {
      // the Fourier-domain syndrome words describe bitwise decisions: with symbol decisions they
      // are written as 0, so that the stop test rests on the GF(2^m) syndrome alone
      if (l == 0) {
        if (sym) sym[(size_t)f * N + v] = static_cast<uint16_t>(best_x);
        if (fsyn) {
          fsyn[(size_t)f * E + e1] = 0;
          fsyn[(size_t)f * E + e2] = 0;
        }
      }
    } else {
      // inverse-direction transform of M as one float vector, P1 -> P0
      float2 mp[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) mp[i] = make_float2(mu[i], mu[i + 8]);
      stage_one<0>(mp);
      stage_one<1>(mp);
      stage_one<2>(mp);
      stage_one<3>(mp);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        sb1[o1 + roff1(i)] = mp[i].x;
        sb1[o1 + roff1(i + 8)] = mp[i].y;
      }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < 8; ++i) mp[i] = make_float2(sb1[o0 + roff0(i)], sb1[o0 + roff0(i + 8)]);
      __syncwarp();
      stage_one<0>(mp);
      stage_one<1>(mp);
      // natural order (x = (j & 3) + 4 l + 16 (j >> 2); j = i in .x, i + 8 in .y)
      float *m_nat = sb1 + g * kNat;
      *reinterpret_cast<float4 *>(m_nat + 4 * l) = make_float4(mp[0].x, mp[1].x, mp[2].x, mp[3].x);
      *reinterpret_cast<float4 *>(m_nat + 4 * l + 16) = make_float4(mp[4].x, mp[5].x, mp[6].x, mp[7].x);
      *reinterpret_cast<float4 *>(m_nat + 4 * l + 32) = make_float4(mp[0].y, mp[1].y, mp[2].y, mp[3].y);
      *reinterpret_cast<float4 *>(m_nat + 4 * l + 48) = make_float4(mp[4].y, mp[5].y, mp[6].y, mp[7].y);
      __syncwarp();
      // TENTATIVE: the signs of M at the read-out points zr, gathered with ballots
      uint32_t word = 0;
#pragma unroll
      for (int round = 0; round < 5; ++round) {
        const bool neg = 4 * round + l < 18 && m_nat[zr[round]] < 0.0f;
        const uint32_t bal = __ballot_sync(kFull, neg);
        word |= ((bal >> (4 * g)) & 0xfu) << (4 * round);
      }
      if (m_nat[0] < 0.0f) word = ~word;
      if (l == 0) {
        if (sym) sym[(size_t)f * N + v] = static_cast<uint16_t>(word & 0x3fu);
        if (fsyn) {
          fsyn[(size_t)f * E + e1] = static_cast<uint8_t>((word >> 6) & 0x3fu);
          fsyn[(size_t)f * E + e2] = static_cast<uint8_t>((word >> 12) & 0x3fu);
        }
      }
    }
    __syncwarp();
  }
  if (failed && lane == 0) {
    if (err) atomicExch(err, NBFD_ETIMEDOUT);
    // the prefetches of the next stages may still be landing in this warp's shared memory
    for (long long k = t + 1; k < t + S && k < n_units; ++k)
      mbar_wait_bounded(&ws.bar[k % S], static_cast<uint32_t>((k / S) & 1));
  }
}

namespace {
// Block shapes: (warps per block, resident blocks per SM). A warp holds 10.5 KB of shared memory
// (two pipeline stages of 8 variables' messages, which the transposes reuse): 4-warp blocks fit
// 5 per SM (20 warps, at most 102 registers), 7-warp blocks 2 (14), one 15-warp block 15.
constexpr int kX8Stages = 2;
constexpr int kX8DefaultWarps = 4;
template <int W>
constexpr int x8_min_blocks() { return W == 4 ? 5 : (W == 7 ? 2 : 1); }
template <int W>
constexpr size_t x8_smem() { return sizeof(X8Stage<kX8Stages>) * W; }
}  // namespace

bool var_fwht6x8_applies(const nbfd_code *c) { return c->m == 6 && c->N % 8 == 0; }

template <int W>
static cudaError_t launch_x8_shape(const nbfd_code *c, FrameSet fs, const float *llr,
                                   const float *c2v, float *v2c, uint16_t *sym, uint8_t *fsyn,
                                   int32_t *err, cudaStream_t s, bool symbol, int blocks_per_sm) {
  constexpr int Mb = x8_min_blocks<W>();
  const long long units = (long long)fs.n_static * c->N / 8;
  long long grid = (units + W - 1) / W;
  const int per_sm = blocks_per_sm > 0
                         ? blocks_per_sm
                         : Mb * oversubscribed_waves(units, (long long)sm_count() * Mb * W);
  const long long cap = (long long)sm_count() * per_sm;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  auto go = [&](auto kern) -> cudaError_t {
    const cudaError_t e = ensure_smem((const void *)kern, x8_smem<W>());
    if (e != cudaSuccess) return e;
    return launch_dependent(kern, dim3((int)grid), dim3(32 * W), x8_smem<W>(), s, llr, c2v, v2c,
                            sym, fsyn, c->d_var_edges, c->d_edge_z, c->N, c->E, fs, err);
  };
  return symbol ? go(k_var_fwht6x8<true, W, kX8Stages, Mb>)
                : go(k_var_fwht6x8<false, W, kX8Stages, Mb>);
}

cudaError_t launch_var_fwht6x8(const nbfd_code *c, FrameSet fs, const float *llr, const float *c2v,
                               float *v2c, uint16_t *sym, uint8_t *fsyn, int32_t *err,
                               cudaStream_t s, bool symbol, VarTune tune) {
  if (!var_fwht6x8_applies(c)) return cudaErrorInvalidValue;
  // default shape: 4-warp blocks, 5 per SM (measured with CUDA events at 2048 / 4096 GF(64) N=1200
  // frames: 0.484 / 0.952 ms, against 0.517 / 0.992 ms for one 15-warp block per SM); the
  // autotuner also times the 7- and 15-warp shapes
  const int dflt = kX8DefaultWarps;
  switch (tune.warps > 0 ? tune.warps : dflt) {
    case 7:
      return launch_x8_shape<7>(c, fs, llr, c2v, v2c, sym, fsyn, err, s, symbol, tune.blocks_per_sm);
    case 15:
      return launch_x8_shape<15>(c, fs, llr, c2v, v2c, sym, fsyn, err, s, symbol, tune.blocks_per_sm);
    case 4:
      return launch_x8_shape<4>(c, fs, llr, c2v, v2c, sym, fsyn, err, s, symbol, tune.blocks_per_sm);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace nbfd
