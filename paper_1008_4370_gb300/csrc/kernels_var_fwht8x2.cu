// VARIABLE TO CHECK + TENTATIVE DECISION, FWHT form (FP32), GF(256): two variables per warp.
//
// The algebra is that of kernels_var_fwht.cu (Section 3.2 boxplus = XOR convolution = pointwise
// product in the x-domain, reached with the Section 2.1 transform). Each half-warp owns one
// variable and each lane 16 entries of a 256-entry vector: 4 index bits in registers, 4 across
// the 16 lanes, so a transform is 4 butterfly stages in registers, one transpose through shared
// memory and 4 more stages -- one transpose per transform instead of the two that 8 entries per
// lane need, which halves the shared-memory traffic that bounds the 8-entry kernel.
//
// Index layouts (x = index of the 256-entry vector, bit i written x_i; j = register, l = lane
// within the half-warp):
//   P0: registers j0..j3 hold x0, x1, x6, x7; lanes l0..l3 hold x2..x5
//       (x = (j & 3) + 4 l + 64 (j >> 2): 16-byte chunks for shared and global memory)
//   P1: registers hold x2..x5; lanes hold x0, x1, x6, x7
// Forward transform (natural input): stages on the registers in P0, transpose, stages in P1.
// Inverse direction: P1 stages, transpose, P0 stages (ends in natural order). Stages on
// different bits commute, so both are the Walsh-Hadamard transform.
//
// Transpose buffer: entry x of a variable's float2 pairs sits at sum_i x_i w_i with
// w = (1, 2, 4, 8, 17, 34, 68, 136). The 16 lanes of a half-warp then hit 16 different 8-byte bank
// pairs for every register in both layouts, and the position splits into a per-lane offset plus
// a compile-time offset per register.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cooperative_groups.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include "bulk_copy.cuh"
#include "check_math.cuh"
#include "device_common.cuh"
#include "nbfd_internal.h"

namespace nbfd {

namespace {

constexpr int kQ = 256;
constexpr int kBuf = 272;  // float2 entries of one variable's transpose buffer (271 used)

__host__ __device__ constexpr int pw(int b) {
  return b == 0 ? 1 : b == 1 ? 2 : b == 2 ? 4 : b == 3 ? 8 : b == 4 ? 17 : b == 5 ? 34 : b == 6 ? 68 : 136;
}
// compile-time register offsets (x bits of register j in P0 / P1)
__host__ __device__ constexpr int roff0(int j) {
  return ((j & 1) ? pw(0) : 0) + ((j & 2) ? pw(1) : 0) + ((j & 4) ? pw(6) : 0) + ((j & 8) ? pw(7) : 0);
}
__host__ __device__ constexpr int roff1(int j) {
  return ((j & 1) ? pw(2) : 0) + ((j & 2) ? pw(3) : 0) + ((j & 4) ? pw(4) : 0) + ((j & 8) ? pw(5) : 0);
}
static_assert(roff0(15) + roff1(15) < kBuf, "buffer");

// buf[stage][variable] first holds the variable's two check messages (bulk-copy targets, edge 1
// then edge 2), then -- once they are decoded into registers -- its transpose buffer and at the
// end M in natural order. Sharing the space keeps a warp at 9 KB, so 5 blocks of 4 warps fit an SM.
template <typename W, int S>
struct X2Stage {
  float2 buf[S][2][kBuf];       // [stage][variable]
  float llr[S][2][8];           // [stage][variable][bit]
  int4 idx[S][2];               // [stage][variable] = (frame, variable, slot e1, slot e2)
  float2 pbt[2][8];             // [variable][bit] = (Pr(b = 0), Pr(b = 1))
  uint64_t bar[S];
  __device__ W *msg(int st, int h, int j) {
    return reinterpret_cast<W *>(&buf[st][h][0]) + j * kQ;
  }
};
static_assert(sizeof(float2) * kBuf >= 2 * kQ * sizeof(float), "messages fit the buffer");

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
__device__ __forceinline__ void stages4(float2 (&v)[16]) {
  stage<0>(v);
  stage<1>(v);
  stage<2>(v);
  stage<3>(v);
}
// P0 -> P1 (TO1) or P1 -> P0 within the half-warp's buffer s
template <bool TO1>
__device__ __forceinline__ void transpose(float2 (&v)[16], float2 *s, int o0, int o1) {
#pragma unroll
  for (int j = 0; j < 16; ++j) s[(TO1 ? o0 + roff0(j) : o1 + roff1(j))] = v[j];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = s[(TO1 ? o1 + roff1(j) : o0 + roff0(j))];
  __syncwarp();
}

// One vector (M) as 8 pairs u[i] = (entry i, entry i + 8): register bits 0..2 pair up across
// the float2 values, register bit 3 lies inside each float2.
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
__device__ __forceinline__ void stages4_one(float2 (&u)[8]) {
  stage_one<0>(u);
  stage_one<1>(u);
  stage_one<2>(u);
  stage_one<3>(u);
}
// P1 -> P0 for one vector per half-warp in 32-bit words: entry x of half-warp h at float
// 2 (sum x_i w_i) + h of the warp's whole scratch, so the two half-warps take the even and the
// odd banks and all 32 lanes hit different banks.
__device__ __forceinline__ void transpose_one_to0(float2 (&u)[8], float *s, int o0, int o1,
                                                  int h) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    s[2 * (o1 + roff1(i)) + h] = u[i].x;
    s[2 * (o1 + roff1(i + 8)) + h] = u[i].y;
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 8; ++i)
    u[i] = make_float2(s[2 * (o0 + roff0(i)) + h], s[2 * (o0 + roff0(i + 8)) + h]);
  __syncwarp();
}

__device__ __forceinline__ float4 load4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float4 load4(const __half *p) {
  const uint2 w = *reinterpret_cast<const uint2 *>(p);
  const float2 a = unpack_half2(w.x), b = unpack_half2(w.y);
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void store4(float *p, float a, float b, float c, float d) {
  *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store4(__half *p, float a, float b, float c, float d) {
  *reinterpret_cast<uint2 *>(p) = make_uint2(pack_half2(a, b), pack_half2(c, d));
}

}  // namespace

// One unit of the variable-node update: variable v (this half-warp, sub = lane / 16) of frame f,
// edges e1 and e2, from its two check messages msg0 / msg1 (Gamma form, natural order, in shared
// memory) and its 8 LLRs: writes V->C on both edges, the tentative decision and the Fourier-domain
// syndrome words when `valid`. Warp-collective (both half-warps call it together). Shared by the
// variable-node kernel and the cluster tail kernel, so both compute bit-identical results.
template <bool SYMBOL, typename W>
__device__ __forceinline__ void x2_unit(const W *msg0, const W *msg1, const float *llr8,
                                        float2 *pbt, float2 *sbuf, float *scratch_all, int f,
                                        int v, int e1, int e2, bool valid, W *__restrict__ v2c,
                                        uint16_t *__restrict__ sym, uint8_t *__restrict__ fsyn,
                                        const uint8_t *__restrict__ edge_z, int N, int E, int lane,
                                        int sub, int l, int o0, int o1, int xl1,
                                        unsigned half_mask) {
  // read-out points of this lane, used at the end: round 0 lanes 0..7 alpha^i, 8..15 H_e1
  // alpha^i; round 1 lanes 0..7 H_e2 alpha^i
  int z0 = 0, z1 = 0;
  if (!SYMBOL) {
    z0 = l < 8 ? (1 << l) : __ldg(edge_z + (size_t)e1 * 8 + (l & 7));
    z1 = l < 8 ? __ldg(edge_z + (size_t)e2 * 8 + l) : 0;
  }
  if (l < 8) {
    const float Li = llr8[l];
    const float e = expf(-fabsf(Li));
    const float big = rcp_ftz(1.0f + e), small = e * big;
    pbt[l] = Li >= 0.0f ? make_float2(big, small) : make_float2(small, big);
  }
  // both check messages in layout P0, decoded from the Gamma form
  float2 c[16];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const float4 a = load4(&msg0[4 * l + 64 * g]);
    const float4 d = load4(&msg1[4 * l + 64 * g]);
    // packed pairs along the 16-byte loads (aligned register pairs)
    const float2 ax = gamma_decode2_ftz(a.x, a.y), az = gamma_decode2_ftz(a.z, a.w);
    const float2 dx = gamma_decode2_ftz(d.x, d.y), dz = gamma_decode2_ftz(d.z, d.w);
    c[4 * g + 0] = make_float2(ax.x, dx.x);
    c[4 * g + 1] = make_float2(ax.y, dx.y);
    c[4 * g + 2] = make_float2(az.x, dz.x);
    c[4 * g + 3] = make_float2(az.y, dz.y);
  }
  // the transpose buffer may be the messages' own (the variable-node kernel): every lane has read
  // its entries before any lane writes
  __syncwarp();
  // forward transforms of the pair (q x-domain check messages), P0 -> P1
  stages4(c);
  transpose<true>(c, sbuf, o0, o1);
  stages4(c);
  // x-domain messages are probability vectors: drop the negative rounding noise
#pragma unroll
  for (int j = 0; j < 16; ++j) c[j] = make_float2(fmaxf(c[j].x, 0.0f), fmaxf(c[j].y, 0.0f));
  // channel term p0(x) in P1 (lane bits x0 x1 x6 x7, register bits x2..x5), then
  // M_v = p0 . c1x . c2x and w = (p0 . c1x, p0 . c2x) = (U of e2, U of e1) in place of c
  float mu[16];
  {
    const float2 q0 = pbt[0], q1 = pbt[1], q6 = pbt[6],
                 q7 = pbt[7];
    const float lf = ((l & 1) ? q0.y : q0.x) * ((l & 2) ? q1.y : q1.x) *
                     ((l & 4) ? q6.y : q6.x) * ((l & 8) ? q7.y : q7.x);
    const float2 q2 = pbt[2], q3 = pbt[3], q4 = pbt[4],
                 q5 = pbt[5];
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
    // symbol decision: argmax over x of the x-domain marginal (ties: lowest x)
    float best = -1.0f;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int x = xl1 | (j << 2);
      if (mu[j] > best || (mu[j] == best && x < best_x)) {
        best = mu[j];
        best_x = x;
      }
    }
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      const float ob = __shfl_xor_sync(kFull, best, o);
      const int oi = __shfl_xor_sync(kFull, best_x, o);
      if (ob > best || (ob == best && oi < best_x)) {
        best = ob;
        best_x = oi;
      }
    }
  }
  // inverse-direction transforms of the pair, P1 -> P0 (natural order)
  stages4(c);
  transpose<false>(c, sbuf, o0, o1);
  stages4(c);
  // normalise to U(0) = 1 (x = 0: register 0 of the half-warp's lane 0); U(0) <= 0 only by
  // underflow: then the message is delta_0
  const float n2 = __shfl_sync(kFull, c[0].x, lane & 16), n1 = __shfl_sync(kFull, c[0].y, lane & 16);
  const float2 r = make_float2(n2 > 0.0f ? rcp_ftz(n2) : 0.0f, n1 > 0.0f ? rcp_ftz(n1) : 0.0f);
  if (valid) {
    W *d2 = v2c + ((size_t)f * E + e2) * kQ, *d1 = v2c + ((size_t)f * E + e1) * kQ;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      float o2[4], o1[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 sc = __ffma2_rn(c[4 * g + i], r, make_float2(0.0f, 0.0f));  // -0 -> +0
        const float2 o = gamma_encode2_ftz(sc);
        o2[i] = o.x;
        o1[i] = o.y;
      }
      if (g == 0 && l == 0) {
        o2[0] = 0.0f;  // Gamma(1)
        o1[0] = 0.0f;
      }
      store4(d2 + 4 * l + 64 * g, o2[0], o2[1], o2[2], o2[3]);
      store4(d1 + 4 * l + 64 * g, o1[0], o1[1], o1[2], o1[3]);
    }
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
  } else {
    // inverse-direction transform of M, P1 -> P0, then stored in natural order for the read-out
    float2 mp[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) mp[i] = make_float2(mu[i], mu[i + 8]);
    stages4_one(mp);
    transpose_one_to0(mp, scratch_all, o0, o1, sub);
    stages4_one(mp);
    float *m_nat = reinterpret_cast<float *>(sbuf);
    *reinterpret_cast<float4 *>(m_nat + 4 * l) = make_float4(mp[0].x, mp[1].x, mp[2].x, mp[3].x);
    *reinterpret_cast<float4 *>(m_nat + 4 * l + 64) = make_float4(mp[4].x, mp[5].x, mp[6].x, mp[7].x);
    *reinterpret_cast<float4 *>(m_nat + 4 * l + 128) = make_float4(mp[0].y, mp[1].y, mp[2].y, mp[3].y);
    *reinterpret_cast<float4 *>(m_nat + 4 * l + 192) = make_float4(mp[4].y, mp[5].y, mp[6].y, mp[7].y);
    __syncwarp();
    // TENTATIVE: signs of M at alpha^{i-1}, H_e1 alpha^{i-1} (round 0) and H_e2 alpha^{i-1}
    // (round 1), gathered with ballots; bit 16 sub + l belongs to this half-warp
    const bool neg0 = m_nat[z0] < 0.0f;
    const bool neg1 = l < 8 && m_nat[z1] < 0.0f;
    const uint32_t bal0 = __ballot_sync(kFull, neg0), bal1 = __ballot_sync(kFull, neg1);
    const bool flip = m_nat[0] < 0.0f;
    if (valid && l == 0) {
      uint32_t w0 = (bal0 & half_mask) >> (16 * sub), w1 = (bal1 & half_mask) >> (16 * sub);
      if (flip) {
        w0 = ~w0 & 0xffffu;
        w1 = ~w1 & 0xffu;
      }
      if (sym) sym[(size_t)f * N + v] = static_cast<uint16_t>(w0 & 0xffu);
      if (fsyn) {
        fsyn[(size_t)f * E + e1] = static_cast<uint8_t>((w0 >> 8) & 0xffu);
        fsyn[(size_t)f * E + e2] = static_cast<uint8_t>(w1 & 0xffu);
      }
    }
  }
}

template <bool SYMBOL, typename W, int WARPS, int S, int MINB>
__global__ void __launch_bounds__(32 * WARPS, MINB)
    k_var_fwht8x2(const float *__restrict__ llr, const W *__restrict__ c2v, W *__restrict__ v2c,
                  uint16_t *__restrict__ sym, uint8_t *__restrict__ fsyn,
                  const int32_t *__restrict__ var_edges, const uint8_t *__restrict__ edge_z, int N,
                  int E, FrameSet fs, int32_t *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane >> 4, l = lane & 15;
  X2Stage<W, S> &ws = reinterpret_cast<X2Stage<W, S> *>(smem_raw)[wib];
  griddep_wait();
  griddep_release();
  const int F = fs.list ? __ldg(fs.count) : fs.n_static;
  const long long total = (long long)F * N;           // variables
  const long long units = (total + 1) >> 1;            // pairs of consecutive variables
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  if (gw >= units) return;
  const long long n_units = (units - gw + nw - 1) / nw;
  // lane 0 walks the first variable of this warp's units (2 gw, 2 gw + 2 nw, ...) as
  // (slot, variable) without a division per unit, one unit ahead of its bulk copies
  long long cur_slot = (2 * gw) / N;
  int cur_v = static_cast<int>(2 * gw - cur_slot * N);
  const long long step_s = (2 * nw) / N;
  const int step_v = static_cast<int>(2 * nw - step_s * N);
  long long cur_item = 2 * gw;
  int4 pf[2];
  int pf_n = 0;
  auto load_next = [&]() {
    long long sl = cur_slot;
    int v = cur_v;
    pf_n = cur_item + 1 < total ? 2 : 1;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h < pf_n) {
        const int f = fs.list ? __ldg(fs.list + sl) : static_cast<int>(sl);
        const int2 e = __ldg(reinterpret_cast<const int2 *>(var_edges) + v);
        pf[h] = make_int4(f, v, e.x, e.y);
      } else {
        pf[h] = pf[0];  // a stand-in: the second half-warp computes it and stores nothing
      }
      if (++v == N) {
        v = 0;
        ++sl;
      }
    }
    cur_item += 2 * nw;
    cur_slot += step_s;
    cur_v += step_v;
    if (cur_v >= N) {
      cur_v -= N;
      ++cur_slot;
    }
  };
  auto issue = [&](int st) {
    constexpr uint32_t vb = kQ * sizeof(W);
    mbar_expect_tx(&ws.bar[st], static_cast<uint32_t>(pf_n) * (2u * vb + 32u));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      ws.idx[st][h] = pf[h];
      if (h < pf_n) {
        const int4 ix = pf[h];
        bulk_load(ws.msg(st, h, 0), c2v + ((size_t)ix.x * E + ix.z) * kQ, vb, &ws.bar[st]);
        bulk_load(ws.msg(st, h, 1), c2v + ((size_t)ix.x * E + ix.w) * kQ, vb, &ws.bar[st]);
        bulk_load(ws.llr[st][h], llr + ((size_t)ix.x * N + ix.y) * 8, 32u, &ws.bar[st]);
      }
    }
  };
  if (lane == 0) {
#pragma unroll
    for (int st = 0; st < S; ++st) mbar_init(&ws.bar[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int k = 0; k < S - 1 && k < n_units; ++k) {
      load_next();
      issue(k);
    }
    if (S - 1 < n_units) load_next();
  }
  __syncwarp();
  // per-lane transpose offsets: P0 lanes hold x2..x5, P1 lanes x0, x1, x6, x7
  const int o0 = ((l & 1) ? pw(2) : 0) + ((l & 2) ? pw(3) : 0) + ((l & 4) ? pw(4) : 0) +
                 ((l & 8) ? pw(5) : 0);
  const int o1 = ((l & 1) ? pw(0) : 0) + ((l & 2) ? pw(1) : 0) + ((l & 4) ? pw(6) : 0) +
                 ((l & 8) ? pw(7) : 0);
  // lane part of x in P1 (lanes hold x0, x1, x6, x7)
  const int xl1 = (l & 3) | ((l >> 2) & 3) << 6;
  const unsigned half_mask = sub ? 0xffff0000u : 0x0000ffffu;
  long long t = 0;
  bool failed = false;
  for (; t < n_units; ++t) {
    const int b = static_cast<int>(t % S);
    if (lane == 0 && t + S - 1 < n_units) {
      fence_proxy_async_smem();
      issue(static_cast<int>((t + S - 1) % S));
      if (t + S < n_units) load_next();
    }
    const bool ok = mbar_wait_bounded(&ws.bar[b], static_cast<uint32_t>((t / S) & 1));
    if (__any_sync(kFull, !ok)) {
      failed = true;
      break;
    }
    const long long item = 2 * (gw + t * nw) + sub;
    const bool valid = item < total;
    const int4 ix = ws.idx[b][sub];
    const int f = ix.x, v = ix.y, e1 = ix.z, e2 = ix.w;
    x2_unit<SYMBOL, W>(ws.msg(b, sub, 0), ws.msg(b, sub, 1), ws.llr[b][sub], ws.pbt[sub],
                       ws.buf[b][sub], reinterpret_cast<float *>(ws.buf[b]), f, v, e1, e2, valid,
                       v2c, sym, fsyn,
                       edge_z, N, E, lane, sub, l, o0, o1, xl1, half_mask);
    // every lane wrote this stage (transposes, M): its writes are ordered before the bulk copies
    // that refill the stage (issued by lane 0 after this barrier)
    fence_proxy_async_smem();
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
// launch shape: warps per block, pipeline depth, blocks per SM
constexpr int kX2Warps = 4, kX2Stages = 2, kX2MinBlocks = 5;
template <typename W>
constexpr size_t x2_smem() {
  return sizeof(X2Stage<W, kX2Stages>) * kX2Warps;
}
}  // namespace

cudaError_t launch_var_fwht8x2(const nbfd_code *c, FrameSet fs, const float *llr, const float *c2v,
                               float *v2c, uint16_t *sym, uint8_t *fsyn, int32_t *err,
                               cudaStream_t s, bool symbol, VarTune tune, bool f16) {
  if (c->m != 8) return cudaErrorInvalidValue;
  const long long units = ((long long)fs.n_static * c->N + 1) / 2;
  long long g = (units + kX2Warps - 1) / kX2Warps;
  const int per_sm =
      tune.blocks_per_sm > 0
          ? tune.blocks_per_sm
          : kX2MinBlocks * oversubscribed_waves(units, (long long)sm_count() * kX2MinBlocks * kX2Warps);
  const long long cap = (long long)sm_count() * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  auto go = [&](auto kern, auto tag) -> cudaError_t {
    using W = decltype(tag);
    const cudaError_t e = ensure_smem((const void *)kern, x2_smem<W>());
    if (e != cudaSuccess) return e;
    return launch_dependent(kern, dim3((int)g), dim3(32 * kX2Warps), x2_smem<W>(), s, llr,
                            reinterpret_cast<const W *>(c2v), reinterpret_cast<W *>(v2c), sym,
                            fsyn, c->d_var_edges, c->d_edge_z, c->N, c->E, fs, err);
  };
  constexpr int Wp = kX2Warps, St = kX2Stages, Mb = kX2MinBlocks;
  if (f16)
    return symbol ? go(k_var_fwht8x2<true, __half, Wp, St, Mb>, __half())
                  : go(k_var_fwht8x2<false, __half, Wp, St, Mb>, __half());
  return symbol ? go(k_var_fwht8x2<true, float, Wp, St, Mb>, 0.0f)
                : go(k_var_fwht8x2<false, float, Wp, St, Mb>, 0.0f);
}

// ---- the tail: one thread-block cluster per remaining frame ----------------------------------
// Once few frames are left (those that do not converge run to max_iter), each iteration costs
// three launches whose fixed latency far exceeds their work. k_tail_x2 runs all remaining
// iterations of each remaining frame inside one thread-block cluster: per iteration the variable
// node, a cluster barrier, the stop test's partial syndromes (each CTA's share of the checks,
// sent to every CTA's shared memory) together with the next iteration's check node, and a
// second cluster barrier, after which every CTA takes the same stop decision. Each unit of work
// calls the arithmetic of the iteration kernels (check_lane_inplace, x2_unit), so results are
// bit-identical. Messages written by other CTAs are read with L2-only loads. GF(256), float
// message storage, k <= 8.

namespace {
constexpr int kTailWarps = 16;
constexpr int kTailMaxCtas = 16;

template <int KMAX>
struct TailWarpMem {
  union {
    float tile[KMAX * kQ];  // check node: the k slots of one check
    struct {
      float msg[2][2][kQ];  // variable node: [variable][edge 1, edge 2][z]
      float llr[2][8];
      float2 scratch[2][kBuf];
      float2 pbt[2][8];
    } v;
  };
};
template <int KMAX>
constexpr size_t tail_smem() {
  return sizeof(TailWarpMem<KMAX>) * kTailWarps;
}
}  // namespace

template <bool SYMBOL, int KMAX>
__global__ void __launch_bounds__(32 * kTailWarps, 1)
    k_tail_x2(const float *__restrict__ llr, float *v2c, float *c2v, uint16_t *sym, uint8_t *fsyn,
              const int32_t *__restrict__ var_edges, const int32_t *__restrict__ edge_var,
              const uint8_t *__restrict__ edge_h, const uint8_t *__restrict__ edge_z,
              const uint8_t *__restrict__ perm, const uint8_t *__restrict__ gexp,
              const uint8_t *__restrict__ glog, int N, int M, int k, int E, FrameSet fs, int it0,
              int max_iter, uint8_t *__restrict__ ok, int32_t *__restrict__ iters,
              int32_t *__restrict__ stats) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t flags[kTailMaxCtas];  // per CTA of the cluster: bit 0 Fourier, bit 1 GF
  const int rank = static_cast<int>(cluster.block_rank());
  const int ncta = static_cast<int>(cluster.num_blocks());
  const int slot = static_cast<int>(blockIdx.x) / ncta;
  // the frame count is the same word for every CTA of the cluster: the whole cluster leaves
  if (slot >= (fs.list ? __ldg(fs.count) : fs.n_static)) return;
  const int f = fs.list ? __ldg(fs.list + slot) : slot;
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane >> 4, l = lane & 15;
  TailWarpMem<KMAX> &wm = reinterpret_cast<TailWarpMem<KMAX> *>(smem_raw)[wib];
  const int gwarp = rank * kTailWarps + wib, nwarp = ncta * kTailWarps;
  const int cper = (M + ncta - 1) / ncta;  // checks of this CTA's share of the stop test
  const int cbeg = rank * cper, cend = M < cbeg + cper ? M : cbeg + cper;
  const int units = (N + 1) >> 1;
  const size_t fE = (size_t)f * E;
  const int o0 = ((l & 1) ? pw(2) : 0) + ((l & 2) ? pw(3) : 0) + ((l & 4) ? pw(4) : 0) +
                 ((l & 8) ? pw(5) : 0);
  const int o1 = ((l & 1) ? pw(0) : 0) + ((l & 2) ? pw(1) : 0) + ((l & 4) ? pw(6) : 0) +
                 ((l & 8) ? pw(7) : 0);
  const int xl1 = (l & 3) | ((l >> 2) & 3) << 6;
  const unsigned half_mask = sub ? 0xffff0000u : 0x0000ffffu;
  // Tables that do not change across iterations, loaded once for the warp's first check, unit
  // and stop-test check (each warp has one of each when N <= 2 * 16 * 16): the index words of
  // its check, the edges of its unit's variable, the labels and variables of its stop-test edges.
  CheckIndex<kQ, 8, KMAX> ix0;
  if (gwarp < M) check_index_load<kQ, 8, KMAX>(ix0, gwarp, k, 8 * lane, edge_h, perm);
  int2 e0 = make_int2(0, 0);
  if (gwarp < units) {
    const int v = 2 * gwarp + sub < N ? 2 * gwarp + sub : 2 * gwarp;
    e0 = __ldg(reinterpret_cast<const int2 *>(var_edges) + v);
  }
  int sv0 = 0, sh0 = 0;  // stop test, first check: variable and label of edge `lane`
  if (cbeg + wib < cend && lane < k) {
    sv0 = __ldg(edge_var + (cbeg + wib) * k + lane);
    sh0 = __ldg(edge_h + (cbeg + wib) * k + lane);
  }
  // CHECK TO VARIABLE: one check per warp tile, lane entries z = 8 lane .. 8 lane + 7
  auto check_phase = [&]() {
    for (int c = gwarp; c < M; c += nwarp) {
      const float4 *src = reinterpret_cast<const float4 *>(v2c + (fE + (size_t)c * k) * kQ);
      float4 *t4 = reinterpret_cast<float4 *>(wm.tile);
      for (int i = lane; i < k * (kQ / 4); i += 32) t4[i] = __ldcg(src + i);
      __syncwarp();
      CheckIndex<kQ, 8, KMAX> ix = ix0;
      if (c != gwarp) check_index_load<kQ, 8, KMAX>(ix, c, k, 8 * lane, edge_h, perm);
      check_lane_apply<kQ, 8, KMAX, float, 1>(wm.tile, k, ix);
      __syncwarp();
      float4 *dst = reinterpret_cast<float4 *>(c2v + (fE + (size_t)c * k) * kQ);
      for (int i = lane; i < k * (kQ / 4); i += 32) dst[i] = t4[i];
      __syncwarp();
    }
  };
  check_phase();
  cluster.sync();
  for (int it = it0;; ++it) {
    // VARIABLE TO CHECK + TENTATIVE DECISION: two variables per warp unit
    for (int u = gwarp; u < units; u += nwarp) {
      const bool valid = 2 * u + sub < N;
      const int v = valid ? 2 * u + sub : 2 * u;  // a stand-in computes and stores nothing
      const int2 e = u == gwarp ? e0 : __ldg(reinterpret_cast<const int2 *>(var_edges) + v);
      const float4 *m1 = reinterpret_cast<const float4 *>(c2v + (fE + e.x) * kQ);
      const float4 *m2 = reinterpret_cast<const float4 *>(c2v + (fE + e.y) * kQ);
      float4 *d1 = reinterpret_cast<float4 *>(wm.v.msg[sub][0]);
      float4 *d2 = reinterpret_cast<float4 *>(wm.v.msg[sub][1]);
      for (int i = l; i < kQ / 4; i += 16) {
        d1[i] = __ldcg(m1 + i);
        d2[i] = __ldcg(m2 + i);
      }
      if (l < 8) wm.v.llr[sub][l] = __ldg(llr + ((size_t)f * N + v) * 8 + l);
      __syncwarp();
      x2_unit<SYMBOL, float>(wm.v.msg[sub][0], wm.v.msg[sub][1], wm.v.llr[sub], wm.v.pbt[sub],
                             wm.v.scratch[sub], reinterpret_cast<float *>(wm.v.scratch), f, v,
                             e.x, e.y, valid, v2c, sym, fsyn, edge_z, N, E, lane, sub, l, o0, o1,
                             xl1, half_mask);
      __syncwarp();
    }
    cluster.sync();
    // stop test over this CTA's share of the checks, one check per warp, lane j on edge j:
    // Fourier-domain and GF(2^m) syndromes. The first check's loads are issued before the next
    // iteration's check node and used after it, so that their latency overlaps its work (the
    // check node does not depend on the stop decision: messages of a frame that stops are never
    // read again).
    int ffail = 0, efail = 0;
    uint32_t fb = 0;
    int xv = 0, hv = 0;
    auto stop_load = [&](int cs) {
      fb = 0;
      xv = 0;
      hv = 0;
      if (cs < cend && lane < k) {
        const int ed = cs * k + lane;
        const bool first = cs == cbeg + wib;
        fb = __ldcg(fsyn + fE + ed);
        xv = __ldcg(sym + (size_t)f * N + (first ? sv0 : __ldg(edge_var + ed)));
        hv = first ? sh0 : __ldg(edge_h + ed);
      }
    };
    stop_load(cbeg + wib);
    if (it < max_iter) check_phase();
    for (int cs = cbeg + wib; cs < cend; cs += kTailWarps) {
      if (cs != cbeg + wib) stop_load(cs);
      uint32_t fx = fb;
      int gx = xv == 0 ? 0 : __ldg(gexp + __ldg(glog + hv) + __ldg(glog + xv));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        fx ^= __shfl_xor_sync(0xffffffffu, fx, o);
        gx ^= __shfl_xor_sync(0xffffffffu, gx, o);
      }
      ffail |= fx != 0;
      efail |= gx != 0;
    }
    ffail = __syncthreads_or(ffail);
    efail = __syncthreads_or(efail);
    if (threadIdx.x < (unsigned)ncta)
      *cluster.map_shared_rank(&flags[rank], static_cast<int>(threadIdx.x)) =
          (ffail ? 1u : 0u) | (efail ? 2u : 0u);
    cluster.sync();
    uint32_t all = 0;
    for (int r = 0; r < ncta; ++r) all |= flags[r];
    const bool ff = all & 1u, ef = (all & 2u) != 0;
    const bool stop = (!ff && !ef) || it >= max_iter;
    if (rank == 0 && threadIdx.x == 0) {
      if (!ff && ef) atomicAdd(stats, 1);  // the Fourier-domain syndrome cleared, H x_hat != 0
      if (stop) {
        ok[f] = ef ? 0 : 1;
        iters[f] = it;
      }
    }
    if (stop) break;
  }
}

// Clusters of the tail kernel that can be resident at once (0: the kernel cannot run), and the
// cluster size it uses; computed once per device and shape.
int tail_clusters(const nbfd_code *c, bool symbol, int *ctas) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, bool>, std::pair<int, int>> cache;
  if (c->m != 8 || c->k > 8) return 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const int kmax = c->k <= 4 ? 4 : 8;
  const auto key = std::make_tuple(dev, kmax, symbol);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *ctas = it->second.second;
      return it->second.first;
    }
  }
  auto probe = [&](auto kern, size_t smem) -> std::pair<int, int> {
    if (ensure_smem((const void *)kern, smem) != cudaSuccess) return {0, 0};
    cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int n : {kTailMaxCtas, 8}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(n);
      cfg.blockDim = dim3(32 * kTailWarps);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = n;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, (const void *)kern, &cfg) == cudaSuccess &&
          clusters > 0)
        return {clusters, n};
      cudaGetLastError();  // clear a refusal of this size, try the next
    }
    return {0, 0};
  };
  std::pair<int, int> r;
  if (kmax == 4)
    r = symbol ? probe(k_tail_x2<true, 4>, tail_smem<4>()) : probe(k_tail_x2<false, 4>, tail_smem<4>());
  else
    r = symbol ? probe(k_tail_x2<true, 8>, tail_smem<8>()) : probe(k_tail_x2<false, 8>, tail_smem<8>());
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = r;
  *ctas = r.second;
  return r.first;
}

cudaError_t launch_tail_x2(const nbfd_code *c, FrameSet fs, const float *llr, float *v2c,
                           float *c2v, uint16_t *sym, uint8_t *fsyn, int it0, int max_iter,
                           uint8_t *ok, int32_t *iters, int32_t *stats, cudaStream_t s,
                           bool symbol) {
  int ctas = 0;
  if (tail_clusters(c, symbol, &ctas) <= 0 || fs.n_static < 1) return cudaErrorNotSupported;
  const int kmax = c->k <= 4 ? 4 : 8;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(fs.n_static * ctas);
  cfg.blockDim = dim3(32 * kTailWarps);
  cfg.dynamicSmemBytes = kmax == 4 ? tail_smem<4>() : tail_smem<8>();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  auto go = [&](auto kern) {
    return cudaLaunchKernelEx(&cfg, kern, llr, v2c, c2v, sym, fsyn, c->d_var_edges, c->d_edge_var,
                              c->d_edge_h, c->d_edge_z, c->d_perm, c->d_gf_exp, c->d_gf_log, c->N,
                              c->M, c->k, c->E, fs, it0, max_iter, ok, iters, stats);
  };
  if (kmax == 4) return symbol ? go(k_tail_x2<true, 4>) : go(k_tail_x2<false, 4>);
  return symbol ? go(k_tail_x2<true, 8>) : go(k_tail_x2<false, 8>);
}

}  // namespace nbfd
