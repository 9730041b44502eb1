// VARIABLE TO CHECK + TENTATIVE DECISION, FWHT form (FP32), GF(256): one warp per variable.
//
// The algebra is that of kernels_var_fwht.cu (Section 3.2 boxplus = XOR convolution = pointwise
// product in the x-domain, reached with the Section 2.1 transform). What differs is how the
// 256-point transforms move data between lanes. Each lane holds 8 entries of a vector; the
// butterflies of the 3 index bits held in registers run in registers, and the index bits held
// across lanes are brought into registers by transposes through shared memory (two per
// transform) instead of warp shuffles (five stages per transform). The two check messages of a
// variable travel together as float2 pairs, so every butterfly of the pair is one packed
// f32x2 add and one packed f32x2 fma (a - b as fma(b, -1, a), exact).
//
// Index layouts (x = index of the 256-entry vector, bit i of x written x_i):
//   P0: registers j0, j1, j2 hold x0, x1, x7; lanes L0..L4 hold x2..x6
//       (x = (j & 3) + 4 L + 128 (j >> 2): natural 16-byte chunks for shared and global memory)
//   P1: registers hold x2, x6, x5; lanes hold x0, x3, x4, x7, x1
//   P2: registers hold x2, x3, x4; lanes hold x0, x6, x5, x7, x1
// Forward transform (natural input): butterflies on x0 x1 x7 (P0), transpose, x2 x6 x5 (P1),
// transpose, x3 x4 (P2). The inverse direction starts in P2 (x2 x3 x4), returns to P1 (x6 x5)
// and ends in P0 (x0 x1 x7). Butterfly stages on different bits commute, so both are the
// Walsh-Hadamard transform.
//
// A transpose stores every entry at a padded position sum_i x_i * w_i and reads it back in the
// other layout. The weights w (one set per transpose and element width) were chosen so that
// every store and load of both layouts is free of shared-memory bank conflicts (float2: the
// 16 lanes of each half-warp hit 16 different 8-byte bank pairs; float: 32 different banks),
// and because the position is linear in the bits, it splits into a per-lane offset plus a
// compile-time offset per register.
#include <cuda_runtime.h>

#include <cstdint>

#include "bulk_copy.cuh"
#include "device_common.cuh"
#include "nbfd_internal.h"

namespace nbfd {

namespace {

constexpr int kQ = 256;

// x bit held by register bit i / lane bit i in layout `ph` (0 = P0, 1 = P1, 2 = P2)
__host__ __device__ constexpr int reg_bit(int ph, int i) {
  return ph == 0 ? (i == 0 ? 0 : i == 1 ? 1 : 7)
                 : ph == 1 ? (i == 0 ? 2 : i == 1 ? 6 : 5) : (i == 0 ? 2 : i == 1 ? 3 : 4);
}
__host__ __device__ constexpr int lane_bit(int ph, int i) {
  return ph == 0   ? 2 + i
         : ph == 1 ? (i == 0 ? 0 : i == 1 ? 3 : i == 2 ? 4 : i == 3 ? 7 : 1)
                   : (i == 0 ? 0 : i == 1 ? 6 : i == 2 ? 5 : i == 3 ? 7 : 1);
}

// padded position weight of x bit b in transpose buffer `pad`:
//   0 = first transpose, float2 pairs    1 = first transpose, single floats
//   2 = second transpose, float2 pairs   3 = second transpose, single floats
enum { kT1Pair = 0, kT1One = 1, kT2Pair = 2, kT2One = 3 };
__host__ __device__ constexpr int pad_w(int pad, int b) {
  return b < 4 ? (1 << b)
         : pad == kT1Pair ? (b == 4 ? 18 : b == 5 ? 35 : b == 6 ? 69 : 140)
         : pad == kT1One  ? (b == 4 ? 16 : b == 5 ? 33 : b == 6 ? 66 : 132)
         : pad == kT2Pair ? (b == 4 ? 18 : b == 5 ? 34 : b == 6 ? 72 : 140)
                          : (b == 4 ? 16 : b == 5 ? 40 : b == 6 ? 80 : 156);
}
__host__ __device__ constexpr int reg_off(int ph, int pad, int j) {
  return ((j & 1) ? pad_w(pad, reg_bit(ph, 0)) : 0) + ((j & 2) ? pad_w(pad, reg_bit(ph, 1)) : 0) +
         ((j & 4) ? pad_w(pad, reg_bit(ph, 2)) : 0);
}
__device__ __forceinline__ int lane_off(int ph, int pad, int lane) {
  int o = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i) o += ((lane >> i) & 1) * pad_w(pad, lane_bit(ph, i));
  return o;
}
// largest padded position + 1 per buffer: 278, 263, 280, 308 entries
__host__ __device__ constexpr int pad_size(int pad) {
  return 1 + reg_off(0, pad, 7) + pad_w(pad, 2) + pad_w(pad, 3) + pad_w(pad, 4) + pad_w(pad, 5) +
         pad_w(pad, 6);
}
constexpr int kScratchFloats = 2 * 280;
static_assert(pad_size(kT1Pair) <= 280 && pad_size(kT2Pair) <= 280, "pair scratch");
static_assert(pad_size(kT1One) <= kScratchFloats && pad_size(kT2One) <= kScratchFloats, "scratch");

constexpr int kStages = 3;  // bulk-copy pipeline depth per warp (two variables in flight)
template <typename W>  // stored message entry: float, or __half with NBFD_STORE_F16
struct Var8Stage {
  W msg[kStages][2][kQ];          // [stage][edge 1, edge 2][z], filled by the bulk copy engine
  float llr[kStages][8];          // [stage][bit] channel LLRs of the variable
  float scratch[kScratchFloats];  // transpose buffer; at the end M in natural order
  int4 idx[kStages];              // [stage] = (frame, variable, slot e1, slot e2)
  float2 pbt[8];                  // (Pr(b_i = 0), Pr(b_i = 1)) of the variable's 8 bits
  uint64_t bar[kStages];
  uint64_t pad_;
};
static_assert(sizeof(Var8Stage<float>) % 16 == 0 && sizeof(Var8Stage<__half>) % 16 == 0,
              "stage alignment");
constexpr int kWarps = 8;
template <typename W>
constexpr size_t smem_bytes() {
  return sizeof(Var8Stage<W>) * kWarps;
}

// four consecutive stored entries -> floats
__device__ __forceinline__ float4 load4(const float *p) {
  return *reinterpret_cast<const float4 *>(p);
}
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

__device__ __forceinline__ void bfly(float2 &a, float2 &b) {
  const float2 s = __fadd2_rn(a, b);
  b = __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
  a = s;
}
// butterflies on register bit R of 8 pairs
template <int R>
__device__ __forceinline__ void stage_pair(float2 (&v)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j)
    if (!(j & (1 << R))) bfly(v[j], v[j | (1 << R)]);
}
// one vector held as 4 pairs u[i] = (entry i, entry i + 4): register bits 0, 1 pair up across
// the float2 values, register bit 2 lies inside each float2
template <int R>
__device__ __forceinline__ void stage_one(float2 (&u)[4]) {
  if constexpr (R < 2) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (!(i & (1 << R))) bfly(u[i], u[i | (1 << R)]);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float a = u[i].x, b = u[i].y;
      u[i] = make_float2(a + b, a - b);
    }
  }
}

// Per-lane offsets of the two layouts a transpose connects, packed as lo | hi << 16 (lo = the
// layout with the smaller index: P0 for the first transpose, P1 for the second).
__device__ __forceinline__ uint32_t lane_offs(int lo, int pad, int lane) {
  return static_cast<uint32_t>(lane_off(lo, pad, lane)) |
         (static_cast<uint32_t>(lane_off(lo + 1, pad, lane)) << 16);
}
template <int PH, int LO>
__device__ __forceinline__ int off_of(uint32_t packed) {
  return PH == LO ? static_cast<int>(packed & 0xffffu) : static_cast<int>(packed >> 16);
}

template <int SRC, int DST, int PAD>
__device__ __forceinline__ void transpose_pair(float2 (&v)[8], float2 *s, uint32_t offs) {
  constexpr int LO = SRC < DST ? SRC : DST;
  const int ow = off_of<SRC, LO>(offs), orr = off_of<DST, LO>(offs);
#pragma unroll
  for (int j = 0; j < 8; ++j) s[ow + reg_off(SRC, PAD, j)] = v[j];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = s[orr + reg_off(DST, PAD, j)];
  __syncwarp();
}
template <int SRC, int DST, int PAD>
__device__ __forceinline__ void transpose_one(float2 (&u)[4], float *s, uint32_t offs) {
  constexpr int LO = SRC < DST ? SRC : DST;
  const int ow = off_of<SRC, LO>(offs), orr = off_of<DST, LO>(offs);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    s[ow + reg_off(SRC, PAD, i)] = u[i].x;
    s[ow + reg_off(SRC, PAD, i + 4)] = u[i].y;
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 4; ++i)
    u[i] = make_float2(s[orr + reg_off(DST, PAD, i)], s[orr + reg_off(DST, PAD, i + 4)]);
  __syncwarp();
}

}  // namespace

template <bool SYMBOL, typename W>
__global__ void __launch_bounds__(32 * kWarps, 3)
    k_var_fwht8(const float *__restrict__ llr, const W *__restrict__ c2v,
                W *__restrict__ v2c, uint16_t *__restrict__ sym, uint8_t *__restrict__ fsyn,
                const int32_t *__restrict__ var_edges, const uint8_t *__restrict__ edge_z,
                int N, int E, FrameSet fs, int32_t *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Var8Stage<W> &ws = reinterpret_cast<Var8Stage<W> *>(smem_raw)[wib];
  griddep_wait();
  griddep_release();
  const int F = fs.list ? __ldg(fs.count) : fs.n_static;
  const long long total = (long long)F * N;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  if (gw >= total) return;
  const long long n_items = (total - gw + nw - 1) / nw;  // this warp's variables
  // Lane 0 walks this warp's items gw, gw + nw, ... as (slot, variable) without a division per
  // item, and loads the indices of an item one iteration before its bulk copies are issued.
  long long cur_slot = gw / N;
  int cur_v = static_cast<int>(gw - cur_slot * N);
  const long long step_s = nw / N;
  const int step_v = static_cast<int>(nw - step_s * N);
  int pf_f = 0, pf_v = 0;
  int2 pf_e = make_int2(0, 0);
  auto load_next = [&]() {  // indices of the item at the cursor, then advance the cursor
    pf_f = fs.list ? __ldg(fs.list + cur_slot) : static_cast<int>(cur_slot);
    pf_v = cur_v;
    pf_e = __ldg(reinterpret_cast<const int2 *>(var_edges) + cur_v);
    cur_slot += step_s;
    cur_v += step_v;
    if (cur_v >= N) {
      cur_v -= N;
      ++cur_slot;
    }
  };
  auto issue = [&](int st) {  // bulk copies of the prefetched item into stage st
    ws.idx[st] = make_int4(pf_f, pf_v, pf_e.x, pf_e.y);
    constexpr uint32_t vb = kQ * sizeof(W);
    mbar_expect_tx(&ws.bar[st], 2u * vb + 32u);
    bulk_load(ws.msg[st][0], c2v + ((size_t)pf_f * E + pf_e.x) * kQ, vb, &ws.bar[st]);
    bulk_load(ws.msg[st][1], c2v + ((size_t)pf_f * E + pf_e.y) * kQ, vb, &ws.bar[st]);
    bulk_load(ws.llr[st], llr + ((size_t)pf_f * N + pf_v) * 8, 32u, &ws.bar[st]);
  };
  if (lane == 0) {
#pragma unroll
    for (int st = 0; st < kStages; ++st) mbar_init(&ws.bar[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int k = 0; k < kStages - 1 && k < n_items; ++k) {
      load_next();
      issue(k);
    }
    if (kStages - 1 < n_items) load_next();
  }
  __syncwarp();
  // per-lane transpose offsets
  const uint32_t o_t1p = lane_offs(0, kT1Pair, lane), o_t2p = lane_offs(1, kT2Pair, lane);
  const uint32_t o_t1o = lane_offs(0, kT1One, lane), o_t2o = lane_offs(1, kT2One, lane);
  float2 *s2 = reinterpret_cast<float2 *>(ws.scratch);
  long long t = 0;
  bool failed = false;
  for (; t < n_items; ++t) {
    const int b = static_cast<int>(t % kStages);
    if (lane == 0 && t + kStages - 1 < n_items) {
      fence_proxy_async_smem();
      issue(static_cast<int>((t + kStages - 1) % kStages));
      if (t + kStages < n_items) load_next();
    }
    const bool ok = mbar_wait_bounded(&ws.bar[b], static_cast<uint32_t>((t / kStages) & 1));
    if (__any_sync(kFull, !ok)) {
      failed = true;
      break;
    }
    const int4 ix = ws.idx[b];
    const int f = ix.x, v = ix.y, e1 = ix.z, e2 = ix.w;
    // read-out point of this lane (used at the end): alpha^i, H_e1 alpha^i, H_e2 alpha^i
    int z_pt = 0;
    if (!SYMBOL && lane < 24)
      z_pt = lane < 8 ? (1 << lane) : __ldg(edge_z + (size_t)(lane < 16 ? e1 : e2) * 8 + (lane & 7));
    // channel bit probabilities: lanes 0..7 compute one bit each
    if (lane < 8) {
      const float Li = ws.llr[b][lane];
      const float e = expf(-fabsf(Li));
      const float big = rcp_ftz(1.0f + e), small = e * big;
      ws.pbt[lane] = Li >= 0.0f ? make_float2(big, small) : make_float2(small, big);
    }
    // both check messages in layout P0, decoded from the Gamma form
    float2 c[8];
    {
      const float4 a0 = load4(&ws.msg[b][0][4 * lane]);
      const float4 a1 = load4(&ws.msg[b][0][128 + 4 * lane]);
      const float4 b0 = load4(&ws.msg[b][1][4 * lane]);
      const float4 b1 = load4(&ws.msg[b][1][128 + 4 * lane]);
      c[0] = make_float2(gamma_decode_ftz(a0.x), gamma_decode_ftz(b0.x));
      c[1] = make_float2(gamma_decode_ftz(a0.y), gamma_decode_ftz(b0.y));
      c[2] = make_float2(gamma_decode_ftz(a0.z), gamma_decode_ftz(b0.z));
      c[3] = make_float2(gamma_decode_ftz(a0.w), gamma_decode_ftz(b0.w));
      c[4] = make_float2(gamma_decode_ftz(a1.x), gamma_decode_ftz(b1.x));
      c[5] = make_float2(gamma_decode_ftz(a1.y), gamma_decode_ftz(b1.y));
      c[6] = make_float2(gamma_decode_ftz(a1.z), gamma_decode_ftz(b1.z));
      c[7] = make_float2(gamma_decode_ftz(a1.w), gamma_decode_ftz(b1.w));
    }
    // forward transforms of the pair: q * x-domain check messages (c1x, c2x), ends in P2
    stage_pair<0>(c);
    stage_pair<1>(c);
    stage_pair<2>(c);
    transpose_pair<0, 1, kT1Pair>(c, s2, o_t1p);
    stage_pair<0>(c);
    stage_pair<1>(c);
    stage_pair<2>(c);
    transpose_pair<1, 2, kT2Pair>(c, s2, o_t2p);
    stage_pair<1>(c);
    stage_pair<2>(c);
    // x-domain messages are probability vectors: drop the negative rounding noise
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j] = make_float2(fmaxf(c[j].x, 0.0f), fmaxf(c[j].y, 0.0f));
    // channel term p0(x) in layout P2: x = xl + 4 j with xl from the lane bits (x0 x6 x5 x7 x1)
    float2 p[8];
    {
      float lf = 1.0f;
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        const float2 pb = ws.pbt[lane_bit(2, i)];
        lf *= ((lane >> i) & 1) ? pb.y : pb.x;
      }
      const float2 q2 = ws.pbt[2], q3 = ws.pbt[3], q4 = ws.pbt[4];
      const float a0 = lf * q2.x, a1 = lf * q2.y;
      const float b00 = a0 * q3.x, b01 = a1 * q3.x, b10 = a0 * q3.y, b11 = a1 * q3.y;
      p[0] = make_float2(b00 * q4.x, b00 * q4.x);
      p[1] = make_float2(b01 * q4.x, b01 * q4.x);
      p[2] = make_float2(b10 * q4.x, b10 * q4.x);
      p[3] = make_float2(b11 * q4.x, b11 * q4.x);
      p[4] = make_float2(b00 * q4.y, b00 * q4.y);
      p[5] = make_float2(b01 * q4.y, b01 * q4.y);
      p[6] = make_float2(b10 * q4.y, b10 * q4.y);
      p[7] = make_float2(b11 * q4.y, b11 * q4.y);
    }
    // M_v = p0 . c1x . c2x (all checks of v); w = (p0 . c1x, p0 . c2x) = (U of e2, U of e1)
    float2 mu[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      mu[i] = make_float2(p[i].x * c[i].x * c[i].y, p[i + 4].x * c[i + 4].x * c[i + 4].y);
    float2 w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = __fmul2_rn(p[j], c[j]);
    int best_x = 0;
    if constexpr (SYMBOL) {
      // symbol decision: argmax over x of the x-domain marginal (ties: lowest x)
      const int xl = (lane & 1) | ((lane >> 4) & 1) << 1 | ((lane >> 2) & 1) << 5 |
                     ((lane >> 1) & 1) << 6 | ((lane >> 3) & 1) << 7;
      float best = -1.0f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (mu[i].x > best) {
          best = mu[i].x;
          best_x = xl + 4 * i;
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (mu[i].y > best) {
          best = mu[i].y;
          best_x = xl + 4 * (i + 4);
        }
      }
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float ob = __shfl_xor_sync(kFull, best, o);
        const int oi = __shfl_xor_sync(kFull, best_x, o);
        if (ob > best || (ob == best && oi < best_x)) {
          best = ob;
          best_x = oi;
        }
      }
    }
    // inverse-direction transforms of the pair, P2 -> P0
    stage_pair<0>(w);
    stage_pair<1>(w);
    stage_pair<2>(w);
    transpose_pair<2, 1, kT2Pair>(w, s2, o_t2p);
    stage_pair<1>(w);
    stage_pair<2>(w);
    transpose_pair<1, 0, kT1Pair>(w, s2, o_t1p);
    stage_pair<0>(w);
    stage_pair<1>(w);
    stage_pair<2>(w);
    // normalise to U(0) = 1 (x = 0 is register 0 of lane 0); U(0) <= 0 only by underflow:
    // then the message is delta_0
    const float n2 = __shfl_sync(kFull, w[0].x, 0), n1 = __shfl_sync(kFull, w[0].y, 0);
    const float2 r = make_float2(n2 > 0.0f ? rcp_ftz(n2) : 0.0f, n1 > 0.0f ? rcp_ftz(n1) : 0.0f);
    float o2[8], o1[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float2 sc = __ffma2_rn(w[j], r, make_float2(0.0f, 0.0f));  // + 0 turns -0 into +0
      o2[j] = gamma_encode_ftz(sc.x);
      o1[j] = gamma_encode_ftz(sc.y);
    }
    if (lane == 0) {
      o2[0] = 0.0f;  // Gamma(1)
      o1[0] = 0.0f;
    }
    {
      W *d2 = v2c + ((size_t)f * E + e2) * kQ, *d1 = v2c + ((size_t)f * E + e1) * kQ;
      store4(d2 + 4 * lane, o2[0], o2[1], o2[2], o2[3]);
      store4(d2 + 128 + 4 * lane, o2[4], o2[5], o2[6], o2[7]);
      store4(d1 + 4 * lane, o1[0], o1[1], o1[2], o1[3]);
      store4(d1 + 128 + 4 * lane, o1[4], o1[5], o1[6], o1[7]);
    }
    if constexpr (SYMBOL) {
      // the Fourier-domain syndrome words describe bitwise decisions: with symbol decisions they
      // are written as 0, so that the stop test rests on the GF(2^m) syndrome alone
      if (lane == 0) {
        if (sym) sym[(size_t)f * N + v] = static_cast<uint16_t>(best_x);
        if (fsyn) {
          fsyn[(size_t)f * E + e1] = 0;
          fsyn[(size_t)f * E + e2] = 0;
        }
      }
      __syncwarp();
      continue;
    }
    // inverse-direction transform of M, P2 -> P0, stored in natural order for the read-out
    stage_one<0>(mu);
    stage_one<1>(mu);
    stage_one<2>(mu);
    transpose_one<2, 1, kT2One>(mu, ws.scratch, o_t2o);
    stage_one<1>(mu);
    stage_one<2>(mu);
    transpose_one<1, 0, kT1One>(mu, ws.scratch, o_t1o);
    stage_one<0>(mu);
    stage_one<1>(mu);
    stage_one<2>(mu);
    *reinterpret_cast<float4 *>(&ws.scratch[4 * lane]) = make_float4(mu[0].x, mu[1].x, mu[2].x, mu[3].x);
    *reinterpret_cast<float4 *>(&ws.scratch[128 + 4 * lane]) =
        make_float4(mu[0].y, mu[1].y, mu[2].y, mu[3].y);
    __syncwarp();
    // TENTATIVE: signs of M at alpha^{i-1} (lanes 0..7), H_e1 alpha^{i-1} (8..15) and
    // H_e2 alpha^{i-1} (16..23), gathered with one ballot
    const bool neg_pt = lane < 24 && ws.scratch[z_pt] < 0.0f;
    uint32_t word = __ballot_sync(kFull, neg_pt);
    if (ws.scratch[0] < 0.0f) word = ~word;
    if (lane == 0) {
      if (sym) sym[(size_t)f * N + v] = static_cast<uint16_t>(word & 0xffu);
      if (fsyn) {
        fsyn[(size_t)f * E + e1] = static_cast<uint8_t>((word >> 8) & 0xffu);
        fsyn[(size_t)f * E + e2] = static_cast<uint8_t>((word >> 16) & 0xffu);
      }
    }
    __syncwarp();
  }
  if (failed && lane == 0) {
    if (err) atomicExch(err, NBFD_ETIMEDOUT);
    // the prefetches of the next stages may still be landing in this warp's shared memory
    for (long long k = t + 1; k < t + kStages && k < n_items; ++k)
      mbar_wait_bounded(&ws.bar[k % kStages], static_cast<uint32_t>((k / kStages) & 1));
  }
}

cudaError_t launch_var_fwht8(const nbfd_code *c, FrameSet fs, const float *llr, const float *c2v,
                             float *v2c, uint16_t *sym, uint8_t *fsyn, int32_t *err,
                             cudaStream_t s, bool symbol, VarTune tune, bool f16) {
  if (c->m != 8) return cudaErrorInvalidValue;
  const long long total = (long long)fs.n_static * c->N;
  long long g = (total + kWarps - 1) / kWarps;
  const int per_sm = tune.blocks_per_sm > 0 && tune.blocks_per_sm < 3 ? tune.blocks_per_sm : 3;
  const long long cap = (long long)sm_count() * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  auto go = [&](auto kern, auto tag) -> cudaError_t {
    using W = decltype(tag);
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(smem_bytes<W>()));
    if (e != cudaSuccess) return e;
    return launch_dependent(kern, dim3((int)g), dim3(32 * kWarps), smem_bytes<W>(), s, llr,
                            reinterpret_cast<const W *>(c2v), reinterpret_cast<W *>(v2c), sym,
                            fsyn, c->d_var_edges, c->d_edge_z, c->N, c->E, fs, err);
  };
  if (f16)
    return symbol ? go(k_var_fwht8<true, __half>, __half()) : go(k_var_fwht8<false, __half>, __half());
  return symbol ? go(k_var_fwht8<true, float>, 0.0f) : go(k_var_fwht8<false, float>, 0.0f);
}

}  // namespace nbfd
