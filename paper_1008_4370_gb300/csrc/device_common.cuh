// Device helpers shared by the kernels: the one-word Gamma encoding of Section 3.2 and the
// channel message of the INITIALIZATION step (p0 from bit LLRs, then the Section 2.1 transform
// computed with register and warp-shuffle butterflies).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace nbfd {

constexpr unsigned kFull = 0xffffffffu;

// Message storage. A Gamma word is a float whose sign bit is the GF(2) sign and whose magnitude
// is -ln|P|; stored as float (FP32 forms) or rounded to IEEE half (NBFD_STORE_F16: same sign
// bit, magnitude with an 11-bit significand, +inf kept). Arithmetic is FP32 either way.
template <typename T>
__device__ __forceinline__ float msg_load(T x);
template <>
__device__ __forceinline__ float msg_load<float>(float x) {
  return x;
}
template <>
__device__ __forceinline__ float msg_load<__half>(__half x) {
  return __half2float(x);
}
// two Gamma words stored as halves, packed low | high << 16 (lower address first)
__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ float2 unpack_half2(uint32_t w) {
  __half2 h;
  *reinterpret_cast<uint32_t *>(&h) = w;
  return __half22float2(h);
}
template <typename T>
__device__ __forceinline__ T msg_store(float x);
template <>
__device__ __forceinline__ float msg_store<float>(float x) {
  return x;
}
template <>
__device__ __forceinline__ __half msg_store<__half>(float x) {
  return __float2half_rn(x);
}

// Programmatic dependent launch (sm_90 and later). A kernel launched as a dependent of the
// previous kernel in its stream may become resident before that kernel ends; griddep_wait()
// blocks until the previous kernel has completed and its memory operations are visible, so it
// comes before the first access to anything an earlier kernel wrote. griddep_release() lets the
// next kernel in the stream start launching (the data it reads is still protected by its own
// wait). Both are no-ops for a kernel launched normally.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Gamma(r) for |r| <= 1 packed in one float: sign bit = sgn_GF(2)(r) (0 for r == 0),
// magnitude = -ln|r| (+inf for r == 0). |r| > 1 (a rounding excess over P(0)) clamps to 0.
__device__ __forceinline__ float gamma_encode(float r) {
  const float a = fabsf(r);
  const float mag = a >= 1.0f ? 0.0f : -logf(a);
  const uint32_t s = (a > 0.0f) ? (__float_as_uint(r) & 0x80000000u) : 0u;
  return __uint_as_float(__float_as_uint(mag) | s);
}

// Gamma^{-1}: (-1)^sign * exp(-magnitude).
__device__ __forceinline__ float gamma_decode(float g) {
  const float e = expf(-fabsf(g));
  return __uint_as_float(__float_as_uint(e) | (__float_as_uint(g) & 0x80000000u));
}

// A length-Q vector held by a group of LPV lanes, VPT consecutive entries per lane (up to 8 in
// registers, so that at most log2(Q) - 3 butterfly stages cross lanes).
template <int MB>
struct ChannelLayout {
  static constexpr int Q = 1 << MB;
  static constexpr int VPT = Q >= 8 ? 8 : Q;        // values per lane
  static constexpr int LPV = Q / VPT;               // lanes per vector (a power of two <= 32)
  static constexpr int VPW = 32 / LPV;              // vectors per warp
  static constexpr int LOG_VPT = MB >= 3 ? 3 : MB;
};

// p0(x) = prod_i Pr(b_i = x_i | L_i) for one variable, at x = l*VPT + j in P[j] (lane l of a
// group of LPV lanes). `L` points at the MB LLRs of this lane's variable.
template <int MB>
__device__ __forceinline__ void channel_probs(const float *__restrict__ L, int l,
                                              float (&P)[ChannelLayout<MB>::VPT]) {
  using CL = ChannelLayout<MB>;
  float pb0[MB], pb1[MB];
#pragma unroll
  for (int i = 0; i < MB; ++i) {
    const float Li = __ldg(L + i);
    const float e = expf(-fabsf(Li));
    const float big = 1.0f / (1.0f + e), small = e / (1.0f + e);
    pb0[i] = Li >= 0.0f ? big : small;  // Pr(b = 0)
    pb1[i] = Li >= 0.0f ? small : big;  // Pr(b = 1)
  }
#pragma unroll
  for (int j = 0; j < CL::VPT; ++j) {
    const int x = l * CL::VPT + j;
    float p = 1.0f;
#pragma unroll
    for (int i = 0; i < MB; ++i) p *= ((x >> i) & 1) ? pb1[i] : pb0[i];
    P[j] = p;
  }
}

// In-place Walsh-Hadamard transform (Section 2.1, without the 1/2^m of the inverse) of one
// length-Q vector spread over a group of LPV lanes, index l*VPT + j in V[j]: butterflies on the
// index bits held in registers, then on the bits spread over lanes (warp shuffles). All 32 lanes
// of the warp must call this together.
template <int MB>
__device__ __forceinline__ void wht_inplace(float (&V)[ChannelLayout<MB>::VPT], int l) {
  using CL = ChannelLayout<MB>;
#pragma unroll
  for (int b = 0; b < CL::LOG_VPT; ++b) {
#pragma unroll
    for (int j = 0; j < CL::VPT; ++j) {
      if (!(j & (1 << b))) {
        const float u = V[j], w = V[j | (1 << b)];
        V[j] = u + w;
        V[j | (1 << b)] = u - w;
      }
    }
  }
#pragma unroll
  for (int b = CL::LOG_VPT; b < MB; ++b) {
    const int lb = 1 << (b - CL::LOG_VPT);
    const float sg = (l & lb) ? -1.0f : 1.0f;  // lower partner keeps V + o, upper o - V
#pragma unroll
    for (int j = 0; j < CL::VPT; ++j) {
      const float o = __shfl_xor_sync(kFull, V[j], lb);
      V[j] = fmaf(sg, V[j], o);  // exact: a product with +-1 is not rounded
    }
  }
}

// Single MUFU instructions (PTX ex2/lg2/rcp .approx.ftz): about 2 ulp of relative error; inputs
// and results below the smallest normal FP32 number are taken as 0.
__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_ftz(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_ftz(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float kLog2E = 1.4426950408889634f;  // log2(e)
constexpr float kLn2 = 0.6931471805599453f;     // ln(2)

// Gamma^{-1} as exp(-m) = 2^(-m log2 e) on the ex2 unit
__device__ __forceinline__ float gamma_decode_ftz(float g) {
  const float e = ex2_ftz(-fabsf(g) * kLog2E);
  return __uint_as_float(__float_as_uint(e) | (__float_as_uint(g) & 0x80000000u));
}
// Gamma(r) for |r| <= 1 as -ln|r| = -ln 2 * log2|r| on the lg2 unit; r = 0 gives magnitude +inf.
// A rounding excess |r| = 1 + d gives magnitude |ln|r||, about d (the sign bit of the word must
// stay the sign of r). r = -0 must not occur (callers add +0 first).
__device__ __forceinline__ float gamma_encode_ftz(float r) {
  const float mag = lg2_ftz(fabsf(r)) * -kLn2;
  return __uint_as_float((__float_as_uint(mag) & 0x7fffffffu) | (__float_as_uint(r) & 0x80000000u));
}

// The two above on a pair of words, their constant multiplies as one packed f32x2 instruction:
// bit-identical to calling them on each word (IEEE products are symmetric in sign, so
// -(|g| log2 e) = -|g (-log2 e)|).
__device__ __forceinline__ float2 gamma_decode2_ftz(float g0, float g1) {
  const float2 t = __fmul2_rn(make_float2(g0, g1), make_float2(-kLog2E, -kLog2E));
  const float e0 = ex2_ftz(-fabsf(t.x)), e1 = ex2_ftz(-fabsf(t.y));
  return make_float2(__uint_as_float(__float_as_uint(e0) | (__float_as_uint(g0) & 0x80000000u)),
                     __uint_as_float(__float_as_uint(e1) | (__float_as_uint(g1) & 0x80000000u)));
}
__device__ __forceinline__ float2 gamma_encode2_ftz(float2 r) {
  const float2 m =
      __fmul2_rn(make_float2(lg2_ftz(fabsf(r.x)), lg2_ftz(fabsf(r.y))), make_float2(-kLn2, -kLn2));
  return make_float2(
      __uint_as_float((__float_as_uint(m.x) & 0x7fffffffu) | (__float_as_uint(r.x) & 0x80000000u)),
      __uint_as_float((__float_as_uint(m.y) & 0x7fffffffu) | (__float_as_uint(r.y) & 0x80000000u)));
}

// Gamma^{-1} with the fast exponential (ex2 unit); a few ulp of relative error per entry.
__device__ __forceinline__ float gamma_decode_fast(float g) {
  const float e = __expf(-fabsf(g));
  return __uint_as_float(__float_as_uint(e) | (__float_as_uint(g) & 0x80000000u));
}

// Gamma(r) for |r| <= 1 with the fast logarithm (lg2 unit).
__device__ __forceinline__ float gamma_encode_fast(float r) {
  const float a = fabsf(r);
  const float mag = a >= 1.0f ? 0.0f : -__logf(a);
  const uint32_t s = (a > 0.0f) ? (__float_as_uint(r) & 0x80000000u) : 0u;
  return __uint_as_float(__float_as_uint(mag) | s);
}

// channel_probs with the MB logistic pairs computed once per group (lane i < MB computes bit i,
// then shuffles share them) and p(x) factored as p_low(j) * p_high(l) over the index bits held
// in registers and across lanes. `L` points at the MB LLRs of this group's variable.
template <int MB>
__device__ __forceinline__ void channel_probs_shared(const float *__restrict__ L, int l,
                                                     float (&P)[ChannelLayout<MB>::VPT]) {
  using CL = ChannelLayout<MB>;
  if constexpr (CL::LPV < MB) {  // fewer lanes than bits: each lane computes its own
    channel_probs<MB>(L, l, P);
    return;
  }
  const int lane = threadIdx.x & 31;
  const int base = lane - l;
  float my0 = 1.0f, my1 = 0.0f;
  if (l < MB) {
    const float Li = __ldg(L + l);
    const float e = expf(-fabsf(Li));
    const float big = 1.0f / (1.0f + e), small = e / (1.0f + e);
    my0 = Li >= 0.0f ? big : small;
    my1 = Li >= 0.0f ? small : big;
  }
  float pb0[MB], pb1[MB];
#pragma unroll
  for (int i = 0; i < MB; ++i) {
    pb0[i] = __shfl_sync(kFull, my0, base + i);
    pb1[i] = __shfl_sync(kFull, my1, base + i);
  }
  float hi = 1.0f;
#pragma unroll
  for (int b = CL::LOG_VPT; b < MB; ++b) hi *= ((l >> (b - CL::LOG_VPT)) & 1) ? pb1[b] : pb0[b];
#pragma unroll
  for (int j = 0; j < CL::VPT; ++j) {
    float p = hi;
#pragma unroll
    for (int b = 0; b < CL::LOG_VPT; ++b) p *= ((j >> b) & 1) ? pb1[b] : pb0[b];
    P[j] = p;
  }
}

// INITIALIZATION in closed form: Gamma(P0) of one variable, entry z = l*VPT + j in g[j] (lane l of
// a group of LPV lanes; `L` points at the MB LLRs of the group's variable). p0 is a product over
// the m bits, so its transform (Section 2.1) is the product of the bits' own transforms,
//   P0(z) = prod over the bits i set in z of (Pr(b_i = 0) - Pr(b_i = 1)) = prod tanh(L_i / 2),
// and Gamma(P0)(z) = (XOR of [L_i < 0], sum of -ln|tanh(L_i / 2)|) over those bits, with
// -ln|tanh(|L| / 2)| = ln(1 + t) - ln(1 - t), t = exp(-|L|) (+inf at L = 0: P0 vanishes there).
// P0(0) = 1, so the message is already normalised. The same values as the transform followed by
// Gamma, with m FP32 additions of non-negative terms per entry instead of exp, butterflies, a
// division and a logarithm.
template <int MB>
__device__ __forceinline__ void channel_gamma(const float *__restrict__ L, int l,
                                              float (&g)[ChannelLayout<MB>::VPT]) {
  using CL = ChannelLayout<MB>;
  float a[MB];
  uint32_t s[MB];
  if constexpr (CL::LPV >= MB) {  // lane i < MB of the group computes bit i, shuffles share them
    const int lane = threadIdx.x & 31;
    const int base = lane - l;
    float am = 0.0f;
    uint32_t sm = 0u;
    if (l < MB) {
      const float Li = __ldg(L + l);
      const float t = expf(-fabsf(Li));
      am = log1pf(t) - log1pf(-t);
      sm = Li < 0.0f ? 0x80000000u : 0u;
    }
#pragma unroll
    for (int i = 0; i < MB; ++i) {
      a[i] = __shfl_sync(kFull, am, base + i);
      s[i] = __shfl_sync(kFull, sm, base + i);
    }
  } else {
#pragma unroll
    for (int i = 0; i < MB; ++i) {
      const float Li = __ldg(L + i);
      const float t = expf(-fabsf(Li));
      a[i] = log1pf(t) - log1pf(-t);
      s[i] = Li < 0.0f ? 0x80000000u : 0u;
    }
  }
  float A = 0.0f;
  uint32_t S = 0u;
#pragma unroll
  for (int b = CL::LOG_VPT; b < MB; ++b) {
    if ((l >> (b - CL::LOG_VPT)) & 1) {
      A += a[b];
      S ^= s[b];
    }
  }
#pragma unroll
  for (int j = 0; j < CL::VPT; ++j) {
    float mag = A;
    uint32_t sg = S;
#pragma unroll
    for (int b = 0; b < CL::LOG_VPT; ++b) {
      if ((j >> b) & 1) {
        mag += a[b];
        sg ^= s[b];
      }
    }
    g[j] = __uint_as_float(__float_as_uint(mag) | sg);
  }
}

// P0(z) = sum_x p0(x) (-1)^{z.x} for one variable (INITIALIZATION of Section 3.2).
template <int MB>
__device__ __forceinline__ void channel_fourier(const float *__restrict__ L, int l,
                                                float (&P)[ChannelLayout<MB>::VPT]) {
  channel_probs<MB>(L, l, P);
  wht_inplace<MB>(P, l);
}

}  // namespace nbfd
