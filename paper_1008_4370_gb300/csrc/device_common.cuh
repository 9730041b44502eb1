// Device helpers shared by the kernels: the one-word Gamma encoding of Section 3.2 and the
// channel message of the INITIALIZATION step (p0 from bit LLRs, then the Section 2.1 transform
// computed with register and warp-shuffle butterflies).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace nbfd {

constexpr unsigned kFull = 0xffffffffu;

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

template <int MB>
struct ChannelLayout {
  static constexpr int Q = 1 << MB;
  static constexpr int VPT = Q >= 32 ? Q / 32 : 1;  // values per lane
  static constexpr int LPV = Q / VPT;               // lanes per vector (a power of two <= 32)
  static constexpr int VPW = 32 / LPV;              // vectors per warp
  static constexpr int LOG_VPT = MB - (Q >= 32 ? 5 : MB);
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
#pragma unroll
    for (int j = 0; j < CL::VPT; ++j) {
      const float o = __shfl_xor_sync(kFull, V[j], lb);
      V[j] = (l & lb) ? (o - V[j]) : (V[j] + o);
    }
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
