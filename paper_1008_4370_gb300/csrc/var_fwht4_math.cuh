// VARIABLE TO CHECK + TENTATIVE DECISION of one GF(16) variable in one lane, FWHT form (FP32).
//
// Section 3.2 boxplus = XOR convolution = pointwise product in the x-domain, reached with the
// Section 2.1 transform. At q = 16 a whole vector fits in one lane's registers: every butterfly
// stage is in registers and the two check messages travel as float2 pairs (packed f32x2
// butterflies). Shared by the streaming kernel (k_var_fwht4: messages in global memory) and the
// fused small-code kernel (k_fused_gf16: messages in shared memory), so both compute
// bit-identical results.
#pragma once

#include <cstdint>

#include "device_common.cuh"

namespace nbfd {

namespace fwht4 {

__device__ __forceinline__ void bfly(float2 &a, float2 &b) {
  const float2 s = __fadd2_rn(a, b);
  b = __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
  a = s;
}
__device__ __forceinline__ void wht16(float2 (&v)[16]) {
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (!(j & (1 << r))) bfly(v[j], v[j | (1 << r)]);
}
// one vector as 8 pairs (entry i, entry i + 8)
__device__ __forceinline__ void wht16_one(float2 (&u)[8]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (!(i & (1 << r))) bfly(u[i], u[i | (1 << r)]);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float a = u[i].x, b = u[i].y;
    u[i] = make_float2(a + b, a - b);
  }
}

}  // namespace fwht4

// One variable: a[] / d[] = the Gamma-form C->V messages of its edges e1 / e2 (4 float4 each),
// L = its 4 LLRs, z1 / z2 = the Fourier syndrome points H_e alpha^(i-1) of e1 / e2 (bytes 0..3),
// my_m = 16 floats of this lane's scratch (may alias nothing else in use). Out: o1 / o2 = V->C of
// e1 / e2 (Gamma form; o1 = Lambda0 [+] C_e2, o2 = Lambda0 [+] C_e1, both normalised), x = the
// tentative decision, w1 / w2 = the Fourier-domain syndrome words of e1 / e2 (0 with SYMBOL).
template <bool SYMBOL>
__device__ __forceinline__ void fwht4_variable(const float4 (&a4)[4], const float4 (&d4)[4],
                                               float4 L, uint2 z1, uint2 z2, float *my_m,
                                               float4 (&o1v)[4], float4 (&o2v)[4], uint16_t &x,
                                               uint8_t &w1o, uint8_t &w2o) {
  using namespace fwht4;
  float2 c[16];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 a = a4[q], d = d4[q];
    c[4 * q + 0] = make_float2(gamma_decode_ftz(a.x), gamma_decode_ftz(d.x));
    c[4 * q + 1] = make_float2(gamma_decode_ftz(a.y), gamma_decode_ftz(d.y));
    c[4 * q + 2] = make_float2(gamma_decode_ftz(a.z), gamma_decode_ftz(d.z));
    c[4 * q + 3] = make_float2(gamma_decode_ftz(a.w), gamma_decode_ftz(d.w));
  }
  wht16(c);  // q * x-domain check messages
#pragma unroll
  for (int j = 0; j < 16; ++j) c[j] = make_float2(fmaxf(c[j].x, 0.0f), fmaxf(c[j].y, 0.0f));
  // channel term: Pr(b_i = x_i) for the 4 bits, p0(x) as a product tree
  float pb0[4], pb1[4];
  {
    const float Ls[4] = {L.x, L.y, L.z, L.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float ex = expf(-fabsf(Ls[i]));
      const float big = rcp_ftz(1.0f + ex), small = ex * big;
      pb0[i] = Ls[i] >= 0.0f ? big : small;
      pb1[i] = Ls[i] >= 0.0f ? small : big;
    }
  }
  const float lo[4] = {pb0[0] * pb0[1], pb1[0] * pb0[1], pb0[0] * pb1[1], pb1[0] * pb1[1]};
  const float hi[4] = {pb0[2] * pb0[3], pb1[2] * pb0[3], pb0[2] * pb1[3], pb1[2] * pb1[3]};
  float mu[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float pj = lo[j & 3] * hi[j >> 2];
    mu[j] = pj * c[j].x * c[j].y;
    c[j] = __fmul2_rn(make_float2(pj, pj), c[j]);  // (U of e2, U of e1) in the x-domain
  }
  wht16(c);
  const float2 r = make_float2(c[0].x > 0.0f ? rcp_ftz(c[0].x) : 0.0f,
                               c[0].y > 0.0f ? rcp_ftz(c[0].y) : 0.0f);
  {
    float o2[16], o1[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float2 sc = __ffma2_rn(c[j], r, make_float2(0.0f, 0.0f));  // -0 -> +0
      o2[j] = gamma_encode_ftz(sc.x);
      o1[j] = gamma_encode_ftz(sc.y);
    }
    o2[0] = 0.0f;  // Gamma(1)
    o1[0] = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      o2v[q] = make_float4(o2[4 * q], o2[4 * q + 1], o2[4 * q + 2], o2[4 * q + 3]);
      o1v[q] = make_float4(o1[4 * q], o1[4 * q + 1], o1[4 * q + 2], o1[4 * q + 3]);
    }
  }
  if constexpr (SYMBOL) {
    // symbol decision: argmax over x of the x-domain marginal (ties: lowest x); the
    // Fourier-domain syndrome words are 0 (stop test on the GF(2^m) syndrome)
    float best = -1.0f;
    int best_x = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (mu[j] > best) {
        best = mu[j];
        best_x = j;
      }
    }
    x = static_cast<uint16_t>(best_x);
    w1o = 0;
    w2o = 0;
  } else {
    // TENTATIVE: M = WHT(p0 . c1x . c2x), signs at alpha^{i-1}, H_e1 alpha^{i-1}, H_e2 alpha^{i-1}
    float2 mp[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) mp[i] = make_float2(mu[i], mu[i + 8]);
    wht16_one(mp);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      my_m[i] = mp[i].x;
      my_m[i + 8] = mp[i].y;
    }
    const bool flip = my_m[0] < 0.0f;
    uint32_t w0 = 0, w1 = 0, w2 = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      w0 |= (my_m[1 << i] < 0.0f ? 1u : 0u) << i;
      w1 |= (my_m[(z1.x >> (8 * i)) & 0xffu] < 0.0f ? 1u : 0u) << i;
      w2 |= (my_m[(z2.x >> (8 * i)) & 0xffu] < 0.0f ? 1u : 0u) << i;
    }
    if (flip) {
      w0 ^= 0xfu;
      w1 ^= 0xfu;
      w2 ^= 0xfu;
    }
    x = static_cast<uint16_t>(w0);
    w1o = static_cast<uint8_t>(w1);
    w2o = static_cast<uint8_t>(w2);
  }
}

}  // namespace nbfd
