// VARIABLE TO CHECK + TENTATIVE DECISION, FWHT form (FP32), GF(16): one lane per variable.
//
// The algebra is that of kernels_var_fwht.cu (Section 3.2 boxplus = XOR convolution = pointwise
// product in the x-domain, reached with the Section 2.1 transform). At q = 16 a whole vector
// fits in one lane's registers: every butterfly stage is in registers, the two check messages
// travel as float2 pairs (packed f32x2 butterflies), and each lane reads and writes its
// variable's 64-byte vectors with 16-byte loads and stores. Only the tentative-decision points,
// indexed by the variable's H_cv alpha^(i-1), go through shared memory.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "nbfd_internal.h"

namespace nbfd {

namespace {

constexpr int kQ4 = 16;
constexpr int kT4 = 256;  // threads per block
constexpr int kMStride = 17;  // floats per lane of M in shared memory (odd: no bank conflicts)

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

}  // namespace

template <bool SYMBOL>
__global__ void __launch_bounds__(kT4)
    k_var_fwht4(const float *__restrict__ llr, const float *__restrict__ c2v,
                float *__restrict__ v2c, uint16_t *__restrict__ sym, uint8_t *__restrict__ fsyn,
                const int32_t *__restrict__ var_edges, const uint8_t *__restrict__ edge_z, int N,
                int E, FrameSet fs) {
  __shared__ float m_sh[kT4 * kMStride];
  griddep_wait();
  griddep_release();
  const int F = fs.list ? __ldg(fs.count) : fs.n_static;
  const long long total = (long long)F * N;
  const long long start = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  float *my_m = m_sh + threadIdx.x * kMStride;
  for (long long item = start; item < total; item += stride) {
    const long long slot = item / N;
    const int v = static_cast<int>(item - slot * N);
    const int f = fs.list ? __ldg(fs.list + slot) : static_cast<int>(slot);
    const int2 e = __ldg(reinterpret_cast<const int2 *>(var_edges) + v);
    const float4 *a4 = reinterpret_cast<const float4 *>(c2v + ((size_t)f * E + e.x) * kQ4);
    const float4 *b4 = reinterpret_cast<const float4 *>(c2v + ((size_t)f * E + e.y) * kQ4);
    const float4 L = __ldg(reinterpret_cast<const float4 *>(llr + ((size_t)f * N + v) * 4));
    float2 c[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 a = __ldg(a4 + q), d = __ldg(b4 + q);
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
      float4 *d2 = reinterpret_cast<float4 *>(v2c + ((size_t)f * E + e.y) * kQ4);
      float4 *d1 = reinterpret_cast<float4 *>(v2c + ((size_t)f * E + e.x) * kQ4);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        d2[q] = make_float4(o2[4 * q], o2[4 * q + 1], o2[4 * q + 2], o2[4 * q + 3]);
        d1[q] = make_float4(o1[4 * q], o1[4 * q + 1], o1[4 * q + 2], o1[4 * q + 3]);
      }
    }
    if constexpr (SYMBOL) {
      // symbol decision: argmax over x of the x-domain marginal (ties: lowest x); the
      // Fourier-domain syndrome words are written as 0 (stop test on the GF(2^m) syndrome)
      float best = -1.0f;
      int best_x = 0;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (mu[j] > best) {
          best = mu[j];
          best_x = j;
        }
      }
      if (sym) sym[(size_t)f * N + v] = static_cast<uint16_t>(best_x);
      if (fsyn) {
        fsyn[(size_t)f * E + e.x] = 0;
        fsyn[(size_t)f * E + e.y] = 0;
      }
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
      const uint2 z1 = __ldg(reinterpret_cast<const uint2 *>(edge_z) + e.x);
      const uint2 z2 = __ldg(reinterpret_cast<const uint2 *>(edge_z) + e.y);
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
      if (sym) sym[(size_t)f * N + v] = static_cast<uint16_t>(w0);
      if (fsyn) {
        fsyn[(size_t)f * E + e.x] = static_cast<uint8_t>(w1);
        fsyn[(size_t)f * E + e.y] = static_cast<uint8_t>(w2);
      }
    }
  }
}

cudaError_t launch_var_fwht4(const nbfd_code *c, FrameSet fs, const float *llr, const float *c2v,
                             float *v2c, uint16_t *sym, uint8_t *fsyn, cudaStream_t s,
                             bool symbol, VarTune tune) {
  if (c->m != 4) return cudaErrorInvalidValue;
  const long long total = (long long)fs.n_static * c->N;
  long long grid = (total + kT4 - 1) / kT4;
  const long long cap = (long long)sm_count() * (tune.blocks_per_sm > 0 ? tune.blocks_per_sm : 8);
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  if (symbol)
    return launch_dependent(k_var_fwht4<true>, dim3((int)grid), dim3(kT4), 0, s, llr, c2v, v2c,
                            sym, fsyn, c->d_var_edges, c->d_edge_z, c->N, c->E, fs);
  return launch_dependent(k_var_fwht4<false>, dim3((int)grid), dim3(kT4), 0, s, llr, c2v, v2c, sym,
                          fsyn, c->d_var_edges, c->d_edge_z, c->N, c->E, fs);
}

}  // namespace nbfd
