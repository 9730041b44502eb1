// Conventional Log-SP (Section 2.2): the decoder the paper's method reformulates, kept as a
// measurement of Table 1 -- its check node carries the (k-1)-fold log-convolutions and its
// variable node only component-wise additions, the reverse of Log-Fourier SP's split.
//
// Messages are x-domain log-probabilities lambda(x) in [-inf, 0] (no sign), FP32, laid out
// [frame][slot][x] like the Gamma-form messages.
//
// CHECK TO VARIABLE (k_logsp_check): one warp per check. Each incoming lambda_vc is shifted by its
// maximum and exponentiated (the log-convolution is a log-sum-exp, evaluated as a linear XOR
// convolution of the shifted exponentials), permuted by h^{-1} (p~_vc(x) = p_vc(h^{-1} x)),
// combined by prefix and suffix XOR convolutions (3(k-2) q^2-term convolutions per check, each
// output the convolution of the others), normalised to its maximum, brought back to the log
// domain and permuted by h (lambda_cv(x) = lambda~_cv(h x)).
//
// VARIABLE TO CHECK (k_logsp_var): lambda_vc = lambda0 + lambda_c'v, normalised to
// lambda_vc(0) = 0; TENTATIVE DECISION argmax of lambda0 + lambda_c1v + lambda_c2v (ties: lowest
// x). lambda0(x) = sum_i ln Pr(b_i = x_i | L_i).
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "nbfd_internal.h"

namespace nbfd {

namespace {

template <int MB>
struct LspLayout {
  static constexpr int Q = 1 << MB;
  static constexpr int R = Q < 8 ? Q : 8;   // entries per lane
  static constexpr int TPV = Q / R;          // lanes per vector (<= 32)
};

// R consecutive floats (R = 8 or a power of two below): 16-byte accesses where R allows
template <int R>
__device__ __forceinline__ void lsp_load(float (&v)[R], const float *__restrict__ src) {
  if constexpr (R % 4 == 0) {
#pragma unroll
    for (int j = 0; j < R; j += 4) {
      const float4 x = __ldg(reinterpret_cast<const float4 *>(src + j));
      v[j] = x.x;
      v[j + 1] = x.y;
      v[j + 2] = x.z;
      v[j + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = __ldg(src + j);
  }
}
template <int R>
__device__ __forceinline__ void lsp_store(float *dst, const float (&v)[R]) {
  if constexpr (R % 4 == 0) {
#pragma unroll
    for (int j = 0; j < R; j += 4)
      *reinterpret_cast<float4 *>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < R; ++j) dst[j] = v[j];
  }
}

__device__ __forceinline__ int gf_mul_tab(int h, int x, const uint8_t *gexp, const uint8_t *glog) {
  return x == 0 ? 0 : gexp[glog[h] + glog[x]];
}

// out[t R + j] = sum_z1 A(z1) B((t R + j) ^ z1) for the lane's R outputs (lanes t < TPV)
template <int R, int TPV>
__device__ __forceinline__ void xor_conv_lane(const float *A, const float *B, int t, float (&o)[R]) {
#pragma unroll
  for (int j = 0; j < R; ++j) o[j] = 0.0f;
#pragma unroll 4
  for (int b = 0; b < TPV; ++b) {
    float a[R], c[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      a[i] = A[b * R + i];
      c[i] = B[(t ^ b) * R + i];
    }
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) o[j] = fmaf(a[i], c[i ^ j], o[j]);
  }
}

__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(kFull, x, o));
  return x;
}

template <int MB>
__global__ void __launch_bounds__(128)
    k_logsp_check(const float *__restrict__ v2c, float *__restrict__ c2v,
                  const uint8_t *__restrict__ edge_h, const uint8_t *__restrict__ gexp_g,
                  const uint8_t *__restrict__ glog_g, int M, int k, int E, int F) {
  using LL = LspLayout<MB>;
  constexpr int Q = LL::Q, R = LL::R, TPV = LL::TPV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint8_t gexp[512], glog[256];
  for (int i = threadIdx.x; i < 2 * Q; i += blockDim.x) gexp[i] = gexp_g[i];
  for (int i = threadIdx.x; i < Q; i += blockDim.x) glog[i] = glog_g[i];
  __syncthreads();
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = lane < TPV ? lane : 0;  // lanes past TPV shadow lane 0 and store nothing
  const bool act = lane < TPV;
  // per warp: inputs I_0..I_{k-1}, prefixes Pre_1..Pre_{k-2}, suffixes Suf_1..Suf_{k-2}, staging
  const int vecs = 3 * k - 3;
  float *base = reinterpret_cast<float *>(smem_raw) + (size_t)wib * vecs * Q;
  float *in = base, *pre = base + (size_t)k * Q, *suf = pre + (size_t)(k - 2) * Q;
  float *stage = suf + (size_t)(k - 2) * Q;
  auto Pre = [&](int j) -> const float * { return j == 0 ? in : pre + (size_t)(j - 1) * Q; };
  auto Suf = [&](int j) -> const float * { return j == k - 1 ? in + (size_t)(k - 1) * Q : suf + (size_t)(j - 1) * Q; };
  const long long total = (long long)F * M;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long item = gw; item < total; item += nw) {
    const long long f = item / M;
    const int c = static_cast<int>(item - f * M);
    // inputs: max-shifted exponentials, permuted by h^{-1}: I_e[h y] = exp(lambda_e(y) - max)
    for (int e = 0; e < k; ++e) {
      const int h = __ldg(edge_h + (size_t)c * k + e);
      const float *src = v2c + ((size_t)f * E + (size_t)c * k + e) * Q + t * R;
      float l[R];
      lsp_load<R>(l, src);
      float mx = -INFINITY;
#pragma unroll
      for (int j = 0; j < R; ++j) mx = fmaxf(mx, l[j]);
      mx = warp_max(mx);
      if (!(mx > -INFINITY)) mx = 0.0f;  // an all-zero message stays all zero
      __syncwarp();
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (act) in[(size_t)e * Q + gf_mul_tab(h, t * R + j, gexp, glog)] = expf(l[j] - mx);
    }
    __syncwarp();
    float o[R];
    // prefixes Pre_j = I_0 (*) .. (*) I_j, j = 1..k-2
    for (int j = 1; j <= k - 2; ++j) {
      xor_conv_lane<R, TPV>(Pre(j - 1), in + (size_t)j * Q, t, o);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < R; ++i)
        if (act) pre[(size_t)(j - 1) * Q + t * R + i] = o[i];
      __syncwarp();
    }
    // suffixes Suf_j = I_j (*) .. (*) I_{k-1}, j = k-2..1
    for (int j = k - 2; j >= 1; --j) {
      xor_conv_lane<R, TPV>(in + (size_t)j * Q, Suf(j + 1), t, o);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < R; ++i)
        if (act) suf[(size_t)(j - 1) * Q + t * R + i] = o[i];
      __syncwarp();
    }
    // outputs: out_e = Pre_{e-1} (*) Suf_{e+1} (out_0 = Suf_1, out_{k-1} = Pre_{k-2}),
    // normalised to their maximum, logged, permuted by h: lambda_cv[h^{-1} x] = lambda~_cv[x]
    for (int e = 0; e < k; ++e) {
      if (e == 0 || e == k - 1) {
        const float *src = e == 0 ? Suf(1) : Pre(k - 2);
#pragma unroll
        for (int i = 0; i < R; ++i) o[i] = src[t * R + i];
      } else {
        xor_conv_lane<R, TPV>(Pre(e - 1), Suf(e + 1), t, o);
      }
      float mx = 0.0f;
#pragma unroll
      for (int i = 0; i < R; ++i) mx = fmaxf(mx, o[i]);
      mx = warp_max(act ? mx : 0.0f);
      const bool pos = mx > 0.0f;  // divided (not multiplied by 1 / mx): the maximum maps to exactly 1
      const int h = __ldg(edge_h + (size_t)c * k + e);
      const int hinv_log = (Q - 1 - glog[h]) % (Q - 1);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int x = t * R + i;
        const int xp = x == 0 ? 0 : gexp[hinv_log + glog[x]];
        if (act) stage[xp] = pos ? logf(o[i] / mx) : -INFINITY;
      }
      __syncwarp();
      float ov[R];
#pragma unroll
      for (int i = 0; i < R; ++i) ov[i] = stage[t * R + i];
      if (act) lsp_store<R>(c2v + ((size_t)f * E + (size_t)c * k + e) * Q + t * R, ov);
      __syncwarp();
    }
  }
}

template <int MB>
__global__ void __launch_bounds__(256)
    k_logsp_var(const float *__restrict__ llr, const float *__restrict__ c2v,
                float *__restrict__ v2c, uint16_t *__restrict__ sym,
                const int32_t *__restrict__ var_edges, int N, int E, int F, bool init) {
  using LL = LspLayout<MB>;
  constexpr int Q = LL::Q, R = LL::R, TPV = LL::TPV, VPW = 32 / TPV;
  const int lane = threadIdx.x & 31, g = lane / TPV, t = lane % TPV;
  const long long total = (long long)F * N;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = gw * VPW; base < total; base += nw * VPW) {
    const long long item = base + g;
    const bool valid = item < total;
    const long long ic = valid ? item : total - 1;
    const long long f = ic / N;
    const int v = static_cast<int>(ic - f * N);
    // lambda0(x) = sum_i ln Pr(b_i = x_i | L_i): ln Pr(b = 0) = -ln(1 + e^-L), ln Pr(b = 1) =
    // -ln(1 + e^L), both as -max(0, -+L) - log1p(e^-|L|)
    float a0[MB], a1[MB];
#pragma unroll
    for (int i = 0; i < MB; ++i) {
      const float L = __ldg(llr + ((size_t)f * N + v) * MB + i);
      const float sp = log1pf(expf(-fabsf(L)));
      a0[i] = -fmaxf(-L, 0.0f) - sp;
      a1[i] = -fmaxf(L, 0.0f) - sp;
    }
    const int e1 = __ldg(var_edges + 2 * v), e2 = __ldg(var_edges + 2 * v + 1);
    float l0[R], u1[R], u2[R], c1v[R], c2v_[R];
    if (!init) {
      lsp_load<R>(c1v, c2v + ((size_t)f * E + e1) * Q + t * R);
      lsp_load<R>(c2v_, c2v + ((size_t)f * E + e2) * Q + t * R);
    }
    float best = -INFINITY;
    int best_x = 0;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int x = t * R + j;
      float s = 0.0f;
#pragma unroll
      for (int i = 0; i < MB; ++i) s += ((x >> i) & 1) ? a1[i] : a0[i];
      l0[j] = s;
      if (init) {
        u1[j] = u2[j] = s;
      } else {
        const float c1 = c1v[j], c2 = c2v_[j];
        u1[j] = s + c2;  // to the check of e1: excludes it
        u2[j] = s + c1;
        const float mu = s + c1 + c2;
        if (mu > best) {
          best = mu;
          best_x = x;
        }
      }
    }
    // normalisation lambda(0) = 0 (to the maximum where lambda(0) = -inf), argmax over the group
    float n1 = __shfl_sync(kFull, u1[0], g * TPV), n2 = __shfl_sync(kFull, u2[0], g * TPV);
    float m1 = -INFINITY, m2 = -INFINITY;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      m1 = fmaxf(m1, u1[j]);
      m2 = fmaxf(m2, u2[j]);
    }
#pragma unroll
    for (int o = TPV / 2; o > 0; o >>= 1) {
      m1 = fmaxf(m1, __shfl_xor_sync(kFull, m1, o));
      m2 = fmaxf(m2, __shfl_xor_sync(kFull, m2, o));
      const float ob = __shfl_xor_sync(kFull, best, o);
      const int oi = __shfl_xor_sync(kFull, best_x, o);
      if (ob > best || (ob == best && oi < best_x)) {
        best = ob;
        best_x = oi;
      }
    }
    if (!(n1 > -INFINITY)) n1 = m1;
    if (!(n2 > -INFINITY)) n2 = m2;
    if (valid) {
      // INITIALIZATION sends lambda0 itself on both edges; later iterations the normalised sums
      float o1[R], o2[R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        o1[j] = init ? l0[j] : u1[j] - n1;
        o2[j] = init ? l0[j] : u2[j] - n2;
      }
      lsp_store<R>(v2c + ((size_t)f * E + e1) * Q + t * R, o1);
      lsp_store<R>(v2c + ((size_t)f * E + e2) * Q + t * R, o2);
      if (!init && sym && t == 0) sym[(size_t)f * N + v] = static_cast<uint16_t>(best_x);
    }
  }
}

}  // namespace

bool logsp_supported(int m) { return m >= 3 && m <= 8; }

size_t logsp_check_smem(const nbfd_code *c) {
  return (size_t)4 * (3 * c->k - 3) * c->q * sizeof(float);  // 4 warps per block
}

cudaError_t launch_logsp_check(const nbfd_code *c, int F, const float *v2c, float *c2v,
                               cudaStream_t s) {
  if (!logsp_supported(c->m) || c->k < 3) return cudaErrorInvalidValue;
  const size_t smem = logsp_check_smem(c);
  const long long work = ((long long)F * c->M + 3) / 4;
  const long long cap = (long long)sm_count() * 16;
  const int grid = static_cast<int>(work < cap ? (work < 1 ? 1 : work) : cap);
#define NBFD_LSP_C(MB)                                                                        \
  {                                                                                           \
    cudaError_t e = ensure_smem((const void *)k_logsp_check<MB>, smem);                       \
    if (e != cudaSuccess) return e;                                                           \
    k_logsp_check<MB><<<grid, 128, smem, s>>>(v2c, c2v, c->d_edge_h, c->d_gf_exp, c->d_gf_log, \
                                              c->M, c->k, c->E, F);                           \
    return cudaGetLastError();                                                                \
  }
  switch (c->m) {
    case 3: NBFD_LSP_C(3)
    case 4: NBFD_LSP_C(4)
    case 5: NBFD_LSP_C(5)
    case 6: NBFD_LSP_C(6)
    case 7: NBFD_LSP_C(7)
    default: NBFD_LSP_C(8)
  }
#undef NBFD_LSP_C
}

cudaError_t launch_logsp_var(const nbfd_code *c, int F, const float *llr, const float *c2v,
                             float *v2c, uint16_t *sym, bool init, cudaStream_t s) {
  if (!logsp_supported(c->m)) return cudaErrorInvalidValue;
  const int tpv = c->q < 8 ? 1 : c->q / 8;
  const long long warps = ((long long)F * c->N * tpv + 31) / 32;
  const long long cap = (long long)sm_count() * 64;
  long long grid = (warps + 7) / 8;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
#define NBFD_LSP_V(MB)                                                                      \
  k_logsp_var<MB><<<(int)grid, 256, 0, s>>>(llr, c2v, v2c, sym, c->d_var_edges, c->N, c->E, F, \
                                            init);                                          \
  return cudaGetLastError();
  switch (c->m) {
    case 3: NBFD_LSP_V(3)
    case 4: NBFD_LSP_V(4)
    case 5: NBFD_LSP_V(5)
    case 6: NBFD_LSP_V(6)
    case 7: NBFD_LSP_V(7)
    default: NBFD_LSP_V(8)
  }
#undef NBFD_LSP_V
}

}  // namespace nbfd
