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

template <int MB>
__global__ void __launch_bounds__(256, 3)
    k_var_fwht(const float *__restrict__ llr, const float *__restrict__ c2v,
               float *__restrict__ v2c, uint16_t *__restrict__ sym, uint8_t *__restrict__ fsyn,
               const int32_t *__restrict__ var_edges, const uint8_t *__restrict__ edge_h,
               const uint8_t *__restrict__ perm, int N, int E, FrameSet fs) {
  using CL = ChannelLayout<MB>;
  constexpr int Q = CL::Q, VPT = CL::VPT, LPV = CL::LPV, VPW = CL::VPW;
  __shared__ float sM[8][VPW * Q];  // M of each variable of the warp, for the read-out
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / LPV, l = lane % LPV;
  const long long total = (long long)frames_in(fs) * N;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = gw * VPW; base < total; base += nw * VPW) {
    const long long item = base + sub;
    const bool valid = item < total;
    const long long ic = valid ? item : total - 1;
    const long long slot = ic / N;
    const int v = static_cast<int>(ic - slot * N);
    const int f = frame_of(fs, slot);
    const int e1 = __ldg(var_edges + 2 * v), e2 = __ldg(var_edges + 2 * v + 1);
    float c1[VPT], c2[VPT];
    ld_global<VPT>(c1, c2v + ((size_t)f * E + e1) * Q + l * VPT);
    ld_global<VPT>(c2, c2v + ((size_t)f * E + e2) * Q + l * VPT);
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      c1[j] = gamma_decode_fast(c1[j]);
      c2[j] = gamma_decode_fast(c2[j]);
    }
    wht_inplace<MB>(c1, l);  // q * (x-domain check message of e1)
    wht_inplace<MB>(c2, l);
    float p[VPT];
    channel_probs_shared<MB>(llr + ((size_t)f * N + v) * MB, l, p);  // x-domain channel message
    // M_v = p0 . c1x . c2x (all checks), read out below from shared memory
    float *m_sh = sM[wib] + sub * Q;
    float nm;
    {
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
    const float r1 = 1.0f / __shfl_sync(kFull, c2[0], sub * LPV);
    if (valid) {
#pragma unroll
      for (int j = 0; j < VPT; ++j) c2[j] = gamma_encode_fast(c2[j] * r1);
      st_global<VPT>(v2c + ((size_t)f * E + e1) * Q + l * VPT, c2);
    }
#pragma unroll
    for (int j = 0; j < VPT; ++j) c1[j] *= p[j];
    wht_inplace<MB>(c1, l);
    const float r2 = 1.0f / __shfl_sync(kFull, c1[0], sub * LPV);
    if (valid) {
#pragma unroll
      for (int j = 0; j < VPT; ++j) c1[j] = gamma_encode_fast(c1[j] * r2);
      st_global<VPT>(v2c + ((size_t)f * E + e2) * Q + l * VPT, c1);
    }
    // TENTATIVE: signs of M at alpha^{i-1} (t < MB), H_e1 alpha^{i-1} (t < 2MB) and
    // H_e2 alpha^{i-1} (t < 3MB), one read-out point per lane, gathered with ballots.
    __syncwarp();
    const int h1 = __ldg(edge_h + e1), h2 = __ldg(edge_h + e2);
    uint32_t word = 0;
#pragma unroll
    for (int r = 0; r < (3 * MB + LPV - 1) / LPV; ++r) {
      const int t = r * LPV + l;
      bool neg_pt = false;
      if (t < 3 * MB) {
        const int kind = t / MB, i = t - kind * MB;
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
}

cudaError_t launch_var_fwht(const nbfd_code *c, FrameSet fs, const float *llr, const float *c2v,
                            float *v2c, uint16_t *sym, uint8_t *fsyn, cudaStream_t s) {
  const long long total = (long long)fs.n_static * c->N;
  const long long cap = (long long)sm_count() * 8;
#define NBFD_VAR_FWHT(MB)                                                                   \
  {                                                                                         \
    constexpr int VPW = ChannelLayout<MB>::VPW;                                             \
    long long g = (total + 8 * VPW - 1) / (8 * VPW);                                        \
    if (g > cap) g = cap;                                                                   \
    if (g < 1) g = 1;                                                                       \
    k_var_fwht<MB><<<(int)g, 256, 0, s>>>(llr, c2v, v2c, sym, fsyn, c->d_var_edges,         \
                                          c->d_edge_h, c->d_perm, c->N, c->E, fs);          \
  }
  switch (c->m) {
    case 2: NBFD_VAR_FWHT(2) break;
    case 3: NBFD_VAR_FWHT(3) break;
    case 4: NBFD_VAR_FWHT(4) break;
    case 5: NBFD_VAR_FWHT(5) break;
    case 6: NBFD_VAR_FWHT(6) break;
    case 7: NBFD_VAR_FWHT(7) break;
    case 8: NBFD_VAR_FWHT(8) break;
    default: return cudaErrorInvalidValue;
  }
#undef NBFD_VAR_FWHT
  return cudaGetLastError();
}

}  // namespace nbfd
