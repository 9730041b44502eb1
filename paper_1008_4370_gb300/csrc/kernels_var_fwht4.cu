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
#include "var_fwht4_math.cuh"

namespace nbfd {

namespace {

constexpr int kQ4 = 16;
constexpr int kT4 = 256;  // threads per block
constexpr int kMStride = 17;  // floats per lane of M in shared memory (odd: no bank conflicts)

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
  const bool narrow = total < (1ll << 32);  // the usual case: 32-bit division
  for (long long item = start; item < total; item += stride) {
    const long long slot =
        narrow ? static_cast<long long>(static_cast<uint32_t>(item) / static_cast<uint32_t>(N))
               : item / N;
    const int v = static_cast<int>(item - slot * N);
    const int f = fs.list ? __ldg(fs.list + slot) : static_cast<int>(slot);
    const int2 e = __ldg(reinterpret_cast<const int2 *>(var_edges) + v);
    const float4 *a4 = reinterpret_cast<const float4 *>(c2v + ((size_t)f * E + e.x) * kQ4);
    const float4 *b4 = reinterpret_cast<const float4 *>(c2v + ((size_t)f * E + e.y) * kQ4);
    const float4 L = __ldg(reinterpret_cast<const float4 *>(llr + ((size_t)f * N + v) * 4));
    float4 a[4], d[4], o1[4], o2[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = __ldg(a4 + q);
      d[q] = __ldg(b4 + q);
    }
    uint2 z1 = make_uint2(0, 0), z2 = make_uint2(0, 0);
    if (!SYMBOL) {
      z1 = __ldg(reinterpret_cast<const uint2 *>(edge_z) + e.x);
      z2 = __ldg(reinterpret_cast<const uint2 *>(edge_z) + e.y);
    }
    uint16_t x;
    uint8_t w1, w2;
    fwht4_variable<SYMBOL>(a, d, L, z1, z2, my_m, o1, o2, x, w1, w2);
    float4 *d2 = reinterpret_cast<float4 *>(v2c + ((size_t)f * E + e.y) * kQ4);
    float4 *d1 = reinterpret_cast<float4 *>(v2c + ((size_t)f * E + e.x) * kQ4);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      d2[q] = o2[q];
      d1[q] = o1[q];
    }
    if (sym) sym[(size_t)f * N + v] = x;
    if (fsyn) {
      fsyn[(size_t)f * E + e.x] = w1;
      fsyn[(size_t)f * E + e.y] = w2;
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
