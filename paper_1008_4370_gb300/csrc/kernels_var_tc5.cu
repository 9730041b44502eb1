// VARIABLE TO CHECK + TENTATIVE DECISION with the Hadamard transforms on the 5th-generation
// tensor cores (tcgen05, accumulators in tensor memory), q = 256.
//
// The algebra of the FWHT form: the boxplus of Section 3.2 is a pointwise product in the x-domain,
// reached with Walsh-Hadamard transforms (Section 2.1). With x = 16a + b and H_256 = H_16 (x) H_16,
// the transform of a 256-vector seen as a 16x16 matrix X[a][b] is H_16 X H_16. A block of 128
// threads holds 8 variables; thread (v, i) owns one line (16 entries) of vector v:
//   1. 4 butterfly stages along the line, in registers (one factor H_16);
//   2. the 16 results, split into bf16 / fp16 operand parts, go to shared memory transposed: row
//      16 v + j, column i of a K-major 128 x 16 tile (the lines of the 8 vectors stacked);
//   3. one elected thread issues tcgen05.mma (M = 128, N = 16, K = 16) against H_16 (the other
//      factor), accumulating the parts in FP32 in tensor memory, and commits to an mbarrier;
//   4. every thread loads its TMEM lane (tcgen05.ld 32x32b): the perpendicular line of the
//      transform.
// So a transform turns line ownership by 90 degrees: natural rows -> x-domain columns -> natural
// rows; the pointwise products in between need no data movement. Several vectors share a launch of
// the tensor core: the forward transforms of the two check messages (N = 16 each, TMEM columns 0-31)
// and the inverse transforms of U1, U2 and M (columns 0-47).
// Operand precision (FP32 accumulation throughout), as the mma.sync form:
//   NBFD_FORM_BF16_HGEMM  bf16 operands;
//   NBFD_FORM_FP16_HGEMM  fp16 operands after a per-vector power-of-two scale putting the largest
//                         magnitude in [1, 2) (cancelled by the normalisation / sign read-out);
//   NBFD_FORM_FP32_TC     each FP32 operand split exactly into three bf16 parts (hi + mid + lo);
//                         H_16 is exact in bf16, so the products are the FP32 transform up to FP32
//                         accumulation rounding.
// Every wait is bounded; on expiry the block records NBFD_ETIMEDOUT, waits (bounded) once more for
// its tensor-core work, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "bulk_copy.cuh"
#include "device_common.cuh"
#include "nbfd_internal.h"

namespace nbfd {

namespace {

constexpr int kT5 = 128;        // threads per block: 8 vectors x 16 lines
constexpr int kTmemCols = 64;   // tensor-memory columns per block (up to 3 x 16 in use)
// K-major 16-bit tile without swizzle: 8-row x 16-byte core matrices (128 contiguous bytes),
// K-adjacent cores kLbo bytes apart (leading byte offset), row-block-adjacent cores kSbo bytes
// apart (stride byte offset). The 16-byte gaps put the two K-halves of a row 36 words apart and
// the next vector's rows 144 words on, so the transposed stores of a warp (two vectors x 16
// lines, one row each) hit 16 distinct banks instead of 4.
constexpr int kLbo = 144, kSbo = 288;
constexpr int kTile = 16 * kSbo;  // bytes of one 128 x 16 operand tile
__host__ __device__ constexpr int tile_off(int row, int k) {
  return (row >> 3) * kSbo + (k >> 3) * kLbo + (row & 7) * 16 + (k & 7) * 2;
}
static_assert(tile_off(127, 15) < kTile, "tile");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// shared-memory matrix descriptor: start address, leading / stride byte offsets (16-byte units),
// descriptor version 1, base offset 0, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(kLbo >> 4) << 16) |
         ((uint64_t)(kSbo >> 4) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: D = F32, A = B = bf16 (fmt 1) or fp16 (fmt 0), both
// K-major, N = 16, M = 128
__device__ __forceinline__ uint32_t instr_desc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&x)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

constexpr int kBF16 = NBFD_FORM_BF16_HGEMM;
constexpr int kFP16 = NBFD_FORM_FP16_HGEMM;
constexpr int kBF16x3 = NBFD_FORM_FP32_TC;

template <int P>
__device__ __forceinline__ uint16_t to16(float x) {
  if constexpr (P == kFP16) {
    const __half h = __float2half_rn(x);
    return *reinterpret_cast<const uint16_t *>(&h);
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    return *reinterpret_cast<const uint16_t *>(&h);
  }
}
__device__ __forceinline__ float bf16_round(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

__device__ __forceinline__ void bfly(float &a, float &b) {
  const float s = a + b;
  b = a - b;
  a = s;
}
__device__ __forceinline__ void wht16_line(float (&x)[16]) {
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (!(j & (1 << r))) bfly(x[j], x[j | (1 << r)]);
}

template <int P>
struct Tc5Smem {
  static constexpr int NP = P == kBF16x3 ? 3 : 1;
  unsigned char a[3][NP][kTile];  // [set][operand part] 128 x 16 tiles
  unsigned char b[2 * kSbo];      // H_16, 16 x 16, K-major
  float m[8][256];                // M of the 8 variables, natural order, for the read-out
  uint64_t bar;
  uint32_t tmem;
};
template <int P>
constexpr size_t tc5_smem() {
  // at least 26 KB, so that no more than 8 blocks (8 x 64 TMEM columns = 512) share an SM
  return sizeof(Tc5Smem<P>) + 1024 > 26 * 1024 ? sizeof(Tc5Smem<P>) + 1024 : 26 * 1024;
}

// One transform of NS sets (each thread's line of each set): butterflies along the line, the
// transposed operand tiles, the tensor-core products with H_16, back to one line per thread (the
// perpendicular one). Returns false if the bounded wait expired (block-uniform).
template <int P, int NS>
__device__ __forceinline__ bool transform_sets(float (&x)[NS][16], Tc5Smem<P> &sm, uint32_t tb,
                                               uint32_t &phase) {
  constexpr int NP = Tc5Smem<P>::NP;
  const int t = threadIdx.x, i = t & 15, v = t >> 4;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    wht16_line(x[s]);
    if constexpr (P == kFP16) {
      // power-of-two scale of the vector (its 16 lines): largest magnitude into [1, 2)
      float mx = 0.0f;
#pragma unroll
      for (int j = 0; j < 16; ++j) mx = fmaxf(mx, fabsf(x[s][j]));
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
      if (mx > 0.0f) {
        const float sc = __int_as_float((254 - ((__float_as_int(mx) >> 23) & 0xff)) << 23);
#pragma unroll
        for (int j = 0; j < 16; ++j) x[s][j] *= sc;
      }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int off = tile_off(16 * v + j, i);
      if constexpr (NP == 1) {
        *reinterpret_cast<uint16_t *>(sm.a[s][0] + off) = to16<P>(x[s][j]);
      } else {
        const float hi = bf16_round(x[s][j]);
        const float r1 = x[s][j] - hi;
        const float mid = bf16_round(r1);
        *reinterpret_cast<uint16_t *>(sm.a[s][0] + off) = to16<P>(hi);
        *reinterpret_cast<uint16_t *>(sm.a[s][1] + off) = to16<P>(mid);
        *reinterpret_cast<uint16_t *>(sm.a[s][2] + off) = to16<P>(r1 - mid);
      }
    }
  }
  // the tiles, written through the generic proxy, are read by the tensor core (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (t == 0) {
    const uint32_t idesc = instr_desc(P == kFP16 ? 0u : 1u);
    const uint64_t bdesc = smem_desc(smem_u32(sm.b));
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int p = 0; p < NP; ++p)
        mma_f16(tb + 16 * s, smem_desc(smem_u32(sm.a[s][p])), bdesc, idesc, p);
    mma_commit(&sm.bar);
  }
  const bool ok = mbar_wait_bounded(&sm.bar, phase);
  phase ^= 1u;
  if (__syncthreads_or(!ok)) return false;
  tc_fence_after();
  const uint32_t lane_base = tb + ((uint32_t)(32 * (t >> 5)) << 16);
#pragma unroll
  for (int s = 0; s < NS; ++s) tmem_ld16(lane_base + 16 * s, x[s]);
  tmem_wait_ld();
  return true;
}

__device__ __forceinline__ int frames_in(const FrameSet &fs) {
  return fs.list ? __ldg(fs.count) : fs.n_static;
}

}  // namespace

template <int P, bool SYMBOL>
__global__ void __launch_bounds__(kT5)
    k_var_tc5(const float *__restrict__ llr, const float *__restrict__ c2v, float *__restrict__ v2c,
              uint16_t *__restrict__ sym, uint8_t *__restrict__ fsyn,
              const int32_t *__restrict__ var_edges, const uint8_t *__restrict__ edge_h,
              const uint8_t *__restrict__ perm, int N, int E, FrameSet fs, int32_t *err) {
  constexpr int Q = 256;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Tc5Smem<P> &sm = *reinterpret_cast<Tc5Smem<P> *>(
      smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023));
  const int t = threadIdx.x, lane = t & 31, v = t >> 4, i = t & 15;
  const int hbase = lane & 16;  // first lane of this thread's vector within the warp
  griddep_wait();
  griddep_release();
  if (t < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sm.tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t < 16) {  // H_16 as the B operand (K-major; H is symmetric)
#pragma unroll
    for (int k = 0; k < 16; ++k)
      *reinterpret_cast<uint16_t *>(sm.b + tile_off(t, k)) =
          to16<P>((__popc(t & k) & 1) ? -1.0f : 1.0f);
  }
  if (t == 0) {
    mbar_init(&sm.bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = sm.tmem;
  uint32_t phase = 0;
  bool failed = false;
  const long long total = (long long)frames_in(fs) * N;
  const long long batches = (total + 7) / 8;
  for (long long bt = blockIdx.x; bt < batches && !failed; bt += gridDim.x) {
    const long long item = bt * 8 + v;
    const bool valid = item < total;
    const long long ic = valid ? item : total - 1;
    const long long slot = ic / N;
    const int var = static_cast<int>(ic - slot * N);
    const int f = fs.list ? __ldg(fs.list + slot) : static_cast<int>(slot);
    const int e1 = __ldg(var_edges + 2 * var), e2 = __ldg(var_edges + 2 * var + 1);
    // channel bit probabilities: thread i < 8 of the vector computes bit i
    float pb0 = 1.0f, pb1 = 0.0f;
    if (i < 8) {
      const float Li = __ldg(llr + ((size_t)f * N + var) * 8 + i);
      const float e = expf(-fabsf(Li));
      const float big = rcp_ftz(1.0f + e), small = e * big;
      pb0 = Li >= 0.0f ? big : small;
      pb1 = Li >= 0.0f ? small : big;
    }
    // line i of the two check messages (natural order: entries 16 i .. 16 i + 15), decoded
    float x[2][16];
    {
      const float4 *m1 = reinterpret_cast<const float4 *>(c2v + ((size_t)f * E + e1) * Q + 16 * i);
      const float4 *m2 = reinterpret_cast<const float4 *>(c2v + ((size_t)f * E + e2) * Q + 16 * i);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 a = __ldg(m1 + q), d = __ldg(m2 + q);
        x[0][4 * q + 0] = gamma_decode_ftz(a.x);
        x[0][4 * q + 1] = gamma_decode_ftz(a.y);
        x[0][4 * q + 2] = gamma_decode_ftz(a.z);
        x[0][4 * q + 3] = gamma_decode_ftz(a.w);
        x[1][4 * q + 0] = gamma_decode_ftz(d.x);
        x[1][4 * q + 1] = gamma_decode_ftz(d.y);
        x[1][4 * q + 2] = gamma_decode_ftz(d.z);
        x[1][4 * q + 3] = gamma_decode_ftz(d.w);
      }
    }
    // to the x-domain: thread (v, i) now holds entries x = 16 n + i, n = 0..15
    if (!transform_sets<P, 2>(x, sm, tb, phase)) {
      failed = true;
      break;
    }
    // p0(x) = prod over the bits of Pr(b = x_b): bits 0..3 are i, bits 4..7 are n
    float lowp = 1.0f, hi0[4], hi1[4];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const float q0 = __shfl_sync(kFull, pb0, hbase + b), q1 = __shfl_sync(kFull, pb1, hbase + b);
      if (b < 4) {
        lowp *= ((i >> b) & 1) ? q1 : q0;
      } else {
        hi0[b - 4] = q0;
        hi1[b - 4] = q1;
      }
    }
    float y[3][16];  // U of e1 (p0 . c2x), U of e2 (p0 . c1x), M (p0 . c1x . c2x)
    int best_x = 0;
    float best = -1.0f;
#pragma unroll
    for (int n = 0; n < 16; ++n) {
      const float c1 = fmaxf(x[0][n], 0.0f), c2 = fmaxf(x[1][n], 0.0f);  // probability vectors
      const float p0 = lowp * ((n & 1) ? hi1[0] : hi0[0]) * ((n & 2) ? hi1[1] : hi0[1]) *
                       ((n & 4) ? hi1[2] : hi0[2]) * ((n & 8) ? hi1[3] : hi0[3]);
      y[0][n] = p0 * c2;
      y[1][n] = p0 * c1;
      y[2][n] = y[1][n] * c2;
      if (SYMBOL) {
        const int xs = 16 * n + i;
        if (y[2][n] > best || (y[2][n] == best && xs < best_x)) {
          best = y[2][n];
          best_x = xs;
        }
      }
    }
    if constexpr (SYMBOL) {
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(kFull, best, o);
        const int oi = __shfl_xor_sync(kFull, best_x, o);
        if (ob > best || (ob == best && oi < best_x)) {
          best = ob;
          best_x = oi;
        }
      }
    }
    // back to the Fourier domain, natural order: thread (v, i) holds entries 16 i .. 16 i + 15
    bool ok;
    if constexpr (SYMBOL) {
      float y2[2][16];
#pragma unroll
      for (int n = 0; n < 16; ++n) {
        y2[0][n] = y[0][n];
        y2[1][n] = y[1][n];
      }
      ok = transform_sets<P, 2>(y2, sm, tb, phase);
#pragma unroll
      for (int n = 0; n < 16; ++n) {
        y[0][n] = y2[0][n];
        y[1][n] = y2[1][n];
      }
    } else {
      ok = transform_sets<P, 3>(y, sm, tb, phase);
    }
    if (!ok) {
      failed = true;
      break;
    }
    // normalise to U(0) = 1 (entry 0 is on line 0); U(0) <= 0 only by underflow: delta_0
    const float n1 = __shfl_sync(kFull, y[0][0], hbase), n2 = __shfl_sync(kFull, y[1][0], hbase);
    const float r1 = n1 > 0.0f ? rcp_ftz(n1) : 0.0f, r2 = n2 > 0.0f ? rcp_ftz(n2) : 0.0f;
    if (valid) {
      float4 *d1 = reinterpret_cast<float4 *>(v2c + ((size_t)f * E + e1) * Q + 16 * i);
      float4 *d2 = reinterpret_cast<float4 *>(v2c + ((size_t)f * E + e2) * Q + 16 * i);
      float o1[16], o2[16];
#pragma unroll
      for (int n = 0; n < 16; ++n) {
        o1[n] = gamma_encode_ftz(fmaf(y[0][n], r1, 0.0f));  // -0 -> +0
        o2[n] = gamma_encode_ftz(fmaf(y[1][n], r2, 0.0f));
      }
      if (i == 0) {
        o1[0] = 0.0f;  // Gamma(1)
        o2[0] = 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        d1[q] = make_float4(o1[4 * q], o1[4 * q + 1], o1[4 * q + 2], o1[4 * q + 3]);
        d2[q] = make_float4(o2[4 * q], o2[4 * q + 1], o2[4 * q + 2], o2[4 * q + 3]);
      }
    }
    if constexpr (SYMBOL) {
      if (valid && i == 0) {
        if (sym) sym[(size_t)f * N + var] = static_cast<uint16_t>(best_x);
        if (fsyn) {
          fsyn[(size_t)f * E + e1] = 0;
          fsyn[(size_t)f * E + e2] = 0;
        }
      }
    } else {
      // TENTATIVE: signs of M at alpha^{i-1} (points 0..7), H_e1 alpha^{i-1} (8..15) and
      // H_e2 alpha^{i-1} (16..23); thread i reads points i and 16 + i
      float *mv = sm.m[v];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4 *>(mv + 16 * i + 4 * q) =
            make_float4(y[2][4 * q], y[2][4 * q + 1], y[2][4 * q + 2], y[2][4 * q + 3]);
      __syncwarp();
      const int h1 = __ldg(edge_h + e1), h2 = __ldg(edge_h + e2);
      const int za = i < 8 ? (1 << i) : __ldg(perm + h1 * Q + (1 << (i - 8)));
      const bool neg0 = mv[za] < 0.0f;
      const bool neg1 = i < 8 && mv[__ldg(perm + h2 * Q + (1 << i))] < 0.0f;
      const uint32_t b0 = __ballot_sync(kFull, neg0), b1 = __ballot_sync(kFull, neg1);
      const bool flip = mv[0] < 0.0f;
      if (valid && i == 0) {
        uint32_t w0 = (b0 >> hbase) & 0xffffu, w1 = (b1 >> hbase) & 0xffu;
        if (flip) {
          w0 ^= 0xffffu;
          w1 ^= 0xffu;
        }
        if (sym) sym[(size_t)f * N + var] = static_cast<uint16_t>(w0 & 0xffu);
        if (fsyn) {
          fsyn[(size_t)f * E + e1] = static_cast<uint8_t>(w0 >> 8);
          fsyn[(size_t)f * E + e2] = static_cast<uint8_t>(w1);
        }
      }
      __syncwarp();
    }
  }
  if (failed) {
    if (t == 0 && err) atomicExch(err, NBFD_ETIMEDOUT);
    // the tensor core may still be working on the last commit: wait for it once more (bounded)
    mbar_wait_bounded(&sm.bar, phase ^ 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (t < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(kTmemCols));
}

bool var_tc5_available() {
  static int avail = -1;
  if (avail < 0) {
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    avail = major == 10 && minor == 3 ? 1 : 0;  // built for sm_103a
  }
  return avail == 1;
}

cudaError_t launch_var_tc5(const nbfd_code *c, FrameSet fs, int form, const float *llr,
                           const float *c2v, float *v2c, uint16_t *sym, uint8_t *fsyn,
                           int32_t *err, cudaStream_t s, bool symbol, VarTune tune) {
  if (c->m != 8) return cudaErrorNotSupported;
  const long long batches = ((long long)fs.n_static * c->N + 7) / 8;
  const int per_sm = tune.blocks_per_sm > 0 ? tune.blocks_per_sm : 4 * oversubscribed_waves(batches, (long long)sm_count() * 4 * 4);
  long long grid = batches;
  const long long cap = (long long)sm_count() * per_sm;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  auto go = [&](auto kern, size_t smem) -> cudaError_t {
    const cudaError_t e = ensure_smem((const void *)kern, smem);
    if (e != cudaSuccess) return e;
    return launch_dependent(kern, dim3((int)grid), dim3(kT5), smem, s, llr, c2v, v2c, sym, fsyn,
                            c->d_var_edges, c->d_edge_h, c->d_perm, c->N, c->E, fs, err);
  };
#define NBFD_TC5(P)                                                                            \
  return symbol ? go(k_var_tc5<P, true>, tc5_smem<P>()) : go(k_var_tc5<P, false>, tc5_smem<P>())
  switch (form & 0xff) {
    case NBFD_FORM_BF16_HGEMM: NBFD_TC5(kBF16);
    case NBFD_FORM_FP16_HGEMM: NBFD_TC5(kFP16);
    case NBFD_FORM_FP32_TC: NBFD_TC5(kBF16x3);
    default:
      return cudaErrorNotSupported;
  }
#undef NBFD_TC5
}

}  // namespace nbfd
