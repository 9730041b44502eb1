// VARIABLE TO CHECK + TENTATIVE DECISION with the Hadamard transforms on tensor cores (q = 256).
//
// Same algebra as the FWHT form (kernels_var_fwht.cu): the boxplus of Section 3.2 is a pointwise
// product in the x-domain, reached with Walsh-Hadamard transforms (Section 2.1). Here each
// transform of a length-256 vector is a dense contraction: with x = 16a + b, H_256 = H_16 (x) H_16,
// so the transform of the 16x16 matrix X[a][b] is H_16 X H_16 -- two 16x16x16 products, run as
// mma.sync m16n8k16 (FP32 accumulate) on one warp:
//   GEMM1  D1 = X H_16                 (A = X from registers, B = H_16 constant fragments)
//   transpose D1 in registers with movmatrix (the accumulator layout of GEMM1 becomes the
//          A operand of GEMM2 after each 8x8 block is transposed)
//   GEMM2  D2 = D1^T H_16 = (H_16 X H_16)^T.
// A transform therefore returns the transposed matrix; applying it twice (forward to the
// x-domain, then back) returns to the natural order, so the pointwise products in between need
// no data movement. Operand precision (FP32 accumulation throughout):
//   NBFD_FORM_BF16_HGEMM  operands rounded to bf16 (8-bit significand);
//   NBFD_FORM_FP16_HGEMM  operands rounded to fp16 after a per-vector power-of-two scaling that
//                         puts the largest magnitude in [1, 2) (fp16 range);
//   NBFD_FORM_FP32_TC     every FP32 operand split exactly into three bf16 parts (hi + mid + lo,
//                         24 significant bits); H_16 is exact in bf16, so the products are the
//                         FP32 transform up to FP32 accumulation rounding.
//
// Lane layout (g = lane / 4, t = lane % 4, register r = 4j + 2h + c, j, h, c in {0,1}):
//   natural    register r holds z = 16(g + 8h) + 8j + 2t + c
//   transposed register r holds z = 16(8j + 2t + c) + g + 8h
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "bulk_copy.cuh"
#include "device_common.cuh"
#include "nbfd_internal.h"

namespace nbfd {

namespace {

constexpr int kBF16 = NBFD_FORM_BF16_HGEMM;
constexpr int kFP16 = NBFD_FORM_FP16_HGEMM;
constexpr int kBF16x3 = NBFD_FORM_FP32_TC;

template <int P>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if constexpr (P == kFP16) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
}

__device__ __forceinline__ float bf16_round(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

template <int P>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  if constexpr (P == kFP16) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
}

__device__ __forceinline__ uint32_t movmatrix_trans(uint32_t x) {
  uint32_t y;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(y) : "r"(x));
  return y;
}

// H_16 as B fragments: hb[j][0] = (H[2t][n], H[2t+1][n]), hb[j][1] = (H[2t+8][n], H[2t+9][n]),
// n = 8j + g, H[k][n] = (-1)^{popcount(k & n)} (exact in bf16 and fp16).
template <int P>
__device__ __forceinline__ void h16_fragments(uint32_t (&hb)[2][2], int g, int t) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int n = 8 * j + g;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int k = 2 * t + 8 * s;
      const float e0 = (__popc(k & n) & 1) ? -1.0f : 1.0f;
      const float e1 = (__popc((k + 1) & n) & 1) ? -1.0f : 1.0f;
      hb[j][s] = pack2<P>(e0, e1);
    }
  }
}

// A operand from 8 values in accumulator / natural order (pairs r = 0..7).
template <int P>
__device__ __forceinline__ void to_a(uint32_t (&a)[4], const float (&v)[8]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = pack2<P>(v[2 * i], v[2 * i + 1]);
}

// One GEMM of the transform: d[j] = A * H_16[:, 8j..8j+7], with A given as 1 (or 3) parts.
template <int P, int NP>
__device__ __forceinline__ void gemm_h(float (&d)[2][4], const uint32_t (&a)[NP][4],
                                       const uint32_t (&hb)[2][2]) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    d[j][0] = d[j][1] = d[j][2] = d[j][3] = 0.0f;
#pragma unroll
    for (int p = 0; p < NP; ++p) mma16816<P>(d[j], a[p], hb[j][0], hb[j][1]);
  }
}

// Split 8 FP32 values into NP operand parts (NP = 3: hi + mid + lo bf16, exact to 24 bits).
template <int P, int NP>
__device__ __forceinline__ void split_parts(uint32_t (&a)[NP][4], const float (&v)[8]) {
  if constexpr (NP == 1) {
    to_a<P>(a[0], v);
  } else {
    float r[8], hi[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      hi[i] = bf16_round(v[i]);
      r[i] = v[i] - hi[i];
    }
    to_a<P>(a[0], hi);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      hi[i] = bf16_round(r[i]);
      r[i] = r[i] - hi[i];
    }
    to_a<P>(a[1], hi);
    to_a<P>(a[2], r);
  }
}

// In-place 2D transform of one 256-vector held by the warp: natural <-> transposed order.
template <int P>
__device__ __forceinline__ void wht256_tc(float (&v)[8], const uint32_t (&hb)[2][2]) {
  constexpr int NP = P == kBF16x3 ? 3 : 1;
  if constexpr (P == kFP16) {
    // power-of-two scale putting max |v| of the vector in [1, 2): exact, and cancelled by the
    // normalisation / sign read-out downstream
    float mx = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) mx = fmaxf(mx, fabsf(v[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    if (mx > 0.0f) {
      const float sc = __int_as_float((254 - ((__float_as_int(mx) >> 23) & 0xff)) << 23);
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] *= sc;
    }
  }
  uint32_t a[NP][4];
  split_parts<P, NP>(a, v);
  float d[2][4];
  gemm_h<P, NP>(d, a, hb);
  // D1 blocks (rows g / g+8 of tiles 0 / 1) -> transposed blocks -> A operand of D1^T
  float w[8];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) w[4 * j + i] = d[j][i];
  uint32_t a2[NP][4];
  split_parts<P, NP>(a2, w);  // a2[p] = {tile0 rows g, tile0 rows g+8, tile1 rows g, tile1 rows g+8}
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const uint32_t t00 = movmatrix_trans(a2[p][0]);  // D1 block (0,0)^T -> block (0,0) of D1^T
    const uint32_t t01 = movmatrix_trans(a2[p][1]);  // D1 block (1,0)^T -> block (0,1) of D1^T
    const uint32_t t10 = movmatrix_trans(a2[p][2]);  // D1 block (0,1)^T -> block (1,0) of D1^T
    const uint32_t t11 = movmatrix_trans(a2[p][3]);  // D1 block (1,1)^T -> block (1,1)
    a2[p][0] = t00;
    a2[p][1] = t10;
    a2[p][2] = t01;
    a2[p][3] = t11;
  }
  gemm_h<P, NP>(d, a2, hb);
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) v[4 * j + i] = d[j][i];
}

__device__ __forceinline__ int z_natural(int r, int g, int t) {
  const int j = r >> 2, h = (r >> 1) & 1, c = r & 1;
  return 16 * (g + 8 * h) + 8 * j + 2 * t + c;
}
__device__ __forceinline__ int z_transposed(int r, int g, int t) {
  const int j = r >> 2, h = (r >> 1) & 1, c = r & 1;
  return 16 * (8 * j + 2 * t + c) + g + 8 * h;
}

__device__ __forceinline__ int frames_of(const FrameSet &fs) {
  return fs.list ? __ldg(fs.count) : fs.n_static;
}
__device__ __forceinline__ int frame_nr(const FrameSet &fs, long long slot) {
  return fs.list ? __ldg(fs.list + slot) : static_cast<int>(slot);
}

struct TcStage {
  float msg[2][2][256];  // [stage][edge 1, edge 2][z]
  int4 idx[2];           // [stage] = (frame, variable, slot e1, slot e2)
  float m[256];          // M of the variable, for the read-out
  uint64_t bar[2];
};

__device__ __forceinline__ void tc_issue(TcStage &ws, int st, long long item, long long total,
                                         int N, int E, const FrameSet &fs,
                                         const int32_t *__restrict__ var_edges,
                                         const float *__restrict__ c2v) {
  const long long slot = item / N;
  const int v = static_cast<int>(item - slot * N);
  const int f = frame_nr(fs, slot);
  const int e1 = __ldg(var_edges + 2 * v), e2 = __ldg(var_edges + 2 * v + 1);
  ws.idx[st] = make_int4(f, v, e1, e2);
  mbar_expect_tx(&ws.bar[st], 2u * 256u * 4u);
  bulk_load(ws.msg[st][0], c2v + ((size_t)f * E + e1) * 256, 256u * 4u, &ws.bar[st]);
  bulk_load(ws.msg[st][1], c2v + ((size_t)f * E + e2) * 256, 256u * 4u, &ws.bar[st]);
  (void)total;
}

}  // namespace

template <int P, bool SYMBOL>
__global__ void __launch_bounds__(256, 3)
    k_var_tc(const float *__restrict__ llr, const float *__restrict__ c2v, float *__restrict__ v2c,
             uint16_t *__restrict__ sym, uint8_t *__restrict__ fsyn,
             const int32_t *__restrict__ var_edges, const uint8_t *__restrict__ edge_h,
             const uint8_t *__restrict__ perm, int N, int E, FrameSet fs, int32_t *err) {
  constexpr int Q = 256, MB = 8;
  __shared__ TcStage stage_mem[8];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  TcStage &ws = stage_mem[wib];
  const long long total = (long long)frames_of(fs) * N;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  if (gw >= total) return;
  uint32_t hb[2][2];
  h16_fragments<P>(hb, g, t);
  if (lane == 0) {
    mbar_init(&ws.bar[0], 1);
    mbar_init(&ws.bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tc_issue(ws, 0, gw, total, N, E, fs, var_edges, c2v);
  }
  __syncwarp();
  long long it = 0;
  bool failed = false, next_issued = false;
  for (long long item = gw; item < total; item += nw, ++it) {
    const int b = static_cast<int>(it & 1);
    const long long next = item + nw;
    next_issued = next < total;
    if (lane == 0 && next_issued) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_issue(ws, b ^ 1, next, total, N, E, fs, var_edges, c2v);
    }
    const bool ok = mbar_wait_bounded(&ws.bar[b], static_cast<uint32_t>((it >> 1) & 1));
    if (__any_sync(kFull, !ok)) {
      failed = true;
      break;
    }
    const int4 ix = ws.idx[b];
    const int f = ix.x, v = ix.y, e1 = ix.z, e2 = ix.w;
    // check messages of e1 and e2, natural order, to the x-domain (transposed order)
    float c1[8], c2[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int z = z_natural(r, g, t);
      c1[r] = gamma_decode_fast(ws.msg[b][0][z]);
      c2[r] = gamma_decode_fast(ws.msg[b][1][z]);
    }
    wht256_tc<P>(c1, hb);
    wht256_tc<P>(c2, hb);
    // x-domain messages are probability vectors (non-negative in exact arithmetic): drop the
    // negative rounding noise of the transform
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      c1[r] = fmaxf(c1[r], 0.0f);
      c2[r] = fmaxf(c2[r], 0.0f);
    }
    // channel probabilities p0(x) at the transposed positions: low nibble g + 8h, high 8j+2t+c
    float pr[8];
    {
      const float *L = llr + ((size_t)f * N + v) * MB;
      float my0 = 1.0f, my1 = 0.0f;
      if (lane < MB) {
        const float Li = __ldg(L + lane);
        const float e = expf(-fabsf(Li));
        const float big = 1.0f / (1.0f + e), small = e / (1.0f + e);
        my0 = Li >= 0.0f ? big : small;
        my1 = Li >= 0.0f ? small : big;
      }
      float pb0[MB], pb1[MB];
#pragma unroll
      for (int i = 0; i < MB; ++i) {
        pb0[i] = __shfl_sync(kFull, my0, i);
        pb1[i] = __shfl_sync(kFull, my1, i);
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int x = z_transposed(r, g, t);
        float p = 1.0f;
#pragma unroll
        for (int i = 0; i < MB; ++i) p *= ((x >> i) & 1) ? pb1[i] : pb0[i];
        pr[r] = p;
      }
    }
    // M_v = p0 . c1x . c2x back to the Fourier domain (natural order), kept for the read-out;
    // with symbol decisions only its argmax over x (ties: lowest x) is needed
    float nm = 0.0f;
    int best_x = 0;
    if constexpr (SYMBOL) {
      float best = -1.0f;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float mv = pr[r] * c1[r] * c2[r];
        const int x = z_transposed(r, g, t);
        if (mv > best || (mv == best && x < best_x)) {
          best = mv;
          best_x = x;
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
    } else {
      float mm[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) mm[r] = pr[r] * c1[r] * c2[r];
      wht256_tc<P>(mm, hb);
      nm = __shfl_sync(kFull, mm[0], 0);
#pragma unroll
      for (int r = 0; r < 8; r += 2)
        *reinterpret_cast<float2 *>(&ws.m[z_natural(r, g, t)]) = make_float2(mm[r], mm[r + 1]);
    }
    // V->C on e1: U1 = WHT(p0 . c2x); on e2: U2 = WHT(p0 . c1x); normalised to U(0) = 1
#pragma unroll
    for (int r = 0; r < 8; ++r) c2[r] *= pr[r];
    wht256_tc<P>(c2, hb);
    const float n1 = __shfl_sync(kFull, c2[0], 0);
    const float r1 = n1 > 0.0f ? 1.0f / n1 : 0.0f;  // U(0) <= 0 only by underflow: send delta_0
    float *o1 = v2c + ((size_t)f * E + e1) * Q;
#pragma unroll
    for (int r = 0; r < 8; r += 2)
      *reinterpret_cast<float2 *>(o1 + z_natural(r, g, t)) =
          make_float2(gamma_encode_fast((r == 0 && lane == 0) ? 1.0f : c2[r] * r1),
                      gamma_encode_fast(c2[r + 1] * r1));
#pragma unroll
    for (int r = 0; r < 8; ++r) c1[r] *= pr[r];
    wht256_tc<P>(c1, hb);
    const float n2 = __shfl_sync(kFull, c1[0], 0);
    const float r2 = n2 > 0.0f ? 1.0f / n2 : 0.0f;
    float *o2 = v2c + ((size_t)f * E + e2) * Q;
#pragma unroll
    for (int r = 0; r < 8; r += 2)
      *reinterpret_cast<float2 *>(o2 + z_natural(r, g, t)) =
          make_float2(gamma_encode_fast((r == 0 && lane == 0) ? 1.0f : c1[r] * r2),
                      gamma_encode_fast(c1[r + 1] * r2));
    if constexpr (SYMBOL) {
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
    // TENTATIVE: signs of M at alpha^{i-1}, H_e1 alpha^{i-1}, H_e2 alpha^{i-1} (lane = point)
    __syncwarp();
    bool neg_pt = false;
    if (lane < 3 * MB) {
      const int kind = lane / MB, i = lane - kind * MB;
      const int h = kind == 1 ? __ldg(edge_h + e1) : __ldg(edge_h + e2);
      const int z = kind == 0 ? (1 << i) : __ldg(perm + h * Q + (1 << i));
      neg_pt = ws.m[z] < 0.0f;
    }
    uint32_t word = __ballot_sync(kFull, neg_pt);
    if (nm < 0.0f) word = ~word;
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
    if (next_issued)
      mbar_wait_bounded(&ws.bar[(it + 1) & 1], static_cast<uint32_t>(((it + 1) >> 1) & 1));
  }
}

cudaError_t launch_var_tc(const nbfd_code *c, FrameSet fs, int form, const float *llr,
                          const float *c2v, float *v2c, uint16_t *sym, uint8_t *fsyn, int32_t *err,
                          cudaStream_t s, bool symbol, VarTune tune) {
  if (c->m != 8) return cudaErrorNotSupported;
  const long long total = (long long)fs.n_static * c->N;
  long long grid = (total + 7) / 8;
  const long long cap = (long long)sm_count() * (tune.blocks_per_sm > 0 ? tune.blocks_per_sm : 3);
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
#define NBFD_TC(P)                                                                          \
  {                                                                                         \
    if (symbol)                                                                             \
      k_var_tc<P, true><<<(int)grid, 256, 0, s>>>(llr, c2v, v2c, sym, fsyn, c->d_var_edges,  \
                                                  c->d_edge_h, c->d_perm, c->N, c->E, fs,  \
                                                  err);                                    \
    else                                                                                    \
      k_var_tc<P, false><<<(int)grid, 256, 0, s>>>(llr, c2v, v2c, sym, fsyn, c->d_var_edges, \
                                                   c->d_edge_h, c->d_perm, c->N, c->E, fs, \
                                                   err);                                   \
  }
  switch (form) {
    case NBFD_FORM_BF16_HGEMM: NBFD_TC(kBF16) break;
    case NBFD_FORM_FP16_HGEMM: NBFD_TC(kFP16) break;
    case NBFD_FORM_FP32_TC: NBFD_TC(kBF16x3) break;
    default:
      return cudaErrorNotSupported;
  }
#undef NBFD_TC
  return cudaGetLastError();
}

}  // namespace nbfd
