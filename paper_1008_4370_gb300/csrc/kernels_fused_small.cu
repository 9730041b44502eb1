// Whole decodes of small GF(16) codes in one launch, each frame's messages resident in shared
// memory for all of its iterations.
//
// A GF(16) frame of a short code holds E * 16 Gamma words per direction (12 KiB at N = 96), so
// one thread block keeps a frame on chip from its INITIALIZATION to its stop: per iteration the
// check node (CHECK TO VARIABLE, Section 3.2), the variable node with its tentative decision
// (VARIABLE TO CHECK, TENTATIVE DECISION) and the stop test (the Fourier-domain syndrome and the
// GF(2^m) syndrome, Section 2 / 3.2) follow one another inside the block, separated by block
// barriers. Both node updates work in place on ONE message buffer: a check's lanes read and
// write only that check's k slots (z -> H_e z is a bijection), and a variable's lane reads and
// writes only its own two slots. HBM then carries the LLRs in and the decisions out, once per
// frame, instead of 36 N q bytes per frame and iteration.
//
// The per-entry arithmetic is that of the streaming kernels (the check kernel's prefix / suffix
// passes over a check's slots, fwht4_variable of k_var_fwht4, the stop rule of k_stop), so the results are
// bit-identical to nbfd_decode's per-iteration path. The block runs frames blockIdx.x,
// blockIdx.x + gridDim.x, ... (one resident wave of blocks, as many as fit per SM).
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "nbfd_internal.h"
#include "var_fwht4_math.cuh"

namespace nbfd {

namespace {

constexpr int kQs = 16;
constexpr int kMStrideS = 17;  // floats per lane of the M read-out buffer (odd: no bank conflicts)
// 96 threads per block (one GF(16) N = 96 frame has 96 variables and 96 check lanes; larger
// frames loop), with registers bounded so that 6 blocks fit on an SM
constexpr int kFusedThreads = 96, kFusedMinBlocks = 6;
// Messages are kept variable-major, [variable][edge 1, edge 2][z] with 4 floats of padding per
// variable (36 floats): a lane's float4 accesses of its variable then start 4 banks after its
// neighbour's, so a quarter-warp's 16-byte accesses hit distinct banks.
constexpr int kVarStride = 36;

struct FusedLayout {
  int threads;
  // byte offsets into the dynamic shared memory, and its total
  size_t msg, m, xs, ws, llr, gexp, glog, perm, edge_h, edge_var, var_edges, edge_z, pos, bytes;
};

__host__ __device__ inline size_t up16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline FusedLayout fused_layout(int N, int E, int threads) {
  FusedLayout L{};
  L.threads = threads;
  L.msg = 0;                                               // [N][kVarStride] float, in place
  L.m = up16(L.msg + (size_t)N * kVarStride * 4);          // [threads][17] float, M read-out
  L.xs = up16(L.m + (size_t)threads * kMStrideS * 4);      // [N] u16 tentative decisions
  L.ws = up16(L.xs + (size_t)N * 2);                       // [E] u8 syndrome words
  L.llr = up16(L.ws + (size_t)E);                          // [N][4] float, this frame's LLRs
  L.gexp = up16(L.llr + (size_t)N * 16);                   // [32] u8
  L.glog = L.gexp + 32;                                    // [16] u8
  L.perm = up16(L.glog + 16);                              // [16][16] u8 index map
  L.edge_h = L.perm + 256;                                 // [E] u8
  L.edge_var = up16(L.edge_h + (size_t)E);                 // [E] u16
  L.var_edges = up16(L.edge_var + (size_t)E * 2);          // [N] (u16 e1, u16 e2)
  L.edge_z = up16(L.var_edges + (size_t)N * 4);            // [E] 4 x u8 points
  L.pos = up16(L.edge_z + (size_t)E * 4);                  // [E][16] u16: offset of H_e z
  L.bytes = up16(L.pos + (size_t)E * kQs * 2);
  return L;
}

// CHECK TO VARIABLE for entry z of check c: the check kernel's per-entry arithmetic (the same
// prefix and suffix passes over the k slots in the same order, so the same FP32 results), one
// entry per thread; pos[e][z] locates entry H_e z of slot e.
template <int KMAX>
__device__ __forceinline__ void check_entry_inplace(float *msg, const uint16_t *pos_tab, int c,
                                                    int k, int z) {
  float mag[KMAX];
  uint32_t sg[KMAX];
  int pos[KMAX];
  uint32_t sx = 0;
#pragma unroll
  for (int e = 0; e < KMAX; ++e) {
    if (e < k) {
      pos[e] = pos_tab[(c * k + e) * kQs + z];
      const float x = msg[pos[e]];
      mag[e] = fabsf(x);
      sg[e] = __float_as_uint(x) & 0x80000000u;
      sx ^= sg[e];
    }
  }
  float suf[KMAX];
  float run = 0.0f;
#pragma unroll
  for (int e = KMAX - 1; e >= 0; --e) {
    if (e < k) {
      suf[e] = run;
      run += mag[e];
    }
  }
  float pre = 0.0f;
#pragma unroll
  for (int e = 0; e < KMAX; ++e) {
    if (e < k) {
      const float o = pre + suf[e];
      pre += mag[e];
      msg[pos[e]] = __uint_as_float(__float_as_uint(o) | (sx ^ sg[e]));
    }
  }
}

template <bool SYMBOL, int KMAX>
__global__ void __launch_bounds__(kFusedThreads, KMAX <= 4 ? kFusedMinBlocks : 1) k_fused_gf16(const float *__restrict__ llr, uint16_t *__restrict__ sym_out,
                             uint8_t *__restrict__ ok, int32_t *__restrict__ iters,
                             int32_t *__restrict__ stats, const int32_t *__restrict__ var_edges_g,
                             const int32_t *__restrict__ edge_var_g,
                             const uint8_t *__restrict__ edge_h_g,
                             const uint8_t *__restrict__ perm_g,
                             const uint8_t *__restrict__ edge_z_g,
                             const uint8_t *__restrict__ gexp_g,
                             const uint8_t *__restrict__ glog_g, int N, int M, int k, int E,
                             int F, int max_iter, int32_t *__restrict__ next_frame) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FusedLayout L = fused_layout(N, E, blockDim.x);
  float *msg = reinterpret_cast<float *>(smem_raw + L.msg);
  float *my_m = reinterpret_cast<float *>(smem_raw + L.m) + threadIdx.x * kMStrideS;
  uint16_t *xs = reinterpret_cast<uint16_t *>(smem_raw + L.xs);
  uint8_t *ws = smem_raw + L.ws;
  float *llr_s = reinterpret_cast<float *>(smem_raw + L.llr);
  uint8_t *gexp = smem_raw + L.gexp, *glog = smem_raw + L.glog, *perm = smem_raw + L.perm;
  uint8_t *edge_h = smem_raw + L.edge_h;
  uint16_t *edge_var = reinterpret_cast<uint16_t *>(smem_raw + L.edge_var);
  uint32_t *var_edges = reinterpret_cast<uint32_t *>(smem_raw + L.var_edges);
  uint32_t *edge_z = reinterpret_cast<uint32_t *>(smem_raw + L.edge_z);
  uint16_t *pos = reinterpret_cast<uint16_t *>(smem_raw + L.pos);
  // the code's tables, once per block
  for (int i = threadIdx.x; i < 32; i += blockDim.x) gexp[i] = gexp_g[i];
  for (int i = threadIdx.x; i < 16; i += blockDim.x) glog[i] = glog_g[i];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) perm[i] = perm_g[i];
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    edge_h[e] = edge_h_g[e];
    edge_var[e] = static_cast<uint16_t>(edge_var_g[e]);
    edge_z[e] = __ldg(reinterpret_cast<const uint2 *>(edge_z_g) + e).x;
  }
  for (int v = threadIdx.x; v < N; v += blockDim.x) {
    const int2 ev = __ldg(reinterpret_cast<const int2 *>(var_edges_g) + v);
    var_edges[v] = static_cast<uint32_t>(ev.x) | static_cast<uint32_t>(ev.y) << 16;
  }
  __syncthreads();
  // pos[e][z]: where entry H_e z of slot e sits in the variable-major message buffer
  for (int t = threadIdx.x; t < E * kQs; t += blockDim.x) {
    const int e = t >> 4, z = t & (kQs - 1);
    const int v = edge_var[e];
    const int side = (var_edges[v] & 0xffffu) == static_cast<uint32_t>(e) ? 0 : kQs;
    pos[t] = static_cast<uint16_t>(v * kVarStride + side + perm[edge_h[e] * kQs + z]);
  }
  __syncthreads();
  // frames are handed out one at a time from a counter (frames that run to max_iter take many
  // times the average; a static split would leave some blocks with several of them)
  __shared__ int f_next;
  if (threadIdx.x == 0) f_next = blockIdx.x;
  __syncthreads();
  for (int f = f_next; f < F; f = f_next) {
    // the frame's LLRs, and the INITIALIZATION: V->C on both edges of a variable = Lambda0
    // (closed form, 8 entries per thread)
    for (int i = threadIdx.x; i < N; i += blockDim.x)
      reinterpret_cast<float4 *>(llr_s)[i] = __ldg(reinterpret_cast<const float4 *>(llr) + (size_t)f * N + i);
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
      const int v = t >> 1, l = t & 1;
      float g[8];
      channel_gamma<4>(llr + ((size_t)f * N + v) * 4, l, g);
      float4 *d1 = reinterpret_cast<float4 *>(msg + v * kVarStride + l * 8);
      float4 *d2 = reinterpret_cast<float4 *>(msg + v * kVarStride + kQs + l * 8);
      d1[0] = d2[0] = make_float4(g[0], g[1], g[2], g[3]);
      d1[1] = d2[1] = make_float4(g[4], g[5], g[6], g[7]);
    }
    __syncthreads();
    int it = 1;
    bool good = false;
    for (;; ++it) {
      // CHECK TO VARIABLE in place: 16 threads per check, one z each (z -> H_e z is a
      // bijection, so a check's 16 threads read 16 distinct words of each slot)
      for (int t = threadIdx.x; t < kQs * M; t += blockDim.x)
        check_entry_inplace<KMAX>(msg, pos, t >> 4, k, t & (kQs - 1));
      __syncthreads();
      // VARIABLE TO CHECK + TENTATIVE DECISION in place: one lane per variable
      for (int v = threadIdx.x; v < N; v += blockDim.x) {
        const uint32_t ev = var_edges[v];
        const int e1 = ev & 0xffffu, e2 = ev >> 16;
        const float4 *a4 = reinterpret_cast<const float4 *>(msg + v * kVarStride);
        const float4 *b4 = reinterpret_cast<const float4 *>(msg + v * kVarStride + kQs);
        float4 a[4], d[4], o1[4], o2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a[q] = a4[q];
          d[q] = b4[q];
        }
        const float4 Lv = reinterpret_cast<const float4 *>(llr_s)[v];
        uint2 z1 = make_uint2(0, 0), z2 = make_uint2(0, 0);
        if (!SYMBOL) {
          z1.x = edge_z[e1];
          z2.x = edge_z[e2];
        }
        uint16_t x;
        uint8_t w1, w2;
        fwht4_variable<SYMBOL>(a, d, Lv, z1, z2, my_m, o1, o2, x, w1, w2);
        float4 *d2 = reinterpret_cast<float4 *>(msg + v * kVarStride + kQs);
        float4 *d1 = reinterpret_cast<float4 *>(msg + v * kVarStride);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          d2[q] = o2[q];
          d1[q] = o1[q];
        }
        xs[v] = x;
        ws[e1] = w1;
        ws[e2] = w2;
      }
      __syncthreads();
      // stop test: the Fourier-domain syndrome (XOR of the per-edge words) and H x_hat
      int ffail = 0, efail = 0;
      for (int c = threadIdx.x; c < M; c += blockDim.x) {
        int fsv = 0, esv = 0;
        for (int j = 0; j < k; ++j) {
          const int e = c * k + j;
          fsv ^= ws[e];
          const int xv = xs[edge_var[e]];
          esv ^= xv == 0 ? 0 : gexp[glog[edge_h[e]] + glog[xv]];
        }
        ffail |= fsv != 0;
        efail |= esv != 0;
      }
      ffail = __syncthreads_or(ffail);
      efail = __syncthreads_or(efail);
      // (frame, iteration) pairs whose Fourier-domain syndrome cleared while H x_hat != 0
      if (threadIdx.x == 0 && !ffail && efail) atomicAdd(stats, 1);
      if ((!ffail && !efail) || it >= max_iter) {
        good = !efail;
        break;
      }
    }
    for (int v = threadIdx.x; v < N; v += blockDim.x) sym_out[(size_t)f * N + v] = xs[v];
    if (threadIdx.x == 0) {
      ok[f] = good ? 1 : 0;
      iters[f] = it;
      f_next = gridDim.x + atomicAdd(next_frame, 1);
    }
    __syncthreads();  // the next frame reuses every buffer
  }
}

int fused_threads(const nbfd_code *) { return kFusedThreads; }

template <bool SYMBOL, int KMAX>
cudaError_t launch_fused_t(const nbfd_code *c, int F, const float *llr, uint16_t *sym,
                           uint8_t *ok, int32_t *iters, int32_t *stats, int max_iter,
                           cudaStream_t s) {
  auto kern = k_fused_gf16<SYMBOL, KMAX>;
  const int threads = fused_threads(c);
  const size_t smem = fused_layout(c->N, c->E, threads).bytes;
  cudaError_t e = ensure_smem((const void *)kern, smem);
  if (e != cudaSuccess) return e;
  // as much shared memory as the SM offers: residency is bounded by it and by registers
  e = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)sm_count() * per_sm;
  if (grid > F) grid = F;
  kern<<<(int)grid, threads, smem, s>>>(llr, sym, ok, iters, stats, c->d_var_edges, c->d_edge_var,
                                         c->d_edge_h, c->d_perm, c->d_edge_z, c->d_gf_exp,
                                         c->d_gf_log, c->N, c->M, c->k, c->E, F, max_iter,
                                         stats + 2);
  return cudaGetLastError();
}

}  // namespace

bool fused_small_applies(const nbfd_code *c, int form) {
  if ((form & 0xff) != NBFD_FORM_FP32_FWHT || stores_f16(form) || (form & NBFD_UNFUSED)) return false;
  if (c->m != 4 || c->k > 32 || (long long)c->N * kVarStride >= 65536) return false;
  return fused_layout(c->N, c->E, fused_threads(c)).bytes <= 96 * 1024;
}

size_t fused_small_smem(const nbfd_code *c) {
  return fused_layout(c->N, c->E, fused_threads(c)).bytes;
}

cudaError_t launch_fused_small(const nbfd_code *c, int F, const float *llr, uint16_t *sym,
                               uint8_t *ok, int32_t *iters, int32_t *stats, int max_iter,
                               bool symbol, cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
#define NBFD_FUSED_K(KM)                                                                   \
  return symbol ? launch_fused_t<true, KM>(c, F, llr, sym, ok, iters, stats, max_iter, s)  \
                : launch_fused_t<false, KM>(c, F, llr, sym, ok, iters, stats, max_iter, s)
  if (c->k <= 4) NBFD_FUSED_K(4);
  if (c->k <= 8) NBFD_FUSED_K(8);
  if (c->k <= 16) NBFD_FUSED_K(16);
  NBFD_FUSED_K(32);
#undef NBFD_FUSED_K
}

}  // namespace nbfd
