// Kernels of one Log-Fourier decoding iteration (Section 3.2) on sm_103a.
//
//   k_init        INITIALIZATION: p0 from bit LLRs, transform with butterflies, Gamma form.
//   (CHECK TO VARIABLE is the bulk-copy pipeline of kernels_check.cu.)
//   k_var_direct  VARIABLE TO CHECK (boxplus of the channel message with the other check's
//                 message, as q^2 signed products in FP32) + TENTATIVE DECISION (bits and
//                 Fourier syndrome words from M_v at 3m points).
//   k_syndrome    Fourier-domain and GF(2^m) syndromes per check.
//   k_stop        per-frame stop test of one decoding iteration + compaction of active frames.
//
// Layouts: messages [frame][slot][z] float32 (Gamma form, see device_common.cuh), slots
// check-major (slot = c*k + j); LLRs [frame][variable][bit].
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "nbfd_internal.h"

namespace nbfd {

template <int N>
__device__ __forceinline__ void store_vec(float *dst, const float (&v)[N]) {
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

template <int N>
__device__ __forceinline__ void load_vec(float (&v)[N], const float *src) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int j = 0; j < N; j += 4) {
      const float4 x = *reinterpret_cast<const float4 *>(src + j);
      v[j] = x.x;
      v[j + 1] = x.y;
      v[j + 2] = x.z;
      v[j + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = src[j];
  }
}

template <int N>
__device__ __forceinline__ void load_vec_global(float (&v)[N], const float *__restrict__ src) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int j = 0; j < N; j += 4) {
      const float4 x = __ldg(reinterpret_cast<const float4 *>(src + j));
      v[j] = x.x;
      v[j + 1] = x.y;
      v[j + 2] = x.z;
      v[j + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = __ldg(src + j);
  }
}

__device__ __forceinline__ int frame_count(const FrameSet &fs) {
  return fs.list ? __ldg(fs.count) : fs.n_static;
}
__device__ __forceinline__ int frame_at(const FrameSet &fs, long long slot) {
  return fs.list ? __ldg(fs.list + slot) : static_cast<int>(slot);
}

// ---------------------------------------------------------------------------------------
// INITIALIZATION
// ---------------------------------------------------------------------------------------
template <int MB, typename W>
__global__ void __launch_bounds__(256)
    k_init(const float *__restrict__ llr, float *__restrict__ lambda0, W *__restrict__ v2c,
           const int32_t *__restrict__ var_edges, int N, int E, int F, int32_t *list_out,
           int32_t *count_out) {
  using CL = ChannelLayout<MB>;
  constexpr int Q = CL::Q, VPT = CL::VPT;
  const int lane = threadIdx.x & 31, sub = lane / CL::LPV, l = lane % CL::LPV;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  if (list_out) {
    for (long long i = gtid; i < F; i += nthr) list_out[i] = static_cast<int32_t>(i);
    if (gtid == 0) *count_out = F;
  }
  const long long total = (long long)F * N;
  for (long long base = (gtid >> 5) * CL::VPW; base < total; base += (nthr >> 5) * CL::VPW) {
    const long long item = base + sub;
    const bool valid = item < total;
    const long long ic = valid ? item : total - 1;
    float g[VPT];
    channel_gamma<MB>(llr + ic * MB, l, g);
    if (valid) {
      if (lambda0) store_vec<VPT>(lambda0 + item * Q + l * VPT, g);
      if (v2c) {
        const long long f = item / N;
        const int v = static_cast<int>(item - f * N);
        const int e1 = __ldg(var_edges + 2 * v), e2 = __ldg(var_edges + 2 * v + 1);
        if constexpr (sizeof(W) == 4) {
          store_vec<VPT>(reinterpret_cast<float *>(v2c) + ((size_t)f * E + e1) * Q + l * VPT, g);
          store_vec<VPT>(reinterpret_cast<float *>(v2c) + ((size_t)f * E + e2) * Q + l * VPT, g);
        } else {  // 8 halves per lane: one 16-byte store per edge
          static_assert(VPT == 8, "half storage needs 8 entries per lane");
          uint4 h;
          h.x = pack_half2(g[0], g[1]);
          h.y = pack_half2(g[2], g[3]);
          h.z = pack_half2(g[4], g[5]);
          h.w = pack_half2(g[6], g[7]);
          *reinterpret_cast<uint4 *>(v2c + ((size_t)f * E + e1) * Q + l * VPT) = h;
          *reinterpret_cast<uint4 *>(v2c + ((size_t)f * E + e2) * Q + l * VPT) = h;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// VARIABLE TO CHECK + TENTATIVE DECISION, FP32 direct form
// ---------------------------------------------------------------------------------------
// A group of TPV = Q/R lanes handles one variable; lane t owns the R outputs z = t*R + j.
// U1 = P0 (*) C2 and U2 = P0 (*) C1 (XOR convolution, U(z) = sum_z1 P0(z1) C(z ^ z1)) are
// accumulated as R x R XOR outer products of 16-byte shared-memory blocks, so each step does
// 2R^2 FMAs for 3R loads. M_v = U1 (*) C1 is then evaluated only at the 3m points the bit and
// syndrome read-out needs.
// A = float: the plain FP32 form. A = double (NBFD_FORM_FP64_DIRECT): the same step with the
// check messages decoded, the channel transform taken in closed form (P0(z) = prod over the bits
// of z of tanh(L_i / 2)), the q^2-term sums, the normalisation and the read-out all in FP64; only
// the stored messages are FP32.
template <typename A>
__device__ __forceinline__ float gamma_encode_t(A r) {
  if constexpr (sizeof(A) == 8) {
    const double a = fabs(r);
    const float mag = a >= 1.0 ? 0.0f : static_cast<float>(-log(a));
    const uint32_t sg = (a > 0.0) ? ((__double2hiint(r) < 0) ? 0x80000000u : 0u) : 0u;
    return __uint_as_float(__float_as_uint(mag) | sg);
  } else {
    return gamma_encode(r);
  }
}
template <typename A>
__device__ __forceinline__ A gamma_decode_t(float g) {
  if constexpr (sizeof(A) == 8) {
    const double e = exp(-static_cast<double>(fabsf(g)));
    return signbit(g) ? -e : e;
  } else {
    return gamma_decode(g);
  }
}

template <int MB, typename A>
__global__ void __launch_bounds__(sizeof(A) == 8 ? 128 : 256)
    k_var_direct(const float *__restrict__ llr, const float *__restrict__ c2v,
                 float *__restrict__ v2c, uint16_t *__restrict__ sym,
                 uint8_t *__restrict__ fsyn, const int32_t *__restrict__ var_edges,
                 const uint8_t *__restrict__ edge_h, const uint8_t *__restrict__ perm, int N,
                 int E, FrameSet fs) {
  using CL = ChannelLayout<MB>;
  constexpr int Q = 1 << MB;
  constexpr int R = Q < 8 ? Q : 8;
  constexpr int TPV = Q / R;
  constexpr int VPW = 32 / TPV;
  constexpr int LOG_R = R == 8 ? 3 : (R == 4 ? 2 : 1);
  constexpr int W = sizeof(A) == 8 ? 4 : 8;  // warps per block (FP64: the same shared bytes)
  __shared__ __align__(16) A sm[W][3][VPW * Q];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / TPV, t = lane % TPV;
  A *sa_w = sm[wib][0];
  A *sa = sm[wib][0] + g * Q;
  A *sc1 = sm[wib][1] + g * Q;
  A *sc2 = sm[wib][2] + g * Q;
  const long long total = (long long)frame_count(fs) * N;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = gw * VPW; base < total; base += nw * VPW) {
    // channel message P0 (linear, P0(0) = 1) of the warp's VPW variables
    if constexpr (sizeof(A) == 8) {
      for (int k = lane; k < VPW * Q; k += 32) {
        const int gi = k / Q, z = k % Q;
        long long item = base + gi;
        if (item >= total) item = total - 1;
        const long long slot = item / N;
        const int v = static_cast<int>(item - slot * N);
        const int f = frame_at(fs, slot);
        const float *L = llr + ((size_t)f * N + v) * MB;
        double p = 1.0;
#pragma unroll
        for (int i = 0; i < MB; ++i)
          if ((z >> i) & 1) p *= tanh(0.5 * static_cast<double>(__ldg(L + i)));
        sa_w[k] = p;
      }
    } else {
#pragma unroll
      for (int r = 0; r < VPW / CL::VPW; ++r) {
        const int gi = r * CL::VPW + lane / CL::LPV;
        long long item = base + gi;
        if (item >= total) item = total - 1;
        const long long slot = item / N;
        const int v = static_cast<int>(item - slot * N);
        const int f = frame_at(fs, slot);
        float P[CL::VPT];
        channel_fourier<MB>(llr + ((size_t)f * N + v) * MB, lane % CL::LPV, P);
        const float p0 = __shfl_sync(kFull, P[0], (lane / CL::LPV) * CL::LPV);
#pragma unroll
        for (int j = 0; j < CL::VPT; ++j)
          sa_w[gi * Q + (lane % CL::LPV) * CL::VPT + j] = P[j] / p0;
      }
    }
    const long long item = base + g;
    const bool valid = item < total;
    const long long ic = valid ? item : total - 1;
    const long long slot = ic / N;
    const int v = static_cast<int>(ic - slot * N);
    const int f = frame_at(fs, slot);
    const int e1 = __ldg(var_edges + 2 * v), e2 = __ldg(var_edges + 2 * v + 1);
    {
      float x1[R], x2[R];
      load_vec_global<R>(x1, c2v + ((size_t)f * E + e1) * Q + t * R);
      load_vec_global<R>(x2, c2v + ((size_t)f * E + e2) * Q + t * R);
      if constexpr (sizeof(A) == 8) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          sc1[t * R + j] = gamma_decode_t<A>(x1[j]);
          sc2[t * R + j] = gamma_decode_t<A>(x2[j]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          x1[j] = gamma_decode(x1[j]);
          x2[j] = gamma_decode(x2[j]);
        }
        store_vec<R>(sc1 + t * R, x1);
        store_vec<R>(sc2 + t * R, x2);
      }
    }
    __syncwarp();
    A u1[R], u2[R];
#pragma unroll
    for (int j = 0; j < R; ++j) u1[j] = u2[j] = A(0);
#pragma unroll 4
    for (int b = 0; b < TPV; ++b) {
      A av[R], c1v[R], c2v_[R];
      if constexpr (sizeof(A) == 8) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          av[i] = sa[b * R + i];
          c1v[i] = sc1[(t ^ b) * R + i];
          c2v_[i] = sc2[(t ^ b) * R + i];
        }
      } else {
        load_vec<R>(av, sa + b * R);
        load_vec<R>(c1v, sc1 + (t ^ b) * R);
        load_vec<R>(c2v_, sc2 + (t ^ b) * R);
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          u1[j] = fma(av[i], c2v_[i ^ j], u1[j]);  // fmaf for A = float
          u2[j] = fma(av[i], c1v[i ^ j], u2[j]);
        }
      }
    }
    const A n1 = __shfl_sync(kFull, u1[0], g * TPV);
    const A n2 = __shfl_sync(kFull, u2[0], g * TPV);
    if (valid) {
      float o1[R], o2[R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        o1[j] = gamma_encode_t<A>(u1[j] / n1);
        o2[j] = gamma_encode_t<A>(u2[j] / n2);
      }
      store_vec<R>(v2c + ((size_t)f * E + e1) * Q + t * R, o1);  // excludes check of e1
      store_vec<R>(v2c + ((size_t)f * E + e2) * Q + t * R, o2);  // excludes check of e2
    }
    // TENTATIVE: M(z) = sum_z1 U1(z1) C1(z ^ z1) at z = alpha^{i-1}, H_e1 alpha^{i-1},
    // H_e2 alpha^{i-1}. Lane t holds U1 on its block; C1 is read from shared memory.
    const int h1 = __ldg(edge_h + e1), h2 = __ldg(edge_h + e2);
    uint32_t bits = 0, w1 = 0, w2 = 0;
    const uint32_t neg1 = n1 < A(0) ? 1u : 0u;
#pragma unroll 1
    for (int i = 0; i < MB; ++i) {
#pragma unroll
      for (int kind = 0; kind < 3; ++kind) {
        const int zp = kind == 0 ? (1 << i) : __ldg(perm + (kind == 1 ? h1 : h2) * Q + (1 << i));
        const int zb = zp >> LOG_R, zl = zp & (R - 1);
        const A *cb = sc1 + (t ^ zb) * R;
        A part = A(0);
#pragma unroll
        for (int j = 0; j < R; ++j) part = fma(u1[j], cb[j ^ zl], part);
#pragma unroll
        for (int o = TPV / 2; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
        const uint32_t bit = (part < A(0) ? 1u : 0u) ^ neg1;
        if (kind == 0) bits |= bit << i;
        else if (kind == 1) w1 |= bit << i;
        else w2 |= bit << i;
      }
    }
    if (valid && t == 0) {
      if (sym) sym[(size_t)f * N + v] = static_cast<uint16_t>(bits);
      if (fsyn) {
        fsyn[(size_t)f * E + e1] = static_cast<uint8_t>(w1);
        fsyn[(size_t)f * E + e2] = static_cast<uint8_t>(w2);
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------
// syndromes
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int gf_mul(int h, int x, const uint8_t *gexp, const uint8_t *glog) {
  return x == 0 ? 0 : gexp[glog[h] + glog[x]];
}

__global__ void k_syndrome(const uint16_t *__restrict__ sym, const uint8_t *__restrict__ fsyn,
                           uint16_t *__restrict__ fourier, uint16_t *__restrict__ exact,
                           const int32_t *__restrict__ edge_var, const uint8_t *__restrict__ edge_h,
                           const uint8_t *__restrict__ gexp, const uint8_t *__restrict__ glog,
                           int N, int M, int k, int E, int F) {
  const long long total = (long long)F * M;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long f = idx / M;
    const int c = static_cast<int>(idx - f * M);
    int fsv = 0, esv = 0;
    for (int j = 0; j < k; ++j) {
      const int e = c * k + j;
      if (fsyn) fsv ^= fsyn[f * E + e];
      esv ^= gf_mul(edge_h[e], sym[f * N + edge_var[e]], gexp, glog);
    }
    if (fourier) fourier[idx] = static_cast<uint16_t>(fsv);
    if (exact) exact[idx] = static_cast<uint16_t>(esv);
  }
}

// One block per active frame: the frame stops when every check's Fourier-domain syndrome word
// and GF(2^m) syndrome are 0 (or at max_iter); otherwise it is appended to next_list.
__global__ void __launch_bounds__(128)
    k_stop(FrameSet fs, const uint16_t *__restrict__ sym, const uint8_t *__restrict__ fsyn,
           const int32_t *__restrict__ edge_var, const uint8_t *__restrict__ edge_h,
           const uint8_t *__restrict__ gexp_g, const uint8_t *__restrict__ glog_g, int q, int N,
           int M, int k, int E, int iter_arg, const int32_t *__restrict__ iter_dev, int max_iter,
           int32_t *__restrict__ next_list,
           int32_t *__restrict__ next_count, uint8_t *__restrict__ ok, int32_t *__restrict__ iters,
           int32_t *__restrict__ stats) {
  __shared__ uint8_t gexp[512];
  __shared__ uint8_t glog[256];
  // the field tables are constant: load them while the previous kernel drains
  for (int i = threadIdx.x; i < 2 * q; i += blockDim.x) gexp[i] = gexp_g[i];
  for (int i = threadIdx.x; i < q; i += blockDim.x) glog[i] = glog_g[i];
  griddep_wait();
  griddep_release();
  const int iter = iter_dev ? *iter_dev : iter_arg;
  __syncthreads();
  const int nf = frame_count(fs);
  for (int s = blockIdx.x; s < nf; s += gridDim.x) {
    const int f = frame_at(fs, s);
    // Fourier-domain syndrome first (one byte per edge); the GF(2^m) syndrome, which gathers
    // the decisions, only where the outcome depends on it: when the Fourier-domain syndrome
    // clears, and at max_iter (the flag of a frame that never stopped)
    int ffail = 0;
    for (int c = threadIdx.x; c < M; c += blockDim.x) {
      int fsv = 0;
      for (int j = 0; j < k; ++j) fsv ^= fsyn[(size_t)f * E + c * k + j];
      ffail |= fsv != 0;
    }
    ffail = __syncthreads_or(ffail);
    int efail = 1;
    if (!ffail || iter >= max_iter) {
      efail = 0;
      for (int c = threadIdx.x; c < M; c += blockDim.x) {
        int esv = 0;
        for (int j = 0; j < k; ++j) {
          const int e = c * k + j;
          esv ^= gf_mul(__ldg(edge_h + e), sym[(size_t)f * N + __ldg(edge_var + e)], gexp, glog);
        }
        efail |= esv != 0;
      }
      efail = __syncthreads_or(efail);
    }
    if (threadIdx.x == 0) {
      if (!ffail && !efail) {
        ok[f] = 1;
        iters[f] = iter;
      } else if (iter >= max_iter) {
        ok[f] = efail ? 0 : 1;
        iters[f] = iter;
      } else {
        next_list[atomicAdd(next_count, 1)] = f;
      }
      // frames whose Fourier-domain syndrome cleared while H x_hat != 0 (the two differ)
      if (!ffail && efail) atomicAdd(stats, 1);
    }
  }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
static int grid_for(long long work_blocks, int per_sm) {
  const long long cap = (long long)sm_count() * per_sm;
  long long g = work_blocks < cap ? work_blocks : cap;
  return g < 1 ? 1 : static_cast<int>(g);
}

#define NBFD_DISPATCH_M(m, FN) \
  switch (m) {                 \
    case 2: FN(2); break;      \
    case 3: FN(3); break;      \
    case 4: FN(4); break;      \
    case 5: FN(5); break;      \
    case 6: FN(6); break;      \
    case 7: FN(7); break;      \
    case 8: FN(8); break;      \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_init(const nbfd_code *c, int F, const float *llr, float *lambda0, float *v2c,
                        int32_t *list_out, int32_t *count_out, cudaStream_t s, bool f16) {
  const long long total = (long long)F * c->N;
  if (f16) {  // half storage: GF(256) only, no lambda0 output
    if (c->m != 8 || lambda0) return cudaErrorNotSupported;
    const int grid = grid_for((total + 7) / 8, 8 * oversubscribed_waves(total, 64LL * sm_count()));
    k_init<8, __half><<<grid, 256, 0, s>>>(llr, nullptr, reinterpret_cast<__half *>(v2c),
                                           c->d_var_edges, c->N, c->E, F, list_out, count_out);
    return cudaGetLastError();
  }
#define NBFD_INIT(MB)                                                                        \
  {                                                                                          \
    using CL = ChannelLayout<MB>;                                                            \
    const int grid = grid_for((total + 8 * CL::VPW - 1) / (8 * CL::VPW),                     \
                              8 * oversubscribed_waves(total / CL::VPW, 64LL * sm_count()));  \
    k_init<MB, float><<<grid, 256, 0, s>>>(llr, lambda0, v2c, c->d_var_edges, c->N, c->E, F, \
                                           list_out, count_out);                             \
  }
  NBFD_DISPATCH_M(c->m, NBFD_INIT)
#undef NBFD_INIT
  return cudaGetLastError();
}

// Tensor-core forms: tcgen05 where asked for, or by default where it measured faster (the FP32
// form's three operand parts per product; 942 against 989 us per 1024-frame launch, while the
// single-part BF16 / FP16 forms measured 25-35% slower on tcgen05)
bool tc_uses_tcgen05(int form) {
  if (form & NBFD_TCGEN05) return true;
  if (form & NBFD_MMA_SYNC) return false;
  return (form & 0xff) == NBFD_FORM_FP32_TC && var_tc5_available();
}

bool form_supported(int form, int m) {
  if (form & ~(0xff | NBFD_DECIDE_SYMBOL | NBFD_STORE_F16 | NBFD_UNFUSED | NBFD_TCGEN05 | NBFD_MMA_SYNC))
    return false;
  const bool symbol = (form & NBFD_DECIDE_SYMBOL) != 0;
  if (form & (NBFD_TCGEN05 | NBFD_MMA_SYNC)) {
    const int b = form & 0xff;
    if (b != NBFD_FORM_BF16_HGEMM && b != NBFD_FORM_FP16_HGEMM && b != NBFD_FORM_FP32_TC) return false;
    if ((form & NBFD_TCGEN05) && (form & NBFD_MMA_SYNC)) return false;
    if ((form & NBFD_TCGEN05) && !var_tc5_available()) return false;
  }
  if (stores_f16(form)) return (form & 0xff) == NBFD_FORM_FP32_FWHT && m == 8;
  switch (form & 0xff) {
    case NBFD_FORM_FP32_DIRECT:
    case NBFD_FORM_FP64_DIRECT:
      return !symbol;  // its M_v is evaluated only at the 3m read-out points
    case NBFD_FORM_FP32_FWHT:
      return true;
    case NBFD_FORM_BF16_HGEMM:
    case NBFD_FORM_FP16_HGEMM:
    case NBFD_FORM_FP32_TC:
      return m == 8;
    default:
      return false;
  }
}

cudaError_t launch_var(const nbfd_code *c, FrameSet fs, int form, const float *llr,
                       const float *c2v, float *v2c, uint16_t *sym, uint8_t *fsyn,
                       cudaStream_t s, int32_t *err, VarTune tune) {
  if (!form_supported(form, c->m)) return cudaErrorNotSupported;
  const bool symbol = (form & NBFD_DECIDE_SYMBOL) != 0;
  const int base = form & 0xff;
  if (base == NBFD_FORM_FP32_FWHT)
    return c->m == 8 ? launch_var_fwht8x2(c, fs, llr, c2v, v2c, sym, fsyn, err, s, symbol, tune,
                                          stores_f16(form))
                     : launch_var_fwht(c, fs, llr, c2v, v2c, sym, fsyn, err, s, symbol, tune);
  if (base == NBFD_FORM_BF16_HGEMM || base == NBFD_FORM_FP16_HGEMM || base == NBFD_FORM_FP32_TC)
    return tc_uses_tcgen05(form)
               ? launch_var_tc5(c, fs, base, llr, c2v, v2c, sym, fsyn, err, s, symbol, tune)
               : launch_var_tc(c, fs, base, llr, c2v, v2c, sym, fsyn, err, s, symbol, tune);
  const long long total = (long long)fs.n_static * c->N;
  const int per_sm = tune.blocks_per_sm > 0 ? tune.blocks_per_sm : 8;
  const bool fp64 = base == NBFD_FORM_FP64_DIRECT;
#define NBFD_VAR(MB)                                                                       \
  {                                                                                        \
    constexpr int Q = 1 << MB, R = Q < 8 ? Q : 8, VPW = 32 / (Q / R);                      \
    if (fp64) {                                                                            \
      const int grid = grid_for((total + 4 * VPW - 1) / (4 * VPW), 2 * per_sm);            \
      k_var_direct<MB, double><<<grid, 128, 0, s>>>(llr, c2v, v2c, sym, fsyn,              \
                                                    c->d_var_edges, c->d_edge_h, c->d_perm, \
                                                    c->N, c->E, fs);                       \
    } else {                                                                               \
      const int grid = grid_for((total + 8 * VPW - 1) / (8 * VPW), per_sm);                \
      k_var_direct<MB, float><<<grid, 256, 0, s>>>(llr, c2v, v2c, sym, fsyn,               \
                                                   c->d_var_edges, c->d_edge_h, c->d_perm, \
                                                   c->N, c->E, fs);                        \
    }                                                                                      \
  }
  NBFD_DISPATCH_M(c->m, NBFD_VAR)
#undef NBFD_VAR
  return cudaGetLastError();
}

cudaError_t launch_syndrome(const nbfd_code *c, int F, const uint16_t *sym, const uint8_t *fsyn,
                            uint16_t *fourier, uint16_t *exact, cudaStream_t s) {
  const long long total = (long long)F * c->M;
  const int grid = grid_for((total + 255) / 256, 8);
  k_syndrome<<<grid, 256, 0, s>>>(sym, fsyn, fourier, exact, c->d_edge_var, c->d_edge_h,
                                  c->d_gf_exp, c->d_gf_log, c->N, c->M, c->k, c->E, F);
  return cudaGetLastError();
}

cudaError_t launch_stop(const nbfd_code *c, FrameSet fs, const uint16_t *sym, const uint8_t *fsyn,
                        int iter, int max_iter, int32_t *next_list, int32_t *next_count,
                        uint8_t *ok, int32_t *iters, int32_t *stats, cudaStream_t s,
                        const int32_t *iter_dev) {
  const int grid = grid_for(fs.n_static, 16);
  return launch_dependent(k_stop, dim3(grid), dim3(128), 0, s, fs, sym, fsyn, c->d_edge_var,
                          c->d_edge_h, c->d_gf_exp, c->d_gf_log, c->q, c->N, c->M, c->k, c->E,
                          iter, iter_dev, max_iter, next_list, next_count, ok, iters, stats);
}

}  // namespace nbfd
