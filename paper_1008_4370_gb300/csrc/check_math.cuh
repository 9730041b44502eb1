// CHECK TO VARIABLE (Section 3.2) for the entries of one lane: the k slots of check c sit in
// shared memory at s[e * Q + z] (Gamma form); the lane owns the EPL consecutive entries z0 ..
// z0 + EPL - 1 of the permuted frame. It gathers H_e z of every slot e through the index map row
// of h_ce, forms the leave-one-out sums of the log-magnitudes (prefix and suffix passes: no
// subtraction, so +inf magnitudes stay exact) and the XOR of the signs, and writes output H_e z of
// slot e back to the same word (z -> H_e z is a bijection: each word has one reader and writer).
// Shared by the check kernel and the cluster tail kernel, so both compute bit-identical messages.
#pragma once

#include <cstdint>

#include "device_common.cuh"

namespace nbfd {

template <int Q, int EPL, int KMAX, typename W>
__device__ __forceinline__ void check_lane_inplace(W *s, int c, int k, int z0,
                                                   const uint8_t *__restrict__ edge_h,
                                                   const uint8_t *__restrict__ perm) {
  // index maps of the k edges at this lane's EPL entries
  uint32_t pw[KMAX][(EPL + 3) / 4];
#pragma unroll
  for (int e = 0; e < KMAX; ++e) {
    if (e < k) {
      const int h = __ldg(edge_h + (size_t)c * k + e);
      const uint8_t *row = perm + h * Q + z0;
      if constexpr (EPL == 8) {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(row));
        pw[e][0] = w.x;
        pw[e][1] = w.y;
      } else if constexpr (EPL == 4) {
        pw[e][0] = __ldg(reinterpret_cast<const uint32_t *>(row));
      } else {
        uint32_t w = 0;
#pragma unroll
        for (int jj = 0; jj < EPL; ++jj) w |= (uint32_t)__ldg(row + jj) << (8 * jj);
        pw[e][0] = w;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < EPL; ++j) {
    float mag[KMAX];
    uint32_t sg[KMAX];
    int pos[KMAX];
    uint32_t sx = 0;
#pragma unroll
    for (int e = 0; e < KMAX; ++e) {
      if (e < k) {
        pos[e] = (pw[e][j >> 2] >> (8 * (j & 3))) & 0xff;
        const float x = msg_load<W>(s[e * Q + pos[e]]);
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
        s[e * Q + pos[e]] = msg_store<W>(__uint_as_float(__float_as_uint(o) | (sx ^ sg[e])));
      }
    }
  }
}

}  // namespace nbfd
