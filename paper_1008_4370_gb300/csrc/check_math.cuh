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

// Entries of a lane gathered together: up to 4 for row weights up to 6 (measured on GB300: the
// GF(64) k = 6 check goes from 0.77 to 0.99 of HBM bandwidth, GF(32) k = 6 from 0.74 to 0.98).
// From k = 8 on, one entry's k loads already keep the lane busy and the registers of a group cost
// occupancy (GF(64) k = 8: 0.87 with one entry, 0.75 with two), so entries go one at a time --
// for k = 8 still gathered before any arithmetic (0.87, against 0.69 with the loads interleaved
// with the magnitude and sign work as for k > 8, where that form needs fewer registers).
__host__ __device__ constexpr int check_gather_group(int epl, int kmax) {
  return kmax > 6 ? 1 : (epl < 4 ? epl : 4);
}

// One entry's outputs from its k gathered inputs x[e] (words e * Q + pos[e]): leave-one-out sums of the
// log-magnitudes by prefix and suffix passes, the XOR of the other signs.
template <int Q, int KMAX, typename W>
__device__ __forceinline__ void check_entry_store(W *s, int k, const float (&x)[KMAX],
                                                  const int (&pos)[KMAX]) {
  float mag[KMAX];
  uint32_t sg[KMAX];
  uint32_t sx = 0;
#pragma unroll
  for (int e = 0; e < KMAX; ++e) {
    if (e < k) {
      mag[e] = fabsf(x[e]);
      sg[e] = __float_as_uint(x[e]) & 0x80000000u;
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

// The index-map words of check c at a lane's EPL entries z0 .. z0 + EPL - 1: byte j of pw[e]
// holds H_e (z0 + j) for edge e (they do not depend on the messages, so a caller may load the
// next check's words while it works on the current one).
template <int Q, int EPL, int KMAX>
struct CheckIndex {
  uint32_t pw[KMAX][(EPL + 3) / 4];
};
// One edge's index-map word(s) from its label h.
template <int Q, int EPL>
__device__ __forceinline__ void check_index_row(uint32_t (&w)[(EPL + 3) / 4], int h, int z0,
                                                const uint8_t *__restrict__ perm) {
  const uint8_t *row = perm + h * Q + z0;
  if constexpr (EPL == 8) {
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(row));
    w[0] = v.x;
    w[1] = v.y;
  } else if constexpr (EPL == 4) {
    w[0] = __ldg(reinterpret_cast<const uint32_t *>(row));
  } else if constexpr (EPL == 2) {
    w[0] = __ldg(reinterpret_cast<const uint16_t *>(row));
  } else {
    uint32_t x = 0;
#pragma unroll
    for (int jj = 0; jj < EPL; ++jj) x |= (uint32_t)__ldg(row + jj) << (8 * jj);
    w[0] = x;
  }
}

template <int Q, int EPL, int KMAX>
__device__ __forceinline__ void check_index_load(CheckIndex<Q, EPL, KMAX> &ix, int c, int k, int z0,
                                                 const uint8_t *__restrict__ edge_h,
                                                 const uint8_t *__restrict__ perm) {
  auto &pw = ix.pw;
  if constexpr (KMAX == 4 || KMAX == 8 || KMAX == 16) {
    if (k == KMAX) {  // the check's KMAX labels as one aligned 4-, 8- or 16-byte load
      uint32_t hw[KMAX / 4];
      const uint8_t *p = edge_h + (size_t)c * KMAX;
      if constexpr (KMAX == 4) {
        hw[0] = __ldg(reinterpret_cast<const uint32_t *>(p));
      } else if constexpr (KMAX == 8) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        hw[0] = v.x;
        hw[1] = v.y;
      } else {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        hw[0] = v.x;
        hw[1] = v.y;
        hw[2] = v.z;
        hw[3] = v.w;
      }
#pragma unroll
      for (int e = 0; e < KMAX; ++e)
        check_index_row<Q, EPL>(pw[e], (hw[e >> 2] >> (8 * (e & 3))) & 0xff, z0, perm);
      return;
    }
  }
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
      } else if constexpr (EPL == 2) {
        pw[e][0] = __ldg(reinterpret_cast<const uint16_t *>(row));
      } else {
        uint32_t w = 0;
#pragma unroll
        for (int jj = 0; jj < EPL; ++jj) w |= (uint32_t)__ldg(row + jj) << (8 * jj);
        pw[e][0] = w;
      }
    }
  }
}

// The lane's entries of check (slots at s[e * Q + z], Gamma form) in place, given its index words.
// MAXG caps the gather group (1 for a caller whose register budget has no room for it).
template <int Q, int EPL, int KMAX, typename W, int MAXG = EPL>
__device__ __forceinline__ void check_lane_apply(W *s, int k, const CheckIndex<Q, EPL, KMAX> &ix) {
  const auto &pw = ix.pw;
  // The words of a lane's entries are read and written by that lane alone, so a group of G
  // entries is gathered before any of them is written back: the compiler cannot prove that a
  // store of one entry misses the next entry's loads, and would otherwise serialise the entries.
  // Both branches compute every output with the same operations in the same order.
  constexpr int G = check_gather_group(EPL, KMAX) < MAXG ? check_gather_group(EPL, KMAX) : MAXG;
  if constexpr (G == 1 && (KMAX > 8 || MAXG == 1)) {  // one entry at a time, loads interleaved
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
  } else {
#pragma unroll
    for (int j0 = 0; j0 < EPL; j0 += G) {
      float x[G][KMAX];
      int pos[G][KMAX];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int j = j0 + g;
#pragma unroll
        for (int e = 0; e < KMAX; ++e) {
          if (e < k) {
            pos[g][e] = static_cast<int>((pw[e][j >> 2] >> (8 * (j & 3))) & 0xff);
            x[g][e] = msg_load<W>(s[e * Q + pos[g][e]]);
          }
        }
      }
#pragma unroll
      for (int g = 0; g < G; ++g) check_entry_store<Q, KMAX, W>(s, k, x[g], pos[g]);
    }
  }
}

template <int Q, int EPL, int KMAX, typename W, int MAXG = EPL>
__device__ __forceinline__ void check_lane_inplace(W *s, int c, int k, int z0,
                                                   const uint8_t *__restrict__ edge_h,
                                                   const uint8_t *__restrict__ perm) {
  CheckIndex<Q, EPL, KMAX> ix;
  check_index_load<Q, EPL, KMAX>(ix, c, k, z0, edge_h, perm);
  check_lane_apply<Q, EPL, KMAX, W, MAXG>(s, k, ix);
}

}  // namespace nbfd
