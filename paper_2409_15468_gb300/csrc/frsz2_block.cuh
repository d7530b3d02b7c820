// FRSZ2 block arithmetic shared by the codec, the streamed basis kernels and the on-chip cycle:
// the code of one value (Compression steps 2-5) and the exact integer dot of one block's codes
// with a block-fixed-point copy of w.
#pragma once

#include "basis_common.cuh"

namespace cbg {

// Code of one value (Compression steps 2-5) given the block's effective maximum exponent.
template <int L>
__device__ __forceinline__ uint32_t make_code(uint64_t u, int ebar) {
  const int e = static_cast<int>((u >> 52) & 0x7FF);
  uint64_t m = u & ((1ull << 52) - 1);
  if (e) m |= 1ull << 52;                     // step 2: explicit leading 1 (none for subnormals)
  const int k = ebar - (e > 1 ? e : 1);       // step 3: number of prefixed zeros
  const int sh = k + 54 - L;                  // steps 3-5: keep the first l-1 significand bits
  const uint32_t S = sh < 64 ? static_cast<uint32_t>(m >> sh) : 0u;
  return (static_cast<uint32_t>(u >> 63) << (L - 1)) | S;  // step 4: sign on the left
}

// Integer dot of one block's codes with the thread's W registers; four independent accumulator
// chains (even/odd values for each half of W).
template <int L>
__device__ __forceinline__ void block_dot(const uint32_t* cw, int t, const int32_t (&W1)[32], const int32_t (&W0)[32],
                                          long long& a1, long long& a0) {
  long long a1e = 0, a0e = 0, a1o = 0, a0o = 0;
  if (L == 32) {
    // 8 chunks of 16 bytes, visited in an order rotated by t so that the 8 threads of a
    // shared-memory phase hit distinct banks; W was loaded in the same rotated order.
    const uint4* c4 = reinterpret_cast<const uint4*>(cw);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const uint4 q = c4[(c + t) & 7];
      const int32_t s0 = code_to_int<32>(q.x), s1 = code_to_int<32>(q.y);
      const int32_t s2 = code_to_int<32>(q.z), s3 = code_to_int<32>(q.w);
      mac_wide(a1e, s0, W1[4 * c + 0]);
      mac_wide(a0e, s0, W0[4 * c + 0]);
      mac_wide(a1o, s1, W1[4 * c + 1]);
      mac_wide(a0o, s1, W0[4 * c + 1]);
      mac_wide(a1e, s2, W1[4 * c + 2]);
      mac_wide(a0e, s2, W0[4 * c + 2]);
      mac_wide(a1o, s3, W1[4 * c + 3]);
      mac_wide(a0o, s3, W0[4 * c + 3]);
    }
  } else if (L == 16) {
    // 4 chunks of 8 codes, rotated by t/2 (two threads share a 128-byte bank row)
    const uint4* c4 = reinterpret_cast<const uint4*>(cw);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint4 q = c4[(c + (t >> 1)) & 3];
      const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int32_t lo = code_to_int<16>(wv[h] & 0xFFFFu);
        const int32_t hi = code_to_int<16>(wv[h] >> 16);
        mac_wide(a1e, lo, W1[8 * c + 2 * h]);
        mac_wide(a0e, lo, W0[8 * c + 2 * h]);
        mac_wide(a1o, hi, W1[8 * c + 2 * h + 1]);
        mac_wide(a0o, hi, W0[8 * c + 2 * h + 1]);
      }
    }
  } else {
    // 21 words; word i of thread t is in bank (21 t + i) mod 32, distinct across a warp
    uint32_t wd[22];
#pragma unroll
    for (int i = 0; i < 21; ++i) wd[i] = cw[i];
    wd[21] = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int bit = 21 * k, a = bit >> 5, o = bit & 31;
      const int32_t s = code_to_int<21>(__funnelshift_r(wd[a], wd[a + 1], o) & 0x1FFFFFu);
      if (k & 1) {
        mac_wide(a1o, s, W1[k]);
        mac_wide(a0o, s, W0[k]);
      } else {
        mac_wide(a1e, s, W1[k]);
        mac_wide(a0e, s, W0[k]);
      }
    }
  }
  a1 = a1e + a1o;
  a0 = a0e + a0o;
}

// A binary16 value (its bit pattern in bits 0-15) below 2 in magnitude as an exact integer in
// units of 2^-24: m 2^(E-1) for a normal value (E the exponent field, m the significand with its
// hidden bit), m for a subnormal one; |V| < 2^25. emax receives the largest exponent field seen: a
// value with E > 15 (|v| >= 2) does not fit and its block is summed on the FP64 path instead.
__device__ __forceinline__ int32_t fp16_fixed(uint32_t h, uint32_t& emax) {
  const uint32_t e = (h >> 10) & 0x1Fu;
  emax = max(emax, e);
  const uint32_t m = (h & 0x3FFu) | (e != 0u ? 0x400u : 0u);
  const uint32_t mag = m << (e != 0u ? e - 1u : 0u);
  const uint32_t s = 0u - ((h >> 15) & 1u);  // 0 or all ones
  return static_cast<int32_t>((mag ^ s) - s);
}

// Integer dot of one block of 32 binary16 values (64 bytes, the layout of an l = 16 block) with
// the thread's W registers, in the order and with the bank rotation of block_dot<16>.
__device__ __forceinline__ void block_dot_fp16(const uint32_t* cw, int t, const int32_t (&W1)[32],
                                               const int32_t (&W0)[32], long long& a1, long long& a0,
                                               uint32_t& emax) {
  long long a1e = 0, a0e = 0, a1o = 0, a0o = 0;
  const uint4* c4 = reinterpret_cast<const uint4*>(cw);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint4 q = c4[(c + (t >> 1)) & 3];
    const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int32_t lo = fp16_fixed(wv[h], emax);
      const int32_t hi = fp16_fixed(wv[h] >> 16, emax);
      mac_wide(a1e, lo, W1[8 * c + 2 * h]);
      mac_wide(a0e, lo, W0[8 * c + 2 * h]);
      mac_wide(a1o, hi, W1[8 * c + 2 * h + 1]);
      mac_wide(a0o, hi, W0[8 * c + 2 * h + 1]);
    }
  }
  a1 = a1e + a1o;
  a0 = a0e + a0o;
}

// Register slot r of the thread's W holds block value w_index(L, t, r) (the order block_dot reads).
template <int L>
__device__ __forceinline__ int w_index(int t, int r) {
  const int c = r >> 2, q = r & 3;
  if (L == 32) return 4 * ((c + t) & 7) + q;
  if (L == 16) return 8 * (((c >> 1) + (t >> 1)) & 3) + 4 * (c & 1) + q;
  return r;
}

}  // namespace cbg
