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

// Integer dot of one block of 32 bfloat16 values (64 bytes, the layout of an l = 16 block) with the
// thread's W registers, in the order and with the bank rotation of block_dot<16>. The block goes on
// a fixed point on the fly. With E the largest exponent field of the block, every value v becomes
// the integer c = v 2^(148 - E), |c| < 2^22: an 8-bit significand lands on an integer exactly when
// its exponent field is at least E - 14.
// - Pass 1 finds E and the smallest nonzero magnitude. When a nonzero value lies lower than
//   E - 14, or E is below 21 (the scale 2^(148 - E) then leaves the binary32 range), the block
//   takes the wide path instead, as long as every nonzero value lies within 54 binades of the
//   largest: c = M 2^(max(e, 1) - E + 54) < 2^62 (M the 8-bit significand, e the exponent field,
//   E now the effective largest, at least 1), so v = c 2^(E - 188); c in 31-bit pieces, four
//   exact products; it returns 1 with the exact sum tot in units of 2^(E + ew - 1263). It returns
//   2, leaving the block to the caller's FP64 path, when a value lies further down or the block
//   holds an infinity or NaN.
// - Pass 2 forms each c with one binary32 FMA, v 2^(148 - E) + 1.5 2^23, exact in the binade
//   [2^23, 2^24), whose bits minus those of 1.5 2^23 are c. The products are block_dot's.
// On 0 the block's sum is (a1 2^27 + a0) 2^(E + ew - 1223), with W in units of 2^(ew - 1075).
__device__ __forceinline__ int block_dot_bf16(const uint32_t* cw, int t, const int32_t (&W1)[32],
                                              const int32_t (&W0)[32], long long& a1, long long& a0,
                                              __int128& tot, int& E) {
  const uint4* c4 = reinterpret_cast<const uint4*>(cw);
  uint32_t mx = 0, mn = 0xFFFFFFFFu;  // largest magnitude bits; smallest nonzero one, minus 1
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint4 q = c4[(c + (t >> 1)) & 3];
    const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const uint32_t lo = wv[h] & 0x7FFFu, hi = (wv[h] >> 16) & 0x7FFFu;
      mx = max(mx, max(lo, hi));
      mn = min(mn, min(lo - 1u, hi - 1u));  // a zero wraps to the largest value
    }
  }
  a1 = a0 = 0;
  E = static_cast<int>(mx >> 7);
  if (mx == 0) return 0;  // every value is zero
  const int emin = max(static_cast<int>((mn + 1u) >> 7), 1);
  if (E > 254) return 2;
  if (E < 21 || emin + 14 < E) {
    E = max(E, 1);
    if (emin + 54 < E) return 2;
    // the wide path: c = M 2^(max(e, 1) - E + 54) < 2^62 in 31-bit pieces, four exact products
    long long s11 = 0, s10 = 0, s01 = 0, s00 = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint4 q = c4[(c + (t >> 1)) & 3];
      const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t h = (k & 1) ? wv[k >> 1] >> 16 : wv[k >> 1] & 0xFFFFu;
        const int e = static_cast<int>((h >> 7) & 0xFFu);
        const uint64_t M = (h & 0x7Fu) | (e ? 0x80u : 0u);
        const uint64_t cc = M ? M << (max(e, 1) - E + 54) : 0;
        const int32_t sg = (h & 0x8000u) ? -1 : 0;
        const int32_t c1 = (static_cast<int32_t>(cc >> 31) ^ sg) - sg;
        const int32_t c0 = (static_cast<int32_t>(cc & 0x7FFFFFFFu) ^ sg) - sg;
        mac_wide(s11, c1, W1[8 * c + k]);
        mac_wide(s10, c1, W0[8 * c + k]);
        mac_wide(s01, c0, W1[8 * c + k]);
        mac_wide(s00, c0, W0[8 * c + k]);
      }
    }
    tot = (static_cast<__int128>(s11) << 58) + (static_cast<__int128>(s10) << 31) +
          (static_cast<__int128>(s01) << 27) + static_cast<__int128>(s00);
    return 1;
  }
  const float S = __uint_as_float(static_cast<uint32_t>(275 - E) << 23);  // 2^(148 - E)
  constexpr float kMagic = 12582912.0f;                                   // 1.5 2^23
  constexpr int32_t kMagicBits = 0x4B400000;
  long long a1e = 0, a0e = 0, a1o = 0, a0o = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint4 q = c4[(c + (t >> 1)) & 3];
    const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int32_t lo = __float_as_int(fmaf(__uint_as_float(wv[h] << 16), S, kMagic)) - kMagicBits;
      const int32_t hi = __float_as_int(fmaf(__uint_as_float(wv[h] & 0xFFFF0000u), S, kMagic)) - kMagicBits;
      mac_wide(a1e, lo, W1[8 * c + 2 * h]);
      mac_wide(a0e, lo, W0[8 * c + 2 * h]);
      mac_wide(a1o, hi, W1[8 * c + 2 * h + 1]);
      mac_wide(a0o, hi, W0[8 * c + 2 * h + 1]);
    }
  }
  a1 = a1e + a1o;
  a0 = a0e + a0o;
  return 0;
}

// Integer dot of one block of 32 binary32 values (128 bytes, the layout of an l = 32 block) with
// the thread's W registers, in the order and with the bank rotation of block_dot<32>. The block
// goes on a fixed point on the fly. With E the largest exponent field of the block, a normal value
// with significand M (24 bits, leading 1 included) and exponent field e becomes the integer
// c = M 2^(e - E + 38) < 2^62, so v = c 2^(E - 188).
// - Pass 1 finds E and the smallest nonzero magnitude. It returns false, leaving the block to the
//   caller's FP64 path, when a nonzero value lies more than 38 binades below the largest, when
//   the block holds a subnormal, or when it holds an infinity or NaN.
// - Pass 2 splits each c into 31-bit pieces, c1 = c >> 31 and c0 = c mod 2^31, signs them, and
//   forms the four exact products c1 W1, c1 W0, c0 W1 and c0 W0 in 64-bit sums.
// On true, tot is the block's exact sum in units of 2^(E + ew - 1263) (|tot| < 2^121), with W in
// units of 2^(ew - 1075).
__device__ __forceinline__ bool block_dot_f32(const uint32_t* cw, int t, const int32_t (&W1)[32],
                                              const int32_t (&W0)[32], __int128& tot, int& E) {
  const uint4* c4 = reinterpret_cast<const uint4*>(cw);
  uint32_t mx = 0, mn = 0xFFFFFFFFu;  // largest magnitude bits; smallest nonzero one, minus 1
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint4 q = c4[(c + t) & 7];
    const uint32_t f[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t m = f[j] & 0x7FFFFFFFu;
      mx = max(mx, m);
      mn = min(mn, m - 1u);  // a zero wraps to the largest value
    }
  }
  tot = 0;
  E = static_cast<int>(mx >> 23);
  if (mx == 0) return true;  // every value is zero
  const int emin = static_cast<int>((mn + 1u) >> 23);
  if (E > 254 || emin == 0 || emin + 38 < E) return false;
  long long s11 = 0, s10 = 0, s01 = 0, s00 = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint4 q = c4[(c + t) & 7];
    const uint32_t f[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = static_cast<int>((f[j] >> 23) & 0xFFu);
      // a zero has e = 0: no leading 1 and a zero shift, so c = 0
      const uint64_t M = (f[j] & 0x7FFFFFu) | (e ? 0x800000u : 0u);
      const uint64_t cc = M << (e ? e - E + 38 : 0);
      const int32_t sg = static_cast<int32_t>(f[j]) >> 31;  // 0 or -1
      const int32_t c1 = (static_cast<int32_t>(cc >> 31) ^ sg) - sg;
      const int32_t c0 = (static_cast<int32_t>(cc & 0x7FFFFFFFu) ^ sg) - sg;
      const int r = 4 * c + j;
      mac_wide(s11, c1, W1[r]);
      mac_wide(s10, c1, W0[r]);
      mac_wide(s01, c0, W1[r]);
      mac_wide(s00, c0, W0[r]);
    }
  }
  // c W = (c1 2^31 + c0)(W1 2^27 + W0): each 64-bit sum is below 2^63 (32 terms below 2^58)
  tot = (static_cast<__int128>(s11) << 58) + (static_cast<__int128>(s10) << 31) +
        (static_cast<__int128>(s01) << 27) + static_cast<__int128>(s00);
  return true;
}

// tot rounded once to 61 bits: returns th with tot = th 2^u (nearest, ties up), u >= 0 in *u.
__device__ __forceinline__ long long round_i128(__int128 tot, int& u) {
  const unsigned __int128 A = tot < 0 ? -static_cast<unsigned __int128>(tot) : static_cast<unsigned __int128>(tot);
  const uint64_t hi = static_cast<uint64_t>(A >> 64), lo = static_cast<uint64_t>(A);
  const int bl = hi ? 128 - __clzll(static_cast<long long>(hi)) : (lo ? 64 - __clzll(static_cast<long long>(lo)) : 0);
  u = bl > 61 ? bl - 61 : 0;
  return u ? static_cast<long long>((tot + (static_cast<__int128>(1) << (u - 1))) >> u) : static_cast<long long>(tot);
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
