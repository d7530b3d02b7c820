// Decoding of stored basis values to FP64 with integer operations only (no FP64 conversion
// instruction, so none of GB300's scarce FP64 issue slots): the FRSZ2 decompression steps of the
// Decompression subsection and the widening of the cast formats, subnormals included.
#pragma once

#include "common.cuh"

namespace cbg {

// Value k of an FRSZ2 vector (exponent words `exps`, code words `codes`), l = L.
template <int L>
__device__ __forceinline__ double frsz2_decode(const uint32_t* __restrict__ exps, const uint32_t* __restrict__ codes,
                                               int64_t k) {
  const int64_t b = k >> 5;
  const int i = static_cast<int>(k & 31);
  const uint32_t emax = exps[b];  // step 1
  uint32_t c;
  if (L == 32) {
    c = codes[b * 32 + i];
  } else if (L == 16) {
    c = reinterpret_cast<const uint16_t*>(codes)[b * 32 + i];
  } else {
    const int bit = 21 * i, a = bit >> 5;
    const uint32_t lo = codes[b * 21 + a];
    const uint32_t hi = a + 1 < 21 ? codes[b * 21 + a + 1] : 0u;
    c = __funnelshift_r(lo, hi, bit & 31) & 0x1FFFFFu;
  }
  const uint64_t s = c >> (L - 1);  // step 2: sign and significand
  const uint32_t S = c & ((1u << (L - 1)) - 1u);
  if (S == 0) return __longlong_as_double(static_cast<long long>(s << 63));
  const int ebar = emax > 1 ? static_cast<int>(emax) : 1;
  const int k0 = __clz(S) - (32 - (L - 1));  // step 2: inserted zeros
  const int p = L - 2 - k0;                   // position of the leading 1
  const int e = ebar - k0;                    // step 3: e = e_max - k
  uint64_t bits;
  if (e >= 1) {  // step 4: reassemble; the leading 1 becomes implicit again
    bits = (s << 63) | (static_cast<uint64_t>(e) << 52) | (static_cast<uint64_t>(S ^ (1u << p)) << (52 - p));
  } else {       // below the normal range: an IEEE subnormal S * 2^(ebar - 1023 - (l-2))
    bits = (s << 63) | (static_cast<uint64_t>(S) << (ebar + 53 - L));
  }
  return __longlong_as_double(static_cast<long long>(bits));
}

// Widening of IEEE binary32 / binary16 bit patterns to FP64 (bfloat16 is the high half of a
// binary32).
__device__ __forceinline__ double widen_f32(uint32_t f) {
  const uint32_t e = (f >> 23) & 0xFFu, m = f & 0x7FFFFFu;
  const uint64_t sgn = static_cast<uint64_t>(f >> 31) << 63;
  uint64_t d;
  if (e != 0) {
    d = sgn | (static_cast<uint64_t>(e + 896) << 52) | (static_cast<uint64_t>(m) << 29);
  } else if (m == 0) {
    d = sgn;
  } else {  // subnormal m 2^-149: normalise with the position p of its leading 1
    const int p = 31 - __clz(m);
    d = sgn | (static_cast<uint64_t>(p + 874) << 52) | (static_cast<uint64_t>(m ^ (1u << p)) << (52 - p));
  }
  return __longlong_as_double(static_cast<long long>(d));
}

__device__ __forceinline__ double widen_f16(uint32_t h) {
  const uint32_t e = (h >> 10) & 0x1Fu, m = h & 0x3FFu;
  const uint64_t sgn = static_cast<uint64_t>((h >> 15) & 1u) << 63;
  uint64_t d;
  if (e != 0) {
    d = sgn | (static_cast<uint64_t>(e + 1008) << 52) | (static_cast<uint64_t>(m) << 42);
  } else if (m == 0) {
    d = sgn;
  } else {  // subnormal m 2^-24
    const int p = 31 - __clz(m);
    d = sgn | (static_cast<uint64_t>(p + 999) << 52) | (static_cast<uint64_t>(m ^ (1u << p)) << (52 - p));
  }
  return __longlong_as_double(static_cast<long long>(d));
}

}  // namespace cbg
