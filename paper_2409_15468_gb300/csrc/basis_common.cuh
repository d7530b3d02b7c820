// Device helpers shared by the basis kernels (FRSZ2 and cast formats).
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace cbg {

// Range of 32-value blocks handled by CTA c of G: balanced, starting at multiples of 4 blocks so
// that every bulk copy starts 16-byte aligned.
__device__ __forceinline__ void cta_block_range(int64_t nb, int G, int c, int64_t* b0, int64_t* b1) {
  const int64_t nu = (nb + 3) / 4;
  const int64_t u0 = nu * c / G, u1 = nu * (c + 1) / G;
  *b0 = u0 * 4 < nb ? u0 * 4 : nb;
  *b1 = u1 * 4 < nb ? u1 * 4 : nb;
}

// Slice y of `slices` holds vectors [floor(nvec y / slices), floor(nvec (y + 1) / slices)); the
// slice of vector v.
__device__ __forceinline__ int vector_slice(int v, int nvec, int slices) {
  int y = static_cast<int>(((int64_t)(v + 1) * slices - 1) / nvec);
  while (y + 1 < slices && (int64_t)nvec * (y + 1) / slices <= v) ++y;
  while (y > 0 && (int64_t)nvec * y / slices > v) --y;
  return y;
}

// The dots' final sums, in the CTA that arrives last: out[v] for every v < nvec is the sum of
// vector v's partials (partials[(y gx + x) nvec + v] over the gx CTAs x of its slice y). Warp w of
// `warps` takes vectors w, w + warps, w + 2 warps, ..., K at a time. Each sum is formed in
// warp_sum_strided's order (lane-strided sums, then the xor tree), so it is bit-identical to that;
// the K sums of a warp are independent, and the lane loop is unrolled U times (0: the compiler's
// choice), so that their loads and adds overlap.
// the FRSZ2 and integer-pipeline dots' shape (4 and 4 measured best against 1 and the compiler's
// unroll, 8 and 2, 2 and 8; the binary64 dot takes 2 and 8)
#ifndef CBG_DOT_SUM_K
#define CBG_DOT_SUM_K 4
#endif
#ifndef CBG_DOT_SUM_U
#define CBG_DOT_SUM_U 4
#endif
template <int K, int U>
__device__ __forceinline__ void slice_sums(const double* partials, int nvec, int gx, int slices, double* out,
                                           int warp, int warps) {
  const int lane = threadIdx.x & 31;
  const int mine = warp < nvec ? (nvec - warp + warps - 1) / warps : 0;  // vectors of this warp
  for (int c0 = 0; c0 < mine; c0 += K) {
    const double* p[K];
    double s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int v = warp + warps * (c0 + k < mine ? c0 + k : c0);  // past the end: a repeat, not stored
      p[k] = partials + (size_t)vector_slice(v, nvec, slices) * gx * nvec + v;
      s[k] = 0.0;
    }
    if constexpr (U == 0) {
      for (int i = lane; i < gx; i += 32) {
#pragma unroll
        for (int k = 0; k < K; ++k) s[k] += __ldcg(p[k] + (size_t)i * nvec);
      }
    } else {
#pragma unroll U
      for (int i = lane; i < gx; i += 32) {
#pragma unroll
        for (int k = 0; k < K; ++k) s[k] += __ldcg(p[k] + (size_t)i * nvec);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < K; ++k) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (c0 + k < mine) out[warp + warps * (c0 + k)] = s[k];
    }
  }
}

__device__ __forceinline__ bool gate_skip(const Gate& g) {
  if (g.stop && *(volatile const int*)g.stop) return true;
  if (g.need && !*(volatile const int*)g.need) return true;
  return false;
}

__device__ __forceinline__ int flag_read(const int* f) { return *(volatile const int*)f; }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// acc += a * b exactly: a 32x32 -> 64-bit signed product, then a 64-bit add. On sm_103a this form
// executes ~1.5 instructions per product, against ~2.5 for a fused mad.wide.s32 with a 64-bit
// accumulator (measured with varying operands).
__device__ __forceinline__ void mac_wide(long long& acc, int32_t a, int32_t b) {
  long long p;
  asm("mul.wide.s32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
  acc += p;
}

// *p += v on a shared-memory counter with acquire-release ordering at CTA scope; returns the old
// value. The warp whose increment completes a count sees every access the other warps made before
// theirs.
__device__ __forceinline__ unsigned atom_add_acq_rel_cta(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;"
               : "=r"(old)
               : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))), "r"(v)
               : "memory");
  return old;
}

// x / 2^d rounded to nearest (ties up) for |x| < 2^62 and d >= 0.
__device__ __forceinline__ long long round_shift_right(long long x, int d) {
  if (d <= 0) return x;
  if (d > 62) return 0;
  return (x + (1ll << (d - 1))) >> d;
}

// A finite double as th * 2^xb exactly (th carries the significand, at most 53 bits, and the sign).
__device__ __forceinline__ void split_double(double v, long long& th, int& xb) {
  const uint64_t u = static_cast<uint64_t>(__double_as_longlong(v));
  const int e = static_cast<int>((u >> 52) & 0x7FF);
  long long m = static_cast<long long>(u & ((1ull << 52) - 1));
  if (e) m |= 1ll << 52;
  th = (u >> 63) ? -m : m;
  xb = (e ? e : 1) - 1075;
}

// The sum over a warp of its lanes' th * 2^xb (|th| < 2^62), returned as S * 2^X on every lane.
// 2^M bounds the warp's largest term and X = M - 57: each term is rounded once to 2^X units
// (nearest, ties up; an error below 2^-58 of the largest term), and the rounded terms, each at most
// 2^57 in magnitude, add up exactly: three 21-bit slices summed by integer warp reductions, so
// the sum of the 32 terms needs no floating point at all.
__device__ __forceinline__ long long warp_fixed_sum(long long th, int xb, int& X) {
  const unsigned long long A = static_cast<unsigned long long>(th < 0 ? -th : th);
  const int mag = A ? xb + 64 - __clzll(static_cast<long long>(A)) : -(1 << 30);
  const int M = __reduce_max_sync(0xffffffffu, mag);
  X = M - 57;
  long long q = 0;
  if (A) {
    const int d = X - xb;
    if (d <= 0)
      q = static_cast<long long>(static_cast<unsigned long long>(th) << (-d));  // -d <= 57 - bitlength
    else if (d < 63)
      q = (th + (1ll << (d - 1))) >> d;  // |th| < 2^62: no overflow
  }
  const int lo = static_cast<int>(q & 0x1FFFFF), mid = static_cast<int>((q >> 21) & 0x1FFFFF);
  const int hi = static_cast<int>(q >> 42);  // |hi| <= 2^15
  const long long slo = __reduce_add_sync(0xffffffffu, lo);    // < 2^26
  const long long smid = __reduce_add_sync(0xffffffffu, mid);  // < 2^26
  const long long shi = __reduce_add_sync(0xffffffffu, hi);    // |.| <= 2^20
  return shi * (1ll << 42) + smid * (1ll << 21) + slo;
}

// Prefetch `bytes` (multiple of 16, 16-byte aligned) of global memory into L2 with the bulk-copy unit.
__device__ __forceinline__ void bulk_prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Sign-magnitude FRSZ2 code (sign bit NB-1, magnitude below it) to a two's complement integer.
template <int NB>
__device__ __forceinline__ int32_t code_to_int(uint32_t c) {
  const int32_t m = static_cast<int32_t>(c << (32 - NB)) >> 31;  // 0 or -1 from the sign bit
  return static_cast<int32_t>((c & ((1u << (NB - 1)) - 1u)) ^ static_cast<uint32_t>(m)) - m;
}

__device__ __forceinline__ int eff_exp(double x) {
  const int e = static_cast<int>((static_cast<uint64_t>(__double_as_longlong(x)) >> 52) & 0x7FF);
  return e > 1 ? e : 1;
}

// x rounded to the block fixed point with exponent ew (the block's largest effective IEEE
// exponent): W = round(|x| 2^{1075-ew}) with sign, |W| < 2^53, split as W1 * 2^27 + W0 with
// W0 in [0, 2^27) and |W1| <= 2^26.
__device__ __forceinline__ void to_block_fixed(double x, int ew, int32_t& w1, int32_t& w0) {
  const uint64_t u = static_cast<uint64_t>(__double_as_longlong(x));
  const int e = static_cast<int>((u >> 52) & 0x7FF);
  uint64_t m = u & ((1ull << 52) - 1);
  if (e) m |= 1ull << 52;
  const int sh = ew - (e > 1 ? e : 1);
  uint64_t mag;
  if (sh == 0) mag = m;
  else if (sh < 64) mag = ((m >> (sh - 1)) + 1) >> 1;  // round half up
  else mag = 0;
  const int64_t W = (u >> 63) ? -static_cast<int64_t>(mag) : static_cast<int64_t>(mag);
  w1 = static_cast<int32_t>(W >> 27);
  w0 = static_cast<int32_t>(W & ((1ll << 27) - 1));
}

}  // namespace cbg
