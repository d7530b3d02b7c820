// Fused basis kernels: the classical Gram-Schmidt projections h = V^T w and the update
// w -= V h of Fig. 1 step 5 (and steps 8 and 17), reading the stored Krylov basis and decoding
// it in registers.
//
// FRSZ2 path (GB300-specific design). An FRSZ2 block is block fixed point: value k of block b
// of vector i is s_{i,k} * 2^{q_{i,b}} with s a signed integer of l-1 magnitude bits (Eq. 2).
// GB300 runs FP64 at ~1.9 operations per clock per SM (conversions to FP64 included) but 32x32->64
// integer multiply-adds at ~57, so the kernels keep the per-element work on the integer pipe:
//   dot:    sum_{k in b} s_{i,k} w_k is formed exactly as an integer against a 54-bit block-fixed-
//           point copy W of w (W = round(w / 2^{p_b}), p_b from the block's largest exponent),
//           then converted once per (vector, block) and accumulated in FP64 across blocks.
//   update: sum_i s_{i,k} h_i 2^{q_{i,b}} is formed exactly as an integer against a 54-bit
//           fixed-point copy of the per-(vector, block) coefficients h_i 2^{q_{i,b}}, scaled to
//           the block's largest term, and converted once per element.
// The basis is streamed with 1D bulk copies (TMA) into a multi-stage shared-memory ring guarded
// by mbarriers with bounded waits.
//
// Cast formats (fp64, fp32, fp16, bf16) widen to FP64 with integer bit manipulation and use one
// FP64 FMA per element and vector, so they are bound by the FP64 pipe on GB300.
#include <algorithm>
#include <cstdio>

#include "common.cuh"
#include "kernels.cuh"

namespace cbg {

// ------------------------------------------------------------------------------------------------
// Shared helpers
// ------------------------------------------------------------------------------------------------

// Range of 32-value blocks handled by CTA c of G: balanced, starting at multiples of 4 blocks so
// that every bulk copy starts 16-byte aligned.
__device__ __forceinline__ void cta_block_range(int64_t nb, int G, int c, int64_t* b0, int64_t* b1) {
  const int64_t nu = (nb + 3) / 4;
  const int64_t u0 = nu * c / G, u1 = nu * (c + 1) / G;
  *b0 = u0 * 4 < nb ? u0 * 4 : nb;
  *b1 = u1 * 4 < nb ? u1 * 4 : nb;
}

__device__ __forceinline__ bool gate_skip(const Gate& g) {
  if (g.stop && *(volatile const int*)g.stop) return true;
  if (g.need && !*(volatile const int*)g.need) return true;
  return false;
}

// Sign-magnitude FRSZ2 code (sign bit nb-1, magnitude below it) to a two's complement integer.
template <int NB>
__device__ __forceinline__ int32_t code_to_int(uint32_t c) {
  const int32_t m = static_cast<int32_t>(c << (32 - NB)) >> 31;  // 0 or -1 from the sign bit
  return static_cast<int32_t>((c & ((1u << (NB - 1)) - 1u)) ^ static_cast<uint32_t>(m)) - m;
}

// w_k rounded to the block fixed point with exponent ew (the block's largest effective IEEE
// exponent): W = round(|w| 2^{1075-ew}) with sign, |W| <= 2^53, split as W1 * 2^27 + W0,
// W0 in [0, 2^27).
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

__device__ __forceinline__ int eff_exp(double x) {
  const int e = static_cast<int>((static_cast<uint64_t>(__double_as_longlong(x)) >> 52) & 0x7FF);
  return e > 1 ? e : 1;
}

// ------------------------------------------------------------------------------------------------
// FRSZ2 dot: one thread per 32-value block
// ------------------------------------------------------------------------------------------------

template <int L>
struct DotCfg {
  static constexpr int kThreads = 128;                 // = blocks per tile
  static constexpr int kStages = 3;
  static constexpr int kRed = 8;                       // vectors per deferred CTA reduction
  static constexpr int kCodeBytes = kThreads * L * 4;  // one vector's codes for a tile
  static constexpr int kExpBytes = kThreads * 4;
  static constexpr int kStageBytes = kCodeBytes + kExpBytes;
  static constexpr int kRedBytes = 2 * kRed * kThreads * 8;
  // dynamic smem: stages | red | hpart[nvec] | mbarriers + flags
  static size_t smem_bytes(int nvec) {
    return (size_t)kStages * kStageBytes + kRedBytes + (size_t)(nvec + 1) * 8 + kStages * 8 + 16;
  }
};

// Integer dot of one block's codes (in shared memory) with the thread's W registers, l = 32.
// The 8 chunks of 16 bytes are visited in an order rotated by the thread index so that the 8
// threads of a shared-memory phase hit distinct banks; W was loaded in the same rotated order.
__device__ __forceinline__ void block_dot32(const uint32_t* cw, int t, const int32_t (&W1)[32],
                                            const int32_t (&W0)[32], long long& a1, long long& a0) {
  const uint4* c4 = reinterpret_cast<const uint4*>(cw);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint4 q = c4[(c + t) & 7];
    const int32_t s0 = code_to_int<32>(q.x), s1 = code_to_int<32>(q.y);
    const int32_t s2 = code_to_int<32>(q.z), s3 = code_to_int<32>(q.w);
    a1 += (long long)s0 * W1[4 * c + 0];
    a0 += (long long)s0 * W0[4 * c + 0];
    a1 += (long long)s1 * W1[4 * c + 1];
    a0 += (long long)s1 * W0[4 * c + 1];
    a1 += (long long)s2 * W1[4 * c + 2];
    a0 += (long long)s2 * W0[4 * c + 2];
    a1 += (long long)s3 * W1[4 * c + 3];
    a0 += (long long)s3 * W0[4 * c + 3];
  }
}

// l = 16: 4 chunks of 8 codes, rotated by t/2 (two threads share a 128-byte bank row).
__device__ __forceinline__ void block_dot16(const uint32_t* cw, int t, const int32_t (&W1)[32],
                                            const int32_t (&W0)[32], long long& a1, long long& a0) {
  const uint4* c4 = reinterpret_cast<const uint4*>(cw);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint4 q = c4[(c + (t >> 1)) & 3];
    const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int32_t lo = code_to_int<16>(wv[h] & 0xFFFFu);
      const int32_t hi = code_to_int<16>(wv[h] >> 16);
      a1 += (long long)lo * W1[8 * c + 2 * h];
      a0 += (long long)lo * W0[8 * c + 2 * h];
      a1 += (long long)hi * W1[8 * c + 2 * h + 1];
      a0 += (long long)hi * W0[8 * c + 2 * h + 1];
    }
  }
}

// l = 21: 21 words per block; word i of thread t sits in bank (21 t + i) mod 32, distinct across a
// warp, so plain 32-bit loads are conflict free. Codes straddling two words use a funnel shift.
__device__ __forceinline__ void block_dot21(const uint32_t* cw, const int32_t (&W1)[32], const int32_t (&W0)[32],
                                            long long& a1, long long& a0) {
  uint32_t wd[22];
#pragma unroll
  for (int i = 0; i < 21; ++i) wd[i] = cw[i];
  wd[21] = 0;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const int bit = 21 * k, a = bit >> 5, o = bit & 31;
    const uint32_t c = __funnelshift_r(wd[a], wd[a + 1], o) & 0x1FFFFFu;
    const int32_t s = code_to_int<21>(c);
    a1 += (long long)s * W1[k];
    a0 += (long long)s * W0[k];
  }
}

template <int L>
__global__ void __launch_bounds__(DotCfg<L>::kThreads) k_dot_frsz2(BasisView B, int nvec, const double* __restrict__ w,
                                                                   double* __restrict__ out,
                                                                   double* __restrict__ partials,
                                                                   unsigned int* counter, int* err, Gate gate) {
  using C = DotCfg<L>;
  constexpr int T = C::kThreads;
  if (gate_skip(gate)) return;
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* stages = smem;
  double* red = reinterpret_cast<double*>(smem + C::kStages * C::kStageBytes);
  double* hpart = red + 2 * C::kRed * T;
  uint64_t* full = reinterpret_cast<uint64_t*>(hpart + nvec + (nvec & 1));
  int* flags = reinterpret_cast<int*>(full + C::kStages);  // [0] abort, [1] last-CTA flag

  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const int64_t nb = (B.n + 31) / 32;
  int64_t b0, b1;
  cta_block_range(nb, gridDim.x, blockIdx.x, &b0, &b1);
  const int ntiles = static_cast<int>((b1 - b0 + T - 1) / T);
  const int total = ntiles * nvec;

  for (int v = t; v < nvec; v += T) hpart[v] = 0.0;
  if (t == 0) {
    for (int s = 0; s < C::kStages; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
    flags[0] = 0;
  }
  __syncthreads();

  auto issue = [&](int it) {
    const int tile = it / nvec, vec = it - tile * nvec, s = it % C::kStages;
    const int64_t tb0 = b0 + (int64_t)tile * T;
    const int nbt = static_cast<int>(min((int64_t)T, b1 - tb0));
    const uint32_t cbytes = static_cast<uint32_t>((nbt * L * 4 + 15) & ~15);
    const uint32_t ebytes = static_cast<uint32_t>((nbt * 4 + 15) & ~15);
    uint8_t* dst = stages + s * C::kStageBytes;
    const uint8_t* src_c = B.vals + (int64_t)vec * B.vstride + tb0 * L * 4;
    const uint8_t* src_e = reinterpret_cast<const uint8_t*>(B.exps) + (int64_t)vec * B.estride + tb0 * 4;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&full[s], cbytes + ebytes);
    bulk_g2s(dst, src_c, cbytes, &full[s]);
    bulk_g2s(dst + C::kCodeBytes, src_e, ebytes, &full[s]);
  };
  if (t == 0) {
    for (int p = 0; p < C::kStages && p < total; ++p) issue(p);
  }

  int it = 0, batch = 0;
  bool aborted = false;
  for (int tile = 0; tile < ntiles && !aborted; ++tile) {
    const int64_t b = b0 + (int64_t)tile * T + t;
    const bool active = b < b1;
    // Block-fixed-point copy of this thread's 32 values of w, kept in registers for all vectors.
    int32_t W1[32], W0[32];
    int ew = 1;
    if (active) {
      const double* wb = w + b * 32;
      const int64_t rem = B.n - b * 32;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const double x = k < rem ? wb[k] : 0.0;
        ew = max(ew, eff_exp(x));
      }
#pragma unroll
      for (int c = 0; c < 32 / 4; ++c) {
        // l = 32 rotates 16-byte chunks by t, l = 16 rotates 32-byte chunks by t/2, l = 21 does not rotate
        const int src_chunk = (L == 32) ? ((c + t) & 7) : c;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          int k;
          if (L == 32) k = 4 * src_chunk + r;
          else if (L == 16) k = 8 * (((c >> 1) + (t >> 1)) & 3) + 4 * (c & 1) + r;
          else k = 4 * c + r;
          const double x = k < rem ? wb[k] : 0.0;
          to_block_fixed(x, ew, W1[4 * c + r], W0[4 * c + r]);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < 32; ++k) W1[k] = W0[k] = 0;
    }
    for (int vec = 0; vec < nvec; ++vec, ++it) {
      const int s = it % C::kStages;
      const uint32_t par = static_cast<uint32_t>((it / C::kStages) & 1);
      const bool ok = mbar_wait_bounded(&full[s], par);
      if (!ok) {
        flags[0] = 1;
        atomicOr(err, kDevErrTimeout);
      }
      double hp = 0.0;
      if (active && ok) {
        const uint8_t* st = stages + s * C::kStageBytes;
        const uint32_t e = reinterpret_cast<const uint32_t*>(st + C::kCodeBytes)[t];
        const uint32_t* cw = reinterpret_cast<const uint32_t*>(st) + t * L;
        long long a1 = 0, a0 = 0;
        if (L == 32) block_dot32(cw, t, W1, W0, a1, a0);
        else if (L == 16) block_dot16(cw, t, W1, W0, a1, a0);
        else block_dot21(cw, W1, W0, a1, a0);
        // value = (a1 2^27 + a0) 2^{x}, x = Ebar + Ew - 2096 - l  (Eq. 2 scale times the W scale)
        const int x = (e > 1 ? (int)e : 1) + ew - 2096 - L;
        hp = fma_pow2(static_cast<double>(a1), x + 27, scale_pow2(static_cast<double>(a0), x));
      }
      red[((batch & 1) * C::kRed + (vec % C::kRed)) * T + t] = hp;
      __syncthreads();
      if (flags[0]) {
        aborted = true;
        break;
      }
      if (vec % C::kRed == C::kRed - 1 || vec == nvec - 1) {
        const int first = vec - (vec % C::kRed);
        for (int vv = first + warp; vv <= vec; vv += T / 32) {
          const double* r = red + ((batch & 1) * C::kRed + (vv % C::kRed)) * T;
          double sacc = 0.0;
          for (int i = lane; i < T; i += 32) sacc += r[i];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
          if (lane == 0) hpart[vv] += sacc;
        }
        ++batch;
      }
      if (t == 0 && it + C::kStages < total) issue(it + C::kStages);
    }
  }
  if (aborted) {
    // Wait (bounded) for the copies still in flight into this CTA's shared memory, then leave.
    if (t == 0) {
      for (int p = it; p < total && p < it + C::kStages; ++p)
        mbar_wait_bounded(&full[p % C::kStages], static_cast<uint32_t>((p / C::kStages) & 1));
    }
    return;
  }
  __syncthreads();
  for (int v = t; v < nvec; v += T) partials[(size_t)blockIdx.x * nvec + v] = hpart[v];
  if (arrive_last(counter, gridDim.x, &flags[1])) {
    for (int v = warp; v < nvec; v += T / 32) {
      const double sum = warp_sum_strided(partials + v, gridDim.x, nvec);
      if (lane == 0) out[v] = sum;
    }
    if (t == 0) *counter = 0;
  }
}

// ------------------------------------------------------------------------------------------------
// FRSZ2 update: 8 consecutive values per thread, 4 threads per block, vectors in groups of 64
// ------------------------------------------------------------------------------------------------

template <int L>
struct UpdCfg {
  static constexpr int kThreads = 128;
  static constexpr int kBlocks = kThreads / 4;           // 32 FRSZ2 blocks per tile
  static constexpr int kStages = 4;
  static constexpr int kGroup = 64;                      // vectors per exact integer group
  static constexpr int kCodeBytes = kBlocks * L * 4;
  static constexpr int kStageBytes = kCodeBytes;
  // dynamic smem: stages | gamma[kGroup][kBlocks] (uint4) | exps[kGroup][kBlocks] | hinfo[nvec] |
  //               rexp[kBlocks] | red[kThreads/32] | mbarriers | flags
  static size_t smem_bytes(int nvec) {
    return (size_t)kStages * kStageBytes + (size_t)kGroup * kBlocks * 16 + (size_t)kGroup * kBlocks * 4 +
           (size_t)nvec * 16 + kBlocks * 4 + (kThreads / 32) * 8 + kStages * 8 + 16;
  }
};

struct HInfo {  // one coefficient h_i as sign, 53-bit integer significand and effective exponent
  unsigned long long mant;
  int eff;
  int neg;
};

template <int L>
__device__ __forceinline__ void load_codes8(const uint32_t* st, int t, uint32_t (&c)[8]) {
  if (L == 32) {
    const uint4* p = reinterpret_cast<const uint4*>(st) + 2 * t;
    const uint4 a = p[0], b = p[1];
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
  } else if (L == 16) {
    const uint4 a = reinterpret_cast<const uint4*>(st)[t];
    c[0] = a.x & 0xFFFFu; c[1] = a.x >> 16; c[2] = a.y & 0xFFFFu; c[3] = a.y >> 16;
    c[4] = a.z & 0xFFFFu; c[5] = a.z >> 16; c[6] = a.w & 0xFFFFu; c[7] = a.w >> 16;
  } else {
    // the 8 codes of quarter q of a block occupy stream bits [168 q, 168 q + 168)
    const int blk = t >> 2, q = t & 3;
    const uint32_t* bw = st + blk * 21;
    const int wbase = (168 * q) >> 5, o = (168 * q) & 31;
    uint32_t raw[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) raw[i] = (wbase + i < 21) ? bw[wbase + i] : 0u;
    uint32_t al[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) al[i] = __funnelshift_r(raw[i], raw[i + 1], o);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int bit = 21 * k, a = bit >> 5, oo = bit & 31;
      c[k] = __funnelshift_r(al[a], a + 1 < 6 ? al[a + 1] : 0u, oo) & 0x1FFFFFu;
    }
  }
}

template <int L>
__global__ void __launch_bounds__(UpdCfg<L>::kThreads) k_update_frsz2(BasisView B, int nvec_arg, const int* nvec_dev,
                                                                      const double* __restrict__ hcoef, int negate,
                                                                      double* __restrict__ w,
                                                                      double* __restrict__ partials,
                                                                      unsigned int* counter, int* err,
                                                                      NormEpilogue epi, Gate gate) {
  using C = UpdCfg<L>;
  constexpr int T = C::kThreads, NBT = C::kBlocks, G = C::kGroup;
  if (gate_skip(gate)) return;
  const int nvec = nvec_dev ? *(volatile const int*)nvec_dev : nvec_arg;
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* stages = smem;
  uint4* gam = reinterpret_cast<uint4*>(smem + C::kStages * C::kStageBytes);
  uint32_t* exq = reinterpret_cast<uint32_t*>(gam + G * NBT);
  HInfo* hinfo = reinterpret_cast<HInfo*>(exq + G * NBT);
  int* rexp = reinterpret_cast<int*>(hinfo + (nvec_dev ? nvec_arg : nvec));
  double* red = reinterpret_cast<double*>(rexp + NBT);
  uint64_t* full = reinterpret_cast<uint64_t*>(red + T / 32);
  int* flags = reinterpret_cast<int*>(full + C::kStages);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t nb = (B.n + 31) / 32;
  int64_t b0, b1;
  cta_block_range(nb, gridDim.x, blockIdx.x, &b0, &b1);
  const int ntiles = static_cast<int>((b1 - b0 + NBT - 1) / NBT);
  const int total = ntiles * nvec;

  for (int i = t; i < nvec; i += T) {
    const double h = negate ? -hcoef[i] : hcoef[i];
    const uint64_t u = static_cast<uint64_t>(__double_as_longlong(h));
    const int e = static_cast<int>((u >> 52) & 0x7FF);
    HInfo hi;
    hi.mant = (u & ((1ull << 52) - 1)) | (e ? (1ull << 52) : 0ull);
    hi.eff = e > 1 ? e : 1;
    hi.neg = static_cast<int>(u >> 63);
    hinfo[i] = hi;
  }
  if (t == 0) {
    for (int s = 0; s < C::kStages; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
    flags[0] = 0;
  }
  __syncthreads();

  auto issue = [&](int it) {
    const int tile = it / nvec, vec = it - tile * nvec, s = it % C::kStages;
    const int64_t tb0 = b0 + (int64_t)tile * NBT;
    const int nbt = static_cast<int>(min((int64_t)NBT, b1 - tb0));
    const uint32_t cbytes = static_cast<uint32_t>((nbt * L * 4 + 15) & ~15);
    const uint8_t* src = B.vals + (int64_t)vec * B.vstride + tb0 * L * 4;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&full[s], cbytes);
    bulk_g2s(stages + s * C::kStageBytes, src, cbytes, &full[s]);
  };
  if (t == 0) {
    for (int p = 0; p < C::kStages && p < total; ++p) issue(p);
  }

  double nrm = 0.0;
  int it = 0;
  bool aborted = false;
  const int blk = t >> 2;  // block of this thread within the tile
  for (int tile = 0; tile < ntiles && !aborted; ++tile) {
    const int64_t tb0 = b0 + (int64_t)tile * NBT;
    const int nbt = static_cast<int>(min((int64_t)NBT, b1 - tb0));
    const int64_t k0 = (tb0 + blk) * 32 + (t & 3) * 8;  // first value of this thread
    const bool active = blk < nbt;
    double dacc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) dacc[k] = 0.0;
    for (int g0 = 0; g0 < nvec && !aborted; g0 += G) {
      const int gn = min(G, nvec - g0);
      // exponents of this group's vectors for the tile's blocks
      for (int idx = t; idx < gn * NBT; idx += T) {
        const int v = idx / NBT, bb = idx - v * NBT;
        exq[idx] = bb < nbt ? __ldg(reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint8_t*>(B.exps) +
                                                                    (int64_t)(g0 + v) * B.estride) + tb0 + bb)
                            : 0u;
      }
      __syncthreads();
      // rexp_b = max over the group of (Eh_i + Ebar_{i,b}): the exponent of the block's largest term
      if (t < NBT) {
        int r = 0;
        for (int v = 0; v < gn; ++v) {
          const uint32_t e = exq[v * NBT + t];
          const int x = hinfo[g0 + v].eff + (e > 1 ? (int)e : 1);
          r = max(r, x);
        }
        rexp[t] = r;
      }
      __syncthreads();
      // Gamma_{i,b} = round(Mh_i 2^{X_{i,b} - rexp_b}) with sign, as three 18-bit pieces
      for (int idx = t; idx < gn * NBT; idx += T) {
        const int v = idx / NBT, bb = idx - v * NBT;
        const uint32_t e = exq[idx];
        const HInfo hi = hinfo[g0 + v];
        const int sh = rexp[bb] - (hi.eff + (e > 1 ? (int)e : 1));
        uint64_t mag;
        if (sh == 0) mag = hi.mant;
        else if (sh < 64) mag = ((hi.mant >> (sh - 1)) + 1) >> 1;
        else mag = 0;
        const int64_t Gm = hi.neg ? -static_cast<int64_t>(mag) : static_cast<int64_t>(mag);
        uint4 p;
        p.x = static_cast<uint32_t>(Gm & 0x3FFFF);
        p.y = static_cast<uint32_t>((Gm >> 18) & 0x3FFFF);
        p.z = static_cast<uint32_t>(static_cast<int32_t>(Gm >> 36));
        p.w = 0;
        gam[idx] = p;
      }
      __syncthreads();
      long long acc0[8], acc1[8], acc2[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc0[k] = acc1[k] = acc2[k] = 0;
      for (int v = 0; v < gn; ++v, ++it) {
        const int s = it % C::kStages;
        const uint32_t par = static_cast<uint32_t>((it / C::kStages) & 1);
        const bool ok = mbar_wait_bounded(&full[s], par);
        if (!ok) {
          flags[0] = 1;
          atomicOr(err, kDevErrTimeout);
        }
        if (active && ok) {
          uint32_t c[8];
          load_codes8<L>(reinterpret_cast<const uint32_t*>(stages + s * C::kStageBytes), t, c);
          const uint4 gp = gam[v * NBT + blk];
          const int32_t g0p = static_cast<int32_t>(gp.x), g1p = static_cast<int32_t>(gp.y);
          const int32_t g2p = static_cast<int32_t>(gp.z);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int32_t sv = code_to_int<L>(c[k]);
            acc0[k] += (long long)sv * g0p;
            acc1[k] += (long long)sv * g1p;
            acc2[k] += (long long)sv * g2p;
          }
        }
        __syncthreads();
        if (flags[0]) {
          aborted = true;
          break;
        }
        if (t == 0 && it + C::kStages < total) issue(it + C::kStages);
      }
      if (aborted) break;
      if (active) {
        // sum_i s Gamma = acc2 2^36 + acc1 2^18 + acc0 exactly; scale 2^{rexp - 2096 - l}
        const int x = rexp[blk] - 2096 - L;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const __int128 tt = ((__int128)acc2[k] << 36) + ((__int128)acc1[k] << 18) + (__int128)acc0[k];
          const long long hi42 = static_cast<long long>(tt >> 42);
          const long long lo42 = static_cast<long long>(tt & ((((__int128)1) << 42) - 1));
          const double d = fma(static_cast<double>(hi42), 4398046511104.0 /* 2^42 */, static_cast<double>(lo42));
          dacc[k] = fma_pow2(d, x, dacc[k]);
        }
      }
    }
    if (aborted) break;
    if (active) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int64_t idx = k0 + k;
        if (idx < B.n) {
          const double nv = w[idx] - dacc[k];
          w[idx] = nv;
          nrm = fma(nv, nv, nrm);
        }
      }
    }
  }
  if (aborted) {
    if (t == 0) {
      for (int p = it; p < total && p < it + C::kStages; ++p)
        mbar_wait_bounded(&full[p % C::kStages], static_cast<uint32_t>((p / C::kStages) & 1));
    }
    return;
  }
  // ||w||^2: CTA partial, then the last CTA reduces all partials in a fixed order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (lane == 0) red[warp] = nrm;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int i = 0; i < T / 32; ++i) s += red[i];
    partials[blockIdx.x] = s;
  }
  if (arrive_last(counter, gridDim.x, &flags[1])) {
    if (warp == 0) {
      const double s = warp_sum_strided(partials, gridDim.x, 1);
      if (lane == 0) norm_epilogue(epi, s, err);
    }
    if (t == 0) *counter = 0;
  }
}

// ------------------------------------------------------------------------------------------------
// Cast formats: widen to FP64 with integer operations, one FP64 FMA per element and vector
// ------------------------------------------------------------------------------------------------

__device__ __forceinline__ double widen_f32(uint32_t f) {
  const uint32_t e = (f >> 23) & 0xFFu;
  if (e != 0) {
    const uint64_t d = (static_cast<uint64_t>(f >> 31) << 63) | (static_cast<uint64_t>(e + 896) << 52) |
                       (static_cast<uint64_t>(f & 0x7FFFFFu) << 29);
    return __longlong_as_double(static_cast<long long>(d));
  }
  return static_cast<double>(__uint_as_float(f));  // zero or subnormal (rare)
}

__device__ __forceinline__ double widen_f16(uint32_t h) {
  const uint32_t e = (h >> 10) & 0x1Fu;
  if (e != 0) {
    const uint64_t d = (static_cast<uint64_t>(h >> 15) << 63) | (static_cast<uint64_t>(e + 1008) << 52) |
                       (static_cast<uint64_t>(h & 0x3FFu) << 42);
    return __longlong_as_double(static_cast<long long>(d));
  }
  const double m = static_cast<double>(static_cast<int>(h & 0x3FFu)) * 5.9604644775390625e-08;  // 2^-24
  return (h >> 15) ? -m : m;
}

template <int F>
struct CastTraits;
template <>
struct CastTraits<CBG_FP64> {
  static constexpr int kBytes = 8;
};
template <>
struct CastTraits<CBG_FP32> {
  static constexpr int kBytes = 4;
};
template <>
struct CastTraits<CBG_FP16> {
  static constexpr int kBytes = 2;
};
template <>
struct CastTraits<CBG_BF16> {
  static constexpr int kBytes = 2;
};

// 8 consecutive values of one vector starting at element k0 (16-byte aligned), widened to FP64.
template <int F>
__device__ __forceinline__ void load8_widen(const uint8_t* base, int64_t k0, double (&v)[8]) {
  if (F == CBG_FP64) {
    const double2* p = reinterpret_cast<const double2*>(base + k0 * 8);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double2 q = __ldcs(p + i);
      v[2 * i] = q.x;
      v[2 * i + 1] = q.y;
    }
  } else if (F == CBG_FP32) {
    const uint4* p = reinterpret_cast<const uint4*>(base + k0 * 4);
    const uint4 a = __ldcs(p), b = __ldcs(p + 1);
    v[0] = widen_f32(a.x); v[1] = widen_f32(a.y); v[2] = widen_f32(a.z); v[3] = widen_f32(a.w);
    v[4] = widen_f32(b.x); v[5] = widen_f32(b.y); v[6] = widen_f32(b.z); v[7] = widen_f32(b.w);
  } else {
    const uint4 a = __ldcs(reinterpret_cast<const uint4*>(base + k0 * 2));
    const uint32_t wv[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (F == CBG_FP16) {
        v[2 * i] = widen_f16(wv[i] & 0xFFFFu);
        v[2 * i + 1] = widen_f16(wv[i] >> 16);
      } else {
        v[2 * i] = widen_f32(wv[i] << 16);
        v[2 * i + 1] = widen_f32(wv[i] & 0xFFFF0000u);
      }
    }
  }
}

struct CastCfg {
  static constexpr int kThreads = 256;
  static constexpr int kPer = 8;                      // values per thread per tile
  static constexpr int kTile = kThreads * kPer;       // 2048 values
  static constexpr int kRed = 8;
  static size_t dot_smem(int nvec) { return (size_t)2 * kRed * kThreads * 8 + (size_t)nvec * 8 + 16; }
};

__device__ __forceinline__ void cta_value_range(int64_t n, int G, int c, int64_t* k0, int64_t* k1) {
  const int64_t nu = (n + 127) / 128;  // units of 128 values keep every chunk 16-byte aligned
  const int64_t u0 = nu * c / G, u1 = nu * (c + 1) / G;
  *k0 = min(u0 * 128, n);
  *k1 = min(u1 * 128, n);
}

template <int F>
__global__ void __launch_bounds__(CastCfg::kThreads) k_dot_cast(BasisView B, int nvec, const double* __restrict__ w,
                                                                 double* __restrict__ out,
                                                                 double* __restrict__ partials, unsigned int* counter,
                                                                 Gate gate) {
  constexpr int T = CastCfg::kThreads, P = CastCfg::kPer, R = CastCfg::kRed;
  if (gate_skip(gate)) return;
  extern __shared__ __align__(128) uint8_t smem[];
  double* red = reinterpret_cast<double*>(smem);
  double* hpart = red + 2 * R * T;
  int* flags = reinterpret_cast<int*>(hpart + nvec + (nvec & 1));
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  int64_t k0, k1;
  cta_value_range(B.n, gridDim.x, blockIdx.x, &k0, &k1);
  for (int v = t; v < nvec; v += T) hpart[v] = 0.0;
  __syncthreads();
  int batch = 0;
  for (int64_t tk = k0; tk < k1; tk += CastCfg::kTile) {
    const int64_t kk = tk + (int64_t)t * P;
    const bool active = kk < k1;
    double wv[P];
#pragma unroll
    for (int i = 0; i < P; ++i) wv[i] = (active && kk + i < B.n) ? w[kk + i] : 0.0;
    double nxt[P];
    if (active) load8_widen<F>(B.vals, kk, nxt);
    for (int vec = 0; vec < nvec; ++vec) {
      double cur[P];
#pragma unroll
      for (int i = 0; i < P; ++i) cur[i] = nxt[i];
      if (active && vec + 1 < nvec) load8_widen<F>(B.vals + (int64_t)(vec + 1) * B.vstride, kk, nxt);
      double hp = 0.0;
      if (active) {
#pragma unroll
        for (int i = 0; i < P; ++i)
          if (kk + i < B.n) hp = fma(cur[i], wv[i], hp);  // the padding past n may hold anything
      }
      red[((batch & 1) * R + (vec % R)) * T + t] = hp;
      __syncthreads();
      if (vec % R == R - 1 || vec == nvec - 1) {
        const int first = vec - (vec % R);
        for (int vv = first + warp; vv <= vec; vv += T / 32) {
          const double* r = red + ((batch & 1) * R + (vv % R)) * T;
          double s = 0.0;
          for (int i = lane; i < T; i += 32) s += r[i];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (lane == 0) hpart[vv] += s;
        }
        ++batch;
      }
    }
  }
  __syncthreads();
  for (int v = t; v < nvec; v += T) partials[(size_t)blockIdx.x * nvec + v] = hpart[v];
  if (arrive_last(counter, gridDim.x, &flags[0])) {
    for (int v = warp; v < nvec; v += T / 32) {
      const double sum = warp_sum_strided(partials + v, gridDim.x, nvec);
      if (lane == 0) out[v] = sum;
    }
    if (t == 0) *counter = 0;
  }
}

template <int F>
__global__ void __launch_bounds__(CastCfg::kThreads) k_update_cast(BasisView B, int nvec_arg, const int* nvec_dev,
                                                                    const double* __restrict__ hcoef, int negate,
                                                                    double* __restrict__ w,
                                                                    double* __restrict__ partials,
                                                                    unsigned int* counter, int* err, NormEpilogue epi,
                                                                    Gate gate) {
  constexpr int T = CastCfg::kThreads, P = CastCfg::kPer;
  if (gate_skip(gate)) return;
  const int nvec = nvec_dev ? *(volatile const int*)nvec_dev : nvec_arg;
  extern __shared__ __align__(128) uint8_t smem[];
  double* hs = reinterpret_cast<double*>(smem);
  double* red = hs + (nvec_dev ? nvec_arg : nvec);
  int* flags = reinterpret_cast<int*>(red + T / 32);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int i = t; i < nvec; i += T) hs[i] = negate ? -hcoef[i] : hcoef[i];
  __syncthreads();
  int64_t k0, k1;
  cta_value_range(B.n, gridDim.x, blockIdx.x, &k0, &k1);
  double nrm = 0.0;
  for (int64_t tk = k0; tk < k1; tk += CastCfg::kTile) {
    const int64_t kk = tk + (int64_t)t * P;
    if (kk >= k1) continue;
    double acc[P];
#pragma unroll
    for (int i = 0; i < P; ++i) acc[i] = (kk + i < B.n) ? w[kk + i] : 0.0;
    double nxt[P];
    if (nvec > 0) load8_widen<F>(B.vals, kk, nxt);
    for (int vec = 0; vec < nvec; ++vec) {
      double cur[P];
#pragma unroll
      for (int i = 0; i < P; ++i) cur[i] = nxt[i];
      if (vec + 1 < nvec) load8_widen<F>(B.vals + (int64_t)(vec + 1) * B.vstride, kk, nxt);
      const double nh = -hs[vec];
#pragma unroll
      for (int i = 0; i < P; ++i) acc[i] = fma(cur[i], nh, acc[i]);
    }
#pragma unroll
    for (int i = 0; i < P; ++i) {
      if (kk + i < B.n) {
        w[kk + i] = acc[i];
        nrm = fma(acc[i], acc[i], nrm);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (lane == 0) red[warp] = nrm;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int i = 0; i < T / 32; ++i) s += red[i];
    partials[blockIdx.x] = s;
  }
  if (arrive_last(counter, gridDim.x, &flags[0])) {
    if (warp == 0) {
      const double s = warp_sum_strided(partials, gridDim.x, 1);
      if (lane == 0) norm_epilogue(epi, s, err);
    }
    if (t == 0) *counter = 0;
  }
}

// ------------------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------------------

namespace {

int ensure_smem(const void* fn, size_t bytes) {
  static thread_local const void* last_fn = nullptr;
  static thread_local size_t last_bytes = 0;
  if (fn == last_fn && bytes <= last_bytes) return CBG_OK;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(max dynamic smem)");
  last_fn = fn;
  last_bytes = bytes;
  return CBG_OK;
}

int grid_for(const void* fn, int threads, size_t smem, int64_t units, int64_t units_per_cta_min, int* grid) {
  DeviceInfo di;
  int st = device_info(&di);
  if (st) return st;
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (occ < 1) occ = 1;
  int64_t g = (int64_t)occ * di.sms;
  int64_t need = (units + units_per_cta_min - 1) / units_per_cta_min;
  if (need < 1) need = 1;
  if (g > need) g = need;
  if (g > kMaxGrid) g = kMaxGrid;
  *grid = static_cast<int>(g);
  return CBG_OK;
}

template <typename K>
const void* fnp(K k) {
  return reinterpret_cast<const void*>(k);
}

}  // namespace

int launch_basis_dot(const BasisView& B, int nvec, const double* w, double* out, double* partials, unsigned int* counter,
                     int* err, const Gate& gate, cudaStream_t stream) {
  if (nvec <= 0 || B.n <= 0) return CBG_OK;
  const void* fn;
  size_t smem;
  int threads;
  int64_t units, per;
  if (B.fmt == CBG_FRSZ2) {
    threads = 128;
    units = (B.n + 31) / 32;
    per = 16;
    switch (B.l) {
      case 32: fn = fnp(k_dot_frsz2<32>); smem = DotCfg<32>::smem_bytes(nvec); break;
      case 21: fn = fnp(k_dot_frsz2<21>); smem = DotCfg<21>::smem_bytes(nvec); break;
      case 16: fn = fnp(k_dot_frsz2<16>); smem = DotCfg<16>::smem_bytes(nvec); break;
      default: return CBG_ERR_INVALID_ARG;
    }
  } else {
    threads = CastCfg::kThreads;
    units = B.n;
    per = 4096;
    smem = CastCfg::dot_smem(nvec);
    switch (B.fmt) {
      case CBG_FP64: fn = fnp(k_dot_cast<CBG_FP64>); break;
      case CBG_FP32: fn = fnp(k_dot_cast<CBG_FP32>); break;
      case CBG_FP16: fn = fnp(k_dot_cast<CBG_FP16>); break;
      case CBG_BF16: fn = fnp(k_dot_cast<CBG_BF16>); break;
      default: return CBG_ERR_INVALID_ARG;
    }
  }
  int st = ensure_smem(fn, smem);
  if (st) return st;
  int grid;
  st = grid_for(fn, threads, smem, units, per, &grid);
  if (st) return st;
  if (B.fmt == CBG_FRSZ2) {
    switch (B.l) {
      case 32: k_dot_frsz2<32><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, err, gate); break;
      case 21: k_dot_frsz2<21><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, err, gate); break;
      default: k_dot_frsz2<16><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, err, gate); break;
    }
  } else {
    switch (B.fmt) {
      case CBG_FP64: k_dot_cast<CBG_FP64><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, gate); break;
      case CBG_FP32: k_dot_cast<CBG_FP32><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, gate); break;
      case CBG_FP16: k_dot_cast<CBG_FP16><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, gate); break;
      default: k_dot_cast<CBG_BF16><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, gate); break;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "basis dot launch");
  return CBG_OK;
}

// The basis dot with the grid limited to max_grid CTAs, for callers whose partial-sum buffer has a
// fixed capacity (max_grid * nvec doubles).
int launch_basis_dot_capped(const BasisView& B, int nvec, const double* w, double* out, double* partials,
                            unsigned int* counter, int* err, int max_grid, cudaStream_t stream) {
  if (nvec <= 0 || B.n <= 0) return CBG_OK;
  const Gate gate{nullptr, nullptr};
  const void* fn;
  size_t smem;
  int threads;
  int64_t units, per;
  if (B.fmt == CBG_FRSZ2) {
    threads = 128;
    units = (B.n + 31) / 32;
    per = 16;
    switch (B.l) {
      case 32: fn = fnp(k_dot_frsz2<32>); smem = DotCfg<32>::smem_bytes(nvec); break;
      case 21: fn = fnp(k_dot_frsz2<21>); smem = DotCfg<21>::smem_bytes(nvec); break;
      case 16: fn = fnp(k_dot_frsz2<16>); smem = DotCfg<16>::smem_bytes(nvec); break;
      default: return CBG_ERR_INVALID_ARG;
    }
  } else {
    threads = CastCfg::kThreads;
    units = B.n;
    per = 4096;
    smem = CastCfg::dot_smem(nvec);
    switch (B.fmt) {
      case CBG_FP64: fn = fnp(k_dot_cast<CBG_FP64>); break;
      case CBG_FP32: fn = fnp(k_dot_cast<CBG_FP32>); break;
      case CBG_FP16: fn = fnp(k_dot_cast<CBG_FP16>); break;
      case CBG_BF16: fn = fnp(k_dot_cast<CBG_BF16>); break;
      default: return CBG_ERR_INVALID_ARG;
    }
  }
  int st = ensure_smem(fn, smem);
  if (st) return st;
  int grid;
  st = grid_for(fn, threads, smem, units, per, &grid);
  if (st) return st;
  if (grid > max_grid) grid = max_grid;
  if (B.fmt == CBG_FRSZ2) {
    switch (B.l) {
      case 32: k_dot_frsz2<32><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, err, gate); break;
      case 21: k_dot_frsz2<21><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, err, gate); break;
      default: k_dot_frsz2<16><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, err, gate); break;
    }
  } else {
    switch (B.fmt) {
      case CBG_FP64: k_dot_cast<CBG_FP64><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, gate); break;
      case CBG_FP32: k_dot_cast<CBG_FP32><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, gate); break;
      case CBG_FP16: k_dot_cast<CBG_FP16><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, gate); break;
      default: k_dot_cast<CBG_BF16><<<grid, threads, smem, stream>>>(B, nvec, w, out, partials, counter, gate); break;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "basis dot launch");
  return CBG_OK;
}

int launch_basis_update(const BasisView& B, int nvec, const int* nvec_dev, const double* h, int negate, double* w,
                        double* partials, unsigned int* counter, int* err, const NormEpilogue& epi, const Gate& gate,
                        cudaStream_t stream) {
  if ((nvec <= 0 && !nvec_dev) || B.n <= 0) return CBG_OK;
  const void* fn;
  size_t smem;
  int threads;
  int64_t units, per;
  if (B.fmt == CBG_FRSZ2) {
    threads = 128;
    units = (B.n + 31) / 32;
    per = 8;
    switch (B.l) {
      case 32: fn = fnp(k_update_frsz2<32>); smem = UpdCfg<32>::smem_bytes(nvec); break;
      case 21: fn = fnp(k_update_frsz2<21>); smem = UpdCfg<21>::smem_bytes(nvec); break;
      case 16: fn = fnp(k_update_frsz2<16>); smem = UpdCfg<16>::smem_bytes(nvec); break;
      default: return CBG_ERR_INVALID_ARG;
    }
  } else {
    threads = CastCfg::kThreads;
    units = B.n;
    per = 2048;
    smem = (size_t)nvec * 8 + (CastCfg::kThreads / 32) * 8 + 16;
    switch (B.fmt) {
      case CBG_FP64: fn = fnp(k_update_cast<CBG_FP64>); break;
      case CBG_FP32: fn = fnp(k_update_cast<CBG_FP32>); break;
      case CBG_FP16: fn = fnp(k_update_cast<CBG_FP16>); break;
      case CBG_BF16: fn = fnp(k_update_cast<CBG_BF16>); break;
      default: return CBG_ERR_INVALID_ARG;
    }
  }
  int st = ensure_smem(fn, smem);
  if (st) return st;
  int grid;
  st = grid_for(fn, threads, smem, units, per, &grid);
  if (st) return st;
  if (B.fmt == CBG_FRSZ2) {
    switch (B.l) {
      case 32: k_update_frsz2<32><<<grid, threads, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate); break;
      case 21: k_update_frsz2<21><<<grid, threads, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate); break;
      default: k_update_frsz2<16><<<grid, threads, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate); break;
    }
  } else {
    switch (B.fmt) {
      case CBG_FP64: k_update_cast<CBG_FP64><<<grid, threads, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate); break;
      case CBG_FP32: k_update_cast<CBG_FP32><<<grid, threads, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate); break;
      case CBG_FP16: k_update_cast<CBG_FP16><<<grid, threads, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate); break;
      default: k_update_cast<CBG_BF16><<<grid, threads, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate); break;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "basis update launch");
  return CBG_OK;
}

}  // namespace cbg
