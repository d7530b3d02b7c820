// FRSZ2 basis kernels: the Gram-Schmidt projections h = V^T w and the update w -= V h of Fig. 1
// step 5 (and steps 8 and 17), decoding the stored FRSZ2 codes in registers.
//
// An FRSZ2 block is block fixed point (Eq. 2): value k of block b of vector i is s_{i,k} 2^{q_{i,b}}
// with s a signed integer of l-1 magnitude bits. GB300 issues FP64 at ~1.9 operations per clock per
// SM (conversions to FP64 included) against ~57 32x32->64 integer multiply-adds, so both kernels do
// the per-element work as exact integer arithmetic and touch FP64 once per block or per element:
//
//   dot     sum_{k in b} s_{i,k} W_k, W a 54-bit block-fixed-point copy of w (rounded to nearest
//           against the block's largest exponent), is exact in two 64-bit accumulators; the sum
//           (at most l+57 bits) is rounded to 2^(l-5) units in integer arithmetic and converted
//           once per (vector, block), then summed in FP64 (per warp, per CTA, across CTAs in a
//           fixed order).
//   update  sum_i s_{i,k} G_{i,b}, G the 54-bit fixed point of h_i 2^{q_{i,b}} against the block's
//           largest term within a group of at most 32 vectors (an integer mantissa shift per
//           (vector, block)), is exact in two 64-bit accumulators (27-bit pieces of G). Groups are
//           combined in a 64-bit integer per element at the larger of their block scales, and the
//           element is converted to FP64 once: FP64 work is per element, not per element and group.
//
// The basis is streamed with 1D bulk copies (TMA) into a ring of shared-memory stages. Each stage
// has a "full" mbarrier (the copy's transaction count) and an "empty" mbarrier (one arrival per
// warp); thread 0 refills the stage released one iteration earlier, so warps never wait on each
// other inside the vector loop. Every wait is bounded (globaltimer); on expiry the kernel records
// kDevErrTimeout, waits (bounded) for its own copies in flight and returns.
#include "decode.cuh"
#include "frsz2_block.cuh"

namespace cbg {

// ================================================================================================
// dot: one thread per 32-value block, 128 blocks per tile (256 at l = 16), two basis vectors per
// pipeline stage;
// CTA (x, y) takes block range x and the y-th slice of the vectors (gridDim.y > 1 only when the
// blocks alone leave the GPU underfilled)
// ================================================================================================

// Pipeline shape of the dot per code width (threads = blocks per tile, vectors per stage, stages);
// the defaults are the measured best, and each can be set at build time (-DCBG_DOT_<knob>_<l>=...)
// for a sweep.
#ifndef CBG_DOT_THREADS_16
#define CBG_DOT_THREADS_16 256
#endif
#ifndef CBG_DOT_THREADS_21
#define CBG_DOT_THREADS_21 128
#endif
#ifndef CBG_DOT_THREADS_32
#define CBG_DOT_THREADS_32 128
#endif
#ifndef CBG_DOT_VPS_16
#define CBG_DOT_VPS_16 2
#endif
#ifndef CBG_DOT_VPS_21
#define CBG_DOT_VPS_21 2
#endif
#ifndef CBG_DOT_VPS_32
#define CBG_DOT_VPS_32 2
#endif
#ifndef CBG_DOT_STAGES_16
#define CBG_DOT_STAGES_16 2
#endif
#ifndef CBG_DOT_STAGES_21
#define CBG_DOT_STAGES_21 2
#endif
#ifndef CBG_DOT_STAGES_32
#define CBG_DOT_STAGES_32 2
#endif
// a dot CTA takes at least 1/CBG_DOT_MIN_DIV of a tile's blocks; vectors are split over CTAs when
// that leaves the GPU underfilled. Whole tiles (1) keep every thread busy at 10^4-10^6 rows, where
// an eighth of a tile per CTA left most threads idle: at 110 592 rows the dot took 28.7 us instead
// of 56 us per launch; unchanged at 2^24 rows
#ifndef CBG_DOT_MIN_DIV
#define CBG_DOT_MIN_DIV 1
#endif
// the update takes the deep pipeline (one CTA per SM) while fewer than one CTA per SM would get
// CBG_UPD_DEEP_BLOCKS blocks (32: up to about 155 000 rows; 23.5 instead of 26.1 us per launch at
// 110 592 rows)
#ifndef CBG_UPD_DEEP_BLOCKS
#define CBG_UPD_DEEP_BLOCKS 32
#endif
// resident CTAs per SM the binary32 dot's registers are capped for
#ifndef CBG_DOT_F32_MINB
#define CBG_DOT_F32_MINB 3
#endif

// FDot<16, K> for K = 1 (binary16) and K = 2 (bfloat16) is the same pipeline over a basis stored as
// 16-bit values (64 bytes per 32-value block, as an l = 16 block, and no exponent words): every
// binary16 value below 2 in magnitude is an exact integer in units of 2^-24 (fp16_fixed), and a
// bfloat16 block goes on a block fixed point on the fly (block_dot_bf16), so a block's dot is the
// same exact integer sum.
template <int L, int K = 0>
struct FDot {
  // 128 threads (blocks) per tile; 256 at l = 16, whose 8 KB per-vector copies then grow to 16 KB
  // (3.7% faster there)
  static constexpr int kThreads = L == 16 ? CBG_DOT_THREADS_16 : (L == 21 ? CBG_DOT_THREADS_21 : CBG_DOT_THREADS_32);
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kVps = L == 16 ? CBG_DOT_VPS_16 : (L == 21 ? CBG_DOT_VPS_21 : CBG_DOT_VPS_32);
  static constexpr int kStages = L == 16 ? CBG_DOT_STAGES_16 : (L == 21 ? CBG_DOT_STAGES_21 : CBG_DOT_STAGES_32);
  static constexpr int kCodeBytes = kThreads * L * 4;
  static constexpr int kVecBytes = kCodeBytes + (K ? 0 : kThreads * 4);  // one vector's codes and exponents
  static constexpr int kStageBytes = kVps * kVecBytes;
  static size_t smem_bytes(int nvec) {
    return (size_t)kStages * kStageBytes + (size_t)kWarps * nvec * 8 + 2 * kStages * 8 + 16;
  }
};

template <int L, int K>
__device__ __forceinline__ void dot_body(const BasisView& B, int nvec, const double* __restrict__ w,
                                         double* __restrict__ out, double* __restrict__ partials,
                                         unsigned int* counter, int* err, const Gate& gate) {
  static_assert(K == 0 || L == (K == 3 ? 32 : 16), "16-bit values use the l = 16 layout, binary32 the l = 32 one");
  constexpr bool H = K != 0;  // a cast format: no exponent words
  using C = FDot<L, K>;
  constexpr int T = C::kThreads, S = C::kStages;
  if (gate_skip(gate)) return;
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* stages = smem;
  double* hpart = reinterpret_cast<double*>(smem + S * C::kStageBytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(hpart + C::kWarps * nvec);
  uint64_t* empty = full + S;
  int* flags = reinterpret_cast<int*>(empty + S);  // [0] abort, [1] last-CTA flag

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t nb = (B.n + 31) / 32;
  int64_t b0, b1;
  cta_block_range(nb, gridDim.x, blockIdx.x, &b0, &b1);
  const int ntiles = static_cast<int>((b1 - b0 + T - 1) / T);
  // this CTA's vectors [v_lo, v_lo + nv)
  const int v_lo = static_cast<int>((int64_t)nvec * blockIdx.y / gridDim.y);
  const int nv = static_cast<int>((int64_t)nvec * (blockIdx.y + 1) / gridDim.y) - v_lo;
  constexpr int VPS = C::kVps;
  const int units = (nv + VPS - 1) / VPS;  // stages per tile
  const int total = ntiles * units;
  const int cid = blockIdx.y * gridDim.x + blockIdx.x, nctas = gridDim.x * gridDim.y;

  for (int i = t; i < C::kWarps * nvec; i += T) hpart[i] = 0.0;
  if (t == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C::kWarps);
    }
    fence_mbar_init();
    flags[0] = 0;
  }
  __syncthreads();

  auto issue = [&](int p) {  // stage unit p: vectors v_lo + VPS u .. of tile p / units
    const int tile = p / units, u = p - tile * units, s = p % S;
    const int v0 = v_lo + u * VPS, cnt = min(VPS, v_lo + nv - v0);
    const int64_t tb0 = b0 + (int64_t)tile * T;
    const int nbt = static_cast<int>(min((int64_t)T, b1 - tb0));
    const uint32_t cbytes = static_cast<uint32_t>((nbt * L * 4 + 15) & ~15);
    const uint32_t ebytes = H ? 0u : static_cast<uint32_t>((nbt * 4 + 15) & ~15);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&full[s], (cbytes + ebytes) * cnt);
    for (int j = 0; j < cnt; ++j) {
      uint8_t* dst = stages + s * C::kStageBytes + j * C::kVecBytes;
      const int vec = v0 + j;
      bulk_g2s(dst, B.vals + (int64_t)vec * B.vstride + tb0 * L * 4, cbytes, &full[s]);
      if (!H)
        bulk_g2s(dst + C::kCodeBytes, reinterpret_cast<const uint8_t*>(B.exps) + (int64_t)vec * B.estride + tb0 * 4,
                 ebytes, &full[s]);
    }
  };
  int issued = 0;  // thread 0 only
  if (t == 0) {
    for (; issued < S && issued < total; ++issued) issue(issued);
  }

  double* myh = hpart + warp * nvec;
  long long ks = 0;  // lane i: the warp's sum for vector 32 k + i of the current batch, ks * 2^kx
  int kx = 0;
  int s = 0;           // stage of the current vector and the phase parity of its barriers
  uint32_t ph = 0;
  int ps = 0;          // stage and parity of the previous vector (refilled by thread 0)
  uint32_t pph = 0;
  bool first = true;
  bool dead = false;   // this warp gave up waiting (warp-uniform); it then runs to the end without waiting
  bool rfail = false;  // thread 0 gave up waiting for a stage to be released
  for (int tile = 0; tile < ntiles; ++tile) {
    const int64_t b = b0 + (int64_t)tile * T + t;
    const bool active = b < b1;
    if (t == 0 && tile + 1 < ntiles) {  // the next tile's w: in L2 by the time it is needed
      const int64_t nb0 = b0 + (int64_t)(tile + 1) * T;
      const int64_t vals = min((int64_t)T, b1 - nb0) * 32;
      const int64_t bytes = min(vals, B.n - nb0 * 32) * 8;
      if (bytes >= 16) bulk_prefetch_l2(w + nb0 * 32, static_cast<uint32_t>(bytes & ~15ll));
    }
    // 54-bit block-fixed-point copy of this thread's 32 values of w, kept in registers
    int32_t W1[32], W0[32];
    int ew = 1;
    if (active) {
      const double* wb = w + b * 32;
      const int64_t rem = B.n - b * 32;
      if (rem >= 32 && L == 32 && K == 0) {
        // one pass: the 32 values in W's order, then their largest exponent, then the conversion in
        // place (2.9% faster at n = 2^24 and 3-5% at 10^5-10^6 rows than the two passes below, which
        // measured faster at l = 16 and 21, where the extra registers cost more)
        double wv[32];
#pragma unroll
        for (int r = 0; r < 32; r += 2) {
          const double2 v = __ldg(reinterpret_cast<const double2*>(wb + w_index<L>(t, r)));
          wv[r] = v.x;
          wv[r + 1] = v.y;
          ew = max(ew, max(eff_exp(v.x), eff_exp(v.y)));
        }
#pragma unroll
        for (int r = 0; r < 32; ++r) to_block_fixed(wv[r], ew, W1[r], W0[r]);
      } else if (rem >= 32) {
        // two passes: the largest exponent over the block, then the values in W's order
        const double2* w2 = reinterpret_cast<const double2*>(wb);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const double2 v = __ldg(w2 + k);
          ew = max(ew, max(eff_exp(v.x), eff_exp(v.y)));
        }
#pragma unroll
        for (int r = 0; r < 32; r += 2) {
          const double2 v = __ldg(reinterpret_cast<const double2*>(wb + w_index<L>(t, r)));
          to_block_fixed(v.x, ew, W1[r], W0[r]);
          to_block_fixed(v.y, ew, W1[r + 1], W0[r + 1]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) ew = max(ew, eff_exp(k < rem ? wb[k] : 0.0));
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int k = w_index<L>(t, r);
          to_block_fixed(k < rem ? wb[k] : 0.0, ew, W1[r], W0[r]);
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < 32; ++r) W1[r] = W0[r] = 0;
    }
    for (int vi = 0; vi < nv; vi += VPS) {
      // lagged refill: the stage released by every warp in the previous iteration
      if (t == 0 && !first && issued < total && !rfail && !dead) {
        if (mbar_wait_bounded(&empty[ps], pph)) {
          issue(issued);
          ++issued;
        } else {
          rfail = true;
          flags[0] = 1;
          atomicOr(err, kDevErrTimeout);
        }
      }
      bool ok = false;
      if (!dead) {
        ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[s], ph));
        if (!ok) {
          dead = true;
          if (lane == 0) {
            flags[0] = 1;
            atomicOr(err, kDevErrTimeout);
          }
        }
      }
      // the warp's 32 block sums th * 2^xb of vector vj at a common scale, exactly in integers;
      // lane vj % 32 keeps vector vj's, and every 32 vectors each lane converts its vector once and
      // adds it to the warp's per-vector sum (one FP64 instruction per 32 vectors)
      auto post = [&](int vj, long long th, int xb) {
        int X;
        const long long sum = warp_fixed_sum(th, xb, X);
        if (lane == (vj & 31)) {
          ks = sum;
          kx = X;
        }
        if ((vj & 31) == 31 || vj == nv - 1) {
          if (lane <= (vj & 31)) {
            double* hv = myh + v_lo + (vj & ~31) + lane;
            *hv = fma_pow2(static_cast<double>(ks), kx, *hv);
          }
        }
      };
#pragma unroll
      for (int j = 0; j < VPS; ++j) {
        const int vj = vi + j;
        if (vj >= nv) break;  // uniform
        long long th = 0;  // this block's sum: th * 2^xb
        int xb = 0;
        if (active && ok) {
          const uint8_t* st = stages + s * C::kStageBytes + j * C::kVecBytes;
          const uint32_t* cw = reinterpret_cast<const uint32_t*>(st) + t * L;
          long long a1, a0;
          if (!H) {
            const uint32_t e = reinterpret_cast<const uint32_t*>(st + C::kCodeBytes)[t];
            block_dot<L>(cw, t, W1, W0, a1, a0);
            // sum = (a1 2^27 + a0) 2^x with x = Ebar + Ew - 2096 - l, |a1 2^27 + a0| < 2^(l+57).
            // Rounded to 2^(l-5) units it fits in 63 bits; the rounding error, at most 2^(l-6)
            // units, is a quarter of the bound 2^-54 max|w| sum|vhat| of a block whose maxima are
            // normal.
            th = (a1 << (32 - L)) + ((a0 + (1ll << (L - 6))) >> (L - 5));
            xb = (e > 1 ? static_cast<int>(e) : 1) + ew - 2101;
          } else if (K == 3) {
            // binary32: sum = tot 2^(E + ew - 1263) exactly, |tot| < 2^121, rounded once to 61 bits.
            // The ragged last block and the blocks that are not exact on the block fixed point
            // take FP64.
            const int64_t rem = B.n - b * 32;
            __int128 tot;
            int E = 0;
            if (rem >= 32 && block_dot_f32(cw, t, W1, W0, tot, E)) {
              const unsigned __int128 A = tot < 0 ? -static_cast<unsigned __int128>(tot) : static_cast<unsigned __int128>(tot);
              const uint64_t hi = static_cast<uint64_t>(A >> 64), lo = static_cast<uint64_t>(A);
              const int bl = hi ? 128 - __clzll(static_cast<long long>(hi))
                                : (lo ? 64 - __clzll(static_cast<long long>(lo)) : 0);
              const int u = bl > 61 ? bl - 61 : 0;
              th = u ? static_cast<long long>((tot + (static_cast<__int128>(1) << (u - 1))) >> u)
                     : static_cast<long long>(tot);
              xb = u + E + ew - 1263;
            } else {
              const float* fv = reinterpret_cast<const float*>(cw);
              const double* wb = w + b * 32;
              double acc = 0.0;
#pragma unroll 1
              for (int k = 0; k < 32; ++k)
                if (k < rem) acc = fma(static_cast<double>(fv[k]), __ldg(wb + k), acc);
              split_double(acc, th, xb);
            }
          } else if (K == 2) {
            // bfloat16: sum = (a1 2^27 + a0) 2^(E + ew - 1223) exactly, |a1|, |a0| < 2^55; kept or
            // rounded to 62 bits as for binary16 below. The ragged last block and the blocks that
            // are not exact on the block fixed point take FP64.
            const int64_t rem = B.n - b * 32;
            int E = 0;
            __int128 tot = 0;
            const int kind = rem >= 32 ? block_dot_bf16(cw, t, W1, W0, a1, a0, tot, E) : 2;
            if (kind == 0) {
              const unsigned long long A = static_cast<unsigned long long>(a1 < 0 ? -a1 : a1);
              const int bl = 64 - __clzll(static_cast<long long>(A));
              const int u = bl > 35 ? bl - 35 : 0;
              th = u == 0 ? (a1 << 27) + a0 : (a1 << (27 - u)) + ((a0 + (1ll << (u - 1))) >> u);
              xb = u + E + ew - 1223;
            } else if (kind == 1) {  // the wide path: tot 2^(E + ew - 1263), rounded once to 61 bits
              const unsigned __int128 A = tot < 0 ? -static_cast<unsigned __int128>(tot) : static_cast<unsigned __int128>(tot);
              const uint64_t hi = static_cast<uint64_t>(A >> 64), lo = static_cast<uint64_t>(A);
              const int bl = hi ? 128 - __clzll(static_cast<long long>(hi))
                                : (lo ? 64 - __clzll(static_cast<long long>(lo)) : 0);
              const int u = bl > 61 ? bl - 61 : 0;
              th = u ? static_cast<long long>((tot + (static_cast<__int128>(1) << (u - 1))) >> u)
                     : static_cast<long long>(tot);
              xb = u + E + ew - 1263;
            } else {
              const uint16_t* hv = reinterpret_cast<const uint16_t*>(cw);
              const double* wb = w + b * 32;
              double acc = 0.0;
#pragma unroll 1
              for (int k = 0; k < 32; ++k)
                if (k < rem) acc = fma(widen_f32(static_cast<uint32_t>(hv[k]) << 16), __ldg(wb + k), acc);
              split_double(acc, th, xb);
            }
          } else {
            uint32_t emax = 0;
            block_dot_fp16(cw, t, W1, W0, a1, a0, emax);
            if (emax <= 15) {
              // sum = (a1 2^27 + a0) 2^(ew - 1099) exactly (V in units of 2^-24, W in units of
              // 2^(ew - 1075)); |a1| < 2^56, |a0| < 2^57. Kept exactly when |a1| < 2^35, else
              // rounded to 2^u units with u chosen so that 62 bits of the sum remain.
              const unsigned long long A = static_cast<unsigned long long>(a1 < 0 ? -a1 : a1);
              const int bl = 64 - __clzll(static_cast<long long>(A));
              const int u = bl > 35 ? bl - 35 : 0;
              th = u == 0 ? (a1 << 27) + a0 : (a1 << (27 - u)) + ((a0 + (1ll << (u - 1))) >> u);
              xb = u + ew - 1099;
            } else {
              // a value of magnitude >= 2 in the block (not a Krylov vector): the FP64 dot of the
              // decoded values with w, read again from memory, taken exactly as th * 2^xb
              const uint16_t* hv = reinterpret_cast<const uint16_t*>(cw);
              const double* wb = w + b * 32;
              const int64_t rem = B.n - b * 32;
              double acc = 0.0;
#pragma unroll 1
              for (int k = 0; k < 32; ++k)
                if (k < rem) acc = fma(widen_f16(hv[k]), __ldg(wb + k), acc);
              split_double(acc, th, xb);
            }
          }
        }
        post(vj, th, xb);
      }
      __syncwarp();
      if (lane == 0 && ok) mbar_arrive(&empty[s]);
      ps = s;
      pph = ph;
      first = false;
      if (++s == S) {
        s = 0;
        ph ^= 1u;
      }
    }
  }
  __syncthreads();
  if (flag_read(&flags[0])) {
    // wait (bounded) for this CTA's copies still in flight, then leave without a result
    if (t == 0) {
      for (int p = max(0, issued - S); p < issued; ++p)
        mbar_wait_bounded(&full[p % S], static_cast<uint32_t>((p / S) & 1));
    }
    return;
  }
  // partials of this CTA's vectors; vector v is then summed over the gridDim.x CTAs of its slice,
  // in a fixed order
  for (int v = v_lo + t; v < v_lo + nv; v += T) {
    double sacc = 0.0;
#pragma unroll
    for (int i = 0; i < C::kWarps; ++i) sacc += hpart[i * nvec + v];
    partials[(size_t)cid * nvec + v] = sacc;
  }
  if (arrive_last(counter, nctas, &flags[1])) {
    slice_sums<CBG_DOT_SUM_K, CBG_DOT_SUM_U>(partials, nvec, gridDim.x, gridDim.y, out, warp, C::kWarps);
    if (t == 0) *counter = 0;
  }
}

template <int L>
__global__ void __launch_bounds__(FDot<L>::kThreads) k_dot_frsz2(BasisView B, int nvec, const double* __restrict__ w,
                                                                 double* __restrict__ out,
                                                                 double* __restrict__ partials,
                                                                 unsigned int* counter, int* err, Gate gate) {
  dot_body<L, 0>(B, nvec, w, out, partials, counter, err, gate);
}

// The binary16 basis (two resident CTAs of 256 threads: registers capped at 128).
__global__ void __launch_bounds__(FDot<16, 1>::kThreads, 2) k_dot_fp16(BasisView B, int nvec,
                                                                          const double* __restrict__ w,
                                                                          double* __restrict__ out,
                                                                          double* __restrict__ partials,
                                                                          unsigned int* counter, int* err, Gate gate) {
  dot_body<16, 1>(B, nvec, w, out, partials, counter, err, gate);
}

__global__ void __launch_bounds__(FDot<32, 3>::kThreads, CBG_DOT_F32_MINB) k_dot_f32(BasisView B, int nvec, const double* __restrict__ w,
                                                                  double* __restrict__ out,
                                                                  double* __restrict__ partials,
                                                                  unsigned int* counter, int* err, Gate gate) {
  dot_body<32, 3>(B, nvec, w, out, partials, counter, err, gate);
}

__global__ void __launch_bounds__(FDot<16, 2>::kThreads, 2) k_dot_bf16(BasisView B, int nvec,
                                                                          const double* __restrict__ w,
                                                                          double* __restrict__ out,
                                                                          double* __restrict__ partials,
                                                                          unsigned int* counter, int* err, Gate gate) {
  dot_body<16, 2>(B, nvec, w, out, partials, counter, err, gate);
}

// ================================================================================================
// update: 8 consecutive values per thread, 4 threads per block, 32 blocks per tile (64 at l = 16),
// four basis vectors per pipeline stage, vectors in groups of at most 32 (the exact integer sums
// are per group)
// ================================================================================================

// S pipeline stages of 4 vectors: 2 when the grid fills the GPU (occupancy matters); 12 when it
// does not (small n: each CTA then has little work per stage, and only more copies in flight hide
// the latency).
// Shape of the full-grid update per code width (threads, resident CTAs the registers are capped
// for); the defaults are the measured best, settable at build time (-DCBG_UPD_<knob>_<l>=...).
#ifndef CBG_UPD_THREADS_16
#define CBG_UPD_THREADS_16 256
#endif
#ifndef CBG_UPD_THREADS_21
#define CBG_UPD_THREADS_21 128
#endif
#ifndef CBG_UPD_THREADS_32
#define CBG_UPD_THREADS_32 128
#endif
#ifndef CBG_UPD_MINB_16
#define CBG_UPD_MINB_16 3
#endif
#ifndef CBG_UPD_MINB_21
#define CBG_UPD_MINB_21 4
#endif
#ifndef CBG_UPD_MINB_32
#define CBG_UPD_MINB_32 5
#endif
#ifndef CBG_UPD_STAGES
#define CBG_UPD_STAGES 2
#endif

template <int L, int S = CBG_UPD_STAGES>
struct FUpd {
  // 128 threads and 32-block tiles (4 KB of l = 32 codes per vector and stage); at l = 16, 256
  // threads and 64-block tiles, whose larger copies measured 2.7% faster there (and 2.3% slower at
  // l = 32); the deep pipeline keeps 128
  static constexpr int kThreads =
      S == 12 ? 128 : (L == 16 ? CBG_UPD_THREADS_16 : (L == 21 ? CBG_UPD_THREADS_21 : CBG_UPD_THREADS_32));
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kBlocks = kThreads / 4;
  static constexpr int kVps = 4;  // basis vectors per stage
  static constexpr int kStages = S;
  // resident CTAs per SM the register allocation is capped for (measured per code width: l = 16,
  // at 256 threads, with a few spills at 3; l = 21 with 4; l = 32 with 5 at 96 registers, 2.4%
  // faster than 4 at 128 with an early load of w); the deep pipeline runs one CTA per SM
  static constexpr int kMinBlocks =
      S == 12 ? 1 : (L == 32 ? CBG_UPD_MINB_32 : (L == 21 ? CBG_UPD_MINB_21 : CBG_UPD_MINB_16));
  // vectors per group; five l = 32 CTAs per SM take groups of 28, whose smaller coefficient and
  // exponent tables (1.5 KB less) let five CTAs' shared memory fit in an SM up to restart 128, and
  // leave out the early load of w, whose 16 registers do not fit under the cap of 96
  static constexpr int kGroup = (L == 32 && kMinBlocks >= 5) ? 28 : 32;
  static constexpr bool kEarlyW = L == 32 && kMinBlocks <= 4;
  static_assert(kGroup % 4 == 0 && kGroup % kVps == 0, "a group is whole stages, split over 4 threads");
  static constexpr int kVecBytes = kBlocks * L * 4;
  static constexpr int kStageBytes = kVps * kVecBytes;
  // dynamic smem: stages | coefficient table [kGroup][kBlocks] (int2) | exponent words of one group
  //               [kGroup][kBlocks] | mantissas of h [nvec_max + 1] (int64) | exponents of h
  //               [nvec_max + 2] (int) | red[kWarps] | full, empty, exps barriers | flags
  static size_t smem_bytes(int nvec_max) {
    return (size_t)kStages * kStageBytes + (size_t)kGroup * kBlocks * 8 + (size_t)kGroup * kBlocks * 4 +
           (size_t)(nvec_max + 1) * 8 + (size_t)((nvec_max + 2) & ~1) * 4 + kWarps * 8 + (2 * kStages + 2) * 8 +
           16;
  }
};

// The 8 codes of this thread (values 8 q .. 8 q + 7 of block t/4, q = t%4) of one vector in a stage.
// For l = 32 the two 16-byte chunks are read in an order swizzled by bit 2 of t so that the 8 threads
// of a shared-memory phase hit distinct banks; slot k then holds value k ^ 4.
template <int L>
__device__ __forceinline__ void load_codes8(const uint32_t* st, int t, uint32_t (&c)[8]) {
  if (L == 32) {
    const int swap = (t >> 2) & 1;
    const uint4* p = reinterpret_cast<const uint4*>(st);
    const uint4 a = p[2 * t + swap], b = p[2 * t + 1 - swap];
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

// w[k0 + k] -= hv * v_k for a thread's 8 binary16 values c (k0 + k < n), in FP64: the rare path of a
// warp range holding a value of 2 or more, kept out of line so that it does not enlarge the
// update's loop body (the loop otherwise stalls on instruction fetch).
__device__ __noinline__ void fp16_axpy8_fp64(double* __restrict__ w, int64_t k0, int64_t n, double hv,
                                             const uint32_t (&c)[8]) {
#pragma unroll 1
  for (int k = 0; k < 8; ++k)
    if (k0 + k < n) w[k0 + k] = fma(-hv, widen_f16(c[k]), w[k0 + k]);
}

// H: the basis is stored as binary16 in the l = 16 layout, without exponent words. Its values below 2
// are exact integers in units of 2^-24 (fp16_fixed), i.e. codes of a block with the fixed exponent
// 1023 and LE = 26 code bits; a vector holding a larger value in a thread's range is subtracted by
// that warp in FP64 instead (global read-modify-write of w, which the tile's end then reads).
template <int L, int SD, bool H>
__device__ __forceinline__ void update_body(const BasisView& B, int nvec_arg, const int* nvec_dev,
                                            const double* __restrict__ hcoef, int negate, double* __restrict__ w,
                                            double* __restrict__ partials, unsigned int* counter, int* err,
                                            const NormEpilogue& epi, const Gate& gate) {
  static_assert(!H || L == 16, "binary16 blocks have the l = 16 layout");
  constexpr int LE = H ? 26 : L;  // code bits, sign included
  using C = FUpd<L, SD>;
  constexpr int T = C::kThreads, NBT = C::kBlocks, G = C::kGroup, S = C::kStages, VPS = C::kVps;
  if (gate_skip(gate)) return;
  const int nvec = nvec_dev ? *(volatile const int*)nvec_dev : nvec_arg;
  const int nvec_cap = nvec_dev ? nvec_arg : nvec;
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* stages = smem;
  int2* gam = reinterpret_cast<int2*>(smem + S * C::kStageBytes);
  uint32_t* exq = reinterpret_cast<uint32_t*>(gam + G * NBT);
  long long* hman = reinterpret_cast<long long*>(exq + G * NBT);  // signed 53-bit mantissa of h_i
  int* hexp = reinterpret_cast<int*>(hman + nvec_cap + 1);        // its effective IEEE exponent
  double* red = reinterpret_cast<double*>(hexp + ((nvec_cap + 2) & ~1));
  uint64_t* full = reinterpret_cast<uint64_t*>(red + C::kWarps);
  uint64_t* empty = full + S;
  uint64_t* ebar = empty + S;  // exponent words of the next group ([1] unused, keeps alignment)
  // per stage s: rel[2 s] counts the warps that released it, rel[2 s + 1] is the last unit issued
  // into it (the "empty" slots hold these counters)
  unsigned* rel = reinterpret_cast<unsigned*>(empty);
  int* flags = reinterpret_cast<int*>(ebar + 2);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int blk = t >> 2, q = t & 3;
  const bool sw = L == 32 && ((t >> 2) & 1);  // slot k holds value k ^ 4 (swizzled l = 32 loads)
  const int64_t nb = (B.n + 31) / 32;
  int64_t b0, b1;
  cta_block_range(nb, gridDim.x, blockIdx.x, &b0, &b1);
  const int ntiles = static_cast<int>((b1 - b0 + NBT - 1) / NBT);
  const int units = (nvec + VPS - 1) / VPS;  // stages per tile
  const int total = ntiles * units;

  // h_i = hman_i 2^{hexp_i - 1075} exactly (subnormals: hexp 1, no implicit bit)
  for (int i = t; i < nvec; i += T) {
    const uint64_t u = static_cast<uint64_t>(__double_as_longlong(hcoef[i]));
    const int e = static_cast<int>((u >> 52) & 0x7FF);
    const long long m = static_cast<long long>((u & ((1ull << 52) - 1)) | (e ? 1ull << 52 : 0ull));
    hman[i] = ((u >> 63) != 0) != (negate != 0) ? -m : m;
    hexp[i] = e > 1 ? e : 1;
  }
  // The group sums are kept in units of 2^(sh) against their block scale, sh = l - 5 + gb, so
  // that up to 2^gb of them add up in 63 bits (binary16: sh from the sums' actual size, below).
  const int ngroups = (nvec + G - 1) / G;
  const int gb = ngroups > 1 ? 32 - __clz(ngroups - 1) : 0;
  const int sh_fixed = L - 5 + gb;
  if (t == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      rel[2 * s] = 0;
      rel[2 * s + 1] = static_cast<unsigned>(s);
    }
    mbar_init(&ebar[0], 1);
    fence_mbar_init();
    flags[0] = 0;
  }
  __syncthreads();

  auto issue = [&](int p) {  // stage unit p: vectors VPS u .. of tile p / units
    const int tile = p / units, u = p - tile * units, s = p % S;
    const int v0 = u * VPS, nv = min(VPS, nvec - v0);
    const int64_t tb0 = b0 + (int64_t)tile * NBT;
    const int nbt = static_cast<int>(min((int64_t)NBT, b1 - tb0));
    const uint32_t cbytes = static_cast<uint32_t>((nbt * L * 4 + 15) & ~15);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&full[s], cbytes * nv);
    for (int j = 0; j < nv; ++j)
      bulk_g2s(stages + s * C::kStageBytes + j * C::kVecBytes, B.vals + (int64_t)(v0 + j) * B.vstride + tb0 * L * 4,
               cbytes, &full[s]);
  };
  // Exponent words of group [g0, g0 + G) for tile `tile`, one bulk copy per vector into exq[v][*],
  // issued by the 32 lanes of warp 0 (lane 0 first posts the expected byte count).
  auto issue_exps = [&](int tile, int g0) {
    const int64_t tb0 = b0 + (int64_t)tile * NBT;
    const int nbt = static_cast<int>(min((int64_t)NBT, b1 - tb0));
    const int gn = min(G, nvec - g0);
    const uint32_t ebytes = static_cast<uint32_t>((nbt * 4 + 15) & ~15);
    if (lane == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&ebar[0], ebytes * gn);
    }
    __syncwarp();
    for (int v = lane; v < gn; v += 32)
      bulk_g2s(exq + v * NBT, reinterpret_cast<const uint8_t*>(B.exps) + (int64_t)(g0 + v) * B.estride + tb0 * 4,
               ebytes, &ebar[0]);
  };
  int issued = 0, eissued = 0;  // the first S code copies (thread 0); exponent-group copies (warp 0)
  if (!H && warp == 0 && ntiles > 0 && nvec > 0) {
    issue_exps(0, 0);
    ++eissued;
  }
  if (t == 0) {
    for (; issued < S && issued < total; ++issued) issue(issued);
  }
  int egroups = 0;  // exponent copies consumed so far (phase of ebar)

  double nrm = 0.0;
  int s = 0;            // stage of the current unit and the phase parity of its barriers
  uint32_t ph = 0;
  int pu = 0;           // the current unit
  bool dead = false;    // this warp gave up waiting (warp-uniform; it then only runs to the next barrier)
  bool aborted = false;
  for (int tile = 0; tile < ntiles && !aborted; ++tile) {
    const int64_t tb0 = b0 + (int64_t)tile * NBT;
    const int nbt = static_cast<int>(min((int64_t)NBT, b1 - tb0));
    const bool active = blk < nbt;
    const int64_t k0 = (tb0 + blk) * 32 + q * 8;  // first of this thread's 8 values
    // l = 32: this thread's 8 values of w are loaded now and arrive while the tile streams (1% at
    // l = 32; at l = 16 and 21 the registers are better spent on the pipeline)
    double wpre[8];
    if (C::kEarlyW && active && k0 + 8 <= B.n) {
      const double2* pw = reinterpret_cast<const double2*>(w + k0);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const double2 v = pw[i];
        wpre[2 * i] = v.x;
        wpre[2 * i + 1] = v.y;
      }
    }
    // sum over the groups so far, in units of 2^xc
    long long tacc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) tacc[k] = 0;
    int xc = 0;
    for (int g0 = 0; g0 < nvec; g0 += G) {
      const int gn = min(G, nvec - g0);
      __syncthreads();  // the previous group's coefficient table is no longer read
      if (flag_read(&flags[0])) {  // read after a barrier: the same decision in every thread
        aborted = true;
        break;
      }
      bool eok = true;
      if (!H) {
        eok = mbar_wait_bounded(&ebar[0], static_cast<uint32_t>(egroups & 1));
        ++egroups;
        if (!eok) {
          flags[0] = 1;
          atomicOr(err, kDevErrTimeout);
        }
      }
      // rexp = max over the group of (Eh_i + Ebar_{i,b}): exponent of the block's largest term;
      // the 4 threads of a block split the group's vectors and combine with shuffles.
      uint32_t ev[G / 4];
      int r = 0;
#pragma unroll
      for (int kk = 0; kk < G / 4; ++kk) {
        const int v = q + 4 * kk;
        const uint32_t e = H ? 1023u : ((v < gn && active && eok) ? exq[v * NBT + blk] : 0u);
        ev[kk] = e;
        if (v < gn) r = max(r, hexp[g0 + v] + (e > 1 ? static_cast<int>(e) : 1));
      }
      r = max(r, __shfl_xor_sync(0xffffffffu, r, 1));
      r = max(r, __shfl_xor_sync(0xffffffffu, r, 2));
      // G_{i,b} = h_i 2^{Ebar_{i,b} + 1075 - rexp} rounded to an integer (half up): the mantissa of
      // h_i shifted right by rexp - hexp_i - Ebar_{i,b} >= 0, which puts the block's largest term at
      // 53 bits, |G| <= 2^53; stored as G0 = G mod 2^27, G1 = floor(G / 2^27)
#pragma unroll
      for (int kk = 0; kk < G / 4; ++kk) {
        const int v = q + 4 * kk;
        if (v < gn) {
          const uint32_t e = ev[kk];
          const int d = r - hexp[g0 + v] - (e > 1 ? static_cast<int>(e) : 1);
          const long long m = hman[g0 + v];
          const long long gm = d == 0 ? m : (d < 64 ? ((m >> (d - 1)) + 1) >> 1 : 0);
          gam[v * NBT + blk] = make_int2(static_cast<int32_t>(gm & ((1ll << 27) - 1)), static_cast<int32_t>(gm >> 27));
        }
      }
      __syncthreads();
      // the exponent words of the next group arrive while this group is processed
      if (!H && warp == 0 && !flag_read(&flags[0])) {
        if (g0 + G < nvec) {
          issue_exps(tile, g0 + G);
          ++eissued;
        } else if (tile + 1 < ntiles) {
          issue_exps(tile + 1, 0);
          ++eissued;
        }
      }
      long long acc0[8], acc1[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc0[k] = acc1[k] = 0;
      for (int v = 0; v < gn; v += VPS) {
        bool ok = false;
        if (!dead) {
          ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[s], ph));
          if (!ok) {
            dead = true;
            if (lane == 0) {
              flags[0] = 1;
              atomicOr(err, kDevErrTimeout);
            }
          }
        }
        if (!H && active && ok) {
          const uint8_t* st = stages + s * C::kStageBytes;
#pragma unroll
          for (int j = 0; j < VPS; ++j) {
            if (v + j < gn) {
              uint32_t c[8];
              load_codes8<L>(reinterpret_cast<const uint32_t*>(st + j * C::kVecBytes), t, c);
              const int2 gp = gam[(v + j) * NBT + blk];
#pragma unroll
              for (int k = 0; k < 8; ++k) {
                const int32_t sv = code_to_int<L>(c[k]);
                mac_wide(acc0[k], sv, gp.x);
                mac_wide(acc1[k], sv, gp.y);
              }
            }
          }
        }
        if (H && ok) {  // every lane takes part: the warp decides together which path a vector takes
          const uint8_t* st = stages + s * C::kStageBytes;
#pragma unroll
          for (int j = 0; j < VPS; ++j) {
            if (v + j < gn) {
              uint32_t c[8];
              load_codes8<L>(reinterpret_cast<const uint32_t*>(st + j * C::kVecBytes), t, c);
              uint32_t emax = 0;
              int32_t sv[8];
#pragma unroll
              for (int k = 0; k < 8; ++k) sv[k] = fp16_fixed(c[k], emax);
              if (!__any_sync(0xffffffffu, active && emax > 15)) {
                if (active) {
                  const int2 gp = gam[(v + j) * NBT + blk];
#pragma unroll
                  for (int k = 0; k < 8; ++k) {
                    mac_wide(acc0[k], sv[k], gp.x);
                    mac_wide(acc1[k], sv[k], gp.y);
                  }
                }
              } else if (active) {  // a value of magnitude >= 2 (not a Krylov vector): FP64
                fp16_axpy8_fp64(w, k0, B.n, negate ? -hcoef[g0 + v + j] : hcoef[g0 + v + j], c);
              }
            }
          }
        }
        // release the stage; the warp that releases it last refills it at once with unit pu + S (a
        // warp that gave up waiting never releases, so the others give up in turn)
        __syncwarp();
        if (lane == 0 && ok && atom_add_acq_rel_cta(&rel[2 * s], 1u) == C::kWarps - 1) {
          rel[2 * s] = 0;
          if (pu + S < total) {
            rel[2 * s + 1] = static_cast<unsigned>(pu + S);
            issue(pu + S);
          }
        }
        ++pu;
        if (++s == S) {
          s = 0;
          ph ^= 1u;
        }
      }
      if (active && !dead) {
        // sum_i s G = acc1 2^27 + acc0 exactly (|.| < 2^(l+57)) at scale 2^{rexp - 2096 - l}, rounded
        // to units of 2^sh (at most 2^(gb-58) of the block's largest possible term, 2^(l+52) units):
        // |th| < 2^(62-gb). It joins the running sum at the larger of the two block scales; every
        // rescaling rounds to nearest, again at most 2^(gb-58) of the larger largest term.
        // binary16: the largest of the thread's sums sets the unit, keeping 61 - gb bits of it (its
        // codes are far below their bound 2^25 for the small values of a Krylov vector)
        int sh = sh_fixed;
        if (H) {
          unsigned long long o1 = 0, o0 = 0;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            o1 |= static_cast<unsigned long long>(acc1[k] < 0 ? -acc1[k] : acc1[k]);
            o0 |= static_cast<unsigned long long>(acc0[k] < 0 ? -acc0[k] : acc0[k]);
          }
          const int bl = max(o1 ? 64 - __clzll(static_cast<long long>(o1)) + 27 : 0,
                             64 - __clzll(static_cast<long long>(o0)));
          sh = max(0, bl - (61 - gb));
        }
        long long th[8];
        if (sh == 0) {
#pragma unroll
          for (int k = 0; k < 8; ++k) th[k] = (acc1[k] << 27) + acc0[k];
        } else if (sh <= 27) {
#pragma unroll
          for (int k = 0; k < 8; ++k) th[k] = (acc1[k] << (27 - sh)) + ((acc0[k] + (1ll << (sh - 1))) >> sh);
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const long long x = acc1[k] + (acc0[k] >> 27);
            const long long y = (acc0[k] & ((1ll << 27) - 1)) + (1ll << (sh - 1));
            th[k] = (x + (y >> 27)) >> (sh - 27);
          }
        }
        // th is in units of 2^xg (sum_i s G in units of 2^(rexp - 2096 - LE))
        const int xg = r - 2096 - LE + sh;
        if (g0 == 0 || xg >= xc) {
          const int dd = g0 == 0 ? 0 : xg - xc;
#pragma unroll
          for (int k = 0; k < 8; ++k) tacc[k] = round_shift_right(tacc[k], dd) + th[k];
          xc = xg;
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) tacc[k] += round_shift_right(th[k], xc - xg);
        }
      }
    }
    if (aborted || dead) continue;
    // value k: w_k - tacc_k 2^x, one conversion and one fused multiply-add (the product tv 2^x is
    // exact in the normal range, so the FMA rounds exactly like the subtraction of the product)
    double tv[8];
    const int x = xc;
    const bool xnorm = x >= -1022 && x <= 1023;
    const double p2 = -pow2_normal(xnorm ? x : 0);
#pragma unroll
    for (int k = 0; k < 8; ++k) tv[k] = static_cast<double>(tacc[k]);
    auto sub = [&](double wk, double t) { return xnorm ? fma(t, p2, wk) : wk - scale_pow2(t, x); };
    if (active) {
      if (k0 + 8 <= B.n) {
        double2* p = reinterpret_cast<double2*>(w + k0);
        double cur[8];
        if (C::kEarlyW) {
#pragma unroll
          for (int i = 0; i < 8; ++i) cur[i] = wpre[i];
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const double2 v = p[i];
            cur[2 * i] = v.x;
            cur[2 * i + 1] = v.y;
          }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) cur[k] = sub(cur[k], sw ? tv[k ^ 4] : tv[k]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          p[i] = make_double2(cur[2 * i], cur[2 * i + 1]);
          nrm = fma(cur[2 * i], cur[2 * i], nrm);
          nrm = fma(cur[2 * i + 1], cur[2 * i + 1], nrm);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int64_t idx = k0 + (sw ? (k ^ 4) : k);
          if (idx < B.n) {
            const double nv = sub(w[idx], tv[k]);
            w[idx] = nv;
            nrm = fma(nv, nv, nrm);
          }
        }
      }
    }
  }
  __syncthreads();
  if (flag_read(&flags[0])) {
    if (t == 0) {
      for (int st = 0; st < S; ++st) {  // the last unit issued into each stage (complete if consumed)
        const int p = static_cast<int>(rel[2 * st + 1]);
        if (p < total) mbar_wait_bounded(&full[st], static_cast<uint32_t>((p / S) & 1));
      }
      if (eissued > egroups) mbar_wait_bounded(&ebar[0], static_cast<uint32_t>(egroups & 1));
    }
    return;
  }
  // ||w||^2: CTA partial, then the last CTA reduces all partials in a fixed order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (lane == 0) red[warp] = nrm;
  __syncthreads();
  if (t == 0) {
    double sacc = 0.0;
    for (int i = 0; i < C::kWarps; ++i) sacc += red[i];
    partials[blockIdx.x] = sacc;
  }
  if (arrive_last(counter, gridDim.x, &flags[1])) {
    if (warp == 0) {
      const double sacc = warp_sum_strided(partials, gridDim.x, 1);
      if (lane == 0) norm_epilogue(epi, sacc, err);
    }
    if (t == 0) *counter = 0;
  }
}

template <int L, int SD>
__global__ void __launch_bounds__(FUpd<L, SD>::kThreads, FUpd<L, SD>::kMinBlocks)
    k_update_frsz2(BasisView B, int nvec_arg, const int* nvec_dev, const double* __restrict__ hcoef, int negate,
                   double* __restrict__ w, double* __restrict__ partials, unsigned int* counter, int* err,
                   NormEpilogue epi, Gate gate) {
  update_body<L, SD, false>(B, nvec_arg, nvec_dev, hcoef, negate, w, partials, counter, err, epi, gate);
}

template <int SD>
__global__ void __launch_bounds__(FUpd<16, SD>::kThreads, FUpd<16, SD>::kMinBlocks)
    k_update_fp16(BasisView B, int nvec_arg, const int* nvec_dev, const double* __restrict__ hcoef, int negate,
                  double* __restrict__ w, double* __restrict__ partials, unsigned int* counter, int* err,
                  NormEpilogue epi, Gate gate) {
  update_body<16, SD, true>(B, nvec_arg, nvec_dev, hcoef, negate, w, partials, counter, err, epi, gate);
}

// ================================================================================================
// launchers
// ================================================================================================

namespace {
template <typename K>
const void* fnp(K k) {
  return reinterpret_cast<const void*>(k);
}
}  // namespace

// The dot of a binary16 basis on the integer pipeline (FDot<16, true>).
int int_dot_launch(const BasisView& B, int nvec, const double* w, double* out, double* partials,
                    unsigned int* counter, int* err, const Gate& gate, int max_grid, cudaStream_t stream) {
  const bool f32 = B.fmt == CBG_FP32, bf = B.fmt == CBG_BF16;
  const int T = f32 ? FDot<32, 3>::kThreads : FDot<16, 1>::kThreads;
  static_assert(FDot<16, 1>::kThreads == FDot<16, 2>::kThreads, "one configuration for the 16-bit formats");
  const void* fn = f32 ? fnp(k_dot_f32) : (bf ? fnp(k_dot_bf16) : fnp(k_dot_fp16));
  const size_t smem = f32 ? FDot<32, 3>::smem_bytes(nvec) : FDot<16, 1>::smem_bytes(nvec);
  int gx, full;
  int st = basis_launch_config(fn, T, smem, (B.n + 31) / 32, T / CBG_DOT_MIN_DIV, max_grid, &gx, &full);
  if (st) return st;
  const dim3 grid(gx, dot_vector_split(gx, full, nvec, max_grid));
  if (f32)
    k_dot_f32<<<grid, T, smem, stream>>>(B, nvec, w, out, partials, counter, err, gate);
  else if (bf)
    k_dot_bf16<<<grid, T, smem, stream>>>(B, nvec, w, out, partials, counter, err, gate);
  else
    k_dot_fp16<<<grid, T, smem, stream>>>(B, nvec, w, out, partials, counter, err, gate);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "integer-pipeline cast dot launch");
}

int frsz2_dot_launch(const BasisView& B, int nvec, const double* w, double* out, double* partials,
                     unsigned int* counter, int* err, const Gate& gate, int max_grid, cudaStream_t stream) {
  const void* fn;
  size_t smem;
  switch (B.l) {
    case 32: fn = fnp(k_dot_frsz2<32>); smem = FDot<32>::smem_bytes(nvec); break;
    case 21: fn = fnp(k_dot_frsz2<21>); smem = FDot<21>::smem_bytes(nvec); break;
    case 16: fn = fnp(k_dot_frsz2<16>); smem = FDot<16>::smem_bytes(nvec); break;
    default: return CBG_ERR_INVALID_ARG;
  }
  int gx, full;
  const int thr = B.l == 16 ? FDot<16>::kThreads : (B.l == 21 ? FDot<21>::kThreads : FDot<32>::kThreads);
  int st = basis_launch_config(fn, thr, smem, (B.n + 31) / 32, thr / CBG_DOT_MIN_DIV, max_grid, &gx, &full);
  if (st) return st;
  const dim3 grid(gx, dot_vector_split(gx, full, nvec, max_grid));
  switch (B.l) {
    case 32: k_dot_frsz2<32><<<grid, thr, smem, stream>>>(B, nvec, w, out, partials, counter, err, gate); break;
    case 21: k_dot_frsz2<21><<<grid, thr, smem, stream>>>(B, nvec, w, out, partials, counter, err, gate); break;
    default: k_dot_frsz2<16><<<grid, thr, smem, stream>>>(B, nvec, w, out, partials, counter, err, gate); break;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "frsz2 dot launch");
}

namespace {

template <int L, int S, bool H>
int frsz2_update_launch_t(const BasisView& B, int nvec, const int* nvec_dev, const double* h, int negate, double* w,
                          double* partials, unsigned int* counter, int* err, const NormEpilogue& epi,
                          const Gate& gate, int grid, cudaStream_t stream) {
  const void* fn = H ? fnp(k_update_fp16<S>) : fnp(k_update_frsz2<L, S>);
  const size_t smem = FUpd<L, S>::smem_bytes(nvec);
  int g;
  constexpr int T = FUpd<L, S>::kThreads;
  int st = basis_launch_config(fn, T, smem, (B.n + 31) / 32, T / 16, kMaxGrid, &g, nullptr);
  if (st) return st;
  if (grid > 0 && grid < g) g = grid;
  if (H)
    k_update_fp16<S><<<g, T, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate);
  else
    k_update_frsz2<L, S><<<g, T, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "frsz2 update launch");
}

template <int L, bool H = false>
int frsz2_update_launch_l(const BasisView& B, int nvec, const int* nvec_dev, const double* h, int negate, double* w,
                          double* partials, unsigned int* counter, int* err, const NormEpilogue& epi,
                          const Gate& gate, cudaStream_t stream) {
  DeviceInfo di;
  int st = device_info(&di);
  if (st) return st;
  // CTAs the blocks need (CBG_UPD_DEEP_BLOCKS at least per CTA): fewer than SMs means an
  // underfilled GPU
  const int64_t need = ((B.n + 31) / 32 + CBG_UPD_DEEP_BLOCKS - 1) / CBG_UPD_DEEP_BLOCKS;
  if (need < di.sms)
    return frsz2_update_launch_t<L, 12, H>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate, 0,
                                           stream);
  return frsz2_update_launch_t<L, CBG_UPD_STAGES, H>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate,
                                                     0, stream);
}

}  // namespace

// The update of a binary16 basis on the integer pipeline (update_body<16, S, true>).
int fp16_update_launch(const BasisView& B, int nvec, const int* nvec_dev, const double* h, int negate, double* w,
                       double* partials, unsigned int* counter, int* err, const NormEpilogue& epi, const Gate& gate,
                       cudaStream_t stream) {
  return frsz2_update_launch_l<16, true>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate, stream);
}

int frsz2_update_launch(const BasisView& B, int nvec, const int* nvec_dev, const double* h, int negate, double* w,
                        double* partials, unsigned int* counter, int* err, const NormEpilogue& epi,
                        const Gate& gate, cudaStream_t stream) {
  switch (B.l) {
    case 32: return frsz2_update_launch_l<32>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate, stream);
    case 21: return frsz2_update_launch_l<21>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate, stream);
    case 16: return frsz2_update_launch_l<16>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate, stream);
    default: return CBG_ERR_INVALID_ARG;
  }
}

}  // namespace cbg
