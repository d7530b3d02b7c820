// The on-chip restart cycle: one launch of one thread-block cluster runs a whole restart cycle of
// CB-GMRES (Fig. 1 steps 1-17) and the residual that starts the next cycle, for systems whose
// compressed Krylov basis fits in the cluster's shared memory.
//
// At a few thousand rows the streamed path is bound by latency, not HBM: an Arnoldi step issues
// about seven kernels and each of them pays a launch and a grid-wide reduction. Here CTA c of the
// cluster owns the 32-aligned row slice [c R, (c + 1) R) and keeps, for every basis slot, its slice
// of the stored vector (FRSZ2 codes and block exponents, or the cast values) in its own shared
// memory: the basis never leaves the SMs. The CTAs exchange only
//  * the SpMV input z_j = M^{-1} v_j (FP64), read by the other CTAs through distributed shared
//    memory (ld.shared::cluster) for the columns they need;
//  * reductions (||w||^2 and V^T w): every CTA writes its partials, one cluster barrier follows,
//    and every CTA sums the partials of all CTAs in the same fixed pairwise tree over the ranks,
//    so every CTA holds the same bits.
// Every CTA then runs the Givens recurrence (step 17's rotations) and the back-substitution itself
// on identical inputs, so the decisions (second pass, breakdown, convergence, step cap) agree in
// every CTA: the cluster's control flow is uniform and every cluster barrier is reached by all of
// its threads. There is no spin-wait: the only waits are the hardware cluster and CTA barriers.
//
// The arithmetic is that of the streamed kernels. The FRSZ2 dot multiplies the codes exactly with
// a 54-bit block fixed point of w and rounds once per (vector, block); the FRSZ2 update forms the
// same per-group integer coefficients, sums and roundings as k_update_frsz2, so every element of
// w - V h is bit-identical to the streamed update; cast formats widen to FP64 and take one FMA per
// (vector, element), in the streamed update's order. Only the order of the FP64 sums over blocks
// and CTAs differs. At the end of the cycle the basis slices are copied to the context's basis
// storage in HBM, in the streamed layout, so the stored vectors can still be read back.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "decode.cuh"
#include "frsz2_block.cuh"
#include "kernels.cuh"

namespace cbg {

namespace {

constexpr int kOcThreads = 256;
constexpr int kOcWarps = kOcThreads / 32;
constexpr int kOcMaxSlots = 128;  // restart + 1: the dot's lanes hold at most four vectors each

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t cluster_ctas() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// Every thread of every CTA of the cluster arrives; shared-memory writes before it are visible to
// distributed shared-memory reads after it. The barrier instructions are .aligned: every lane of a
// warp must execute them together, so the warp is first reconverged (callers reach it straight
// from loops in which only some lanes iterate).
__device__ __forceinline__ void cluster_sync() {
  __syncwarp();
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::
          : "memory");
}

// The value at shared-memory location p of cluster CTA `rank` (p is this CTA's address of it).
// Only read after a cluster barrier: volatile asm keeps it after the barrier's asm, and without a
// memory clobber independent reads can be in flight together.
__device__ __forceinline__ double dsmem_ld(const double* p, uint32_t rank) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_addr(p)), "r"(rank));
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}

// p[0] + ... + p[7 stride] as a fixed pairwise tree (three dependent adds instead of seven).
__device__ __forceinline__ double sum8(const double* p, int stride) {
  const double a = p[0] + p[stride], b = p[2 * stride] + p[3 * stride];
  const double c = p[4 * stride] + p[5 * stride], d = p[6 * stride] + p[7 * stride];
  return (a + b) + (c + d);
}

template <int L>
__device__ __forceinline__ uint32_t code_at(const uint32_t* block_words, int k) {
  if (L == 32) return block_words[k];
  if (L == 16) return reinterpret_cast<const uint16_t*>(block_words)[k];
  const int bit = 21 * k, a = bit >> 5;
  const uint32_t lo = block_words[a], hi = a + 1 < 21 ? block_words[a + 1] : 0u;
  return __funnelshift_r(lo, hi, bit & 31) & 0x1FFFFFu;
}

template <int F>
__device__ __forceinline__ double cast_at(const uint8_t* slot, int i) {
  if (F == CBG_FP64) return reinterpret_cast<const double*>(slot)[i];
  if (F == CBG_FP32) return widen_f32(reinterpret_cast<const uint32_t*>(slot)[i]);
  const uint32_t h = reinterpret_cast<const uint16_t*>(slot)[i];
  return F == CBG_FP16 ? widen_f16(h) : widen_f32(h << 16);
}

// Per-CTA scalars of the cycle (identical in every CTA).
struct OcState {
  double omega2, hn2, hn2_first, rcp, implicit, beta2, xc, hn, hn_first;
  int stop, reorth, m_eff, breakdown, reorth_count, stored, m_ls;
};

struct OcSmem {
  uint8_t* codes;   // slot s at codes + s * slot_bytes
  uint32_t* exq;    // slot s at exq + s * exp_words (FRSZ2)
  double* z;        // [R] SpMV input of this CTA's rows (read by the other CTAs)
  double* w;        // [R]
  double* hp;       // [2][M1 + 1] partials of this CTA (double-buffered)
  double* wpart;    // [warps][M1]
  double* h;        // [M1 + 1] first-pass projections, reduced
  double* u;        // [M1 + 1] second-pass projections, reduced
  double* col;      // [M1 + 1] the column being rotated
  double* cs;       // [M1]
  double* sn;       // [M1]
  double* g;        // [M1 + 1]
  double* y;        // [M1]
  double* Rm;       // [m][M1] the rotated Hessenberg columns (R of step 17)
  long long* hman;  // [M1]
  int* hexp;        // [M1]
  int2* gt;         // [warps][32]
  double* red;      // [warps]
  OcState* st;
};

__device__ __forceinline__ OcSmem oc_carve(uint8_t* smem, const OcLayout& lay, int m) {
  OcSmem s;
  s.codes = smem + lay.off_codes;
  s.exq = reinterpret_cast<uint32_t*>(smem + lay.off_exps);
  s.z = reinterpret_cast<double*>(smem + lay.off_z);
  s.w = s.z + lay.rows;
  s.hp = reinterpret_cast<double*>(smem + lay.off_vec);
  const int M1 = m + 1;
  s.wpart = s.hp + 2 * (M1 + 1);
  s.h = s.wpart + kOcWarps * M1;
  s.u = s.h + (M1 + 1);
  s.col = s.u + (M1 + 1);
  s.cs = s.col + (M1 + 1);
  s.sn = s.cs + M1;
  s.g = s.sn + M1;
  s.y = s.g + (M1 + 1);
  s.Rm = s.y + M1;
  s.red = s.Rm + (size_t)m * M1;
  s.hman = reinterpret_cast<long long*>(s.red + kOcWarps);
  s.gt = reinterpret_cast<int2*>(s.hman + M1);
  s.hexp = reinterpret_cast<int*>(s.gt + kOcWarps * 32);
  s.st = reinterpret_cast<OcState*>(smem + lay.off_state);
  return s;
}

template <int F, int L>
__global__ void __launch_bounds__(kOcThreads, 1) k_cycle_onchip(OnchipArgs a, OcLayout lay) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t rank = cluster_rank(), nctas = cluster_ctas();
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int R = lay.rows, NB = R / 32, m = a.m, M1 = m + 1, n = a.n;
  const int row0 = static_cast<int>(rank) * R;
  OcSmem s = oc_carve(smem, lay, m);
  OcState& S = *s.st;
  SolverCtl* ctl = a.ctl;
  const double eta = ctl->eta, bnorm = ctl->bnorm, tol = ctl->tol;
  int buf = 0;

  // Sum over the CTA's threads of v into hp[buf][slot]: a shuffle tree per warp, then warp 0 adds
  // the eight warp sums as a three-level tree.
  auto cta_sum = [&](double v, int slot) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s.red[warp] = v;
    __syncthreads();
    if (warp == 0) {  // the warp sums, as a three-level tree over lanes 0-7
      double r = lane < kOcWarps ? s.red[lane] : 0.0;
#pragma unroll
      for (int o = 1; o < kOcWarps; o <<= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
      if (lane == 0) s.hp[buf * (M1 + 1) + slot] = r;
    }
  };
  // out[i] = sum over the cluster's CTAs of their hp[buf][i], i < cnt, read through distributed
  // shared memory after the barrier.
  auto cluster_sum = [&](int cnt, double* out) {
    cluster_sync();
    const double* src = s.hp + buf * (M1 + 1);
    // four lanes per value, each over four ranks, then two shuffle levels: a fixed pairwise tree
    // over the 16 ranks (absent ranks add +0.0) in five FP64 instructions per warp
    const int g = t & 3;
    for (int i0 = 0; i0 < cnt; i0 += kOcThreads / 4) {
      const int i = i0 + (t >> 2);
      double v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t c = static_cast<uint32_t>(4 * g + k);
        v[k] = (i < cnt && c < nctas) ? (c == rank ? src[i] : dsmem_ld(src + i, c)) : 0.0;
      }
      double r = (v[0] + v[1]) + (v[2] + v[3]);
      r += __shfl_xor_sync(0xffffffffu, r, 1);
      r += __shfl_xor_sync(0xffffffffu, r, 2);
      if (i < cnt && g == 0) out[i] = r;
    }
    buf ^= 1;
    __syncthreads();
  };

  // v := w / hdiv (correctly rounded; rcp = RN(1 / hdiv)) into basis slot `slot` (Fig. 1 steps
  // 13-14; step 1 for slot 0) and z := M^{-1} v.
  auto store = [&](int slot, double hdiv, double rcp) {
    uint8_t* sb = s.codes + (size_t)slot * lay.slot_bytes;
    for (int b = warp; b < NB; b += kOcWarps) {
      const int i = b * 32 + lane, gi = row0 + i;
      const double v = gi < n ? div_rn(s.w[i], hdiv, rcp) : 0.0;  // rows past n: the padding +0.0
      s.z[i] = gi < n ? (a.dinv ? v * a.dinv[gi] : v) : 0.0;
      if (F == CBG_FRSZ2) {
        const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(v));
        const uint32_t emax = __reduce_max_sync(0xffffffffu, static_cast<uint32_t>((bits >> 52) & 0x7FF));
        const uint32_t c = make_code<L>(bits, emax > 1 ? static_cast<int>(emax) : 1);
        uint32_t* cw = reinterpret_cast<uint32_t*>(sb) + b * L;
        if (lane == 0) s.exq[slot * lay.exp_words + b] = emax;
        if (L == 32) {
          cw[lane] = c;
        } else if (L == 16) {
          reinterpret_cast<uint16_t*>(cw)[lane] = static_cast<uint16_t>(c);
        } else {
          const int i0 = (32 * lane) / 21;
          const uint32_t c0 = __shfl_sync(0xffffffffu, c, i0 < 32 ? i0 : 31);
          const uint32_t c1 = __shfl_sync(0xffffffffu, c, i0 + 1 < 32 ? i0 + 1 : 31);
          const uint32_t c2 = __shfl_sync(0xffffffffu, c, i0 + 2 < 32 ? i0 + 2 : 31);
          const uint64_t win = static_cast<uint64_t>(c0) | (static_cast<uint64_t>(c1) << 21) |
                               (static_cast<uint64_t>(c2) << 42);
          if (lane < 21) cw[lane] = static_cast<uint32_t>(win >> (32 * lane - 21 * i0));
        }
      } else if (F == CBG_FP64) {
        reinterpret_cast<double*>(sb)[i] = v;
      } else if (F == CBG_FP32) {
        reinterpret_cast<float*>(sb)[i] = __double2float_rn(v);
      } else if (F == CBG_FP16) {
        reinterpret_cast<__half*>(sb)[i] = __double2half(v);
      } else {
        reinterpret_cast<__nv_bfloat16*>(sb)[i] = __double2bfloat16(v);
      }
    }
  };

  // The CTA's CSR rows in shared memory when they fit in the space left (once per cycle: the matrix
  // is immutable); otherwise the SpMV reads them from global memory.
  const int rlo = min(n, row0), rhi = min(n, row0 + R);
  const int plo = a.row_ptr[rlo], pcnt = a.row_ptr[rhi] - plo;
  const bool staged = (int64_t)pcnt * 12 + (int64_t)(rhi - rlo + 1) * 4 <= lay.csr_bytes;
  double* svals = reinterpret_cast<double*>(smem + lay.off_csr);
  int32_t* scol = reinterpret_cast<int32_t*>(svals + (staged ? pcnt : 0));
  int32_t* srp = scol + (staged ? pcnt : 0);
  if (staged) {
    for (int p = t; p < pcnt; p += kOcThreads) {
      svals[p] = a.vals[plo + p];
      scol[p] = a.col[plo + p];
    }
    for (int i = t; i <= rhi - rlo; i += kOcThreads) srp[i] = a.row_ptr[rlo + i] - plo;
  }
  const double* mvals = staged ? svals : a.vals + plo;
  const int32_t* mcol = staged ? scol : a.col + plo;

  // This thread's part of ||A z||^2 (Fig. 1 step 3; z of every CTA through distributed shared
  // memory). residual: r := b - A z into a.r (the next cycle's step 1), else w := A z. The products
  // of a row are accumulated in order, as in the streamed thread-per-row SpMV.
  auto spmv = [&](bool residual) {
    double nrm = 0.0;
    bool bad = false;
    for (int i = t; i < R; i += kOcThreads) {
      const int gi = row0 + i;
      if (gi >= n) {
        if (!residual) s.w[i] = 0.0;
        continue;
      }
      const int p0 = staged ? srp[i] : a.row_ptr[gi] - plo, p1 = staged ? srp[i + 1] : a.row_ptr[gi + 1] - plo;
      double acc = 0.0;
      for (int p = p0; p < p1; p += 4) {
        double xv[4], av[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          xv[u] = 0.0;
          av[u] = 0.0;
          if (p + u < p1) {
            const int c = mcol[p + u];
            av[u] = mvals[p + u];
            if (static_cast<unsigned>(c) < static_cast<unsigned>(n)) {  // c < n <= nctas R: owner < nctas
              const uint32_t owner = static_cast<uint32_t>(c / R);
              const int off = c - static_cast<int>(owner) * R;
              xv[u] = owner == rank ? s.z[off] : dsmem_ld(s.z + off, owner);
            } else {
              bad = true;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (p + u < p1) acc = fma(av[u], xv[u], acc);
      }
      if (residual) {
        acc = a.b[gi] - acc;
        a.r[gi] = acc;
      } else {
        s.w[i] = acc;
      }
      nrm = fma(acc, acc, nrm);
    }
    if (bad) atomicOr(&ctl->err, kDevErrBadMatrix);
    return nrm;
  };

  // hp[buf][0..nv) := this CTA's part of V_nv^T w (Fig. 1 steps 5 and 8): warp <-> block,
  // lane <-> vector (lane + 32 q).
  auto dot = [&](int nv) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = warp; b < NB; b += kOcWarps) {
      const double* wb = s.w + b * 32;
      if (F == CBG_FRSZ2) {
        // the block's 54-bit fixed point of w, one value per lane, then read back in the order
        // block_dot visits the codes (the warp that writes block b is the one that reads it)
        const int ew = __reduce_max_sync(0xffffffffu, eff_exp(wb[lane]));
        int2* wt = s.gt + warp * 32;
        {
          int32_t w1, w0;
          to_block_fixed(wb[lane], ew, w1, w0);
          wt[lane] = make_int2(w1, w0);
        }
        __syncwarp();
        int32_t W1[32], W0[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int2 wv = wt[w_index<L>(lane, r)];
          W1[r] = wv.x;
          W0[r] = wv.y;
        }
        __syncwarp();  // the table is rewritten for the warp's next block
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = lane + 32 * q;
          if (i < nv) {
            const uint32_t* cw = reinterpret_cast<const uint32_t*>(s.codes + (size_t)i * lay.slot_bytes) + b * L;
            const uint32_t e = s.exq[i * lay.exp_words + b];
            long long a1, a0;
            block_dot<L>(cw, lane, W1, W0, a1, a0);
            // (a1 2^27 + a0) 2^x, x = Ebar + Ew - 2096 - l, rounded to 2^(l-5) units (as k_dot_frsz2)
            const long long th = (a1 << (32 - L)) + ((a0 + (1ll << (L - 6))) >> (L - 5));
            const int x = (e > 1 ? static_cast<int>(e) : 1) + ew - 2096 - L;
            acc[q] += scale_pow2(static_cast<double>(th), x + L - 5);
          }
        }
      } else if (F == CBG_FP64) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = lane + 32 * q;
          if (i < nv) {
            const uint8_t* sb = s.codes + (size_t)i * lay.slot_bytes;
            double d[4] = {0.0, 0.0, 0.0, 0.0};  // four independent chains (values k mod 4)
#pragma unroll
            for (int k = 0; k < 32; ++k) d[k & 3] = fma(cast_at<F>(sb, b * 32 + k), wb[k], d[k & 3]);
            acc[q] += (d[0] + d[1]) + (d[2] + d[3]);
          }
        }
      } else {
        // binary32, binary16, bfloat16: the streamed dot's exact integer block dot (a block fixed
        // point of the stored values against the 54-bit fixed point of w), one rounding and one
        // conversion per (vector, block); a block it cannot hold exactly takes FP64 FMAs
        constexpr int WL = F == CBG_FP32 ? 32 : 16;
        const int ew = __reduce_max_sync(0xffffffffu, eff_exp(wb[lane]));
        int2* wt = s.gt + warp * 32;
        {
          int32_t w1, w0;
          to_block_fixed(wb[lane], ew, w1, w0);
          wt[lane] = make_int2(w1, w0);
        }
        __syncwarp();
        int32_t W1[32], W0[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int2 wv = wt[w_index<WL>(lane, r)];
          W1[r] = wv.x;
          W0[r] = wv.y;
        }
        __syncwarp();  // the table is rewritten for the warp's next block
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = lane + 32 * q;
          if (i < nv) {
            const uint8_t* sb = s.codes + (size_t)i * lay.slot_bytes;
            const uint32_t* cw = reinterpret_cast<const uint32_t*>(sb) + b * WL;  // WL words per block
            long long th = 0;
            int xb = 0;
            bool exact;
            if (F == CBG_FP16) {
              uint32_t emax = 0;
              long long a1, a0;
              block_dot_fp16(cw, lane, W1, W0, a1, a0, emax);
              exact = emax <= 15;
              if (exact) {  // (a1 2^27 + a0) 2^(ew - 1099), kept or rounded to 62 bits
                const unsigned long long A = static_cast<unsigned long long>(a1 < 0 ? -a1 : a1);
                const int bl = 64 - __clzll(static_cast<long long>(A));
                const int u = bl > 35 ? bl - 35 : 0;
                th = u == 0 ? (a1 << 27) + a0 : (a1 << (27 - u)) + ((a0 + (1ll << (u - 1))) >> u);
                xb = u + ew - 1099;
              }
            } else if (F == CBG_BF16) {
              long long a1, a0;
              __int128 tot = 0;
              int E = 0;
              const int kind = block_dot_bf16(cw, lane, W1, W0, a1, a0, tot, E);
              exact = kind < 2;
              if (kind == 0) {
                const unsigned long long A = static_cast<unsigned long long>(a1 < 0 ? -a1 : a1);
                const int bl = 64 - __clzll(static_cast<long long>(A));
                const int u = bl > 35 ? bl - 35 : 0;
                th = u == 0 ? (a1 << 27) + a0 : (a1 << (27 - u)) + ((a0 + (1ll << (u - 1))) >> u);
                xb = u + E + ew - 1223;
              } else if (kind == 1) {
                th = round_i128(tot, xb);
                xb += E + ew - 1263;
              }
            } else {
              __int128 tot = 0;
              int E = 0;
              exact = block_dot_f32(cw, lane, W1, W0, tot, E);
              if (exact) {
                th = round_i128(tot, xb);
                xb += E + ew - 1263;
              }
            }
            if (exact) {
              acc[q] += scale_pow2(static_cast<double>(th), xb);
            } else {
              double d[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 1
              for (int k = 0; k < 32; ++k) d[k & 3] = fma(cast_at<F>(sb, b * 32 + k), wb[k], d[k & 3]);
              acc[q] += (d[0] + d[1]) + (d[2] + d[3]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = lane + 32 * q;
      if (i < nv) s.wpart[warp * M1 + i] = acc[q];
    }
    __syncthreads();
    for (int i = t; i < nv; i += kOcThreads) s.hp[buf * (M1 + 1) + i] = sum8(s.wpart + i, M1);
  };

  // x := x - V_nv c (negate: x + V_nv c) over this CTA's rows (Fig. 1 steps 5, 10 and 17);
  // returns this thread's part of ||x||^2. warp <-> block, lane <-> value.
  auto update = [&](int nv, const double* c, bool negate, double* x) {
    if (F == CBG_FRSZ2) {
      for (int i = t; i < nv; i += kOcThreads) {  // c_i = hman_i 2^{hexp_i - 1075} exactly
        const uint64_t u = static_cast<uint64_t>(__double_as_longlong(c[i]));
        const int e = static_cast<int>((u >> 52) & 0x7FF);
        const long long mm = static_cast<long long>((u & ((1ull << 52) - 1)) | (e ? 1ull << 52 : 0ull));
        s.hman[i] = ((u >> 63) != 0) != negate ? -mm : mm;
        s.hexp[i] = e > 1 ? e : 1;
      }
    }
    __syncthreads();
    const int ngroups = (nv + 31) / 32;
    const int gb = ngroups > 1 ? 32 - __clz(ngroups - 1) : 0;
    const int sh = L - 5 + gb;
    int2* gtw = s.gt + warp * 32;
    double nrm = 0.0;
    for (int b = warp; b < NB; b += kOcWarps) {
      const int i = b * 32 + lane, gi = row0 + i;
      if (F == CBG_FRSZ2) {
        long long tacc = 0;  // sum over the groups so far, in units of 2^(rc - 2101 + gb)
        int rc = 0;
        for (int g0 = 0; g0 < nv; g0 += 32) {
          const int gn = min(32, nv - g0);
          // the group's coefficients: lane v computes G for vector g0 + v against
          // rexp = max over the group of (Eh_i + Ebar_{i,b})
          uint32_t e = 0;
          int rv = 0;
          if (lane < gn) {
            e = s.exq[(g0 + lane) * lay.exp_words + b];
            rv = s.hexp[g0 + lane] + (e > 1 ? static_cast<int>(e) : 1);
          }
          const int r = __reduce_max_sync(0xffffffffu, rv);
          if (lane < gn) {
            const int d = r - s.hexp[g0 + lane] - (e > 1 ? static_cast<int>(e) : 1);
            const long long mm = s.hman[g0 + lane];
            const long long gm = d == 0 ? mm : (d < 64 ? ((mm >> (d - 1)) + 1) >> 1 : 0);
            gtw[lane] = make_int2(static_cast<int32_t>(gm & ((1ll << 27) - 1)), static_cast<int32_t>(gm >> 27));
          }
          __syncwarp();
          long long acc0 = 0, acc1 = 0;
          for (int v = 0; v < gn; ++v) {
            const uint32_t* bw = reinterpret_cast<const uint32_t*>(s.codes + (size_t)(g0 + v) * lay.slot_bytes) + b * L;
            const int32_t sv = code_to_int<L>(code_at<L>(bw, lane));
            const int2 gp = gtw[v];
            mac_wide(acc0, sv, gp.x);
            mac_wide(acc1, sv, gp.y);
          }
          __syncwarp();  // the table is rewritten by the next group
          long long th;
          if (sh <= 27) {
            th = (acc1 << (27 - sh)) + ((acc0 + (1ll << (sh - 1))) >> sh);
          } else {
            const long long xx = acc1 + (acc0 >> 27);
            const long long yy = (acc0 & ((1ll << 27) - 1)) + (1ll << (sh - 1));
            th = (xx + (yy >> 27)) >> (sh - 27);
          }
          if (g0 == 0 || r >= rc) {
            tacc = round_shift_right(tacc, g0 == 0 ? 0 : r - rc) + th;
            rc = r;
          } else {
            tacc += round_shift_right(th, rc - r);
          }
        }
        if (gi < n) {
          const int xe = rc - 2101 + gb;
          const double tv = static_cast<double>(tacc);
          const double cur = x[i];
          const double nx = (xe >= -1022 && xe <= 1023) ? fma(tv, -pow2_normal(xe), cur) : cur - scale_pow2(tv, xe);
          x[i] = nx;
          nrm = fma(nx, nx, nrm);
        }
      } else if (gi < n) {
        double acc = x[i];
        for (int v = 0; v < nv; ++v) {
          const double nh = -(negate ? -c[v] : c[v]);
          acc = fma(cast_at<F>(s.codes + (size_t)v * lay.slot_bytes, i), nh, acc);
        }
        x[i] = acc;
        nrm = fma(acc, acc, nrm);
      }
    }
    return nrm;
  };

  // Norm reductions: hp[buf][0] of every CTA, summed over the cluster into *dst; a NaN or
  // infinity stops the cycle (the error word reports it). Returns the stop flag.
  auto norm_sum = [&](double part, double* dst) {
    cta_sum(part, 0);
    cluster_sum(1, dst);
    if (t == 0 && !isfinite(*dst)) {
      S.stop = 1;
      if (rank == 0) atomicOr(&ctl->err, kDevErrNonFinite);
    }
    __syncthreads();
    return S.stop != 0;
  };

  // ---- step 1: v_1 = r0 / beta (r0 and beta from the previous residual) -------------------------
  for (int i = t; i < R; i += kOcThreads) s.w[i] = row0 + i < n ? a.r[row0 + i] : 0.0;
  for (int i = t; i <= m; i += kOcThreads) s.g[i] = 0.0;
  __syncthreads();
  if (t == 0) {
    const double beta = ctl->beta;
    s.g[0] = beta;
    S.rcp = ctl->rcp;
    S.stop = beta > 0.0 ? 0 : 1;
    S.reorth = 0;
    S.m_eff = 0;
    S.breakdown = 0;
    S.reorth_count = 0;
    S.stored = 0;
    S.m_ls = 0;
    S.implicit = ctl->implicit;
  }
  __syncthreads();
  store(0, ctl->hdiv, S.rcp);
  cluster_sync();  // every CTA's z is complete

  // ---- Arnoldi steps (steps 3-16) ---------------------------------------------------------------
  // Per step two cluster reductions carry everything the decisions need: [V^T w, ||A z||^2] after
  // the SpMV, and [V^T w', ||w'||^2] after the first update (the second pass's projections are
  // formed with the norm that decides whether they are needed, and dropped when they are not);
  // a third carries ||w''||^2 after a second pass.
  for (int j = 0; j < a.steps_allowed; ++j) {
    if (S.stop) break;  // the same in every CTA
    const int nv = j + 1;
    // steps 3-5: w = A z_j, omega^2 = ||w||^2, h = V^T w
    double part = spmv(false);
    __syncthreads();
    dot(nv);
    cta_sum(part, nv);
    cluster_sum(nv + 1, s.h);
    if (t == 0) {
      S.omega2 = s.h[nv];
      if (!isfinite(S.omega2)) S.stop = 1;
    }
    // step 5: w -= V h; step 6: ||w||; step 8's projections of the updated w
    part = update(nv, s.h, false, s.w);
    __syncthreads();
    dot(nv);
    cta_sum(part, nv);
    cluster_sum(nv + 1, s.u);
    if (t == 0) {
      S.hn2_first = S.hn2 = s.u[nv];
      if (!isfinite(S.hn2)) S.stop = 1;
      S.reorth = sqrt(S.hn2) < eta * sqrt(S.omega2) ? 1 : 0;  // step 7
      if (S.stop && rank == 0) atomicOr(&ctl->err, kDevErrNonFinite);
    }
    __syncthreads();
    if (S.stop) break;
    if (S.reorth) {  // steps 9-10: the second update and its norm
      if (norm_sum(update(nv, s.u, false, s.w), &S.hn2)) break;
    }
    // step 17, one column: h_{1:j+1} (+ u), h_{j+2,j+1} = ||w||, the previous rotations, a new one
    for (int i = t; i <= j; i += kOcThreads) s.col[i] = S.reorth ? s.h[i] + s.u[i] : s.h[i];
    __syncthreads();
    // warp 0 applies the previous rotations while warp 1 takes the square roots: ||w|| and, for
    // the breakdown test, ||w|| after the first pass
    if (warp == 0) {
      const double xr = rotate_column_warp(s.col, s.cs, s.sn, s.wpart, s.wpart + M1, j, lane);
      if (lane == 0) S.xc = xr;
    } else if (warp == 1 && lane < 2) {
      const double q = sqrt(lane == 1 ? S.hn2_first : S.hn2);
      if (lane == 1) S.hn_first = q;
      else S.hn = q;
    }
    __syncthreads();
    // Warp 0 forms the new rotation and 1 / h_{j+2,j+1}, publishes the latter (named barrier 1:
    // warp 0 arrives, the other warps wait), then finishes the column and the stop test while the
    // other warps already store v_{j+2} = w / h_{j+2,j+1} (steps 13-14) into slot j + 1. The store
    // is made on every step: on the last one it fills a slot the cycle does not read (the
    // write-back stops at S.stored).
    if (warp == 0) {
      const bool reorth = S.reorth != 0;
      const double hn = S.hn, hn_first = S.hn_first, xc = S.xc;
      // lane 0 c = x / r, lane 1 s = h / r, lane 2 the next normalisation 1 / h
      const double r = givens_radius(xc, hn);
      const double num = lane == 0 ? xc : (lane == 1 ? hn : 1.0);
      const double den = lane == 2 ? hn : r;
      const double q = (lane < 3 && den != 0.0) ? num / den : 0.0;
      const double c = hn != 0.0 ? __shfl_sync(0xffffffffu, q, 0) : 1.0;
      const double sn = hn != 0.0 ? __shfl_sync(0xffffffffu, q, 1) : 0.0;
      const double rcp = __shfl_sync(0xffffffffu, q, 2);
      if (lane == 0) {
        S.rcp = hn > 0.0 ? rcp : 0.0;
        s.col[j] = hn != 0.0 ? r : xc;
        s.col[j + 1] = 0.0;
        s.cs[j] = c;
        s.sn[j] = sn;
        const double gj = s.g[j];
        s.g[j + 1] = -sn * gj;
        s.g[j] = c * gj;
      }
      __syncwarp();
      asm volatile("bar.arrive 1, %0;" ::"n"(kOcThreads) : "memory");
      if (lane == 0) {
        const bool breakdown = (hn == 0.0) || (reorth && hn < eta * hn_first);  // step 12
        if (reorth) S.reorth_count += 1;
        const double implicit = fabs(s.g[j + 1]) / bnorm;
        S.implicit = implicit;
        if (rank == 0 && a.hist && a.hist_off + j < a.hist_cap) a.hist[a.hist_off + j] = implicit;
        S.m_eff = j + 1;
        if (breakdown) S.breakdown = 1;
        if (!isfinite(implicit)) {
          if (rank == 0) atomicOr(&ctl->err, kDevErrNonFinite);
          S.stop = 1;
        }
        if (breakdown || implicit <= tol || j + 1 >= a.steps_allowed) S.stop = 1;
        if (!S.stop) S.stored = j + 1;
      }
      for (int i = lane; i <= j + 1; i += 32) s.Rm[(size_t)j * M1 + i] = s.col[i];
    } else {
      __syncwarp();  // bar.sync is .aligned
      asm volatile("bar.sync 1, %0;" ::"n"(kOcThreads) : "memory");
    }
    store(j + 1, S.hn, S.rcp);
    cluster_sync();  // every CTA's z is complete, and S.stop is set
  }
  __syncthreads();

  // ---- step 17: y = R^{-1} g over the columns with a nonzero pivot, x += V y -------------------
  if (t == 0) {
    int mls = S.m_eff;
    for (int k = 0; k < S.m_eff; ++k) {
      if (s.Rm[(size_t)k * M1 + k] == 0.0) {
        mls = k;
        break;
      }
    }
    S.m_ls = mls;
  }
  __syncthreads();
  const int mls = S.m_ls;
  if (warp == 0) {
    for (int k = mls - 1; k >= 0; --k) {
      double acc = 0.0;
      for (int i = k + 1 + lane; i < mls; i += 32) acc += s.Rm[(size_t)i * M1 + k] * s.y[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) s.y[k] = (s.g[k] - acc) / s.Rm[(size_t)k * M1 + k];
      __syncwarp();
    }
  }
  // x := x + V y, or x + M^{-1} (V y) with the Jacobi preconditioner (the update of a zero vector)
  for (int i = t; i < R; i += kOcThreads) s.w[i] = (row0 + i < n && !a.dinv) ? a.x[row0 + i] : 0.0;
  __syncthreads();
  update(mls, s.y, true, s.w);
  __syncthreads();
  for (int i = t; i < R; i += kOcThreads) {
    const int gi = row0 + i;
    double xn = 0.0;
    if (gi < n) {
      xn = a.dinv ? fma(a.dinv[gi], s.w[i], a.x[gi]) : s.w[i];
      a.x[gi] = xn;
    }
    s.z[i] = xn;
  }
  cluster_sync();  // every CTA's z = x is complete

  // ---- the next cycle's step 1: r = b - A x, beta = ||r|| ---------------------------------------
  cta_sum(spmv(true), 0);
  cluster_sum(1, &S.beta2);
  if (rank == 0 && t == 0) {
    const double b2 = S.beta2;
    if (!isfinite(b2)) {
      atomicOr(&ctl->err, kDevErrNonFinite);
      S.stop = 1;
    }
    const double nrm = sqrt(b2);
    ctl->beta = nrm;
    ctl->hdiv = nrm;
    ctl->rcp = nrm > 0.0 ? 1.0 / nrm : 0.0;
    ctl->stop = S.stop;
    ctl->reorth = 0;
    ctl->m_eff = S.m_eff;
    ctl->breakdown = S.breakdown;
    ctl->reorth_count = S.reorth_count;
    ctl->m_ls = S.m_ls;
    ctl->steps_allowed = a.steps_allowed;
    ctl->omega2 = S.omega2;
    ctl->hn2_first = S.hn2_first;
    ctl->hn2 = S.hn2;
    ctl->implicit = S.implicit;
  }

  // ---- the basis slices of this cycle to the context's basis storage (streamed layout) ----------
  const int nb_all = (n + 31) / 32;
  const int stored = S.stored;
  if (F == CBG_FRSZ2) {
    const int per_slot = NB * (L + 1);
    for (int idx = t; idx < (stored + 1) * per_slot; idx += kOcThreads) {
      const int slot = idx / per_slot, rem = idx - slot * per_slot;
      const int b = rem / (L + 1), wd = rem - b * (L + 1);
      const int gbk = static_cast<int>(rank) * NB + b;
      if (gbk >= nb_all) continue;
      if (wd < L) {
        const uint32_t* cw = reinterpret_cast<const uint32_t*>(s.codes + (size_t)slot * lay.slot_bytes) + b * L;
        reinterpret_cast<uint32_t*>(a.basis.vals + (int64_t)slot * a.basis.vstride)[(int64_t)gbk * L + wd] = cw[wd];
      } else {
        reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(a.basis.exps) + (int64_t)slot * a.basis.estride)[gbk] =
            s.exq[slot * lay.exp_words + b];
      }
    }
  } else {
    constexpr int ES = F == CBG_FP64 ? 8 : (F == CBG_FP32 ? 4 : 2);
    for (int idx = t; idx < (stored + 1) * R; idx += kOcThreads) {
      const int slot = idx / R, i = idx - slot * R, gi = row0 + i;
      if (gi >= n) continue;
      const uint8_t* src = s.codes + (size_t)slot * lay.slot_bytes + (size_t)i * ES;
      uint8_t* dst = a.basis.vals + (int64_t)slot * a.basis.vstride + (int64_t)gi * ES;
      if (ES == 8) *reinterpret_cast<double*>(dst) = *reinterpret_cast<const double*>(src);
      else if (ES == 4) *reinterpret_cast<uint32_t*>(dst) = *reinterpret_cast<const uint32_t*>(src);
      else *reinterpret_cast<uint16_t*>(dst) = *reinterpret_cast<const uint16_t*>(src);
    }
  }
  cluster_sync();  // no CTA leaves while another may still read its shared memory
}

template <int F, int L>
const void* oc_kernel() {
  return reinterpret_cast<const void*>(k_cycle_onchip<F, L>);
}

const void* oc_pick(int fmt, int l) {
  switch (fmt) {
    case CBG_FP64: return oc_kernel<CBG_FP64, 32>();
    case CBG_FP32: return oc_kernel<CBG_FP32, 32>();
    case CBG_FP16: return oc_kernel<CBG_FP16, 32>();
    case CBG_BF16: return oc_kernel<CBG_BF16, 32>();
    case CBG_FRSZ2:
      return l == 16 ? oc_kernel<CBG_FRSZ2, 16>() : (l == 21 ? oc_kernel<CBG_FRSZ2, 21>() : oc_kernel<CBG_FRSZ2, 32>());
    default: return nullptr;
  }
}

int64_t rup(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// Shared-memory layout of one CTA (the device side carves the same offsets in oc_carve).
OcLayout oc_layout(int32_t n, int m, int fmt, int l, int cl) {
  OcLayout L{};
  const int64_t rows = rup((n + cl - 1) / cl, 32);
  const int64_t nb = rows / 32, M1 = m + 1;
  int64_t slot;
  if (fmt == CBG_FRSZ2) {
    // slot stride = l (mod 32) words: lane i reading slot i meets the bank pattern block_dot's
    // chunk rotation is built for (consecutive 32 l-bit blocks)
    int64_t words = nb * l;
    words += ((l - words) % 32 + 32) % 32;
    slot = words * 4;
  } else if (fmt == CBG_FP64) {
    slot = rup(rows * 8, 128) + 8;  // lane i of a warp reading slot i: distinct banks
  } else {
    // binary32 and the 16-bit formats: the integer block dot reads 16-byte chunks of slot i in lane
    // i in the rotation of block_dot<32>, resp. <16>: the FRSZ2 strides for l = 32, resp. 16
    const int64_t lw = fmt == CBG_FP32 ? 32 : 16;
    int64_t words = rows * (fmt == CBG_FP32 ? 4 : 2) / 4;
    words += ((lw - words) % 32 + 32) % 32;
    slot = words * 4;
  }
  const int64_t expw = fmt == CBG_FRSZ2 ? (nb | 1) : 0;
  const int64_t off_exps = rup(M1 * slot, 16);
  const int64_t off_z = rup(off_exps + M1 * expw * 4, 16);
  const int64_t off_vec = off_z + 2 * rows * 8;
  const int64_t vec8 = 2 * (M1 + 1) + kOcWarps * M1 + 2 * (M1 + 1) + (M1 + 1) + 2 * M1 + (M1 + 1) + M1 +
                       (int64_t)m * M1 + kOcWarps + M1 + kOcWarps * 32;
  const int64_t off_state = rup(off_vec + vec8 * 8 + M1 * 4, 16);
  const int64_t total = rup(off_state + (int64_t)sizeof(OcState), 128);
  L.rows = static_cast<int>(rows);
  L.slot_bytes = static_cast<int>(slot);
  L.exp_words = static_cast<int>(expw);
  L.off_codes = 0;
  L.off_exps = static_cast<int>(off_exps);
  L.off_z = static_cast<int>(off_z);
  L.off_vec = static_cast<int>(off_vec);
  L.off_state = static_cast<int>(off_state);
  L.bytes = total > (1ll << 30) ? (1 << 30) : static_cast<int>(total);
  L.off_csr = L.bytes;  // 128-byte aligned; the size is set by the plan
  L.csr_bytes = 0;
  return L;
}

}  // namespace

int onchip_plan(int32_t n, int64_t nnz, const cbg_opts* o, OnchipPlan* plan) {
  plan->cluster = 0;
  if (o->cycle != CBG_CYCLE_AUTO) return CBG_OK;
  if (o->restart + 1 > kOcMaxSlots) return CBG_OK;
  if (spmv_lanes_per_row(n, nnz) > 1) return CBG_OK;  // long rows: the streamed lanes-per-row SpMV
  DeviceInfo di;
  int st = device_info(&di);
  if (st) return st;
  const int l = o->fmt == CBG_FRSZ2 ? o->frsz2_bits : 32;
  const void* fn = oc_pick(o->fmt, l);
  if (!fn) return CBG_ERR_INVALID_ARG;
  for (int cl = 16; cl >= 8; cl /= 2) {
    const OcLayout lay = oc_layout(n, o->restart, o->fmt, l, cl);
    if (lay.bytes > di.max_smem_optin) continue;
    // the largest opt-in size, so that contexts of any size can launch the same function
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, di.max_smem_optin) != cudaSuccess ||
        (cl > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(kOcThreads);
    cfg.dynamicSmemBytes = static_cast<size_t>(lay.bytes);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess || clusters < 1) {
      cudaGetLastError();
      continue;
    }
    plan->cluster = cl;
    plan->lay = lay;
    // room for the CSR rows of a CTA: twice the mean share, within the opt-in limit
    const int64_t want = 2 * ((nnz * lay.rows + n - 1) / n * 12 + (int64_t)(lay.rows + 1) * 4) + 1024;
    const int64_t room = (di.max_smem_optin - plan->lay.off_csr) / 16 * 16;
    plan->lay.csr_bytes = static_cast<int>(want < room ? rup(want, 16) : (room > 0 ? room : 0));
    plan->lay.bytes = plan->lay.off_csr + plan->lay.csr_bytes;
    return CBG_OK;
  }
  return CBG_OK;
}

int launch_onchip_cycle(const OnchipPlan& plan, const OnchipArgs& a, int fmt, int l, cudaStream_t stream) {
  if (plan.cluster < 1 || a.m + 1 > kOcMaxSlots) return CBG_ERR_INVALID_ARG;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(plan.cluster);
  cfg.blockDim = dim3(kOcThreads);
  cfg.dynamicSmemBytes = static_cast<size_t>(plan.lay.bytes);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = plan.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  switch (fmt) {
    case CBG_FP64: e = cudaLaunchKernelEx(&cfg, k_cycle_onchip<CBG_FP64, 32>, a, plan.lay); break;
    case CBG_FP32: e = cudaLaunchKernelEx(&cfg, k_cycle_onchip<CBG_FP32, 32>, a, plan.lay); break;
    case CBG_FP16: e = cudaLaunchKernelEx(&cfg, k_cycle_onchip<CBG_FP16, 32>, a, plan.lay); break;
    case CBG_BF16: e = cudaLaunchKernelEx(&cfg, k_cycle_onchip<CBG_BF16, 32>, a, plan.lay); break;
    case CBG_FRSZ2:
      if (l == 16) e = cudaLaunchKernelEx(&cfg, k_cycle_onchip<CBG_FRSZ2, 16>, a, plan.lay);
      else if (l == 21) e = cudaLaunchKernelEx(&cfg, k_cycle_onchip<CBG_FRSZ2, 21>, a, plan.lay);
      else e = cudaLaunchKernelEx(&cfg, k_cycle_onchip<CBG_FRSZ2, 32>, a, plan.lay);
      break;
    default: return CBG_ERR_INVALID_ARG;
  }
  if (e != cudaSuccess) return cuda_fail(e, "on-chip cycle launch");
  return CBG_OK;
}

}  // namespace cbg
