// Internal definitions shared by the CUDA translation units of the library (sm_103a only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cbgmres.h"

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ < 1000)
#error "this library targets sm_103a (Blackwell Ultra); build with -gencode arch=compute_103a,code=sm_103a"
#endif

namespace cbg {

constexpr int kBS = 32;  // FRSZ2 block size (fixed to the warp width: Implementation subsection)

// Device-side error bits, OR-ed into a status word that the host reads back.
enum DevErr : int {
  kDevErrTimeout = 1,     // a bounded mbarrier wait expired
  kDevErrNonFinite = 2,   // a norm became NaN or Inf
  kDevErrBadMatrix = 4,   // CSR validation failed
  kDevErrBadDiagonal = 8, // a zero or missing diagonal entry (Jacobi preconditioner)
};

// A wait on a bulk copy gives up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// ---- small integer / FP64 helpers -------------------------------------------------------------

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// 2^x as a double for x in [-1022, 1023], built from its bit pattern (no FP64 instruction).
__device__ __forceinline__ double pow2_normal(int x) {
  return __longlong_as_double((long long)(x + 1023) << 52);
}

// v * 2^x for any integer x; one FP64 multiply when 2^x is a normal double, two otherwise (the
// first of the two is exact, so the result is rounded once).
__device__ __forceinline__ double scale_pow2(double v, int x) {
  if (x > 1023) {
    v *= pow2_normal(1023);
    x -= 1023;
    if (x > 1023) x = 1023;
  } else if (x < -1022) {
    v *= pow2_normal(-1022);
    x += 1022;
    if (x < -1022) x = -1022;
  }
  return v * pow2_normal(x);
}

// acc + v * 2^x with a single FMA in the normal range.
__device__ __forceinline__ double fma_pow2(double v, int x, double acc) {
  if (x >= -1022 && x <= 1023) return fma(v, pow2_normal(x), acc);
  return acc + scale_pow2(v, x);
}

// The correctly rounded quotient w / h (round to nearest even, as IEEE division) for a divisor
// h > 0, given rcp = RN(1/h), at the cost of one FP64 multiply and integer arithmetic. (For h = 0
// the caller passes rcp = 0 and gets w * 0.)
//
// q = RN(w * rcp) lies within 1.5 units in the last place of w / h, so RN(w / h) is q or one of
// its neighbours. With the integer significands (53 bits, hidden bit explicit) w = mw 2^(ew-1075),
// h = mh 2^(eh-1075) and q = mq 2^(eq-1075), the remainder in units of 2^(eq+eh-2150),
//   R = mw 2^(ew+1075-eq-eh) - mq mh,
// is exact in 64-bit integers (|R| < 2^56 for such a q), and (w/h - q) / ulp(q) = R / mh. So q is
// the rounded quotient exactly when -1/2 (-1/4 below a power of two, where the next double down
// is half an ulp away) < R / mh < 1/2; otherwise the neighbour in the direction of R's sign is
// tested the same way. Exact halfway quotients of two 53-bit significands do not exist, so no tie
// arises. Zero, subnormal or non-finite operands, a quotient outside the normal range, and a
// candidate that fails both tests (not expected) take the IEEE division.
__device__ __forceinline__ double div_rn(double w, double h, double rcp) {
  const double q0 = w * rcp;
  const uint64_t uw = static_cast<uint64_t>(__double_as_longlong(w));
  const uint64_t uh = static_cast<uint64_t>(__double_as_longlong(h));
  const uint64_t uq0 = static_cast<uint64_t>(__double_as_longlong(q0));
  const int ew = static_cast<int>((uw >> 52) & 0x7FF), eh = static_cast<int>((uh >> 52) & 0x7FF);
  const int eq0 = static_cast<int>((uq0 >> 52) & 0x7FF);
  if (ew == 0 || ew == 0x7FF || eh == 0 || eh == 0x7FF || eq0 <= 1 || eq0 >= 0x7FE) {
    if (w == 0.0 || !(h > 0.0)) return q0;  // +-0 / h = +-0; a zero divisor (rcp 0) keeps w * rcp
    return w / h;
  }
  constexpr uint64_t kHidden = 1ull << 52, kMant = kHidden - 1;
  const uint64_t mw = (uw & kMant) | kHidden, mh = (uh & kMant) | kHidden;
  const uint64_t sgn = uw & (1ull << 63);
  // true when the magnitude with bits `uq` is RN(|w| / h); *up receives the sign of R
  auto rounded = [&](uint64_t uq, bool* up) {
    const int eq = static_cast<int>(uq >> 52);
    const uint64_t mq = (uq & kMant) | kHidden;
    const int s = ew + 1075 - eq - eh;
    if (s < 0 || s > 63) {
      *up = s > 63;
      return false;
    }
    const long long R = static_cast<long long>((mw << s) - mq * mh);
    *up = R > 0;
    if (R >= 0) return static_cast<uint64_t>(2 * R) < mh;
    const uint64_t a = static_cast<uint64_t>(-R);
    return (mq == kHidden ? 4 * a : 2 * a) < mh;
  };
  const uint64_t m0 = uq0 & ~(1ull << 63);
  bool up = false;
  if (rounded(m0, &up)) return __longlong_as_double(static_cast<long long>(m0 | sgn));
  const uint64_t m1 = up ? m0 + 1 : m0 - 1;  // the next double up or down in magnitude
  bool up1 = false;
  if (rounded(m1, &up1)) return __longlong_as_double(static_cast<long long>(m1 | sgn));
  return w / h;
}

// ---- mbarrier and bulk-copy (TMA) wrappers ---------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Asynchronous global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// that completes on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// One bounded probe of phase `parity`: the thread may be suspended (not spinning) for up to about
// 100 microseconds while the phase is incomplete, and resumes as soon as it completes.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of `bar` to complete, giving up after kWaitLimitNs. Returns false on
// timeout (the caller records kDevErrTimeout and stops using the stage).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
  }
}

// ---- deterministic cross-CTA reduction ----------------------------------------------------------
// Each CTA writes its partial results; the CTA that arrives last (atomic ticket) reduces all of
// them in a fixed order, so the result does not depend on scheduling.

__device__ __forceinline__ bool arrive_last(unsigned int* counter, unsigned int nblocks, int* smem_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int ticket = atomicAdd(counter, 1u);
    *smem_flag = (ticket == nblocks - 1);
  }
  __syncthreads();
  const bool last = *smem_flag != 0;
  if (last) __threadfence();
  return last;
}

// Sum of v[0..count) with stride `stride`, computed by one warp in a fixed order: lane-strided
// sequential sums followed by a shuffle tree. Reads through L2 (values written by other CTAs).
__device__ __forceinline__ double warp_sum_strided(const double* v, int count, int stride) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < count; i += 32) s += __ldcg(v + (size_t)i * stride);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// ---- basis views --------------------------------------------------------------------------------

struct BasisView {
  const uint8_t* vals;
  int64_t vstride;      // bytes
  const uint32_t* exps;
  int64_t estride;      // bytes
  int64_t n;
  int32_t fmt;
  int32_t l;
};

struct BasisMut {
  uint8_t* vals;
  int64_t vstride;
  uint32_t* exps;
  int64_t estride;
  int64_t n;
  int32_t fmt;
  int32_t l;
};

// Solver control block in device memory. The last CTA of a kernel (see arrive_last) or the
// single-CTA kernels update it; later kernels read it to skip work (`stop`, `reorth`).
struct SolverCtl {
  int stop;          // the current cycle has ended (breakdown, implicit convergence, step cap)
  int reorth;        // the second Gram-Schmidt pass is needed at the current step
  int m_eff;         // Arnoldi steps completed in the current cycle
  int breakdown;     // the cycle ended on Fig. 1 step 12
  int err;           // DevErr bits
  int steps_allowed; // steps the host allows in this cycle
  int reorth_count;  // second passes taken in this cycle
  int m_ls;          // columns used by the least-squares solve of the cycle (step 17)
  double omega2;     // ||A v_j||^2 (step 4)
  double hn2_first;  // ||w||^2 after the first pass (step 6)
  double hn2;        // ||w||^2 after the last pass
  double beta;       // ||r0|| at the start of the cycle
  double bnorm;      // ||b||
  double tol;        // target relative residual (Eq. 4)
  double hdiv;       // the norm the next normalisation divides by (step 1: beta; step 13: h_{j+1,j})
  double rcp;        // RN(1 / hdiv)
  double implicit;   // |g_{j+1}| / ||b||
  double eta;
  unsigned int counters[8];  // arrive_last tickets, one per kernel kind
};

enum CounterSlot { kCtrSpmv = 0, kCtrDot = 1, kCtrUpdate = 2, kCtrStandalone = 3 };

// ---- host-side helpers (defined in capi.cu) -----------------------------------------------------

void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

struct DeviceInfo {
  int sms;
  int max_smem_optin;
};
int device_info(DeviceInfo* out);

}  // namespace cbg
