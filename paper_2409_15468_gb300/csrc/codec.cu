// FRSZ2 compression and decompression (Design section of arXiv 2409.15468) and the cast storage
// formats, as standalone kernels and as the "normalise and append to the basis" step of Fig. 1
// (steps 1, 13 and 14).
//
// Compression runs one warp per 32-value block, as the paper's block size 32 is chosen for
// (Implementation subsection): every lane extracts the exponent field of its value, a warp-wide
// integer maximum (redux.sync) gives e_max, and each lane forms its l-bit code with integer shifts
// (steps 1-5). Codes are then packed and stored (step 6): one 32-bit word per lane for l = 32,
// 16-bit stores for l = 16, and for l = 21 each of the block's 21 output words is assembled by one
// lane from the (at most three) codes that overlap it, fetched with warp shuffles.
// Decompression (steps 1-4) is per value: the sign is split off, the leading zeros of the
// significand are counted, and the IEEE double is reassembled from integer fields.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "decode.cuh"
#include "frsz2_block.cuh"
#include "kernels.cuh"

namespace cbg {

namespace {

__device__ __forceinline__ bool gate_skip_c(const Gate& g) {
  if (g.stop && *(volatile const int*)g.stop) return true;
  if (g.need && !*(volatile const int*)g.need) return true;
  return false;
}

}  // namespace

// The divisor of the normalisation v := w / h (Fig. 1 steps 1 and 13) and RN(1/h): read from the
// device when given (the solver computes 1/h once per step), else 1/h by one IEEE division per CTA.
__device__ __forceinline__ void divisor(const double* hdiv_ptr, const double* rcp_ptr, double* h, double* rcp) {
  __shared__ double s_rcp;
  if (!hdiv_ptr) {
    *h = 1.0;
    *rcp = 1.0;
    return;
  }
  *h = *hdiv_ptr;
  if (rcp_ptr) {
    *rcp = *rcp_ptr;
    return;
  }
  if (threadIdx.x == 0) s_rcp = 1.0 / *h;
  __syncthreads();
  *rcp = s_rcp;
}

template <int L, int U>
__global__ void __launch_bounds__(256) k_frsz2_compress(const double* __restrict__ src, int64_t n,
                                                        uint32_t* __restrict__ exps, uint32_t* __restrict__ codes,
                                                        const double* __restrict__ hdiv_ptr,
                                                        const double* __restrict__ rcp_ptr, double* __restrict__ vout,
                                                        const double* __restrict__ dscale, Gate gate) {
  if (gate_skip_c(gate)) return;
  double hdiv, rcp;
  divisor(hdiv_ptr, rcp_ptr, &hdiv, &rcp);
  const int lane = threadIdx.x & 31;
  const int64_t nb = (n + 31) / 32;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int64_t b0 = wg; b0 < nb; b0 += nwarps * U) {
    double x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t k = (b0 + u * nwarps) * 32 + lane;
      x[u] = k < n ? __ldcs(src + k) : 0.0;  // the last block is padded with +0.0
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t b = b0 + u * nwarps;
      if (b >= nb) break;  // uniform across the warp
      const int64_t k = b * 32 + lane;
      double v = x[u];
      if (hdiv_ptr) {
        v = div_rn(v, hdiv, rcp);  // v := w / h, correctly rounded
        if (k < n && vout) vout[k] = dscale ? v * dscale[k] : v;  // the SpMV input M^{-1} v (Fig. 1 step 3)
      }
      const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(v));
      // step 1: block maximum of the exponent fields
      const uint32_t e = static_cast<uint32_t>((bits >> 52) & 0x7FF);
      const uint32_t emax = __reduce_max_sync(0xffffffffu, e);
      const int ebar = emax > 1 ? static_cast<int>(emax) : 1;
      const uint32_t c = make_code<L>(bits, ebar);
      // step 6: store e_max and the codes
      if (lane == 0) exps[b] = emax;
      if (L == 32) {
        codes[b * 32 + lane] = c;
      } else if (L == 16) {
        reinterpret_cast<uint16_t*>(codes)[b * 32 + lane] = static_cast<uint16_t>(c);
      } else {
        // output word wd covers stream bits [32 wd, 32 wd + 32); codes i0..i0+2 can overlap it
        const int wd = lane;
        const int i0 = (32 * wd) / 21;
        const uint32_t c0 = __shfl_sync(0xffffffffu, c, i0 < 32 ? i0 : 31);
        const uint32_t c1 = __shfl_sync(0xffffffffu, c, i0 + 1 < 32 ? i0 + 1 : 31);
        const uint32_t c2 = __shfl_sync(0xffffffffu, c, i0 + 2 < 32 ? i0 + 2 : 31);
        const uint64_t win = static_cast<uint64_t>(c0) | (static_cast<uint64_t>(c1) << 21) |
                             (static_cast<uint64_t>(c2) << 42);
        const int off = 32 * wd - 21 * i0;  // in [0, 20]
        if (wd < 21) codes[b * 21 + wd] = static_cast<uint32_t>(win >> off);
      }
    }
  }
}

// Decompression steps 1-4 (frsz2_decode), one value per thread.
template <int L>
__global__ void k_frsz2_decompress(const uint32_t* __restrict__ exps, const uint32_t* __restrict__ codes, int64_t n,
                                   double* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
    dst[k] = frsz2_decode<L>(exps, codes, k);
}

// Cast storage: round to nearest even directly from FP64 with CUDA's conversion intrinsics.
template <int F>
__global__ void k_cast_store(const double* __restrict__ src, int64_t n, uint8_t* __restrict__ dst,
                             const double* __restrict__ hdiv_ptr, const double* __restrict__ rcp_ptr,
                             double* __restrict__ vout, const double* __restrict__ dscale, Gate gate) {
  if (gate_skip_c(gate)) return;
  double hdiv, rcp;
  divisor(hdiv_ptr, rcp_ptr, &hdiv, &rcp);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    double v = src[k];
    if (hdiv_ptr) {
      v = div_rn(v, hdiv, rcp);  // v := w / h, correctly rounded
      if (vout) vout[k] = dscale ? v * dscale[k] : v;
    }
    if (F == CBG_FP64) {
      reinterpret_cast<double*>(dst)[k] = v;
    } else if (F == CBG_FP32) {
      reinterpret_cast<float*>(dst)[k] = __double2float_rn(v);
    } else if (F == CBG_FP16) {
      reinterpret_cast<__half*>(dst)[k] = __double2half(v);
    } else {
      reinterpret_cast<__nv_bfloat16*>(dst)[k] = __double2bfloat16(v);
    }
  }
}

template <int F>
__global__ void k_cast_load(const uint8_t* __restrict__ src, int64_t n, double* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    double v;
    if (F == CBG_FP64) v = reinterpret_cast<const double*>(src)[k];
    else if (F == CBG_FP32) v = static_cast<double>(reinterpret_cast<const float*>(src)[k]);
    else if (F == CBG_FP16) v = static_cast<double>(__half2float(reinterpret_cast<const __half*>(src)[k]));
    else v = static_cast<double>(__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(src)[k]));
    dst[k] = v;
  }
}

namespace {

int grid_elems(int64_t n, int threads, int per_sm) {
  DeviceInfo di;
  if (device_info(&di)) return 1;
  int64_t g = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)di.sms * per_sm;
  if (g > cap) g = cap;
  return g < 1 ? 1 : static_cast<int>(g);
}

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, what);
}

}  // namespace

int launch_frsz2_compress_impl(const double* src, int64_t n, int l, uint32_t* exps, uint32_t* codes,
                               const double* hdiv, const double* rcp, double* vout, const double* dscale,
                               const Gate& gate, cudaStream_t stream) {
  if (n <= 0) return CBG_OK;
  constexpr int U = 4;
  const int64_t nb = (n + 31) / 32;
  const int grid = grid_elems((nb + U - 1) / U * 32, 256, 16);
  switch (l) {
    case 32: k_frsz2_compress<32, U><<<grid, 256, 0, stream>>>(src, n, exps, codes, hdiv, rcp, vout, dscale, gate); break;
    case 21: k_frsz2_compress<21, U><<<grid, 256, 0, stream>>>(src, n, exps, codes, hdiv, rcp, vout, dscale, gate); break;
    case 16: k_frsz2_compress<16, U><<<grid, 256, 0, stream>>>(src, n, exps, codes, hdiv, rcp, vout, dscale, gate); break;
    default: return CBG_ERR_INVALID_ARG;
  }
  return check_launch("frsz2 compress launch");
}

int launch_frsz2_compress(const double* src, int64_t n, int l, uint32_t* exps, uint32_t* codes, cudaStream_t stream) {
  return launch_frsz2_compress_impl(src, n, l, exps, codes, nullptr, nullptr, nullptr, nullptr, Gate{nullptr, nullptr},
                                    stream);
}

int launch_frsz2_decompress(const uint32_t* exps, const uint32_t* codes, int64_t n, int l, double* dst,
                            cudaStream_t stream) {
  if (n <= 0) return CBG_OK;
  const int grid = grid_elems(n, 256, 16);
  switch (l) {
    case 32: k_frsz2_decompress<32><<<grid, 256, 0, stream>>>(exps, codes, n, dst); break;
    case 21: k_frsz2_decompress<21><<<grid, 256, 0, stream>>>(exps, codes, n, dst); break;
    case 16: k_frsz2_decompress<16><<<grid, 256, 0, stream>>>(exps, codes, n, dst); break;
    default: return CBG_ERR_INVALID_ARG;
  }
  return check_launch("frsz2 decompress launch");
}

int launch_store(const BasisMut& B, int slot, const double* src, const double* hdiv, const double* rcp, double* vout,
                 const double* dscale, const Gate& gate, cudaStream_t stream) {
  if (B.n <= 0) return CBG_OK;
  uint8_t* vals = B.vals + (int64_t)slot * B.vstride;
  if (B.fmt == CBG_FRSZ2) {
    uint32_t* exps = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(B.exps) + (int64_t)slot * B.estride);
    return launch_frsz2_compress_impl(src, B.n, B.l, exps, reinterpret_cast<uint32_t*>(vals), hdiv, rcp, vout, dscale,
                                      gate, stream);
  }
  const int grid = grid_elems(B.n, 256, 16);
  switch (B.fmt) {
    case CBG_FP64: k_cast_store<CBG_FP64><<<grid, 256, 0, stream>>>(src, B.n, vals, hdiv, rcp, vout, dscale, gate); break;
    case CBG_FP32: k_cast_store<CBG_FP32><<<grid, 256, 0, stream>>>(src, B.n, vals, hdiv, rcp, vout, dscale, gate); break;
    case CBG_FP16: k_cast_store<CBG_FP16><<<grid, 256, 0, stream>>>(src, B.n, vals, hdiv, rcp, vout, dscale, gate); break;
    case CBG_BF16: k_cast_store<CBG_BF16><<<grid, 256, 0, stream>>>(src, B.n, vals, hdiv, rcp, vout, dscale, gate); break;
    default: return CBG_ERR_INVALID_ARG;
  }
  return check_launch("cast store launch");
}

int launch_load(const BasisView& B, int slot, double* dst, cudaStream_t stream) {
  if (B.n <= 0) return CBG_OK;
  const uint8_t* vals = B.vals + (int64_t)slot * B.vstride;
  if (B.fmt == CBG_FRSZ2) {
    const uint32_t* exps =
        reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint8_t*>(B.exps) + (int64_t)slot * B.estride);
    return launch_frsz2_decompress(exps, reinterpret_cast<const uint32_t*>(vals), B.n, B.l, dst, stream);
  }
  const int grid = grid_elems(B.n, 256, 16);
  switch (B.fmt) {
    case CBG_FP64: k_cast_load<CBG_FP64><<<grid, 256, 0, stream>>>(vals, B.n, dst); break;
    case CBG_FP32: k_cast_load<CBG_FP32><<<grid, 256, 0, stream>>>(vals, B.n, dst); break;
    case CBG_FP16: k_cast_load<CBG_FP16><<<grid, 256, 0, stream>>>(vals, B.n, dst); break;
    case CBG_BF16: k_cast_load<CBG_BF16><<<grid, 256, 0, stream>>>(vals, B.n, dst); break;
    default: return CBG_ERR_INVALID_ARG;
  }
  return check_launch("cast load launch");
}

}  // namespace cbg
