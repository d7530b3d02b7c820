// The synthetic arithmetic-intensity benchmark of the synthetic-performance discussion (Fig. 3):
// read the consecutive values of one stored basis vector, decode each to FP64 (or read FP32 and
// stay in FP32), apply r fused multiply-adds to it, and sum the results. Sweeping r moves the
// kernel from the memory roof (r = 0) to the arithmetic roof of its precision; on GB300 FP64
// issues ~2 operations per clock per SM, so the FP64 roof is crossed at ~0.2 FLOP per byte.
//
// Value k contributes f^r(x_k) with f(y) = 0.5 y + 0.25: the product by 0.5 is exact, so each
// step rounds once whether or not the multiply-add is fused, and a host reference can follow it
// bit for bit. Each thread carries 4 independent chains so that FMA latency is hidden.
#include "common.cuh"
#include "decode.cuh"
#include "kernels.cuh"

namespace cbg {

namespace {

template <int F, int L>
__device__ __forceinline__ double decode_at(const uint8_t* vals, const uint32_t* exps, int64_t k) {
  if (F == CBG_FRSZ2) return frsz2_decode<L>(exps, reinterpret_cast<const uint32_t*>(vals), k);
  if (F == CBG_FP64) return __ldcs(reinterpret_cast<const double*>(vals) + k);
  if (F == CBG_FP32) return widen_f32(__ldcs(reinterpret_cast<const uint32_t*>(vals) + k));
  const uint32_t h = __ldcs(reinterpret_cast<const unsigned short*>(vals) + k);
  return F == CBG_FP16 ? widen_f16(h) : widen_f32(h << 16);
}

}  // namespace

// F: storage format (L: FRSZ2 code width); F32: FP32 storage read and computed in FP32.
template <int F, int L, bool F32>
__global__ void __launch_bounds__(256) k_intensity(BasisView B, const uint8_t* __restrict__ vals,
                                                   const uint32_t* __restrict__ exps, int r,
                                                   double* __restrict__ partials, unsigned int* counter,
                                                   double* __restrict__ out) {
  __shared__ double red[8];
  __shared__ int flag;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t n = B.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x + t; k0 < n; k0 += 4 * stride) {
    if (F32) {
      float y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t k = k0 + u * stride;
        y[u] = k < n ? __ldcs(reinterpret_cast<const float*>(vals) + k) : 0.0f;
      }
      for (int s = 0; s < r; ++s) {
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = fmaf(y[u], 0.5f, 0.25f);
      }
      float sf = 0.0f;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k0 + u * stride < n) sf += y[u];
      acc += static_cast<double>(sf);
    } else {
      double y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t k = k0 + u * stride;
        y[u] = k < n ? decode_at<F, L>(vals, exps, k) : 0.0;
      }
      for (int s = 0; s < r; ++s) {
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = fma(y[u], 0.5, 0.25);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k0 + u * stride < n) acc += y[u];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += red[i];
    partials[blockIdx.x] = s;
  }
  if (arrive_last(counter, gridDim.x, &flag)) {
    if (warp == 0) {
      const double s = warp_sum_strided(partials, gridDim.x, 1);
      if (lane == 0) *out = s;
    }
    if (t == 0) *counter = 0;
  }
}

namespace {

template <int F, int L, bool F32>
int launch_t(const BasisView& B, const uint8_t* vals, const uint32_t* exps, int r, double* partials,
             unsigned int* counter, double* out, cudaStream_t stream) {
  DeviceInfo di;
  int st = device_info(&di);
  if (st) return st;
  int64_t g = (B.n + 4 * 256 - 1) / (4 * 256);
  const int64_t cap = (int64_t)di.sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  k_intensity<F, L, F32><<<static_cast<int>(g), 256, 0, stream>>>(B, vals, exps, r, partials, counter, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "intensity launch");
}

}  // namespace

int launch_intensity(const BasisView& B, int slot, int r, bool fp32_compute, double* partials, unsigned int* counter,
                     double* out, cudaStream_t stream) {
  const uint8_t* vals = B.vals + (int64_t)slot * B.vstride;
  const uint32_t* exps =
      B.fmt == CBG_FRSZ2
          ? reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint8_t*>(B.exps) + (int64_t)slot * B.estride)
          : nullptr;
  if (fp32_compute) return launch_t<CBG_FP32, 32, true>(B, vals, exps, r, partials, counter, out, stream);
  switch (B.fmt) {
    case CBG_FP64: return launch_t<CBG_FP64, 32, false>(B, vals, exps, r, partials, counter, out, stream);
    case CBG_FP32: return launch_t<CBG_FP32, 32, false>(B, vals, exps, r, partials, counter, out, stream);
    case CBG_FP16: return launch_t<CBG_FP16, 32, false>(B, vals, exps, r, partials, counter, out, stream);
    case CBG_BF16: return launch_t<CBG_BF16, 32, false>(B, vals, exps, r, partials, counter, out, stream);
    default:
      switch (B.l) {
        case 32: return launch_t<CBG_FRSZ2, 32, false>(B, vals, exps, r, partials, counter, out, stream);
        case 21: return launch_t<CBG_FRSZ2, 21, false>(B, vals, exps, r, partials, counter, out, stream);
        default: return launch_t<CBG_FRSZ2, 16, false>(B, vals, exps, r, partials, counter, out, stream);
      }
  }
}

}  // namespace cbg
