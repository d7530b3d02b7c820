// Basis kernels for the cast storage formats (fp64, fp32, fp16, bf16) and the dispatch of the basis
// dot and update to the FRSZ2 kernels (basis_frsz2.cu) or the cast kernels.
//
// Cast formats widen each stored value to FP64 with integer bit manipulation (no FP64 conversion
// instruction, subnormals included) and take one FP64 FMA per value and vector, so on GB300 they
// are bound by the FP64 pipe (~1.9 FMA per clock per SM) rather than by HBM.
#include <mutex>
#include <unordered_map>

#include "basis_common.cuh"
#include "decode.cuh"

namespace cbg {

// ------------------------------------------------------------------------------------------------
// Cast formats: widen to FP64 with integer operations, one FP64 FMA per element and vector
// ------------------------------------------------------------------------------------------------

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
  // this CTA's vectors [v_lo, v_hi) (gridDim.y > 1 only when the values leave the GPU underfilled)
  const int v_lo = static_cast<int>((int64_t)nvec * blockIdx.y / gridDim.y);
  const int v_hi = static_cast<int>((int64_t)nvec * (blockIdx.y + 1) / gridDim.y);
  const int cid = blockIdx.y * gridDim.x + blockIdx.x, nctas = gridDim.x * gridDim.y;
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
    if (active && v_lo < v_hi) load8_widen<F>(B.vals + (int64_t)v_lo * B.vstride, kk, nxt);
    for (int vec = v_lo; vec < v_hi; ++vec) {
      double cur[P];
#pragma unroll
      for (int i = 0; i < P; ++i) cur[i] = nxt[i];
      if (active && vec + 1 < v_hi) load8_widen<F>(B.vals + (int64_t)(vec + 1) * B.vstride, kk, nxt);
      double hp = 0.0;
      if (active) {
#pragma unroll
        for (int i = 0; i < P; ++i)
          if (kk + i < B.n) hp = fma(cur[i], wv[i], hp);  // the padding past n may hold anything
      }
      const int vi = vec - v_lo;
      red[((batch & 1) * R + (vi % R)) * T + t] = hp;
      // one barrier per batch of R vectors: each vector has its own slot, and a buffer is written
      // again two batches later, after every thread has passed the next batch's barrier
      if (vi % R == R - 1 || vec == v_hi - 1) {
        __syncthreads();
        const int first = vec - (vi % R);
        for (int vv = first + warp; vv <= vec; vv += T / 32) {
          const double* r = red + ((batch & 1) * R + ((vv - v_lo) % R)) * T;
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
  for (int v = v_lo + t; v < v_hi; v += T) partials[(size_t)cid * nvec + v] = hpart[v];
  if (arrive_last(counter, nctas, &flags[0])) {
    slice_sums<2, 8>(partials, nvec, gridDim.x, gridDim.y, out, warp, T / 32);  // measured best here
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
// Launch configuration and dispatch
// ------------------------------------------------------------------------------------------------

namespace {

template <typename K>
const void* fnp(K k) {
  return reinterpret_cast<const void*>(k);
}

struct LaunchKey {
  const void* fn;
  size_t smem;
  int dev;
  bool operator==(const LaunchKey& o) const { return fn == o.fn && smem == o.smem && dev == o.dev; }
};
struct LaunchKeyHash {
  size_t operator()(const LaunchKey& k) const {
    return std::hash<const void*>()(k.fn) ^ (k.smem * 1315423911u) ^ (static_cast<size_t>(k.dev) << 48);
  }
};
struct FnKey {
  const void* fn;
  int dev;
  bool operator==(const FnKey& o) const { return fn == o.fn && dev == o.dev; }
};
struct FnKeyHash {
  size_t operator()(const FnKey& k) const { return std::hash<const void*>()(k.fn) ^ (static_cast<size_t>(k.dev) << 48); }
};
std::mutex g_cfg_mu;
std::unordered_map<LaunchKey, int, LaunchKeyHash> g_occ;    // CTAs per SM for (kernel, smem, device)
std::unordered_map<FnKey, size_t, FnKeyHash> g_smem_limit;  // dynamic smem limit raised so far

}  // namespace

int basis_launch_config(const void* fn, int threads, size_t smem, int64_t units, int64_t units_per_cta_min,
                        int max_grid, int* grid, int* full) {
  DeviceInfo di;
  int st = device_info(&di);
  if (st) return st;
  int dev = 0;
  cudaGetDevice(&dev);
  int occ = 0;
  {
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    // the limit only ever grows, so a launch with less shared memory never lowers it below a
    // size that another launch of the same kernel relies on
    size_t& limit = g_smem_limit[FnKey{fn, dev}];
    if (smem > limit) {
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(max dynamic shared memory)");
      limit = smem;
    }
    auto it = g_occ.find(LaunchKey{fn, smem, dev});
    if (it != g_occ.end()) {
      occ = it->second;
    } else {
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      if (occ < 1) {
        set_error("kernel does not fit on an SM with %zu bytes of shared memory", smem);
        return CBG_ERR_INVALID_ARG;
      }
      g_occ[LaunchKey{fn, smem, dev}] = occ;
    }
  }
  int64_t g = (int64_t)occ * di.sms;
  if (full) *full = static_cast<int>(g);
  int64_t need = (units + units_per_cta_min - 1) / units_per_cta_min;
  if (need < 1) need = 1;
  if (g > need) g = need;
  if (g > max_grid) g = max_grid;
  if (g > kMaxGrid) g = kMaxGrid;
  *grid = static_cast<int>(g);
  return CBG_OK;
}

namespace {

int cast_dot_launch(const BasisView& B, int nvec, const double* w, double* out, double* partials,
                    unsigned int* counter, int* err, const Gate& gate, int max_grid, cudaStream_t stream) {
  // binary32 and the 16-bit formats run the dot on the integer pipeline (exact block products, one
  // rounding per block); binary64 stays on FP64 FMAs, which measured faster for it (3.8 against
  // 2.3 TB/s: its 62-bit codes need four products and a 64-bit shift per value)
  if (B.fmt == CBG_FP32 || B.fmt == CBG_FP16 || B.fmt == CBG_BF16)
    return int_dot_launch(B, nvec, w, out, partials, counter, err, gate, max_grid, stream);
  if (B.fmt != CBG_FP64) return CBG_ERR_INVALID_ARG;
  const void* fn = fnp(k_dot_cast<CBG_FP64>);
  const size_t smem = CastCfg::dot_smem(nvec);
  int gx, full;
  int st = basis_launch_config(fn, CastCfg::kThreads, smem, B.n, 4096, max_grid, &gx, &full);
  if (st) return st;
  const dim3 grid(gx, dot_vector_split(gx, full, nvec, max_grid));
  k_dot_cast<CBG_FP64><<<grid, CastCfg::kThreads, smem, stream>>>(B, nvec, w, out, partials, counter, gate);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "cast dot launch");
}

}  // namespace

// Vector slices for a dot whose block grid gx leaves the GPU (full resident CTAs) underfilled: up to
// full / gx slices, at least one vector each, and gx * slices <= max_grid.
int dot_vector_split(int gx, int full, int nvec, int max_grid) {
  int64_t ny = gx > 0 ? full / gx : 1;
  if (ny > nvec) ny = nvec;
  const int64_t cap = (max_grid < kMaxGrid ? max_grid : kMaxGrid) / (gx > 0 ? gx : 1);
  if (ny > cap) ny = cap;
  return ny < 1 ? 1 : static_cast<int>(ny);
}

int launch_basis_dot(const BasisView& B, int nvec, const double* w, double* out, double* partials, unsigned int* counter,
                     int* err, const Gate& gate, cudaStream_t stream) {
  if (nvec <= 0 || B.n <= 0) return CBG_OK;
  if (B.fmt == CBG_FRSZ2) return frsz2_dot_launch(B, nvec, w, out, partials, counter, err, gate, kMaxGrid, stream);
  return cast_dot_launch(B, nvec, w, out, partials, counter, err, gate, kMaxGrid, stream);
}

// The basis dot with the grid limited to max_grid CTAs, for callers whose partial-sum buffer has a
// fixed capacity (max_grid * nvec doubles).
int launch_basis_dot_capped(const BasisView& B, int nvec, const double* w, double* out, double* partials,
                            unsigned int* counter, int* err, int max_grid, cudaStream_t stream) {
  if (nvec <= 0 || B.n <= 0) return CBG_OK;
  const Gate gate{nullptr, nullptr};
  if (B.fmt == CBG_FRSZ2) return frsz2_dot_launch(B, nvec, w, out, partials, counter, err, gate, max_grid, stream);
  return cast_dot_launch(B, nvec, w, out, partials, counter, err, gate, max_grid, stream);
}

int launch_basis_update(const BasisView& B, int nvec, const int* nvec_dev, const double* h, int negate, double* w,
                        double* partials, unsigned int* counter, int* err, const NormEpilogue& epi, const Gate& gate,
                        cudaStream_t stream) {
  if ((nvec <= 0 && !nvec_dev) || B.n <= 0) return CBG_OK;
  if (B.fmt == CBG_FRSZ2)
    return frsz2_update_launch(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate, stream);
  if (B.fmt == CBG_FP16)
    return fp16_update_launch(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate, stream);
  const void* fn;
  switch (B.fmt) {
    case CBG_FP64: fn = fnp(k_update_cast<CBG_FP64>); break;
    case CBG_FP32: fn = fnp(k_update_cast<CBG_FP32>); break;
    case CBG_FP16: fn = fnp(k_update_cast<CBG_FP16>); break;
    case CBG_BF16: fn = fnp(k_update_cast<CBG_BF16>); break;
    default: return CBG_ERR_INVALID_ARG;
  }
  const size_t smem = (size_t)nvec * 8 + (CastCfg::kThreads / 32) * 8 + 16;
  int grid;
  int st = basis_launch_config(fn, CastCfg::kThreads, smem, B.n, 2048, kMaxGrid, &grid, nullptr);
  if (st) return st;
  const int T = CastCfg::kThreads;
  switch (B.fmt) {
    case CBG_FP64: k_update_cast<CBG_FP64><<<grid, T, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate); break;
    case CBG_FP32: k_update_cast<CBG_FP32><<<grid, T, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate); break;
    case CBG_FP16: k_update_cast<CBG_FP16><<<grid, T, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate); break;
    default: k_update_cast<CBG_BF16><<<grid, T, smem, stream>>>(B, nvec, nvec_dev, h, negate, w, partials, counter, err, epi, gate); break;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "cast update launch");
}

}  // namespace cbg
