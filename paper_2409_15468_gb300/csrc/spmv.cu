// CSR sparse matrix-vector product w := A v (Fig. 1 step 3, M = I) with the norm of step 4 fused
// into the epilogue, the residual r := b - A x of step 1, and the CSR validation done once when a
// solver is created. The SpMV reads the uncompressed FP64 vector v: the paper highlights only the
// basis accesses as compressed.
//
// One thread per row for short rows: the stencil matrices have ~7 nonzeros per row, so the rows of a
// warp cover a contiguous stretch of the value and column arrays that L1 serves to the per-nonzero
// loads, and the FP64 work is exactly one FMA per nonzero (GB300's FP64 rate is the other bound of
// this kernel). Rows are strided over a grid sized to the SM count so that the norm partials stay
// few.
//
// Matrices with long rows (mean >= 12 nonzeros, e.g. power-law row lengths): a CTA takes 512
// consecutive rows, sorts them in shared memory by length bucket (floor(log2 len) + 1) and gives
// each bucket its own number G of lanes per row, about 8-16 nonzeros per lane. A warp then serves
// 32/G rows of lengths within a factor of two, so few lanes idle while it iterates to its longest
// row (GB300 issues every FP64 warp instruction at full cost, whatever its active lanes), the row
// sum costs log2(G) shuffle-adds, and the rows of a segment are read close together in time, so the
// sectors that neighbouring rows share come from DRAM once (a global sort by length scattered them:
// 1.47x the algorithmic DRAM bytes).
#include "common.cuh"
#include "kernels.cuh"

namespace cbg {

namespace {
__device__ __forceinline__ bool gate_skip_s(const Gate& g) {
  if (g.stop && *(volatile const int*)g.stop) return true;
  if (g.need && !*(volatile const int*)g.need) return true;
  return false;
}
}  // namespace

__global__ void __launch_bounds__(256) k_spmv(int n, const int32_t* __restrict__ row_ptr,
                                              const int32_t* __restrict__ col, const double* __restrict__ vals,
                                              const double* __restrict__ x, double* __restrict__ y,
                                              const double* __restrict__ bsub, double* __restrict__ partials,
                                              unsigned int* counter, int* err, NormEpilogue epi, Gate gate) {
  if (gate_skip_s(gate)) return;
  __shared__ double red[8];
  __shared__ int flag;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double nrm = 0.0;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + t; i < n; i += stride) {
    const int p0 = __ldg(row_ptr + i), p1 = __ldg(row_ptr + i + 1);
    double s = 0.0;
    for (int p = p0; p < p1; ++p) s = fma(__ldg(vals + p), __ldg(x + __ldg(col + p)), s);
    if (bsub) s = bsub[i] - s;
    y[i] = s;
    nrm = fma(s, s, nrm);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (lane == 0) red[warp] = nrm;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += red[i];
    partials[blockIdx.x] = s;
  }
  if (arrive_last(counter, gridDim.x, &flag)) {
    if (warp == 0) {
      const double s = warp_sum_strided(partials, gridDim.x, 1);
      if (lane == 0) norm_epilogue(epi, s, err);
    }
    if (t == 0) *counter = 0;
  }
}

// ---- long rows: segment-local sort by length, lanes per row by length -------------------------
// Loads in flight per lane and resident CTAs per SM of the long-row kernel (measured best; settable
// at build time for a sweep).
#ifndef CBG_SPMV_LOADS
#define CBG_SPMV_LOADS 8
#endif
#ifndef CBG_SPMV_CTAS_PER_SM
#define CBG_SPMV_CTAS_PER_SM 8
#endif
constexpr int kRowBuckets = 12;  // floor(log2 len) + 1, capped: bucket 0 holds the empty rows
constexpr int kSeg = 512;        // rows a CTA sorts and serves at a time

// Lanes per row for rows of bucket b (lengths [2^(b-1), 2^b)): about 8-16 nonzeros per lane, at
// most a warp per row.
__device__ __forceinline__ int bucket_lanes(int b) {
  const int g = b >= 5 ? 1 << (b - 4) : 1;
  return g < 32 ? g : 32;
}

// The sum of a row over G consecutive lanes (sub = lane % G): each lane keeps U independent
// (column, value, x-gather) loads in flight before its FMAs, one FMA chain per lane, and the G lanes
// combine in a fixed shuffle order (deterministic).
template <int G, int U>
__device__ __forceinline__ double row_sum(int p0, int p1, int sub, const int32_t* __restrict__ col,
                                          const double* __restrict__ vals, const double* __restrict__ x) {
  double s = 0.0;
  for (int p = p0 + sub; p < p1; p += G * U) {
    int c[U];
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = p + u * G;
      c[u] = q < p1 ? __ldg(col + q) : -1;
      v[u] = q < p1 ? __ldg(vals + q) : 0.0;
    }
    double xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u) s = fma(v[u], xv[u], s);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// A CTA serves segments of kSeg rows (grid-strided): the segment's row pointers go to shared
// memory, its rows are ordered by bucket there (within a bucket in any order: each row's sum does
// not depend on it), and warps take work groups of 32/G rows of one bucket in turn. ||y||^2 is
// then summed over the segment in row order, so it is deterministic.
template <int U>
__global__ void __launch_bounds__(256) k_spmv_seg(int n, const int32_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col, const double* __restrict__ vals,
                                                  const double* __restrict__ x, double* __restrict__ y,
                                                  const double* __restrict__ bsub, double* __restrict__ partials,
                                                  unsigned int* counter, int* err, NormEpilogue epi, Gate gate) {
  if (gate_skip_s(gate)) return;
  __shared__ int srp[kSeg + 1];
  __shared__ uint16_t sorder[kSeg];
  __shared__ int cnt[kRowBuckets], fill[kRowBuckets], off[kRowBuckets + 1], gst[kRowBuckets + 1];
  __shared__ double red[8];
  __shared__ int flag;
  constexpr int T = 256, PER = kSeg / T;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double nrm = 0.0;
  const int nseg = (n + kSeg - 1) / kSeg;
  for (int sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    const int r0 = sg * kSeg, rows = min(kSeg, n - r0);
    __syncthreads();  // the previous segment's shared arrays are no longer read
    if (t < kRowBuckets) {
      cnt[t] = 0;
      fill[t] = 0;
    }
    for (int i = t; i <= rows; i += T) srp[i] = __ldg(row_ptr + r0 + i);
    __syncthreads();
    int bk[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = t + k * T;
      bk[k] = -1;
      if (i < rows) {
        const int len = srp[i + 1] - srp[i];
        const int b = min(len > 0 ? 32 - __clz(len) : 0, kRowBuckets - 1);
        bk[k] = b;
        atomicAdd(&cnt[b], 1);
      }
    }
    __syncthreads();
    if (t == 0) {
      int o = 0, g = 0;
      for (int b = 0; b < kRowBuckets; ++b) {
        off[b] = o;
        gst[b] = g;
        const int per = 32 / bucket_lanes(b);
        o += cnt[b];
        g += (cnt[b] + per - 1) / per;
      }
      off[kRowBuckets] = o;
      gst[kRowBuckets] = g;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k)
      if (bk[k] >= 0) sorder[off[bk[k]] + atomicAdd(&fill[bk[k]], 1)] = static_cast<uint16_t>(t + k * T);
    __syncthreads();
    const int ngroups = gst[kRowBuckets];
    for (int gi = warp; gi < ngroups; gi += T / 32) {
      int b = 0;
      while (b + 1 < kRowBuckets && gst[b + 1] <= gi) ++b;  // warp-uniform
      const int G = bucket_lanes(b);
      const int j = off[b] + (gi - gst[b]) * (32 / G) + lane / G;
      const bool valid = j < off[b + 1];
      const int r = valid ? sorder[j] : 0;
      const int p0 = valid ? srp[r] : 0, p1 = valid ? srp[r + 1] : 0;
      const int sub = lane & (G - 1);
      double s;
      switch (G) {
        case 1: s = row_sum<1, U>(p0, p1, sub, col, vals, x); break;
        case 2: s = row_sum<2, U>(p0, p1, sub, col, vals, x); break;
        case 4: s = row_sum<4, U>(p0, p1, sub, col, vals, x); break;
        case 8: s = row_sum<8, U>(p0, p1, sub, col, vals, x); break;
        case 16: s = row_sum<16, U>(p0, p1, sub, col, vals, x); break;
        default: s = row_sum<32, U>(p0, p1, sub, col, vals, x); break;
      }
      if (valid && sub == 0) {
        if (bsub) s = bsub[r0 + r] - s;
        y[r0 + r] = s;
      }
    }
    __syncthreads();  // the segment's y is written (visible within the CTA)
    for (int i = t; i < rows; i += T) {
      const double v = y[r0 + i];
      nrm = fma(v, v, nrm);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (lane == 0) red[warp] = nrm;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += red[i];
    partials[blockIdx.x] = s;
  }
  if (arrive_last(counter, gridDim.x, &flag)) {
    if (warp == 0) {
      const double s = warp_sum_strided(partials, gridDim.x, 1);
      if (lane == 0) norm_epilogue(epi, s, err);
    }
    if (t == 0) *counter = 0;
  }
}

// dinv[i] = 1 / a_ii for the Jacobi preconditioner M = diag(A) (entries of row i in column i are
// summed); a zero, non-finite or missing diagonal sets kDevErrBadDiagonal. Runs only on a
// validated matrix.
__global__ void k_jacobi_diag(int n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                              const double* __restrict__ vals, double* __restrict__ dinv, int* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double d = 0.0;
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
      if (col[p] == i) d += vals[p];
    if (d == 0.0 || !isfinite(d)) {
      atomicOr(err, kDevErrBadDiagonal);
      dinv[i] = 0.0;
    } else {
      dinv[i] = 1.0 / d;
    }
  }
}

// x += d .* z (Fig. 1 step 17 with M^{-1} = diag(d): x_m := x_0 + M^{-1} (V_m y_m)).
__global__ void k_add_scaled(int64_t n, const double* __restrict__ d, const double* __restrict__ z,
                             double* __restrict__ x) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) x[k] = fma(d[k], z[k], x[k]);
}

__global__ void k_validate_csr(int n, int64_t nnz, const int32_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ col, int* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid == 0 && (row_ptr[0] != 0 || (int64_t)row_ptr[n] != nnz)) atomicOr(err, kDevErrBadMatrix);
  for (int64_t i = tid; i < n; i += stride)
    if (row_ptr[i] > row_ptr[i + 1]) atomicOr(err, kDevErrBadMatrix);
  for (int64_t p = tid; p < nnz; p += stride) {
    const int32_t c = col[p];
    if (c < 0 || c >= n) atomicOr(err, kDevErrBadMatrix);
  }
}

__global__ void __launch_bounds__(256) k_sumsq(const double* __restrict__ x, int64_t n, double* __restrict__ partials,
                                               unsigned int* counter, int* err, double* out) {
  __shared__ double red[8];
  __shared__ int flag;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double nrm = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + t; i < n; i += stride) nrm = fma(x[i], x[i], nrm);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (lane == 0) red[warp] = nrm;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += red[i];
    partials[blockIdx.x] = s;
  }
  if (arrive_last(counter, gridDim.x, &flag)) {
    if (warp == 0) {
      const double s = warp_sum_strided(partials, gridDim.x, 1);
      if (lane == 0) {
        *out = s;
        if (!isfinite(s)) atomicOr(err, kDevErrNonFinite);
      }
    }
    if (t == 0) *counter = 0;
  }
}

namespace {
int grid_rows(int64_t n, int per_sm) {
  DeviceInfo di;
  if (device_info(&di)) return 1;
  int64_t g = (n + 255) / 256;
  const int64_t cap = (int64_t)di.sms * per_sm;
  if (g > cap) g = cap;
  if (g > kMaxGrid) g = kMaxGrid;
  return g < 1 ? 1 : static_cast<int>(g);
}
}  // namespace

// Lanes per row from the mean row length: one thread per row below 12 nonzeros per row
// (stencils), else 4 lanes with 8 loads each in flight (measured best for mean row lengths 29 and
// 56 among 2-32 lanes and 2-8 loads).
int spmv_lanes_per_row(int n, int64_t nnz) {
  const double mean = n > 0 ? static_cast<double>(nnz) / n : 0.0;
  return mean < 12.0 ? 1 : 4;
}

int launch_spmv(int n, int64_t nnz, const int32_t* row_ptr, const int32_t* col, const double* vals, const double* x,
                double* y, const double* bsub, double* partials, unsigned int* counter, int* err,
                const NormEpilogue& epi, const Gate& gate, cudaStream_t stream) {
  if (n <= 0) return CBG_OK;
  const int g = spmv_lanes_per_row(n, nnz);
  if (g == 1) {
    const int grid = grid_rows(n, 8);
    k_spmv<<<grid, 256, 0, stream>>>(n, row_ptr, col, vals, x, y, bsub, partials, counter, err, epi, gate);
  } else {
    // one segment of kSeg rows per CTA and turn; as many CTAs as the GPU holds
    const int grid = grid_rows(((int64_t)n + kSeg - 1) / kSeg * 256, CBG_SPMV_CTAS_PER_SM);
    k_spmv_seg<CBG_SPMV_LOADS><<<grid, 256, 0, stream>>>(n, row_ptr, col, vals, x, y, bsub, partials, counter, err,
                                                         epi, gate);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "spmv launch");
}

int launch_jacobi_diag(int n, const int32_t* row_ptr, const int32_t* col, const double* vals, double* dinv, int* err,
                       cudaStream_t stream) {
  if (n <= 0) return CBG_OK;
  k_jacobi_diag<<<grid_rows(n, 8), 256, 0, stream>>>(n, row_ptr, col, vals, dinv, err);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "jacobi diagonal launch");
}

int launch_add_scaled(int64_t n, const double* d, const double* z, double* x, cudaStream_t stream) {
  if (n <= 0) return CBG_OK;
  k_add_scaled<<<grid_rows(n, 8), 256, 0, stream>>>(n, d, z, x);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "scaled add launch");
}

int launch_validate_csr(int n, int64_t nnz, const int32_t* row_ptr, const int32_t* col, int* err,
                        cudaStream_t stream) {
  const int grid = grid_rows(n > nnz ? n : nnz, 8);
  k_validate_csr<<<grid, 256, 0, stream>>>(n, nnz, row_ptr, col, err);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "csr validation launch");
}

int launch_sumsq(const double* x, int64_t n, double* partials, unsigned int* counter, int* err, double* out,
                 cudaStream_t stream) {
  const int grid = grid_rows(n, 4);
  k_sumsq<<<grid, 256, 0, stream>>>(x, n, partials, counter, err, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "sumsq launch");
}

}  // namespace cbg
