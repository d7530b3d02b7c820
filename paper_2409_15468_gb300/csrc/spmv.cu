// CSR sparse matrix-vector product w := A v (Fig. 1 step 3, M = I) with the norm of step 4 fused
// into the epilogue, the residual r := b - A x of step 1, and the CSR validation done once when a
// solver is created. The SpMV reads the uncompressed FP64 vector v: the paper highlights only the
// basis accesses as compressed.
//
// One thread per row for short rows: the stencil matrices have ~7 nonzeros per row, so the rows of a
// warp cover a contiguous stretch of the value and column arrays that L1 serves to the per-nonzero
// loads, and the FP64 work is exactly one FMA per nonzero (GB300's FP64 rate is the other bound of
// this kernel). Matrices with long rows (mean >= 12 nonzeros) use 4 lanes per row instead.
// Rows are strided over a grid sized to the SM count so that the norm partials stay few.
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

// Rows with many nonzeros (power-law matrices): G consecutive lanes per row, so the loads of a
// row's values and column indices are coalesced and a long row is split G ways. Each lane issues
// U independent (column, value, x-gather) loads before it uses any of them, and the next row's
// bounds are loaded before the current row is processed, so several gathers are in flight per
// lane. Each lane keeps one FMA chain and the G lanes of a row combine in a fixed shuffle order
// (deterministic): on GB300 every extra FP64 add costs as much issue time as a gather, so the
// combining work is kept to log2(G) adds per row and lane.
template <int G, int U>
__global__ void __launch_bounds__(256) k_spmv_vec(int n, const int32_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col, const double* __restrict__ vals,
                                                  const double* __restrict__ x, double* __restrict__ y,
                                                  const double* __restrict__ bsub, const int32_t* __restrict__ perm,
                                                  double* __restrict__ partials, unsigned int* counter, int* err,
                                                  NormEpilogue epi, Gate gate) {
  if (gate_skip_s(gate)) return;
  __shared__ double red[8];
  __shared__ int flag;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int sub = lane & (G - 1);
  // position j of the row order holds row perm[j] (rows sorted by length bucket, so the rows a
  // warp handles together have similar lengths), or row j without a permutation
  auto row_at = [&](int64_t j) -> int64_t { return perm ? static_cast<int64_t>(__ldg(perm + j)) : j; };
  double nrm = 0.0;
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  const int64_t g0 = (int64_t)blockIdx.x * (blockDim.x / G) + t / G;
  // every lane of a warp runs the same number of row iterations (rows past n are empty), so the
  // shuffles below always see the whole warp
  const int64_t rows_per_group = ((int64_t)n + groups - 1) / groups;
  int p0 = 0, p1 = 0;
  int64_t i = g0 < n ? row_at(g0) : n;
  if (g0 < n) {
    p0 = __ldg(row_ptr + i);
    p1 = __ldg(row_ptr + i + 1);
  }
  for (int64_t k = 0; k < rows_per_group; ++k) {
    const int64_t jnext = g0 + (k + 1) * groups;
    const int64_t inext = jnext < n ? row_at(jnext) : n;
    int q0 = 0, q1 = 0;
    if (inext < n) {
      q0 = __ldg(row_ptr + inext);
      q1 = __ldg(row_ptr + inext + 1);
    }
    double s = 0.0;  // one chain: the loads of a pass are in flight before its first FMA
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
    if (i < n && sub == 0) {
      if (bsub) s = bsub[i] - s;
      y[i] = s;
      nrm = fma(s, s, nrm);
    }
    p0 = q0;
    p1 = q1;
    i = inext;
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

// ---- row order by length (for the lanes-per-row kernel) ----------------------------------------
// A stable counting sort of the rows by the bucket floor(log2(len)) + 1 (capped at 11), in three
// deterministic passes: counts per 256-row chunk, a per-bucket scan, and the scatter with ranks
// from warp ballots. Rows that a warp then processes together have similar lengths, so a warp
// does not iterate to the length of one long row while its other lanes idle.
constexpr int kRowBuckets = 12;
constexpr int kRowChunk = 256;

__device__ __forceinline__ int row_bucket(const int32_t* row_ptr, int64_t i) {
  const int len = row_ptr[i + 1] - row_ptr[i];
  const int b = len > 0 ? 32 - __clz(len) : 0;
  return b < kRowBuckets - 1 ? b : kRowBuckets - 1;
}

__global__ void __launch_bounds__(kRowChunk) k_row_count(int n, const int32_t* __restrict__ row_ptr,
                                                         int32_t* __restrict__ counts) {
  __shared__ int cnt[kRowBuckets];
  const int t = threadIdx.x;
  if (t < kRowBuckets) cnt[t] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kRowChunk + t;
  if (i < n) atomicAdd(&cnt[row_bucket(row_ptr, i)], 1);
  __syncthreads();
  if (t < kRowBuckets) counts[(int64_t)blockIdx.x * kRowBuckets + t] = cnt[t];
}

// One CTA, one warp per bucket: counts[c][b] becomes the position of chunk c's first row of
// bucket b in the row order (buckets in increasing order, chunks in order within a bucket).
__global__ void __launch_bounds__(32 * kRowBuckets) k_row_scan(int nchunks, int32_t* __restrict__ counts) {
  __shared__ int total[kRowBuckets];
  const int b = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int carry = 0;
  for (int c0 = 0; c0 < nchunks; c0 += 32) {
    const int c = c0 + lane;
    const int v = c < nchunks ? counts[(int64_t)c * kRowBuckets + b] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (c < nchunks) counts[(int64_t)c * kRowBuckets + b] = carry + incl - v;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) total[b] = carry;
  __syncthreads();
  int base = 0;
  for (int bb = 0; bb < b; ++bb) base += total[bb];
  for (int c = lane; c < nchunks; c += 32) counts[(int64_t)c * kRowBuckets + b] += base;
}

__global__ void __launch_bounds__(kRowChunk) k_row_scatter(int n, const int32_t* __restrict__ row_ptr,
                                                           const int32_t* __restrict__ offs,
                                                           int32_t* __restrict__ perm) {
  constexpr int W = kRowChunk / 32;
  __shared__ int wcnt[W][kRowBuckets];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t i = (int64_t)blockIdx.x * kRowChunk + t;
  const bool valid = i < n;
  const int b = valid ? row_bucket(row_ptr, i) : -1;
  int rank = 0;
  for (int bb = 0; bb < kRowBuckets; ++bb) {
    const unsigned m = __ballot_sync(0xffffffffu, b == bb);
    if (lane == 0) wcnt[warp][bb] = __popc(m);
    if (b == bb) rank = __popc(m & ((1u << lane) - 1u));
  }
  __syncthreads();
  if (valid) {
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wcnt[w][b];
    perm[offs[(int64_t)blockIdx.x * kRowBuckets + b] + before + rank] = static_cast<int32_t>(i);
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

size_t row_order_scratch_bytes(int n) { return (size_t)((n + kRowChunk - 1) / kRowChunk) * kRowBuckets * 4; }

int launch_row_order(int n, const int32_t* row_ptr, int32_t* perm, int32_t* scratch, cudaStream_t stream) {
  if (n <= 0) return CBG_OK;
  const int nchunks = (n + kRowChunk - 1) / kRowChunk;
  k_row_count<<<nchunks, kRowChunk, 0, stream>>>(n, row_ptr, scratch);
  k_row_scan<<<1, 32 * kRowBuckets, 0, stream>>>(nchunks, scratch);
  k_row_scatter<<<nchunks, kRowChunk, 0, stream>>>(n, row_ptr, scratch, perm);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "row order launch");
}

int launch_spmv(int n, int64_t nnz, const int32_t* row_ptr, const int32_t* col, const double* vals, const double* x,
                double* y, const double* bsub, const int32_t* perm, double* partials, unsigned int* counter, int* err,
                const NormEpilogue& epi, const Gate& gate, cudaStream_t stream) {
  if (n <= 0) return CBG_OK;
  const int g = spmv_lanes_per_row(n, nnz);
  if (g == 1) {
    const int grid = grid_rows(n, 8);
    k_spmv<<<grid, 256, 0, stream>>>(n, row_ptr, col, vals, x, y, bsub, partials, counter, err, epi, gate);
  } else {
    const int grid = grid_rows((int64_t)n * g, 8);
    k_spmv_vec<4, 8><<<grid, 256, 0, stream>>>(n, row_ptr, col, vals, x, y, bsub, perm, partials, counter, err, epi,
                                               gate);
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
