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
// consecutive rows and sorts them in shared memory by a length key (the exact length below 64,
// eighths of an octave above), longest first. Each length class gets its own number G of lanes per
// row, at most 8 nonzeros per lane up to 255, so a warp serves 32/G rows of nearly equal length,
// each in one round of loads. GB300 issues an FP64 warp instruction at full cost whatever its
// active lanes, and the SpMV's FP64 time is close to its HBM time, so the warp issues exactly as
// many FMAs as its longest lane needs (no chunk padding). The row sum costs log2(G) shuffle-adds; the rows of a segment are read close together
// in time, so the sectors that neighbouring rows share come from DRAM once (a global sort by
// length scattered them: 1.47x the algorithmic DRAM bytes).
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
constexpr int kSeg = 512;                     // rows a CTA sorts and serves at a time
constexpr int kExactKeys = 64;                // rows shorter than this are keyed by their exact length
constexpr int kLenKeys = kExactKeys + 5 * 8;  // then 8 keys per octave up to 2047, the last one capped
constexpr int kLaneClasses = 6;               // G = 32, 16, 8, 4, 2, 1 lanes per row
// the sort keys of lane class c (G = 32 >> c) are [kClassLo[c], kClassLo[c - 1]), kClassLo[-1] = kLenKeys
// at most 8 nonzeros per lane below 256, one chunk of loads: G = 1 up to 8, 2 up to 16, 4 up to 32,
// 8 up to 63, 16 up to 127, else 32
__constant__ int kClassLo[kLaneClasses] = {kExactKeys + 8, kExactKeys, 33, 17, 9, 0};

// Sort key of a row of `len` nonzeros: the length itself below 64, else its octave and the three
// bits after the leading one (lengths within 12.5% share a key); 2048 and more share the top key.
// Keys ascend with the length, and each lane class is a contiguous range of keys: G = 1 up to 8
// nonzeros, 2 up to 16, 4 up to 32, 8 up to 63, 16 up to 127, else 32 (at most 8 nonzeros per lane
// below 256, so that a row's loads are in flight together: one round trip of column and value
// loads, then x gathers).
__device__ __forceinline__ int len_key(int len) {
  if (len < kExactKeys) return len;
  const int b = 31 - __clz(len);
  if (b >= 11) return kLenKeys - 1;
  return kExactKeys + (b - 6) * 8 + ((len >> (b - 3)) & 7);
}

// s + v[0] x[0] + ... + v[K-1] x[K-1], one FMA chain.
template <int K>
__device__ __forceinline__ double fma_chain(const double* v, const double* xv, double s) {
#pragma unroll
  for (int u = 0; u < K; ++u) s = fma(v[u], xv[u], s);
  return s;
}

// U (column, value) loads of one lane from p, p + G, ... (positions past p1 give 0), then the U
// x-gathers: all in flight before the FMAs.
template <int G, int U>
__device__ __forceinline__ void row_chunk(int p, int p1, const int32_t* __restrict__ col,
                                          const double* __restrict__ vals, const double* __restrict__ x, double* v,
                                          double* xv) {
  int c[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int q = p + u * G;
    c[u] = q < p1 ? __ldg(col + q) : -1;
    v[u] = q < p1 ? __ldg(vals + q) : 0.0;
  }
#pragma unroll
  for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : 0.0;
}

// The sum of a row over G consecutive lanes (sub = lane % G), lane sub taking nonzeros p0 + sub,
// p0 + sub + G, ... in order: the full chunks into two FMA chains (even and odd chunk positions),
// added together before the last partial chunk; the G lanes then combine in a fixed shuffle order
// (deterministic). The whole warp runs to the largest per-lane count of its rows, mw, in
// chunks of U loads and then one chunk of exactly mw mod U FMAs, so the warp issues mw FMAs: GB300
// issues an FP64 warp instruction at full cost whatever its active lanes, so no FMA is padded to a
// chunk boundary, and the rows of a warp have nearly equal lengths (sorted by key).
template <int G, int U>
__device__ __forceinline__ double row_sum(int p0, int p1, int sub, const int32_t* __restrict__ col,
                                          const double* __restrict__ vals, const double* __restrict__ x) {
  static_assert(U == 4 || U == 8, "the tail switch covers chunks of 4 or 8 loads");
  const int len = p1 - p0;
  const int m = len > sub ? (len - sub + G - 1) / G : 0;
  const int mw = static_cast<int>(__reduce_max_sync(0xffffffffu, static_cast<unsigned>(m)));
  double s = 0.0;
  double v[U], xv[U];
  int p = p0 + sub;
  double s2 = 0.0;  // GB300's dependent FP64 latency is ~64 cycles: two chains halve the wait
  for (int k = mw / U; k > 0; --k, p += G * U) {
    row_chunk<G, U>(p, p1, col, vals, x, v, xv);
#pragma unroll
    for (int u = 0; u < U; u += 2) {
      s = fma(v[u], xv[u], s);
      s2 = fma(v[u + 1], xv[u + 1], s2);
    }
  }
  s += s2;
  const int rem = mw % U;  // warp-uniform
  if (rem > 0) {
    row_chunk<G, U>(p, p1, col, vals, x, v, xv);
    switch (rem) {
      case 1: s = fma_chain<1>(v, xv, s); break;
      case 2: s = fma_chain<2>(v, xv, s); break;
      case 3: s = fma_chain<3>(v, xv, s); break;
      case 4: s = fma_chain<(U > 4 ? 4 : 1)>(v, xv, s); break;
      case 5: s = fma_chain<(U > 5 ? 5 : 1)>(v, xv, s); break;
      case 6: s = fma_chain<(U > 6 ? 6 : 1)>(v, xv, s); break;
      default: s = fma_chain<(U > 7 ? 7 : 1)>(v, xv, s); break;
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// A CTA serves segments of kSeg rows (grid-strided). The segment's row pointers go to shared
// memory; a counting sort on the length key orders its rows from the longest down; warps then take
// work groups of 32/G rows of one lane class from a shared counter, the longest rows first, so that
// the warps reach the segment's end together. The order within a key is arbitrary: each row's sum
// depends only on the row and its key. ||y||^2 is then summed over the segment in row order, so it
// is deterministic.
template <int U>
__global__ void __launch_bounds__(256) k_spmv_seg(int n, const int32_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col, const double* __restrict__ vals,
                                                  const double* __restrict__ x, double* __restrict__ y,
                                                  const double* __restrict__ bsub, double* __restrict__ partials,
                                                  unsigned int* counter, int* err, NormEpilogue epi, Gate gate) {
  if (gate_skip_s(gate)) return;
  __shared__ int srp[kSeg + 1];
  __shared__ uint16_t sorder[kSeg];
  __shared__ int cnt[kLenKeys], off[kLenKeys];
  __shared__ int cls[kLaneClasses + 1], grp[kLaneClasses + 1];
  __shared__ int next;
  __shared__ double red[8];
  __shared__ int flag;
  constexpr int T = 256, PER = kSeg / T;
  static_assert(kLenKeys <= 4 * 32, "one warp scans the keys, four per lane");
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double nrm = 0.0;
  const int nseg = (n + kSeg - 1) / kSeg;
  for (int sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    const int r0 = sg * kSeg, rows = min(kSeg, n - r0);
    __syncthreads();  // the previous segment's shared arrays are no longer read
    for (int i = t; i < kLenKeys; i += T) cnt[i] = 0;
    if (t == 0) next = 0;
    for (int i = t; i <= rows; i += T) srp[i] = __ldg(row_ptr + r0 + i);
    __syncthreads();
    int key[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = t + k * T;
      key[k] = i < rows ? len_key(srp[i + 1] - srp[i]) : -1;
      if (key[k] >= 0) atomicAdd(&cnt[key[k]], 1);
    }
    __syncthreads();
    if (warp == 0) {
      // off[key] := rows with a larger key (descending order), lane l holding positions 4l .. 4l+3
      int c4[4], s = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int kk = kLenKeys - 1 - (4 * lane + j);
        c4[j] = kk >= 0 ? cnt[kk] : 0;
        s += c4[j];
      }
      int incl = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
      }
      int run = incl - s;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int kk = kLenKeys - 1 - (4 * lane + j);
        if (kk >= 0) off[kk] = run;
        run += c4[j];
      }
      __syncwarp();
      if (lane == 0) {
        // class c's rows are [cls[c], cls[c + 1]) of the sorted order, its work groups start at grp[c]
        int g = 0;
        for (int c = 0; c < kLaneClasses; ++c) {
          cls[c] = off[(c == 0 ? kLenKeys : kClassLo[c - 1]) - 1];
          grp[c] = g;
          const int end = off[kClassLo[c]] + cnt[kClassLo[c]];
          g += (end - cls[c] + (1 << c) - 1) >> c;  // 32 / G = 2^c rows per group
        }
        cls[kLaneClasses] = rows;
        grp[kLaneClasses] = g;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k)
      if (key[k] >= 0) sorder[atomicAdd(&off[key[k]], 1)] = static_cast<uint16_t>(t + k * T);
    __syncthreads();
    const int ngroups = grp[kLaneClasses];
    for (;;) {
      int gi = 0;
      if (lane == 0) gi = atomicAdd(&next, 1);
      gi = __shfl_sync(0xffffffffu, gi, 0);
      if (gi >= ngroups) break;
      int c = 0;
      while (grp[c + 1] <= gi) ++c;  // warp-uniform; gi < grp[kLaneClasses]
      const int G = 32 >> c;
      const int j = cls[c] + ((gi - grp[c]) << c) + (lane >> (5 - c));
      const bool valid = j < cls[c + 1];
      const int r = valid ? sorder[j] : 0;
      const int p0 = valid ? srp[r] : 0, p1 = valid ? srp[r + 1] : 0;
      const int sub = lane & (G - 1);
      double s;
      switch (c) {
        case 0: s = row_sum<32, U>(p0, p1, sub, col, vals, x); break;
        case 1: s = row_sum<16, U>(p0, p1, sub, col, vals, x); break;
        case 2: s = row_sum<8, U>(p0, p1, sub, col, vals, x); break;
        case 3: s = row_sum<4, U>(p0, p1, sub, col, vals, x); break;
        case 4: s = row_sum<2, U>(p0, p1, sub, col, vals, x); break;
        default: s = row_sum<1, U>(p0, p1, sub, col, vals, x); break;
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
