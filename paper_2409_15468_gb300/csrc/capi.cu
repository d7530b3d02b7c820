// C ABI of the library (include/cbgmres.h): argument validation, the error state, and the
// standalone codec, basis and SpMV entry points. The solver entry points live in solver.cu.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace cbg {

namespace {
thread_local char g_last_error[512] = "";

struct DevCache {
  std::once_flag once;
  DeviceInfo info;
  int status;
};
DevCache g_dev[64];
}  // namespace

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  if (e == cudaErrorMemoryAllocation) return CBG_ERR_OOM;
  return CBG_ERR_CUDA;
}

int device_info(DeviceInfo* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice (is a CUDA device available?)");
  if (dev < 0 || dev >= 64) {
    set_error("device index %d out of range", dev);
    return CBG_ERR_CUDA;
  }
  DevCache& c = g_dev[dev];
  std::call_once(c.once, [&]() {
    c.status = CBG_OK;
    cudaDeviceProp p;
    cudaError_t err = cudaGetDeviceProperties(&p, dev);
    if (err != cudaSuccess) {
      c.status = cuda_fail(err, "cudaGetDeviceProperties");
      return;
    }
    c.info.sms = p.multiProcessorCount;
    c.info.max_smem_optin = static_cast<int>(p.sharedMemPerBlockOptin);
    if (p.major < 10) {
      set_error("device %d is sm_%d%d; this library is built for sm_103a", dev, p.major, p.minor);
      c.status = CBG_ERR_CUDA;
    }
  });
  if (c.status != CBG_OK) {
    set_error("device %d is not usable by this library (needs an sm_103a GPU)", dev);
    return c.status;
  }
  *out = c.info;
  return CBG_OK;
}

}  // namespace cbg

using namespace cbg;

namespace {

constexpr int kMaxVecs = 1025;

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int bad(const char* msg) {
  set_error("%s", msg);
  return CBG_ERR_INVALID_ARG;
}

bool valid_l(int32_t l) { return l == 16 || l == 21 || l == 32; }

}  // namespace

// CBG_OK for an implemented FRSZ2 code width; CBG_ERR_UNIMPLEMENTED for another width the format
// admits (2..32 bits); CBG_ERR_INVALID_ARG otherwise.
int cbg::l_status(int32_t l, const char* what) {
  if (valid_l(l)) return CBG_OK;
  if (l >= 2 && l <= 32) {
    set_error("%s: FRSZ2 code width %d is not implemented (16, 21 or 32)", what, l);
    return CBG_ERR_UNIMPLEMENTED;
  }
  set_error("%s: FRSZ2 code width %d outside [2, 32]", what, l);
  return CBG_ERR_INVALID_ARG;
}

namespace {

int value_bytes(int32_t fmt) {
  switch (fmt) {
    case CBG_FP64: return 8;
    case CBG_FP32: return 4;
    case CBG_FP16:
    case CBG_BF16: return 2;
    default: return 0;
  }
}

}  // namespace

namespace cbg {

int check_basis(const cbg_basis* b, int32_t nvec_hi) {
  if (!b) return bad("null basis");
  if (b->fmt < CBG_FP64 || b->fmt > CBG_FRSZ2) return bad("basis: unknown format");
  if (b->fmt == CBG_FRSZ2) {
    const int st = l_status(b->frsz2_bits, "basis");
    if (st) return st;
  }
  if (b->n < 0 || b->n > (int64_t(1) << 40)) return bad("basis: n out of range");
  if (nvec_hi < 0 || nvec_hi > kMaxVecs) return bad("basis: vector index or count out of range (at most 1025)");
  if (b->n == 0) return CBG_OK;
  int64_t vs = 0, es = 0;
  cbg_basis_layout(b->n, b->fmt, b->fmt == CBG_FRSZ2 ? b->frsz2_bits : 32, &vs, &es);
  if (!b->vals || !aligned(b->vals, 256)) return bad("basis: vals must be a 256-byte aligned device pointer");
  if (b->vals_stride < vs || b->vals_stride % 256) return bad("basis: vals_stride too small or not a multiple of 256");
  if (b->fmt == CBG_FRSZ2) {
    if (!b->exps || !aligned(b->exps, 256)) return bad("basis: exps must be a 256-byte aligned device pointer");
    if (b->exps_stride < es || b->exps_stride % 256) return bad("basis: exps_stride too small or not a multiple of 256");
  }
  return CBG_OK;
}

BasisView view(const cbg_basis* b) {
  BasisView v;
  v.vals = static_cast<const uint8_t*>(b->vals);
  v.vstride = b->vals_stride;
  v.exps = b->exps;
  v.estride = b->exps_stride;
  v.n = b->n;
  v.fmt = b->fmt;
  v.l = b->fmt == CBG_FRSZ2 ? b->frsz2_bits : 32;
  return v;
}

BasisMut mut(const cbg_basis* b) {
  BasisMut v;
  v.vals = static_cast<uint8_t*>(b->vals);
  v.vstride = b->vals_stride;
  v.exps = b->exps;
  v.estride = b->exps_stride;
  v.n = b->n;
  v.fmt = b->fmt;
  v.l = b->fmt == CBG_FRSZ2 ? b->frsz2_bits : 32;
  return v;
}

}  // namespace cbg

namespace {

// Work buffer of the standalone reducing calls: partial sums, then one 256-byte control region
// (arrive_last ticket, error word).
struct Work {
  double* partials;
  unsigned int* counter;
  int* err;
};

size_t partial_bytes(int32_t nvec) { return (size_t)round_up((int64_t)kMaxGrid * (nvec > 0 ? nvec : 1) * 8, 256); }

int take_work(void* d_work, size_t work_bytes, int32_t nvec, cudaStream_t s, Work* w) {
  const size_t need = partial_bytes(nvec) + 256;
  if (!d_work || !aligned(d_work, 256)) return bad("work buffer must be a 256-byte aligned device pointer");
  if (work_bytes < need) {
    set_error("work buffer too small: %zu bytes given, %zu needed", work_bytes, need);
    return CBG_ERR_INVALID_ARG;
  }
  uint8_t* base = static_cast<uint8_t*>(d_work);
  w->partials = reinterpret_cast<double*>(base);
  w->counter = reinterpret_cast<unsigned int*>(base + partial_bytes(nvec));
  w->err = reinterpret_cast<int*>(base + partial_bytes(nvec) + 16);
  cudaError_t e = cudaMemsetAsync(base + partial_bytes(nvec), 0, 256, s);
  if (e != cudaSuccess) return cuda_fail(e, "work buffer reset");
  return CBG_OK;
}

}  // namespace

extern "C" {

const char* cbg_last_error(void) { return g_last_error; }

const char* cbgmres_last_error(void) { return g_last_error; }

size_t frsz2_bytes(int64_t n, int32_t l) {
  const int64_t b = cbg_frsz2_bytes(n, l);
  return b < 0 ? 0 : static_cast<size_t>(b);
}

int frsz2_compress(const double* d_src, int64_t n, int32_t l, uint32_t* d_exp, uint32_t* d_codes, void* stream) {
  return cbg_frsz2_compress(d_src, n, l, d_exp, d_codes, stream);
}

int frsz2_decompress(const uint32_t* d_exp, const uint32_t* d_codes, int64_t n, int32_t l, double* d_dst,
                     void* stream) {
  return cbg_frsz2_decompress(d_exp, d_codes, n, l, d_dst, stream);
}

const char* cbg_version(void) { return "cbgmres-gb300 0.1 (sm_103a)"; }

int64_t cbg_frsz2_bytes(int64_t n, int32_t l) {
  if (n < 0 || !valid_l(l)) return -1;
  const int64_t nb = (n + 31) / 32;
  return nb * ((32 * (int64_t)l + 31) / 32) * 4 + nb * 4;
}

int cbg_frsz2_compress(const double* d_src, int64_t n, int32_t l, uint32_t* d_exps, uint32_t* d_codes, void* stream) {
  if (const int lst = l_status(l, "cbg_frsz2_compress")) return lst;
  if (n < 0) return bad("cbg_frsz2_compress: negative n");
  if (n == 0) return CBG_OK;
  if (!d_src || !d_exps || !d_codes) return bad("cbg_frsz2_compress: null pointer");
  if (!aligned(d_src, 8) || !aligned(d_exps, 4) || !aligned(d_codes, 4))
    return bad("cbg_frsz2_compress: misaligned pointer");
  DeviceInfo di;
  int st = device_info(&di);
  if (st) return st;
  return launch_frsz2_compress(d_src, n, l, d_exps, d_codes, static_cast<cudaStream_t>(stream));
}

int cbg_frsz2_decompress(const uint32_t* d_exps, const uint32_t* d_codes, int64_t n, int32_t l, double* d_dst,
                         void* stream) {
  if (const int lst = l_status(l, "cbg_frsz2_decompress")) return lst;
  if (n < 0) return bad("cbg_frsz2_decompress: negative n");
  if (n == 0) return CBG_OK;
  if (!d_exps || !d_codes || !d_dst) return bad("cbg_frsz2_decompress: null pointer");
  if (!aligned(d_dst, 8) || !aligned(d_exps, 4) || !aligned(d_codes, 4))
    return bad("cbg_frsz2_decompress: misaligned pointer");
  DeviceInfo di;
  int st = device_info(&di);
  if (st) return st;
  return launch_frsz2_decompress(d_exps, d_codes, n, l, d_dst, static_cast<cudaStream_t>(stream));
}

int cbg_basis_layout(int64_t n, int32_t fmt, int32_t l, int64_t* vals_stride, int64_t* exps_stride) {
  if (!vals_stride || !exps_stride) return bad("cbg_basis_layout: null output");
  if (n < 0) return bad("cbg_basis_layout: negative n");
  const int64_t nb4 = round_up((n + 31) / 32, 4);  // blocks rounded up to 4 (128 values)
  if (fmt == CBG_FRSZ2) {
    if (!valid_l(l)) return bad("cbg_basis_layout: l must be 16, 21 or 32");
    *vals_stride = round_up(nb4 * l * 4, 256);
    *exps_stride = round_up(nb4 * 4, 256);
    return CBG_OK;
  }
  const int vb = value_bytes(fmt);
  if (!vb) return bad("cbg_basis_layout: unknown format");
  *vals_stride = round_up(nb4 * 32 * vb, 256);
  *exps_stride = 0;
  return CBG_OK;
}

int cbg_basis_store(const cbg_basis* basis, int32_t slot, const double* d_src, void* stream) {
  int st = check_basis(basis, slot + 1);
  if (st) return st;
  if (slot < 0) return bad("cbg_basis_store: negative slot");
  if (basis->n == 0) return CBG_OK;
  if (!d_src || !aligned(d_src, 8)) return bad("cbg_basis_store: bad source pointer");
  DeviceInfo di;
  st = device_info(&di);
  if (st) return st;
  return launch_store(mut(basis), slot, d_src, nullptr, nullptr, nullptr, nullptr, Gate{nullptr, nullptr},
                      static_cast<cudaStream_t>(stream));
}

int cbg_basis_append(const cbg_basis* basis, int32_t slot, const double* d_w, const double* d_h, double* d_v,
                     void* stream) {
  int st = check_basis(basis, slot + 1);
  if (st) return st;
  if (slot < 0) return bad("cbg_basis_append: negative slot");
  if (basis->n == 0) return CBG_OK;
  if (!d_w || !aligned(d_w, 8) || !d_h || !aligned(d_h, 8) || (d_v && !aligned(d_v, 8)))
    return bad("cbg_basis_append: bad w, h or v pointer");
  DeviceInfo di;
  st = device_info(&di);
  if (st) return st;
  return launch_store(mut(basis), slot, d_w, d_h, nullptr, d_v, nullptr, Gate{nullptr, nullptr},
                      static_cast<cudaStream_t>(stream));
}

int cbg_basis_load(const cbg_basis* basis, int32_t slot, double* d_dst, void* stream) {
  int st = check_basis(basis, slot + 1);
  if (st) return st;
  if (slot < 0) return bad("cbg_basis_load: negative slot");
  if (basis->n == 0) return CBG_OK;
  if (!d_dst || !aligned(d_dst, 8)) return bad("cbg_basis_load: bad destination pointer");
  DeviceInfo di;
  st = device_info(&di);
  if (st) return st;
  return launch_load(view(basis), slot, d_dst, static_cast<cudaStream_t>(stream));
}

size_t cbg_basis_work_bytes(int64_t n, int32_t nvec) {
  (void)n;
  if (nvec < 0 || nvec > kMaxVecs) return 0;
  return partial_bytes(nvec) + 256;
}

int cbg_basis_dot(const cbg_basis* basis, int32_t nvec, const double* d_w, double* d_h, void* d_work,
                  size_t work_bytes, void* stream) {
  int st = check_basis(basis, nvec);
  if (st) return st;
  if (nvec == 0 || basis->n == 0) {
    if (nvec > 0 && d_h) {
      cudaError_t e = cudaMemsetAsync(d_h, 0, sizeof(double) * nvec, static_cast<cudaStream_t>(stream));
      if (e != cudaSuccess) return cuda_fail(e, "cbg_basis_dot: zero fill");
    }
    return CBG_OK;
  }
  if (!d_w || !d_h || !aligned(d_w, 16) || !aligned(d_h, 8)) return bad("cbg_basis_dot: bad w or h pointer");
  DeviceInfo di;
  st = device_info(&di);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w;
  st = take_work(d_work, work_bytes, nvec, s, &w);
  if (st) return st;
  return launch_basis_dot(view(basis), nvec, d_w, d_h, w.partials, w.counter, w.err, Gate{nullptr, nullptr}, s);
}

int cbg_basis_update(const cbg_basis* basis, int32_t nvec, const double* d_h, double* d_w, double* d_norm2,
                     void* d_work, size_t work_bytes, void* stream) {
  int st = check_basis(basis, nvec);
  if (st) return st;
  if (basis->n == 0) {  // an empty w: nothing to update, ||w||^2 = 0
    if (d_norm2) {
      if (!aligned(d_norm2, 8)) return bad("cbg_basis_update: misaligned norm pointer");
      cudaError_t e = cudaMemsetAsync(d_norm2, 0, sizeof(double), static_cast<cudaStream_t>(stream));
      if (e != cudaSuccess) return cuda_fail(e, "cbg_basis_update: zero fill");
    }
    return CBG_OK;
  }
  if (!d_w || !aligned(d_w, 16) || (nvec > 0 && (!d_h || !aligned(d_h, 8))))
    return bad("cbg_basis_update: bad w or h pointer");
  DeviceInfo di;
  st = device_info(&di);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w;
  st = take_work(d_work, work_bytes, nvec, s, &w);
  if (st) return st;
  NormEpilogue epi{d_norm2, nullptr, kEpiNone};
  if (nvec == 0) {  // nothing to subtract; still report ||w||^2
    return d_norm2 ? launch_sumsq(d_w, basis->n, w.partials, w.counter, w.err, d_norm2, s) : CBG_OK;
  }
  return launch_basis_update(view(basis), nvec, nullptr, d_h, 0, d_w, w.partials, w.counter, w.err, epi,
                             Gate{nullptr, nullptr}, s);
}

int cbg_intensity(const cbg_basis* basis, int32_t slot, int32_t fma_per_value, int32_t compute_fp32, double* d_out,
                  void* d_work, size_t work_bytes, void* stream) {
  int st = check_basis(basis, 1);
  if (st) return st;
  if (slot < 0) return bad("cbg_intensity: negative slot");
  if (fma_per_value < 0 || fma_per_value > (1 << 20)) return bad("cbg_intensity: fma_per_value outside [0, 2^20]");
  if (compute_fp32 && basis->fmt != CBG_FP32) return bad("cbg_intensity: compute_fp32 needs fp32 storage");
  if (!d_out || !aligned(d_out, 8)) return bad("cbg_intensity: bad output pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (basis->n == 0) {
    cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(double), s);
    return e == cudaSuccess ? CBG_OK : cuda_fail(e, "cbg_intensity: zero fill");
  }
  DeviceInfo di;
  st = device_info(&di);
  if (st) return st;
  Work w;
  st = take_work(d_work, work_bytes, 1, s, &w);
  if (st) return st;
  return launch_intensity(view(basis), slot, fma_per_value, compute_fp32 != 0, w.partials, w.counter, d_out, s);
}

int cbg_csr_validate(int32_t n, int64_t nnz, const int32_t* d_row_ptr, const int32_t* d_col, void* stream) {
  if (n < 1 || nnz < 0 || nnz > INT32_MAX) return bad("cbg_csr_validate: n or nnz out of range");
  if (!d_row_ptr || (nnz > 0 && !d_col)) return bad("cbg_csr_validate: null pointer");
  DeviceInfo di;
  int st = device_info(&di);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* d_err = nullptr;
  int h_err = 0;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d_err), sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "cbg_csr_validate: allocation");
  e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) st = launch_validate_csr(n, nnz, d_row_ptr, d_col, d_err, s);
  if (e == cudaSuccess && st == CBG_OK) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d_err, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cbg_csr_validate");
  if (st) return st;
  if (h_err & kDevErrBadMatrix) {
    set_error("invalid CSR: row pointers not monotone, row_ptr[0] != 0, row_ptr[n] != nnz, or a column outside [0, n)");
    return CBG_ERR_BAD_MATRIX;
  }
  return CBG_OK;
}

size_t cbg_spmv_work_bytes(int32_t n) {
  (void)n;
  return partial_bytes(1) + 256;
}

int cbg_spmv(int32_t n, int64_t nnz, const int32_t* d_row_ptr, const int32_t* d_col, const double* d_vals,
             const double* d_x, double* d_y, double* d_norm2, void* d_work, size_t work_bytes, void* stream) {
  if (n < 0 || nnz < 0 || nnz > INT32_MAX) return bad("cbg_spmv: negative n or nnz outside [0, 2^31)");
  if (n == 0) return CBG_OK;
  if (!d_row_ptr || !d_x || !d_y || (nnz > 0 && (!d_col || !d_vals))) return bad("cbg_spmv: null pointer");
  DeviceInfo di;
  int st = device_info(&di);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (work_bytes < cbg_spmv_work_bytes(n)) {
    set_error("cbg_spmv: work buffer too small: %zu bytes given, %zu needed", work_bytes, cbg_spmv_work_bytes(n));
    return CBG_ERR_INVALID_ARG;
  }
  Work w;
  st = take_work(d_work, work_bytes, 1, s, &w);
  if (st) return st;
  NormEpilogue epi{d_norm2, nullptr, kEpiNone};
  return launch_spmv(n, nnz, d_row_ptr, d_col, d_vals, d_x, d_y, nullptr, w.partials, w.counter, w.err, epi,
                     Gate{nullptr, nullptr}, s);
}

}  // extern "C"
