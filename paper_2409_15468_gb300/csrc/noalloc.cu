// cbg_basis_dot_noalloc: the basis dot product (h = V^T w over stored basis vectors) for callers
// that cannot allocate device memory.
//
// cbg_basis_dot needs a caller-provided scratch buffer for its cross-CTA partial sums. Some callers
// have no way to provide one: a plugin whose host application has reserved all device memory in
// its own pool, or a latency-critical path that must not call cudaMalloc (which can synchronise the
// whole device). This variant takes no scratch argument and allocates nothing: its partial sums and
// its completion counter live in a fixed array in device memory that this library defines and every
// GPU that loads the library keeps until the process exits.
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int kNoAllocMaxVecs = 128;   // largest nvec accepted
constexpr int kNoAllocMaxGrid = 1024;  // CTAs of one call at most (GB300 uses 456)
constexpr size_t kPartialDoubles = (size_t)kNoAllocMaxVecs * kNoAllocMaxGrid;
constexpr size_t kControlDoubles = 32;  // 256 bytes: completion counter, error word

// Scratch shared by every call on a device: kNoAllocMaxGrid x kNoAllocMaxVecs partial sums (1 MiB)
// followed by a 256-byte control region. Host code must not use this name as an address; it looks
// the address up with cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kPartialDoubles + kControlDoubles];

struct DeviceScratch {
  std::once_flag once;
  double* ptr = nullptr;
  cudaError_t status = cudaSuccess;
};
DeviceScratch g_scratch[64];

}  // namespace

using namespace cbg;

extern "C" int cbg_basis_dot_noalloc(const cbg_basis* b, int32_t nvec, const double* d_w, double* d_h,
                                     void* stream) {
  if (!b) {
    set_error("cbg_basis_dot_noalloc: null basis");
    return CBG_ERR_INVALID_ARG;
  }
  if (nvec < 0 || nvec > kNoAllocMaxVecs) {
    set_error("cbg_basis_dot_noalloc: nvec = %d is outside [0, %d], the capacity of its fixed scratch array "
              "(use cbg_basis_dot with a caller-provided work buffer for more vectors)",
              nvec, kNoAllocMaxVecs);
    return CBG_ERR_INVALID_ARG;
  }
  if (b->fmt < CBG_FP64 || b->fmt > CBG_FRSZ2 ||
      (b->fmt == CBG_FRSZ2 && b->frsz2_bits != 16 && b->frsz2_bits != 21 && b->frsz2_bits != 32) || b->n < 0 ||
      b->n > (int64_t(1) << 40)) {
    set_error("cbg_basis_dot_noalloc: bad basis format, code width or n");
    return CBG_ERR_INVALID_ARG;
  }
  if (nvec == 0 || b->n == 0) return CBG_OK;
  int64_t vs = 0, es = 0;
  cbg_basis_layout(b->n, b->fmt, b->fmt == CBG_FRSZ2 ? b->frsz2_bits : 32, &vs, &es);
  const bool frsz2 = b->fmt == CBG_FRSZ2;
  if (!b->vals || reinterpret_cast<uintptr_t>(b->vals) % 256 || b->vals_stride < vs || b->vals_stride % 256 ||
      (frsz2 && (!b->exps || reinterpret_cast<uintptr_t>(b->exps) % 256 || b->exps_stride < es ||
                 b->exps_stride % 256))) {
    set_error("cbg_basis_dot_noalloc: basis pointers must be 256-byte aligned with strides from cbg_basis_layout");
    return CBG_ERR_INVALID_ARG;
  }
  if (!d_w || !d_h || reinterpret_cast<uintptr_t>(d_w) % 16 || reinterpret_cast<uintptr_t>(d_h) % 8) {
    set_error("cbg_basis_dot_noalloc: bad w or h pointer");
    return CBG_ERR_INVALID_ARG;
  }
  DeviceInfo di;
  int st = device_info(&di);
  if (st) return st;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cbg_basis_dot_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    set_error("cbg_basis_dot_noalloc: device index %d out of range", dev);
    return CBG_ERR_CUDA;
  }
  // One-time set-up per device, with that device current: the device address of the scratch array.
  DeviceScratch& ds = g_scratch[dev];
  std::call_once(ds.once, [&]() {
    void* p = nullptr;
    ds.status = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    ds.ptr = static_cast<double*>(p);
  });
  if (ds.status != cudaSuccess || !ds.ptr) return cuda_fail(ds.status, "cbg_basis_dot_noalloc: cudaGetSymbolAddress");

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* partials = ds.ptr;
  double* control = ds.ptr + kPartialDoubles;
  // The completion counter must start at zero; the array keeps whatever the previous call left.
  e = cudaMemsetAsync(control, 0, kControlDoubles * sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(e, "cbg_basis_dot_noalloc: control reset");
  BasisView v;
  v.vals = static_cast<const uint8_t*>(b->vals);
  v.vstride = b->vals_stride;
  v.exps = b->exps;
  v.estride = b->exps_stride;
  v.n = b->n;
  v.fmt = b->fmt;
  v.l = frsz2 ? b->frsz2_bits : 32;
  return launch_basis_dot_capped(v, nvec, d_w, d_h, partials, reinterpret_cast<unsigned int*>(control),
                                 reinterpret_cast<int*>(control) + 4, kNoAllocMaxGrid, s);
}
