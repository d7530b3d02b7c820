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

// Device address of the scratch array per device index, looked up once with that device current.
// A failed lookup (for example one attempted during a stream capture) is not remembered: the next
// call tries again.
std::mutex g_scratch_mu;
double* g_scratch_ptr[64] = {};

}  // namespace

using namespace cbg;

extern "C" int cbg_basis_dot_noalloc(const cbg_basis* b, int32_t nvec, const double* d_w, double* d_h,
                                     void* stream) {
  int st = check_basis(b, nvec);
  if (st) return st;
  if (nvec > kNoAllocMaxVecs) {
    set_error("cbg_basis_dot_noalloc: nvec = %d is above %d, the capacity of its fixed scratch array "
              "(use cbg_basis_dot with a caller-provided work buffer for more vectors)",
              nvec, kNoAllocMaxVecs);
    return CBG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (nvec == 0) return CBG_OK;
  if (!d_h || reinterpret_cast<uintptr_t>(d_h) % 8) {
    set_error("cbg_basis_dot_noalloc: bad h pointer");
    return CBG_ERR_INVALID_ARG;
  }
  if (b->n == 0) {  // the empty sums
    cudaError_t e = cudaMemsetAsync(d_h, 0, sizeof(double) * nvec, s);
    return e == cudaSuccess ? CBG_OK : cuda_fail(e, "cbg_basis_dot_noalloc: zero fill");
  }
  if (!d_w || reinterpret_cast<uintptr_t>(d_w) % 16) {
    set_error("cbg_basis_dot_noalloc: bad w pointer");
    return CBG_ERR_INVALID_ARG;
  }
  DeviceInfo di;
  st = device_info(&di);
  if (st) return st;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cbg_basis_dot_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    set_error("cbg_basis_dot_noalloc: device index %d out of range", dev);
    return CBG_ERR_CUDA;
  }
  // Set-up per device, with that device current: the device address of the scratch array (the
  // array's name is only a host-side stand-in in host code).
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cbg_basis_dot_noalloc: cudaGetSymbolAddress");
      }
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    base = g_scratch_ptr[dev];
  }
  double* partials = base;
  double* control = base + kPartialDoubles;
  // The completion counter must start at zero; the array keeps whatever the previous call left.
  e = cudaMemsetAsync(control, 0, kControlDoubles * sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(e, "cbg_basis_dot_noalloc: control reset");
  return launch_basis_dot_capped(view(b), nvec, d_w, d_h, partials, reinterpret_cast<unsigned int*>(control),
                                 reinterpret_cast<int*>(control) + 4, kNoAllocMaxGrid, s);
}
