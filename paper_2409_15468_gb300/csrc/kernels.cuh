// Internal kernel launchers of the library (host side) and the small device structs they share.
#pragma once

#include "common.cuh"

namespace cbg {

constexpr int kMaxGrid = 4096;  // upper bound on CTAs of the reducing kernels (sizes partial buffers)

// Skip a kernel (uniformly, at entry) when *stop != 0 or when *need == 0. Null pointers never skip.
struct Gate {
  const int* stop;
  const int* need;
};

// What the last CTA of a norm-producing kernel does with the reduced ||.||^2.
enum EpiMode { kEpiNone = 0, kEpiOmega = 1, kEpiPass1 = 2, kEpiPass2 = 3, kEpiResidual = 4 };

struct NormEpilogue {
  double* out;     // receives ||.||^2 when not null
  SolverCtl* ctl;  // solver control block to update, or null
  int mode;        // EpiMode
};

__device__ __forceinline__ void norm_epilogue(const NormEpilogue& e, double norm2, int* err) {
  if (e.out) *e.out = norm2;
  if (!e.ctl) return;
  SolverCtl* c = e.ctl;
  if (!isfinite(norm2)) {
    atomicOr(err, kDevErrNonFinite);
    c->stop = 1;
  }
  const double nrm = sqrt(norm2);
  switch (e.mode) {
    case kEpiOmega:  // Fig. 1 step 4
      c->omega2 = norm2;
      break;
    case kEpiPass1: {  // step 6 and the test of step 7
      c->hn2_first = norm2;
      c->hn2 = norm2;
      c->reorth = nrm < c->eta * sqrt(c->omega2) ? 1 : 0;
      break;
    }
    case kEpiPass2:  // step 10
      c->hn2 = norm2;
      break;
    case kEpiResidual:  // step 1: beta = ||r0||, v = r0 / beta
      c->beta = nrm;
      c->hdiv = nrm;
      c->rcp = nrm > 0.0 ? 1.0 / nrm : 0.0;
      break;
    default:
      break;
  }
}

// ---- capi.cu: argument checks shared by the C entry points ----------------------------------
// CBG_OK when `b` describes a basis the fused kernels can read for vector indices below nvec_hi
// (format, code width, n, 256-byte aligned pointers and strides from cbg_basis_layout); the
// CBG_ERR_* status otherwise, with the message set.
int check_basis(const cbg_basis* b, int32_t nvec_hi);
BasisView view(const cbg_basis* b);
BasisMut mut(const cbg_basis* b);
// CBG_OK for FRSZ2 code widths 16, 21, 32; CBG_ERR_UNIMPLEMENTED for another width in [2, 32];
// CBG_ERR_INVALID_ARG otherwise (message set, prefixed with `what`).
int l_status(int32_t l, const char* what);

// ---- basis.cu / basis_frsz2.cu -----------------------------------------------------------------
// Grid for a reducing basis kernel: occupancy x SMs, at most one CTA per units_per_cta_min units,
// at most max_grid (and kMaxGrid); *full (if not null) receives occupancy x SMs. Raises the
// kernel's dynamic shared memory limit once.
int basis_launch_config(const void* fn, int threads, size_t smem, int64_t units, int64_t units_per_cta_min,
                        int max_grid, int* grid, int* full);
int dot_vector_split(int gx, int full, int nvec, int max_grid);
int frsz2_dot_launch(const BasisView& B, int nvec, const double* w, double* out, double* partials,
                     unsigned int* counter, int* err, const Gate& gate, int max_grid, cudaStream_t stream);
// The dot of a binary32, binary16 or bfloat16 basis (B.fmt) on the FRSZ2 kernels' integer pipeline.
int int_dot_launch(const BasisView& B, int nvec, const double* w, double* out, double* partials,
                    unsigned int* counter, int* err, const Gate& gate, int max_grid, cudaStream_t stream);
int fp16_update_launch(const BasisView& B, int nvec, const int* nvec_dev, const double* h, int negate, double* w,
                       double* partials, unsigned int* counter, int* err, const NormEpilogue& epi, const Gate& gate,
                       cudaStream_t stream);
int frsz2_update_launch(const BasisView& B, int nvec, const int* nvec_dev, const double* h, int negate, double* w,
                        double* partials, unsigned int* counter, int* err, const NormEpilogue& epi,
                        const Gate& gate, cudaStream_t stream);
// ---- basis.cu -----------------------------------------------------------------------------------
// out[i] = <vhat_i, w> for i < nvec. partials: kMaxGrid * nvec doubles. *counter must be 0.
int launch_basis_dot(const BasisView& B, int nvec, const double* w, double* out, double* partials,
                     unsigned int* counter, int* err, const Gate& gate, cudaStream_t stream);
// The same with at most max_grid CTAs (partials: max_grid * nvec doubles).
int launch_basis_dot_capped(const BasisView& B, int nvec, const double* w, double* out, double* partials,
                            unsigned int* counter, int* err, int max_grid, cudaStream_t stream);
// w -= sum_i vhat_i h_i (h negated when `negate`), nvec from *nvec_dev when not null (then
// nvec is the upper bound used to size shared memory). ||w||^2 goes to the epilogue.
int launch_basis_update(const BasisView& B, int nvec, const int* nvec_dev, const double* h, int negate, double* w,
                        double* partials, unsigned int* counter, int* err, const NormEpilogue& epi,
                        const Gate& gate, cudaStream_t stream);

// ---- codec.cu -----------------------------------------------------------------------------------
// Stores src into basis vector `slot`; when hdiv is not null, stores v = src / *hdiv instead
// (correctly rounded; *rcp = RN(1 / *hdiv) when rcp is not null, else computed), and writes v to
// vout when vout is not null, multiplied elementwise by dscale when dscale is not null (the SpMV
// input M^{-1} v of a right preconditioner M = diag^{-1}(dscale)).
int launch_store(const BasisMut& B, int slot, const double* src, const double* hdiv, const double* rcp, double* vout,
                 const double* dscale, const Gate& gate, cudaStream_t stream);
int launch_frsz2_compress(const double* src, int64_t n, int l, uint32_t* exps, uint32_t* codes, cudaStream_t stream);
int launch_frsz2_decompress(const uint32_t* exps, const uint32_t* codes, int64_t n, int l, double* dst,
                            cudaStream_t stream);
int launch_load(const BasisView& B, int slot, double* dst, cudaStream_t stream);

// ---- spmv.cu ------------------------------------------------------------------------------------
// y = A x (or y = bsub - A x when bsub is not null); ||y||^2 to the epilogue. partials: kMaxGrid.
int launch_spmv(int n, int64_t nnz, const int32_t* row_ptr, const int32_t* col, const double* vals, const double* x,
                double* y, const double* bsub, double* partials, unsigned int* counter, int* err,
                const NormEpilogue& epi, const Gate& gate, cudaStream_t stream);
// Lanes per row of the SpMV for this matrix shape (1: one thread per row; else the long-row kernel).
int spmv_lanes_per_row(int n, int64_t nnz);
// dinv := 1 / diag(A) (kDevErrBadDiagonal on a zero or missing entry); x += d .* z.
int launch_jacobi_diag(int n, const int32_t* row_ptr, const int32_t* col, const double* vals, double* dinv, int* err,
                       cudaStream_t stream);
int launch_add_scaled(int64_t n, const double* d, const double* z, double* x, cudaStream_t stream);
int launch_validate_csr(int n, int64_t nnz, const int32_t* row_ptr, const int32_t* col, int* err,
                        cudaStream_t stream);
int launch_sumsq(const double* x, int64_t n, double* partials, unsigned int* counter, int* err, double* out,
                 cudaStream_t stream);

// ---- solver.cu ----------------------------------------------------------------------------------
struct GivensArgs {
  SolverCtl* ctl;
  double* H;     // (m+1) x m column-major, ld m+1: the Hessenberg matrix (before rotations)
  double* R;     // the rotated copy
  double* cs;
  double* sn;
  double* g;     // rotated right-hand side beta e1
  const double* u;  // second-pass coefficients
  double* hist;  // implicit RRN history (may be null)
  int64_t hist_off;
  int64_t hist_cap;
  int m;
};
int launch_givens(const GivensArgs& a, int j, cudaStream_t stream);
int launch_cycle_init(SolverCtl* ctl, double* g, int m, int steps_allowed, cudaStream_t stream);

// The length r = sqrt(a*a + b*b) of the Givens rotation that zeroes b against a (Fig. 1 step 17),
// as IEEE operations in that order (no fused multiply-add), after an exact power-of-two scaling when
// the larger exponent field is above 1523 or below 523. The oracle evaluates the same expression,
// so both round r identically; it is also cheaper than a library hypot on GB300 (one square root
// and two dependent FP64 operations against ~1 000 cycles).
__device__ __forceinline__ double givens_radius(double a, double b) {
  const int ea = static_cast<int>((static_cast<unsigned long long>(__double_as_longlong(a)) >> 52) & 0x7FF);
  const int eb = static_cast<int>((static_cast<unsigned long long>(__double_as_longlong(b)) >> 52) & 0x7FF);
  const int e = ea > eb ? ea : eb;
  if (e <= 1523 && e >= 523) return sqrt(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)));
  const double scale = e > 1523 ? 0x1p-600 : 0x1p600;
  const double as = __dmul_rn(a, scale), bs = __dmul_rn(b, scale);
  return __ddiv_rn(sqrt(__dadd_rn(__dmul_rn(as, as), __dmul_rn(bs, bs))), scale);
}

// Applies the rotations 0..j-1 of the least-squares update (Fig. 1 step 17) to col[0..j], called
// by all 32 lanes of one warp: col[i] := c_i x_i + s_i y_i with x_0 = col[0],
// x_{i+1} = -s_i x_i + c_i y_i and y_i the entry col[i+1] before the rotations. Returns x_j
// (col[j] holds it too). p and q are j doubles of scratch each.
//
// GB300's FP64 pipe spends ~64 cycles on every warp instruction however few lanes are active, so
// the carried recurrence, an affine map per rotation, runs as a warp scan rather than a chain of
// j FMAs. Lane l composes the maps of its K = ceil(j/32) consecutive rotations, five shuffle
// levels compose them across the lanes, and each lane replays its rotations from the composed
// start value: about 4K + 11 FP64 instructions per warp instead of j + 3. Every output and every
// x_{i+1} is still one FMA on the products c_i y_i and s_i y_i. Only the start of each lane's
// chunk is rounded in a different order than in a sequential pass.
__device__ __forceinline__ double rotate_column_warp(double* col, const double* cs, const double* sn, double* p,
                                                     double* q, int j, int lane) {
  const double x0 = col[0];
  if (j <= 0) return x0;
  for (int i = lane; i < j; i += 32) {
    const double y = col[i + 1];
    p[i] = cs[i] * y;
    q[i] = sn[i] * y;
  }
  __syncwarp();
  const int K = (j + 31) >> 5;
  const int i0 = lane * K, i1 = min(j, i0 + K);
  double A = 1.0, B = 0.0;  // this lane's rotations as x -> A x + B
  for (int i = i0; i < i1; ++i) {
    const double a = -sn[i];
    B = fma(a, B, p[i]);
    A = a * A;
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {  // inclusive scan: the maps of lanes <= l, earlier ones first
    const double Ap = __shfl_up_sync(0xffffffffu, A, d), Bp = __shfl_up_sync(0xffffffffu, B, d);
    if (lane >= d) {
      B = fma(A, Bp, B);
      A = A * Ap;
    }
  }
  double Ae = __shfl_up_sync(0xffffffffu, A, 1), Be = __shfl_up_sync(0xffffffffu, B, 1);
  double x = lane == 0 ? x0 : fma(Ae, x0, Be);  // x at the start of this lane's rotations
  for (int i = i0; i < i1; ++i) {
    col[i] = fma(cs[i], x, q[i]);
    x = fma(-sn[i], x, p[i]);
  }
  const double xj = __shfl_sync(0xffffffffu, x, (j - 1) / K);
  __syncwarp();
  if (lane == 0) col[j] = xj;
  __syncwarp();
  return xj;
}

// ---- intensity.cu -------------------------------------------------------------------------------
// *out = sum_k f^r(x_k) over stored vector `slot` (see cbg_intensity). partials: kMaxGrid doubles.
int launch_intensity(const BasisView& B, int slot, int r, bool fp32_compute, double* partials, unsigned int* counter,
                     double* out, cudaStream_t stream);

// ---- onchip.cu: a whole restart cycle in one thread-block cluster ------------------------------
// Shared-memory layout of one CTA of the on-chip cycle (byte offsets; rows per CTA a multiple of 32).
struct OcLayout {
  int rows;
  int slot_bytes;  // stride between basis slots
  int exp_words;   // stride between slots' exponent words (FRSZ2)
  int off_codes, off_exps, off_z, off_vec, off_state;
  int off_csr;     // the CTA's CSR rows (values, columns, row offsets) when they fit in csr_bytes
  int csr_bytes;
  int bytes;       // dynamic shared memory per CTA
};
struct OnchipPlan {
  int cluster;  // CTAs per cluster (16 or 8); 0: the system takes the streamed cycle
  OcLayout lay;
};
struct OnchipArgs {
  int n;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* vals;
  const double* b;
  double* x;           // x0 in, x_m out
  const double* dinv;  // Jacobi M^{-1} = 1 / diag(A), or null
  double* r;           // r0 = b - A x0 in (its norm and reciprocal in ctl), the next r out
  BasisMut basis;      // receives the cycle's basis vectors (streamed layout)
  SolverCtl* ctl;
  double* hist;
  int64_t hist_off;
  int64_t hist_cap;
  int m;
  int steps_allowed;
};
// Decides whether the system (n rows, nnz nonzeros, options o) runs its cycles on chip: short
// rows, restart + 1 <= 128, one CTA's slice of the basis within the opt-in shared memory and a
// cluster of that size schedulable on the device. plan->cluster = 0 otherwise.
int onchip_plan(int32_t n, int64_t nnz, const cbg_opts* o, OnchipPlan* plan);
// One restart cycle (Fig. 1 steps 1-17) and the next residual: r and x updated, ctl's beta, rcp,
// m_eff, reorth_count, m_ls, breakdown, implicit and err set, the basis written back.
int launch_onchip_cycle(const OnchipPlan& plan, const OnchipArgs& a, int fmt, int l, cudaStream_t stream);

// ---- solver contexts over caller-provided memory (solver.cu), used by the serving runtime ----
size_t ctx_pinned_bytes();
size_t ctx_device_bytes(int32_t n, const cbg_opts* opts);
int ctx_create_in(cbg_ctx** out, int32_t n, int64_t nnz, const int32_t* d_row_ptr, const int32_t* d_col,
                  const double* d_vals, const cbg_opts* opts, cudaStream_t stream, void* dmem, size_t dbytes,
                  void* pinned);
int ctx_validated(cbg_ctx* c);
void ctx_release(cbg_ctx* c);
cudaStream_t ctx_stream(const cbg_ctx* c);

}  // namespace cbg
