// Restarted CB-GMRES (Fig. 1 of arXiv 2409.15468) on one GPU: the solver context, its device
// workspace, the small single-CTA kernels (Givens rotations, back substitution) and the host state
// machine behind cbgmres_solve and the stepwise calls.
//
// One Arnoldi step j enqueues, on the context's stream:
//   spmv     w := A v_j, ||w||                                  (steps 3-4)
//   dot      h_{0..j} := V^T w   into column j of Hbar          (step 5)
//   update   w := w - V h, ||w||, decide the second pass        (steps 5-7)
//   dot      u := V^T w          (skipped unless needed)        (step 8)
//   update   w := w - V u, ||w|| (skipped unless needed)        (steps 8-10)
//   givens   h += u, h_{j+1,j}, rotations, implicit residual, breakdown and stop tests (9, 12, 17)
//   store    v_{j+1} := w / h_{j+1,j} into the FP64 v and basis slot j+1   (steps 13-14)
// All decisions live in a device control block (SolverCtl); kernels of a finished cycle return at
// entry, so a cycle is enqueued without host round trips. The host synchronises once per cycle,
// on an event after the restart's residual (step 1 of the next cycle), reading a pinned copy of
// the control block. The wait is non-blocking in cbgmres_advance, which lets a serving loop
// interleave many solves on their own streams.
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "common.cuh"
#include "kernels.cuh"

namespace cbg {

// ---- single-CTA kernels -------------------------------------------------------------------------

__global__ void k_cycle_init(SolverCtl* ctl, double* g, int m, int steps_allowed) {
  // g := beta e1; reset the per-cycle state (step 1)
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = i == 0 ? ctl->beta : 0.0;
  if (threadIdx.x == 0) {
    ctl->stop = ctl->beta > 0.0 ? 0 : 1;
    ctl->reorth = 0;
    ctl->m_eff = 0;
    ctl->breakdown = 0;
    ctl->reorth_count = 0;
    ctl->m_ls = 0;
    ctl->steps_allowed = steps_allowed;
  }
}

__global__ void k_set_bnorm(SolverCtl* ctl, const double* bnorm2, double tol, double eta) {
  ctl->bnorm = sqrt(*bnorm2);
  ctl->tol = tol;
  ctl->eta = eta;
  ctl->stop = 0;
  ctl->err = 0;
}

// Column j of the least-squares problem (step 17, one column at a time): finish h with the second
// pass (step 9), set h_{j+1,j} (steps 6/10), test for breakdown (step 12), apply the previous
// Givens rotations, form the new one and rotate beta e1. |g_{j+1}| / ||b|| is the implicit residual.
// One warp stages the column and the previous rotations in shared memory; lane 0 then runs the
// sequential recurrence on shared memory (no dependent global loads in the loop).
constexpr int kMaxRestart = 1024;
__global__ void __launch_bounds__(32) k_givens(GivensArgs a, int j) {
  __shared__ double col[kMaxRestart + 2];
  __shared__ double scs[kMaxRestart], ssn[kMaxRestart], sp[kMaxRestart], sq[kMaxRestart];
  SolverCtl* c = a.ctl;
  if (*(volatile const int*)&c->stop) return;  // every lane reads it before lane 0 may write it
  const int lane = threadIdx.x;
  const int ld = a.m + 1;
  double* hcol = a.H + (size_t)j * ld;
  const int reorth = c->reorth;
  for (int i = lane; i <= j; i += 32) {
    double h = hcol[i];
    if (reorth) {
      h += a.u[i];
      hcol[i] = h;
    }
    col[i] = h;
  }
  for (int i = lane; i < j; i += 32) {
    scs[i] = a.cs[i];
    ssn[i] = a.sn[i];
  }
  __syncwarp();
  // lanes 0 and 1: ||w|| and, for the breakdown test, ||w|| after the first pass (one instruction
  // stream for both); then the previous rotations, across the warp
  const double sqv = sqrt(lane == 1 ? c->hn2_first : c->hn2);
  const double hn = __shfl_sync(0xffffffffu, sqv, 0), hn_first = __shfl_sync(0xffffffffu, sqv, 1);
  const double x = rotate_column_warp(col, scs, ssn, sp, sq, j, lane), y = hn;
  // the new rotation: lane 0 c = x / r, lane 1 s = y / r, lane 2 the next normalisation 1 / h
  const double r = givens_radius(x, y);
  const double num = lane == 0 ? x : (lane == 1 ? y : 1.0);
  const double den = lane == 2 ? hn : r;
  const double qv = (lane < 3 && den != 0.0) ? num / den : 0.0;
  const double cs = y != 0.0 ? __shfl_sync(0xffffffffu, qv, 0) : 1.0;
  const double sn = y != 0.0 ? __shfl_sync(0xffffffffu, qv, 1) : 0.0;
  const double rcp = __shfl_sync(0xffffffffu, qv, 2);
  if (lane == 0) {
    if (reorth) c->reorth_count += 1;
    hcol[j + 1] = hn;
    const bool breakdown = (hn == 0.0) || (reorth && hn < c->eta * hn_first);
    col[j] = y != 0.0 ? r : x;
    col[j + 1] = 0.0;
    a.cs[j] = cs;
    a.sn[j] = sn;
    a.g[j + 1] = -sn * a.g[j];
    a.g[j] = cs * a.g[j];
    const double implicit = fabs(a.g[j + 1]) / c->bnorm;
    c->implicit = implicit;
    if (a.hist && a.hist_off + j < a.hist_cap) a.hist[a.hist_off + j] = implicit;
    c->m_eff = j + 1;
    if (breakdown) c->breakdown = 1;
    if (!isfinite(implicit)) {
      c->err |= kDevErrNonFinite;
      c->stop = 1;
    }
    if (breakdown || implicit <= c->tol || j + 1 >= c->steps_allowed) c->stop = 1;
    c->hdiv = hn;
    c->rcp = hn > 0.0 ? rcp : 0.0;
    c->reorth = 0;
  }
  __syncwarp();
  double* Rj = a.R + (size_t)j * ld;
  for (int i = lane; i <= j + 1; i += 32) Rj[i] = col[i];
}

// y := R^{-1} g over the leading columns with a nonzero diagonal (step 17). The CTA finds the first
// zero pivot in parallel and, for restarts up to kBacksubStaged, stages the upper triangle of R
// transposed in shared memory (rows contiguous); one warp then runs the substitution.
constexpr int kBacksubStaged = 128;
__global__ void __launch_bounds__(256) k_backsub(GivensArgs a, double* y) {
  extern __shared__ double sT[];  // [mls][mls] rows of R, then y[mls] (staged case only)
  __shared__ int s_mls;
  SolverCtl* c = a.ctl;
  const int t = threadIdx.x, lane = t & 31;
  const int ld = a.m + 1;
  const int m_eff = c->m_eff;
  if (t == 0) s_mls = m_eff;
  __syncthreads();
  for (int k = t; k < m_eff; k += blockDim.x)
    if (a.R[(size_t)k * ld + k] == 0.0) atomicMin(&s_mls, k);
  __syncthreads();
  const int mls = s_mls;
  const bool staged = a.m <= kBacksubStaged;
  if (staged) {
    for (int idx = t; idx < mls * mls; idx += blockDim.x) {
      const int cl = idx / mls, r = idx - cl * mls;  // consecutive threads read down a column
      if (r <= cl) sT[r * mls + cl] = a.R[(size_t)cl * ld + r];
    }
    __syncthreads();
  }
  if (t >= 32) return;
  double* sy = sT + mls * mls;
  for (int k = mls - 1; k >= 0; --k) {
    double s = 0.0;
    if (staged) {
      for (int i = k + 1 + lane; i < mls; i += 32) s += sT[k * mls + i] * sy[i];
    } else {
      for (int i = k + 1 + lane; i < mls; i += 32) s += a.R[(size_t)i * ld + k] * y[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const double yk = (a.g[k] - s) / (staged ? sT[k * mls + k] : a.R[(size_t)k * ld + k]);
      y[k] = yk;
      if (staged) sy[k] = yk;
    }
    __syncwarp();
  }
  if (lane == 0) c->m_ls = mls;
}

int launch_backsub(const GivensArgs& a, double* y, cudaStream_t stream) {
  size_t smem = 0;
  if (a.m <= kBacksubStaged) {
    smem = (size_t)(a.m * a.m + a.m) * sizeof(double);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_backsub, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
      if (e != cudaSuccess) return cuda_fail(e, "back substitution smem attribute");
    }
  }
  k_backsub<<<1, 256, smem, stream>>>(a, y);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "back substitution launch");
}

int launch_givens(const GivensArgs& a, int j, cudaStream_t stream) {
  k_givens<<<1, 32, 0, stream>>>(a, j);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "givens launch");
}

int launch_cycle_init(SolverCtl* ctl, double* g, int m, int steps_allowed, cudaStream_t stream) {
  k_cycle_init<<<1, 128, 0, stream>>>(ctl, g, m, steps_allowed);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBG_OK : cuda_fail(e, "cycle init launch");
}

}  // namespace cbg

// ---- the context --------------------------------------------------------------------------------

using namespace cbg;

namespace {

enum Phase { kValidating = -1, kIdle = 0, kWaitResidual = 1, kInCycle = 2, kDone = 3 };

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct cbg_ctx {
  int32_t n;
  int64_t nnz;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* vals;
  cbg_opts opts;
  cudaStream_t stream;
  // device workspace (one block) and pinned control-block mirror; owned unless provided by a server
  void* dmem;
  size_t dbytes;
  bool owns_dmem;
  bool owns_pinned;
  BasisMut basis;
  double *v, *w, *H, *R, *cs, *sn, *g, *u, *y, *partials, *hist, *bnorm2;
  double *dinv, *z;  // Jacobi preconditioner: 1 / diag(A) and the restart's V y (null without)
  OnchipPlan oc;  // oc.cluster > 0: every cycle is one cluster launch (onchip.cu)
  SolverCtl* ctl;
  SolverCtl* ctl_host;  // pinned mirror
  double* bnorm2_host;  // pinned
  cudaEvent_t ev;
  // solve state
  const double* b;
  double* x;
  int phase;
  int j;
  int steps_allowed;
  int64_t iters, restarts, reorths, breakdowns;
  double bnorm, true_rrn, implicit;
  int status, converged, first_residual;
  std::chrono::steady_clock::time_point t0;
  double seconds;
};

namespace {

struct Layout {
  int64_t vstride, estride;
  size_t off_basis_vals, off_basis_exps, off_v, off_w, off_H, off_R, off_cs, off_sn, off_g, off_u, off_y,
      off_partials, off_hist, off_ctl, off_bnorm2, off_dinv, off_z, total;
};

// CBG_OK, CBG_ERR_UNIMPLEMENTED (an FRSZ2 code width in [2, 32] other than 16, 21 and 32) or
// CBG_ERR_INVALID_ARG; does not set the error message.
int opts_status(int32_t n, const cbg_opts* o) {
  if (!o) return CBG_ERR_INVALID_ARG;
  if (n < 1) return CBG_ERR_INVALID_ARG;
  if (o->restart < 1 || o->restart > 1024 || o->restart > n) return CBG_ERR_INVALID_ARG;
  if (!(o->tol > 0.0) || !std::isfinite(o->tol)) return CBG_ERR_INVALID_ARG;
  if (o->max_iters < 0) return CBG_ERR_INVALID_ARG;
  if (!(o->eta >= 0.0) || !std::isfinite(o->eta)) return CBG_ERR_INVALID_ARG;
  if (o->fmt < CBG_FP64 || o->fmt > CBG_FRSZ2) return CBG_ERR_INVALID_ARG;
  if (o->precond != CBG_PRECOND_NONE && o->precond != CBG_PRECOND_JACOBI) return CBG_ERR_INVALID_ARG;
  if (o->cycle != CBG_CYCLE_AUTO && o->cycle != CBG_CYCLE_STREAMED) return CBG_ERR_INVALID_ARG;
  if (o->fmt == CBG_FRSZ2 && o->frsz2_bits != 16 && o->frsz2_bits != 21 && o->frsz2_bits != 32)
    return (o->frsz2_bits >= 2 && o->frsz2_bits <= 32) ? CBG_ERR_UNIMPLEMENTED : CBG_ERR_INVALID_ARG;
  return CBG_OK;
}

bool opts_valid(int32_t n, const cbg_opts* o) { return opts_status(n, o) == CBG_OK; }

int opts_fail(int32_t n, const cbg_opts* o) {
  const int st = opts_status(n, o);
  if (st == CBG_ERR_UNIMPLEMENTED)
    set_error("cbgmres_create: FRSZ2 code width %d is not implemented (16, 21 or 32)", o->frsz2_bits);
  else
    set_error("cbgmres_create: invalid n or options (1 <= restart <= min(n, 1024), tol > 0, l in {16,21,32})");
  return st;
}

Layout layout_of(int32_t n, const cbg_opts* o) {
  Layout L;
  cbg_basis_layout(n, o->fmt, o->fmt == CBG_FRSZ2 ? o->frsz2_bits : 32, &L.vstride, &L.estride);
  const int64_t m1 = o->restart + 1;
  size_t off = 0;
  auto take = [&](int64_t bytes) {
    size_t at = off;
    off += (size_t)round_up(bytes, 256);
    return at;
  };
  L.off_basis_vals = take(L.vstride * m1);
  L.off_basis_exps = take(L.estride * m1);
  L.off_v = take(8ll * n);
  L.off_w = take(8ll * n);
  L.off_H = take(8 * m1 * o->restart);
  L.off_R = take(8 * m1 * o->restart);
  L.off_cs = take(8 * m1);
  L.off_sn = take(8 * m1);
  L.off_g = take(8 * m1);
  L.off_u = take(8 * m1);
  L.off_y = take(8 * m1);
  L.off_partials = take(8ll * kMaxGrid * m1);
  L.off_hist = take(o->history ? 8 * (o->max_iters + 1) : 0);
  L.off_ctl = take(sizeof(SolverCtl));
  L.off_bnorm2 = take(8);
  const bool jac = o->precond == CBG_PRECOND_JACOBI;
  L.off_dinv = take(jac ? 8ll * n : 0);
  L.off_z = take(jac ? 8ll * n : 0);
  L.total = off;
  return L;
}

int ctx_fail(cbg_ctx* c, int status) {
  c->status = status;
  c->phase = kDone;
  return status;
}

BasisView view_of(const cbg_ctx* c) {
  BasisView B;
  B.vals = c->basis.vals;
  B.vstride = c->basis.vstride;
  B.exps = c->basis.exps;
  B.estride = c->basis.estride;
  B.n = c->basis.n;
  B.fmt = c->basis.fmt;
  B.l = c->basis.l;
  return B;
}

GivensArgs givens_args(cbg_ctx* c) {
  GivensArgs a;
  a.ctl = c->ctl;
  a.H = c->H;
  a.R = c->R;
  a.cs = c->cs;
  a.sn = c->sn;
  a.g = c->g;
  a.u = c->u;
  a.hist = c->hist;
  a.hist_off = c->iters;
  a.hist_cap = c->opts.history ? c->opts.max_iters : 0;
  a.m = c->opts.restart;
  return a;
}

// A pinned copy of the control block and an event the host polls.
int enqueue_readback(cbg_ctx* c) {
  cudaError_t e = cudaMemcpyAsync(c->ctl_host, c->ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "control block copy");
  e = cudaEventRecord(c->ev, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "event record");
  return CBG_OK;
}

// Residual r := b - A x into w with beta = ||r|| (step 1), then the control-block readback.
int enqueue_residual(cbg_ctx* c) {
  NormEpilogue epi{nullptr, c->ctl, kEpiResidual};
  int st = launch_spmv(c->n, c->nnz, c->row_ptr, c->col, c->vals, c->x, c->w, c->b, c->partials,
                       &c->ctl->counters[kCtrSpmv], &c->ctl->err, epi, Gate{nullptr, nullptr}, c->stream);
  if (st) return st;
  return enqueue_readback(c);
}

// A whole cycle as one cluster launch, ending with the next residual, then the readback.
int enqueue_onchip_cycle(cbg_ctx* c) {
  OnchipArgs a;
  a.n = c->n;
  a.row_ptr = c->row_ptr;
  a.col = c->col;
  a.vals = c->vals;
  a.b = c->b;
  a.x = c->x;
  a.dinv = c->dinv;
  a.r = c->w;
  a.basis = c->basis;
  a.ctl = c->ctl;
  a.hist = c->hist;
  a.hist_off = c->iters;
  a.hist_cap = c->opts.history ? c->opts.max_iters : 0;
  a.m = c->opts.restart;
  a.steps_allowed = c->steps_allowed;
  int st = launch_onchip_cycle(c->oc, a, c->opts.fmt, c->opts.frsz2_bits, c->stream);
  if (st) return st;
  return enqueue_readback(c);
}

// One Arnoldi step j (see the file comment).
int enqueue_step(cbg_ctx* c, int j) {
  const BasisView B = view_of(c);
  SolverCtl* ctl = c->ctl;
  const Gate run{&ctl->stop, nullptr};
  const Gate second{&ctl->stop, &ctl->reorth};
  const int ld = c->opts.restart + 1;
  double* hcol = c->H + (size_t)j * ld;
  int st;
  NormEpilogue e_omega{nullptr, ctl, kEpiOmega};
  st = launch_spmv(c->n, c->nnz, c->row_ptr, c->col, c->vals, c->v, c->w, nullptr, c->partials,
                   &ctl->counters[kCtrSpmv],
                   &ctl->err, e_omega, run, c->stream);
  if (st) return st;
  st = launch_basis_dot(B, j + 1, c->w, hcol, c->partials, &ctl->counters[kCtrDot], &ctl->err, run, c->stream);
  if (st) return st;
  NormEpilogue e_p1{nullptr, ctl, kEpiPass1};
  st = launch_basis_update(B, j + 1, nullptr, hcol, 0, c->w, c->partials, &ctl->counters[kCtrUpdate], &ctl->err,
                           e_p1, run, c->stream);
  if (st) return st;
  st = launch_basis_dot(B, j + 1, c->w, c->u, c->partials, &ctl->counters[kCtrDot], &ctl->err, second, c->stream);
  if (st) return st;
  NormEpilogue e_p2{nullptr, ctl, kEpiPass2};
  st = launch_basis_update(B, j + 1, nullptr, c->u, 0, c->w, c->partials, &ctl->counters[kCtrUpdate], &ctl->err,
                           e_p2, second, c->stream);
  if (st) return st;
  st = launch_givens(givens_args(c), j, c->stream);
  if (st) return st;
  if (j + 1 <= c->opts.restart) {
    st = launch_store(c->basis, j + 1, c->w, &ctl->hdiv, &ctl->rcp, c->v, c->dinv, run, c->stream);
    if (st) return st;
  }
  return CBG_OK;
}

// Step 17 and the next step 1: y := R^{-1} g, x := x + V y, r := b - A x.
int enqueue_restart(cbg_ctx* c) {
  const BasisView B = view_of(c);
  SolverCtl* ctl = c->ctl;
  GivensArgs a = givens_args(c);
  int st = launch_backsub(a, c->y, c->stream);
  if (st) return st;
  NormEpilogue none{nullptr, nullptr, kEpiNone};
  if (c->dinv) {
    // x := x + M^{-1} (V y): z := V y (the update of a zero vector by -y), then x += dinv .* z
    cudaError_t ez = cudaMemsetAsync(c->z, 0, sizeof(double) * c->n, c->stream);
    if (ez != cudaSuccess) return cuda_fail(ez, "restart scratch clear");
    st = launch_basis_update(B, c->opts.restart, &ctl->m_ls, c->y, 1, c->z, c->partials, &ctl->counters[kCtrUpdate],
                             &ctl->err, none, Gate{nullptr, nullptr}, c->stream);
    if (st) return st;
    st = launch_add_scaled(c->n, c->dinv, c->z, c->x, c->stream);
    if (st) return st;
    return enqueue_residual(c);
  }
  st = launch_basis_update(B, c->opts.restart, &ctl->m_ls, c->y, 1, c->x, c->partials, &ctl->counters[kCtrUpdate],
                           &ctl->err, none, Gate{nullptr, nullptr}, c->stream);
  if (st) return st;
  return enqueue_residual(c);
}

int status_from_err(int err) {
  if (err & kDevErrTimeout) {
    set_error("a bounded device-side wait expired (bulk copy did not complete)");
    return CBG_ERR_TIMEOUT;
  }
  if (err & kDevErrNonFinite) {
    set_error("a norm or residual became NaN or infinite");
    return CBG_ERR_NONFINITE;
  }
  if (err & kDevErrBadMatrix) {
    set_error("invalid CSR matrix");
    return CBG_ERR_BAD_MATRIX;
  }
  if (err & kDevErrBadDiagonal) {
    set_error("the Jacobi preconditioner needs a finite nonzero diagonal entry in every row");
    return CBG_ERR_BAD_MATRIX;
  }
  return CBG_OK;
}

// The residual of a cycle start is on the host: account the finished cycle and decide what next.
int after_residual(cbg_ctx* c) {
  const SolverCtl& h = *c->ctl_host;
  bool broke_down = false;  // the cycle that just ended did so on the breakdown test (step 12)
  if (c->first_residual) {
    c->first_residual = 0;
  } else {
    c->iters += h.m_eff;
    c->reorths += h.reorth_count;
    c->restarts += 1;
    c->implicit = h.implicit;
    broke_down = h.breakdown != 0;
    if (broke_down) c->breakdowns += 1;
  }
  int st = status_from_err(h.err);
  if (st) return ctx_fail(c, st);
  const double cycle_start_rrn = c->true_rrn;
  c->true_rrn = c->bnorm > 0.0 ? h.beta / c->bnorm : 0.0;
  if (!std::isfinite(c->true_rrn)) {
    set_error("the residual became NaN or infinite");
    return ctx_fail(c, CBG_ERR_NONFINITE);
  }
  if (c->true_rrn <= c->opts.tol) {
    c->converged = 1;
    c->status = CBG_OK;
    c->phase = kDone;
    return CBG_OK;
  }
  // A breakdown that left the residual where the cycle started: the Krylov space stopped growing,
  // and repeating the cycle would give the same result (the oracle's reading R18).
  if (broke_down && c->true_rrn >= cycle_start_rrn) {
    set_error("breakdown (Fig. 1 step 12) without progress: relative residual %.3e at restart %lld",
              c->true_rrn, static_cast<long long>(c->restarts));
    c->status = CBG_ERR_BREAKDOWN_NOT_CONVERGED;
    c->phase = kDone;
    return CBG_OK;
  }
  if (c->iters >= c->opts.max_iters) {
    c->status = CBG_ERR_NOT_CONVERGED;
    c->phase = kDone;
    return CBG_OK;
  }
  const int64_t left = c->opts.max_iters - c->iters;
  c->steps_allowed = static_cast<int>(left < c->opts.restart ? left : c->opts.restart);
  if (c->oc.cluster > 0) {
    st = enqueue_onchip_cycle(c);
    if (st) return ctx_fail(c, st);
    c->phase = kWaitResidual;
    return CBG_OK;
  }
  st = launch_cycle_init(c->ctl, c->g, c->opts.restart, c->steps_allowed, c->stream);
  if (st) return ctx_fail(c, st);
  // v_1 := r0 / beta, stored as basis vector 0 (step 1)
  st = launch_store(c->basis, 0, c->w, &c->ctl->hdiv, &c->ctl->rcp, c->v, c->dinv, Gate{nullptr, nullptr}, c->stream);
  if (st) return ctx_fail(c, st);
  c->j = 0;
  c->phase = kInCycle;
  return CBG_OK;
}

}  // namespace

namespace cbg {

size_t ctx_pinned_bytes() { return (sizeof(SolverCtl) + 64 + 255) / 256 * 256; }

size_t ctx_device_bytes(int32_t n, const cbg_opts* opts) { return opts_valid(n, opts) ? layout_of(n, opts).total : 0; }

// A context over caller-provided memory: dbytes >= ctx_device_bytes(n, opts) of device memory
// (256-byte aligned) and ctx_pinned_bytes() of pinned host memory. Nothing is allocated but the
// host object and an event, and nothing waits: the workspace is cleared and the CSR validated on
// `stream`, and ctx_validated() reports the outcome once that work has run.
int ctx_create_in(cbg_ctx** out, int32_t n, int64_t nnz, const int32_t* d_row_ptr, const int32_t* d_col,
                  const double* d_vals, const cbg_opts* opts, cudaStream_t stream, void* dmem, size_t dbytes,
                  void* pinned) {
  *out = nullptr;
  if (!opts_valid(n, opts)) return opts_fail(n, opts);
  if (nnz < 0 || nnz > INT32_MAX || !d_row_ptr || (nnz > 0 && (!d_col || !d_vals))) {
    set_error("cbgmres_create: invalid CSR arguments");
    return CBG_ERR_INVALID_ARG;
  }
  const Layout L = layout_of(n, opts);
  if (!dmem || dbytes < L.total || reinterpret_cast<uintptr_t>(dmem) % 256 || !pinned) {
    set_error("cbgmres_create: workspace too small or misaligned");
    return CBG_ERR_INVALID_ARG;
  }
  DeviceInfo di;
  int st = device_info(&di);
  if (st) return st;
  cbg_ctx* c = new (std::nothrow) cbg_ctx();
  if (!c) {
    set_error("cbgmres_create: host allocation failed");
    return CBG_ERR_OOM;
  }
  c->n = n;
  c->nnz = nnz;
  c->row_ptr = d_row_ptr;
  c->col = d_col;
  c->vals = d_vals;
  c->opts = *opts;
  if (c->opts.fmt != CBG_FRSZ2) c->opts.frsz2_bits = 32;
  c->stream = stream;
  c->dmem = dmem;
  c->dbytes = L.total;
  c->owns_dmem = false;
  c->owns_pinned = false;
  uint8_t* base = static_cast<uint8_t*>(c->dmem);
  c->basis.vals = base + L.off_basis_vals;
  c->basis.vstride = L.vstride;
  c->basis.exps = reinterpret_cast<uint32_t*>(base + L.off_basis_exps);
  c->basis.estride = L.estride;
  c->basis.n = n;
  c->basis.fmt = c->opts.fmt;
  c->basis.l = c->opts.frsz2_bits;
  c->v = reinterpret_cast<double*>(base + L.off_v);
  c->w = reinterpret_cast<double*>(base + L.off_w);
  c->H = reinterpret_cast<double*>(base + L.off_H);
  c->R = reinterpret_cast<double*>(base + L.off_R);
  c->cs = reinterpret_cast<double*>(base + L.off_cs);
  c->sn = reinterpret_cast<double*>(base + L.off_sn);
  c->g = reinterpret_cast<double*>(base + L.off_g);
  c->u = reinterpret_cast<double*>(base + L.off_u);
  c->y = reinterpret_cast<double*>(base + L.off_y);
  c->partials = reinterpret_cast<double*>(base + L.off_partials);
  c->hist = c->opts.history ? reinterpret_cast<double*>(base + L.off_hist) : nullptr;
  c->ctl = reinterpret_cast<SolverCtl*>(base + L.off_ctl);
  c->bnorm2 = reinterpret_cast<double*>(base + L.off_bnorm2);
  const bool jac = c->opts.precond == CBG_PRECOND_JACOBI;
  c->dinv = jac ? reinterpret_cast<double*>(base + L.off_dinv) : nullptr;
  c->z = jac ? reinterpret_cast<double*>(base + L.off_z) : nullptr;
  st = onchip_plan(n, nnz, &c->opts, &c->oc);
  if (st) {
    delete c;
    return st;
  }
  c->ctl_host = static_cast<SolverCtl*>(pinned);
  c->bnorm2_host = reinterpret_cast<double*>(static_cast<uint8_t*>(pinned) + sizeof(SolverCtl) + 16);
  cudaError_t e = cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->dmem, 0, L.total, c->stream);
  if (e != cudaSuccess) {
    st = cuda_fail(e, "cbgmres_create setup");
    ctx_release(c);
    return st;
  }
  st = launch_validate_csr(n, nnz, d_row_ptr, d_col, &c->ctl->err, c->stream);
  if (st) {
    ctx_release(c);
    return st;
  }
  e = cudaMemcpyAsync(c->ctl_host, c->ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev, c->stream);
  if (e != cudaSuccess) {
    st = cuda_fail(e, "cbgmres_create validation");
    ctx_release(c);
    return st;
  }
  c->phase = kValidating;
  *out = c;
  return CBG_OK;
}

// 1: validated (the context is idle), 0: the validation has not run yet, < 0: CBG_ERR_* (a bad
// matrix or a CUDA error). Never waits.
int ctx_validated(cbg_ctx* c) {
  if (c->phase != kValidating) return 1;
  cudaError_t q = cudaEventQuery(c->ev);
  if (q == cudaErrorNotReady) return 0;
  if (q != cudaSuccess) return cuda_fail(q, "CSR validation");
  if (c->ctl_host->err & kDevErrBadMatrix) {
    set_error("cbgmres_create: CSR row pointers not monotone, row_ptr[0] != 0, row_ptr[n] != nnz, or a column "
              "index outside [0, n)");
    return CBG_ERR_BAD_MATRIX;
  }
  c->phase = kIdle;
  return 1;
}

// Waits for the context's stream, then frees what the context owns (not caller-provided memory).
void ctx_release(cbg_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->owns_dmem && c->dmem) cudaFree(c->dmem);
  if (c->owns_pinned && c->ctl_host) cudaFreeHost(c->ctl_host);
  if (c->ev) cudaEventDestroy(c->ev);
  delete c;
}

// The stream the context enqueues on.
cudaStream_t ctx_stream(const cbg_ctx* c) { return c->stream; }

}  // namespace cbg

extern "C" {

int cbg_opts_default(cbg_opts* o) {
  if (!o) {
    set_error("cbg_opts_default: null opts");
    return CBG_ERR_INVALID_ARG;
  }
  o->restart = 100;
  o->fmt = CBG_FRSZ2;
  o->frsz2_bits = 32;
  o->history = 0;
  o->tol = 1e-10;
  o->max_iters = 20000;
  o->eta = 0.70710678118654752440;
  o->precond = CBG_PRECOND_NONE;
  o->cycle = CBG_CYCLE_AUTO;
  return CBG_OK;
}

size_t cbgmres_workspace_bytes(int32_t n, const cbg_opts* o) {
  if (!opts_valid(n, o)) return 0;
  return layout_of(n, o).total + 3 * sizeof(SolverCtl);
}

int cbgmres_create(cbg_ctx** out, int32_t n, int64_t nnz, const int32_t* d_row_ptr, const int32_t* d_col,
                   const double* d_vals, const cbg_opts* opts, void* stream) {
  if (!out) {
    set_error("cbgmres_create: null output pointer");
    return CBG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (!opts_valid(n, opts)) return opts_fail(n, opts);
  const size_t total = layout_of(n, opts).total;
  void* dmem = nullptr;
  cudaError_t e = cudaMalloc(&dmem, total);
  if (e != cudaSuccess) {
    set_error("cbgmres_create: cudaMalloc of %zu bytes failed: %s", total, cudaGetErrorString(e));
    cudaGetLastError();
    return CBG_ERR_OOM;
  }
  void* pinned = nullptr;
  e = cudaMallocHost(&pinned, ctx_pinned_bytes());
  if (e != cudaSuccess) {
    cudaFree(dmem);
    return cuda_fail(e, "cbgmres_create: pinned control block");
  }
  cbg_ctx* c = nullptr;
  int st = ctx_create_in(&c, n, nnz, d_row_ptr, d_col, d_vals, opts, static_cast<cudaStream_t>(stream), dmem, total,
                         pinned);
  if (st) {
    cudaFree(dmem);
    cudaFreeHost(pinned);
    return st;
  }
  c->owns_dmem = true;
  c->owns_pinned = true;
  // wait for the CSR validation enqueued by ctx_create_in
  e = cudaEventSynchronize(c->ev);
  if (e != cudaSuccess) {
    st = cuda_fail(e, "cbgmres_create validation");
    cbgmres_destroy(c);
    return st;
  }
  st = ctx_validated(c);
  if (st != 1) {
    cbgmres_destroy(c);
    return st < 0 ? st : CBG_ERR_CUDA;
  }
  *out = c;
  return CBG_OK;
}

int cbgmres_start(cbg_ctx* c, const double* d_b, double* d_x) {
  if (!c || !d_b || !d_x) {
    set_error("cbgmres_start: null argument");
    return CBG_ERR_INVALID_ARG;
  }
  if (c->phase == kValidating) {
    // a context made over server memory: its matrix must be known valid before any SpMV runs
    cudaError_t e = cudaEventSynchronize(c->ev);
    if (e != cudaSuccess) return cuda_fail(e, "CSR validation wait");
    int v = ctx_validated(c);
    if (v != 1) return v < 0 ? v : CBG_ERR_CUDA;
  }
  if (c->phase != kIdle && c->phase != kDone) {
    set_error("cbgmres_start: a solve is in progress on this context");
    return CBG_ERR_STATE;
  }
  c->b = d_b;
  c->x = d_x;
  c->iters = c->restarts = c->reorths = c->breakdowns = 0;
  c->bnorm = c->true_rrn = c->implicit = 0.0;
  c->status = CBG_OK;
  c->converged = 0;
  c->first_residual = 1;
  c->seconds = 0.0;
  c->t0 = std::chrono::steady_clock::now();
  // ||b|| (Eq. 4), then the initial residual
  int st = launch_sumsq(d_b, c->n, c->partials, &c->ctl->counters[kCtrStandalone], &c->ctl->err, c->bnorm2, c->stream);
  if (st) return ctx_fail(c, st);
  k_set_bnorm<<<1, 1, 0, c->stream>>>(c->ctl, c->bnorm2, c->opts.tol, c->opts.eta);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_fail(c, cuda_fail(e, "set bnorm launch"));
  if (c->dinv) {  // M^{-1} = 1 / diag(A), after k_set_bnorm has cleared the error word
    st = launch_jacobi_diag(c->n, c->row_ptr, c->col, c->vals, c->dinv, &c->ctl->err, c->stream);
    if (st) return ctx_fail(c, st);
  }
  e = cudaMemcpyAsync(c->bnorm2_host, c->bnorm2, 8, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return ctx_fail(c, cuda_fail(e, "bnorm copy"));
  st = enqueue_residual(c);
  if (st) return ctx_fail(c, st);
  c->phase = kWaitResidual;
  return CBG_OK;
}

int cbgmres_advance(cbg_ctx* c, int32_t max_steps, int32_t* done) {
  if (!c || !done) {
    set_error("cbgmres_advance: null argument");
    return CBG_ERR_INVALID_ARG;
  }
  *done = 0;
  if (c->phase == kIdle || c->phase == kValidating) {
    set_error("cbgmres_advance: no solve started");
    return CBG_ERR_STATE;
  }
  int budget = max_steps < 1 ? 1 : max_steps;
  while (c->phase != kDone) {
    if (c->phase == kWaitResidual) {
      cudaError_t q = cudaEventQuery(c->ev);
      if (q == cudaErrorNotReady) return CBG_OK;  // keep the host free: poll again later
      if (q != cudaSuccess) {
        int st = cuda_fail(q, "solver event");
        ctx_fail(c, st);
        break;
      }
      if (c->first_residual) {
        c->bnorm = std::sqrt(*c->bnorm2_host);
        if (!std::isfinite(c->bnorm)) {
          set_error("||b|| is NaN or infinite");
          ctx_fail(c, CBG_ERR_NONFINITE);
          break;
        }
        if (c->bnorm == 0.0) {  // b = 0: x = 0 is the solution
          cudaMemsetAsync(c->x, 0, sizeof(double) * c->n, c->stream);
          cudaStreamSynchronize(c->stream);
          c->first_residual = 0;
          c->converged = 1;
          c->true_rrn = 0.0;
          c->phase = kDone;
          break;
        }
      }
      after_residual(c);
      continue;
    }
    if (c->phase == kInCycle) {
      if (budget <= 0) return CBG_OK;
      while (c->j < c->steps_allowed && budget > 0) {
        int st = enqueue_step(c, c->j);
        if (st) return ctx_fail(c, st);
        ++c->j;
        --budget;
      }
      if (c->j >= c->steps_allowed) {
        int st = enqueue_restart(c);
        if (st) return ctx_fail(c, st);
        c->phase = kWaitResidual;
      }
    }
  }
  c->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - c->t0).count();
  *done = 1;
  return c->status;
}

int cbgmres_finish(cbg_ctx* c, cbg_result* r) {
  if (!c) {
    set_error("cbgmres_finish: null context");
    return CBG_ERR_INVALID_ARG;
  }
  if (c->phase != kDone) {
    set_error("cbgmres_finish: the solve has not finished");
    return CBG_ERR_STATE;
  }
  if (r) {
    r->iters = c->iters;
    r->restarts = c->restarts;
    r->reorths = c->reorths;
    r->converged = c->converged;
    r->status = c->status;
    r->true_rrn = c->true_rrn;
    r->implicit_rrn = c->implicit;
    r->seconds = c->seconds;
    r->breakdowns = c->breakdowns;
  }
  return c->status;
}

int cbgmres_solve(cbg_ctx* c, const double* d_b, double* d_x, cbg_result* r) {
  int st = cbgmres_start(c, d_b, d_x);
  if (st) return st;
  int32_t done = 0;
  while (!done) {
    st = cbgmres_advance(c, 1 << 30, &done);
    if (st && st != CBG_ERR_NOT_CONVERGED && st != CBG_ERR_BREAKDOWN_NOT_CONVERGED) break;
    if (!done) {
      cudaError_t e = cudaEventSynchronize(c->ev);
      if (e != cudaSuccess) return ctx_fail(c, cuda_fail(e, "solver event wait"));
    }
  }
  return cbgmres_finish(c, r);
}

int cbgmres_history(cbg_ctx* c, double* h_out, int64_t cap, int64_t* count) {
  if (!c || !count || (cap > 0 && !h_out)) {
    set_error("cbgmres_history: null argument");
    return CBG_ERR_INVALID_ARG;
  }
  *count = 0;
  if (!c->hist) return CBG_OK;
  int64_t k = c->iters < cap ? c->iters : cap;
  if (k > c->opts.max_iters) k = c->opts.max_iters;
  if (k > 0) {
    cudaError_t e = cudaMemcpyAsync(h_out, c->hist, sizeof(double) * k, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "history copy");
  }
  *count = k;
  return CBG_OK;
}

int cbgmres_basis_vector(cbg_ctx* c, int32_t slot, double* d_out) {
  if (!c || !d_out) {
    set_error("cbgmres_basis_vector: null argument");
    return CBG_ERR_INVALID_ARG;
  }
  if (slot < 0 || slot > c->opts.restart) {
    set_error("cbgmres_basis_vector: slot %d outside [0, %d]", slot, c->opts.restart);
    return CBG_ERR_INVALID_ARG;
  }
  if (c->phase == kValidating) {
    set_error("cbgmres_basis_vector: the context has not been validated yet");
    return CBG_ERR_STATE;
  }
  return launch_load(view_of(c), slot, d_out, c->stream);
}

int32_t cbgmres_cycle_cluster(const cbg_ctx* c) { return c ? c->oc.cluster : -1; }

int cbgmres_destroy(cbg_ctx* c) {
  ctx_release(c);
  return CBG_OK;
}

}  // extern "C"
