/* cbgmres.h - C ABI of the GB300 (sm_103a) Compressed-Basis GMRES library with the FRSZ2 block
 * compressor of arXiv 2409.15468 ("FRSZ2 for In-Register Block Compression Inside GMRES on GPUs").
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are CUDA device pointers on the current device; h_* are host pointers.
 *     The library never frees or retains caller memory beyond the call, except the CSR arrays
 *     handed to cbgmres_create, which the context borrows until cbgmres_destroy.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is enqueued on it; calls
 *     return without synchronising unless stated otherwise.
 *   - Every call returns CBG_OK (0) or a negative CBG_ERR_* status and never throws. The message
 *     of the last failure on the calling thread is available from cbg_last_error().
 *   - There is no CPU fallback: without a usable CUDA device every compute call fails with
 *     CBG_ERR_CUDA.
 *
 * Storage formats of the Krylov basis (Compression Configuration: float64, float32 and float16
 * storage with FP64 arithmetic; bfloat16 is one more cast; FRSZ2 per the Design section). All
 * arithmetic is FP64 or exact integer arithmetic on the stored codes; the format only changes
 * how the basis sits in memory.
 */
#ifndef CBGMRES_H
#define CBGMRES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------------------------- */
#define CBG_OK 0
#define CBG_ERR_INVALID_ARG (-1)  /* an argument failed validation; nothing was enqueued */
#define CBG_ERR_CUDA (-2)         /* a CUDA runtime call failed (no device, launch failure, ...) */
#define CBG_ERR_OOM (-3)          /* device allocation failed */
#define CBG_ERR_NONFINITE (-4)    /* a norm or residual became NaN or infinite during a solve */
#define CBG_ERR_NOT_CONVERGED (-5) /* max_iters reached; x and the result are still written */
#define CBG_ERR_TIMEOUT (-6)      /* a bounded device-side wait expired; the context is unusable */
#define CBG_ERR_BAD_MATRIX (-7)   /* CSR row pointers not monotone or a column index out of range;
                                     with the Jacobi preconditioner also a zero or missing
                                     diagonal entry */
#define CBG_ERR_STATE (-8)        /* stepwise call out of order (advance before start, ...) */
#define CBG_ERR_BREAKDOWN_NOT_CONVERGED (-9) /* a restart cycle ended on Fig. 1 step 12 (breakdown) and
                                     the explicit residual at the next restart was no smaller than at
                                     the start of that cycle: the Krylov space stopped growing without
                                     reaching tol (e.g. an inconsistent singular system). x and the
                                     result are still written. */
#define CBG_ERR_UNIMPLEMENTED (-10) /* a well-formed request this library does not implement: an
                                     FRSZ2 code width l in [2, 32] other than 16, 21 and 32 */

/* ---- basis storage formats ------------------------------------------------------------------ */
typedef enum cbg_format {
  CBG_FP64 = 0,  /* IEEE binary64 */
  CBG_FP32 = 1,  /* IEEE binary32, round-to-nearest-even from FP64 */
  CBG_FP16 = 2,  /* IEEE binary16, round-to-nearest-even from FP64 */
  CBG_BF16 = 3,  /* bfloat16, round-to-nearest-even from FP64 */
  CBG_FRSZ2 = 4  /* FRSZ2 with block size 32 and l-bit codes, l in {16, 21, 32} */
} cbg_format;

/* ---- FRSZ2 codec (Design section: Eq. 2, Eq. 3, Compression steps 1-6, Decompression 1-4) -----
 * Layout of n values: ceil(n/32) exponent words (uint32, the raw biased IEEE exponent field of
 * the block maximum) and, separately, ceil(n/32)*l code words (uint32). Code i of a block occupies
 * bits [i*l, (i+1)*l) of the block's little-endian bit stream; bit l-1 is the sign, bit l-2 the
 * integer bit, then l-2 fraction bits (Eq. 2); values are truncated toward zero to the block's
 * quantum 2^(max(e_max,1) - 1023 - (l-2)). The last block is padded with +0.0. */

/* Bytes of Eq. 3 for n values at code width l (code-size term read as ceil(32*l/32) words per
 * block, consistent with the paper's 33 bits per value for l = 32). Returns -1 for a bad l or n. */
int64_t cbg_frsz2_bytes(int64_t n, int32_t l);

/* Compresses d_src[0..n) into d_exps[ceil(n/32)] and d_codes[ceil(n/32)*l] (Compression,
 * steps 1-6: one warp per 32-value block, warp-wide maximum of the exponent fields).
 * Inputs must be finite (Krylov values lie in [-1, 1]); the output for NaN or Inf is unspecified.
 * d_src must be 8-byte aligned, d_exps and d_codes 4-byte aligned. Errors: CBG_ERR_UNIMPLEMENTED
 * for a code width in [2, 32] other than 16, 21 and 32 (the format admits them; this library
 * implements those three), CBG_ERR_INVALID_ARG for any other l or a negative n. */
int cbg_frsz2_compress(const double* d_src, int64_t n, int32_t l, uint32_t* d_exps, uint32_t* d_codes,
                       void* stream);

/* Decompresses into d_dst[0..n) (Decompression, steps 1-4; random access by block). Errors as for
 * cbg_frsz2_compress. */
int cbg_frsz2_decompress(const uint32_t* d_exps, const uint32_t* d_codes, int64_t n, int32_t l, double* d_dst,
                         void* stream);

/* The codec under the plain names of the problem statement: the same functions as cbg_frsz2_bytes
 * (returned as size_t, 0 for a bad n or l), cbg_frsz2_compress and cbg_frsz2_decompress. */
size_t frsz2_bytes(int64_t n, int32_t l);
int frsz2_compress(const double* d_src, int64_t n, int32_t l, uint32_t* d_exp, uint32_t* d_codes, void* stream);
int frsz2_decompress(const uint32_t* d_exp, const uint32_t* d_codes, int64_t n, int32_t l, double* d_dst,
                     void* stream);

/* ---- basis layout --------------------------------------------------------------------------- *
 * A basis is nvec vectors of n values stored in one format. Vector i keeps its values (cast bits
 * or FRSZ2 codes) at vals + i*vals_stride bytes and, for FRSZ2, its exponent words at
 * exps + i*exps_stride bytes. The fused basis kernels stream the basis with 16-byte bulk copies,
 * so: vals, exps and both strides must be multiples of 256 bytes, and each vector's arrays must
 * hold ceil(n/128)*4 blocks of 32 values (the format's block rounded up to 4 blocks), the
 * padding being readable memory (its contents are ignored). cbg_basis_layout gives the minimal
 * strides. */
typedef struct cbg_basis {
  int32_t fmt;         /* cbg_format */
  int32_t frsz2_bits;  /* l when fmt == CBG_FRSZ2, ignored otherwise */
  int64_t n;           /* values per vector */
  void* vals;          /* device pointer to vector 0's values / codes */
  int64_t vals_stride; /* bytes between consecutive vectors' values */
  uint32_t* exps;      /* device pointer to vector 0's exponent words (FRSZ2), else NULL */
  int64_t exps_stride; /* bytes between consecutive vectors' exponent arrays */
} cbg_basis;

/* Minimal strides (bytes) of one basis vector; exps_stride is 0 for cast formats. */
int cbg_basis_layout(int64_t n, int32_t fmt, int32_t l, int64_t* vals_stride, int64_t* exps_stride);

/* Stores d_src[0..n) as vector `slot` of the basis: FRSZ2 compression or a round-to-nearest-even
 * cast from FP64 (Fig. 1 steps 1 and 14, highlighted: appending a vector to the compressed basis). */
int cbg_basis_store(const cbg_basis* basis, int32_t slot, const double* d_src, void* stream);

/* Normalises and appends (Fig. 1 steps 13-14, and step 1 with h = beta): v := d_w / *d_h, each
 * element the correctly rounded IEEE quotient (as the oracle divides), stored as vector `slot`
 * exactly as cbg_basis_store would store v. d_h points to one double on the device, positive and
 * finite (a norm); for other values of h the elements are d_w * RN(1/h). If d_v is not NULL it
 * receives the FP64 v (the input of the next SpMV, step 3). d_w and d_v may be the same vector. */
int cbg_basis_append(const cbg_basis* basis, int32_t slot, const double* d_w, const double* d_h, double* d_v,
                     void* stream);

/* Decodes basis vector `slot` into d_dst[0..n) (a read through the accessor: Implementation and
 * synthetic performance subsection). */
int cbg_basis_load(const cbg_basis* basis, int32_t slot, double* d_dst, void* stream);

/* Scratch bytes that cbg_basis_dot / cbg_basis_update need for up to nvec vectors of n values. */
size_t cbg_basis_work_bytes(int64_t n, int32_t nvec);

/* d_h[i] = sum_k vhat_i[k] * d_w[k] for i in [0, nvec): the classical Gram-Schmidt projections
 * h_{1:j} := V_j^T w of Fig. 1 step 5 (highlighted), reading the stored basis and decoding it in
 * registers. FRSZ2 blocks are multiplied exactly in integer arithmetic against a 54-bit
 * block-fixed-point copy of w and accumulated in FP64 across blocks; cast formats accumulate in
 * FP64. Error bound: 2^-53 * sum_b max_{k in b}|w_k| * sum_{k in b}|vhat_k| plus FP64 summation
 * error over at most about 2^6 sequential terms. d_work: cbg_basis_work_bytes(n, nvec) bytes,
 * 256-byte aligned, no initial contents required, not used concurrently by another call. Empty
 * inputs: nvec = 0 writes nothing; n = 0 sets d_h[0..nvec) to 0 (the empty sums). */
int cbg_basis_dot(const cbg_basis* basis, int32_t nvec, const double* d_w, double* d_h, void* d_work,
                  size_t work_bytes, void* stream);

/* The same dot product as cbg_basis_dot for callers that cannot allocate device memory: a plugin
 * whose host application has reserved all device memory in its own pool, or a latency-critical
 * path that must not call cudaMalloc (which can synchronise the whole device). The paper has no
 * counterpart; this is a convenience of the library. It takes no work buffer and allocates nothing:
 * its partial sums live in a fixed 1 MiB array in device memory that the library defines, which
 * every GPU that loads the library holds until the process exits.
 *   - nvec must be at most 128; larger values return CBG_ERR_INVALID_ARG with nothing enqueued.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *     that device current; make that first call before any stream capture on the device.
 *   - Every call on a device uses the same array. Calls whose kernels overlap on the GPU (for
 *     example on two streams at once) race and produce wrong results; order them on one stream.
 *     Each call clears the array's completion counter before its kernel runs; the partial sums
 *     need no clearing (every slot a call reads is written by that call first).
 *   - Empty inputs as for cbg_basis_dot: nvec = 0 writes nothing, n = 0 sets d_h[0..nvec) to 0.
 *   - The FRSZ2 kernel bounds every wait on its bulk copies; should one expire, d_h is left
 *     incomplete and, as for cbg_basis_dot, the device-side error word is not reported (the
 *     copies complete with any valid basis, so this only happens on a faulting device).
 * Other arguments, results and the error bound are those of cbg_basis_dot. */
int cbg_basis_dot_noalloc(const cbg_basis* basis, int32_t nvec, const double* d_w, double* d_h, void* stream);

/* d_w[k] -= sum_i vhat_i[k] * d_h[i] over i in [0, nvec): the update w := w - V_j h of Fig. 1
 * step 5 (highlighted). The sum over i is exact in integer arithmetic for FRSZ2 (h scaled per
 * block to a 54-bit fixed point), FP64 otherwise. If d_norm2 is not NULL it receives ||w||^2 after
 * the update (the norm of step 6). d_work as for cbg_basis_dot. Empty inputs: with nvec = 0, w
 * is left unchanged and *d_norm2 still receives ||w||^2; with n = 0, *d_norm2 receives 0. */
int cbg_basis_update(const cbg_basis* basis, int32_t nvec, const double* d_h, double* d_w, double* d_norm2,
                     void* d_work, size_t work_bytes, void* stream);

/* The synthetic arithmetic-intensity benchmark of the synthetic-performance discussion (Fig. 3):
 * every value x_k of stored vector `slot` is read and decoded to FP64 (as cbg_basis_load does),
 * then r = fma_per_value fused multiply-adds f(y) = 0.5 y + 0.25 are applied to it, and
 * *d_out = sum_k f^r(x_k) (FP64, fixed reduction order). The multiplication by 0.5 is exact, so
 * every step rounds once. compute_fp32 != 0 (fmt CBG_FP32 only) reads the binary32 values and
 * computes and sums in FP32 per thread, the paper's native float baseline. Per value: 2 r + 1
 * floating-point operations over the format's bytes per value. d_work as for cbg_basis_dot with
 * nvec = 1. Errors: CBG_ERR_INVALID_ARG (bad basis, slot < 0, r < 0 or > 2^20, compute_fp32 on
 * another format). */
int cbg_intensity(const cbg_basis* basis, int32_t slot, int32_t fma_per_value, int32_t compute_fp32, double* d_out,
                  void* d_work, size_t work_bytes, void* stream);

/* ---- sparse matrix ---------------------------------------------------------------------------- */
/* Checks a CSR matrix on the device: row_ptr[0] == 0, row_ptr[n] == nnz, row pointers monotone,
 * every column in [0, n). Returns CBG_ERR_BAD_MATRIX otherwise. Synchronises the stream.
 * cbg_spmv assumes a valid matrix (it does not check), cbgmres_create runs this check itself. */
int cbg_csr_validate(int32_t n, int64_t nnz, const int32_t* d_row_ptr, const int32_t* d_col, void* stream);

/* d_y = A d_x for the CSR matrix (int32 row pointers and columns, FP64 values): Fig. 1 step 3,
 * w := A M^{-1} v with M = I (no preconditioner: Solver Configuration). If d_norm2 is not NULL it
 * receives ||y||^2 (step 4). nnz = row_ptr[n]; it chooses the kernel (one thread per row for
 * short rows; when the mean row length is 12 or more, segments of 512 rows sorted by length in
 * shared memory, with 1 to 32 lanes per row by length) and must match the matrix. d_work:
 * cbg_spmv_work_bytes(n) bytes, 256-byte aligned. */
size_t cbg_spmv_work_bytes(int32_t n);
int cbg_spmv(int32_t n, int64_t nnz, const int32_t* d_row_ptr, const int32_t* d_col, const double* d_vals,
             const double* d_x, double* d_y, double* d_norm2, void* d_work, size_t work_bytes, void* stream);

/* ---- solver ----------------------------------------------------------------------------------- */
typedef struct cbg_opts {
  int32_t restart;    /* m, the number of basis vectors before a restart (Methodology: m = 100) */
  int32_t fmt;        /* cbg_format of the Krylov basis */
  int32_t frsz2_bits; /* l for CBG_FRSZ2: 16, 21 or 32 (another l in [2, 32]: CBG_ERR_UNIMPLEMENTED) */
  int32_t history;    /* nonzero: record the implicit relative residual after every Arnoldi step */
  double tol;         /* target relative residual ||b - A x|| / ||b|| (Eq. 4) */
  int64_t max_iters;  /* cap on Arnoldi steps */
  double eta;         /* re-orthogonalisation threshold of Fig. 1 step 7 (default 1/sqrt(2)) */
  int32_t precond;    /* the M of Fig. 1 steps 3 and 17, applied on the right: CBG_PRECOND_NONE
                         (M = I, the paper's setting, default) or CBG_PRECOND_JACOBI (M = diag(A);
                         a zero or missing diagonal entry ends the solve with CBG_ERR_BAD_MATRIX) */
  int32_t cycle;      /* how a restart cycle runs: CBG_CYCLE_AUTO (default) runs it as one
                         thread-block cluster launch with the compressed basis in shared memory
                         when the system is small enough (see cbgmres_cycle_cluster), else as
                         the streamed kernels over the basis in device memory;
                         CBG_CYCLE_STREAMED always streams. Both compute Fig. 1 with the same
                         per-element arithmetic; only the order of FP64 sums differs. */
} cbg_opts;

enum { CBG_PRECOND_NONE = 0, CBG_PRECOND_JACOBI = 1 };
enum { CBG_CYCLE_AUTO = 0, CBG_CYCLE_STREAMED = 1 };

typedef struct cbg_result {
  int64_t iters;       /* Arnoldi steps (new basis vectors) */
  int64_t restarts;    /* completed restart cycles */
  int64_t reorths;     /* steps that took the second Gram-Schmidt pass (Fig. 1 steps 7-11) */
  int32_t converged;   /* explicit ||b - A x|| <= tol ||b|| reached */
  int32_t status;      /* CBG_OK or the CBG_ERR_* the solve ended with */
  double true_rrn;     /* last explicit ||b - A x|| / ||b|| (Eq. 4) */
  double implicit_rrn; /* last |g_{j+1}| / ||b|| of the Givens recurrence */
  double seconds;      /* wall time of the solve as seen by the host */
  int64_t breakdowns;  /* restart cycles that ended on the breakdown test of Fig. 1 step 12 */
} cbg_result;

typedef struct cbg_ctx cbg_ctx;

/* Fills defaults: restart 100, FRSZ2 with l = 32, tol 1e-10, max_iters 20000, eta 1/sqrt(2),
 * no preconditioner. */
int cbg_opts_default(cbg_opts* opts);

/* Device bytes a context of size n with these options allocates (HBM admission control). */
size_t cbgmres_workspace_bytes(int32_t n, const cbg_opts* opts);

/* Creates a solver for the n x n CSR matrix A (Solver Configuration: A and b are immutable inputs).
 * The CSR arrays are borrowed and must stay valid until cbgmres_destroy. Validates the matrix on
 * the device (monotone row pointers, columns in [0, n)) and returns CBG_ERR_BAD_MATRIX otherwise.
 * Allocates cbgmres_workspace_bytes(n, opts) of device memory. `stream` is the stream all of the
 * context's work goes to. Synchronises the stream. */
int cbgmres_create(cbg_ctx** out, int32_t n, int64_t nnz, const int32_t* d_row_ptr, const int32_t* d_col,
                   const double* d_vals, const cbg_opts* opts, void* stream);

/* Solves A x = b (Fig. 1: restarted GMRES with the basis stored in opts->fmt). d_x holds x0 on
 * entry (the paper starts from x0 = 0) and the approximation on exit. Synchronises the stream.
 * Returns CBG_OK when converged, CBG_ERR_NOT_CONVERGED when max_iters was reached,
 * CBG_ERR_BREAKDOWN_NOT_CONVERGED when a cycle that ended on a breakdown (step 12) left the
 * explicit residual no smaller than it was at that cycle's start (x and *result still valid in
 * both cases), or another CBG_ERR_*. *result may be NULL. */
int cbgmres_solve(cbg_ctx* ctx, const double* d_b, double* d_x, cbg_result* result);

/* Stepwise form of cbgmres_solve for a serving loop that interleaves several solves:
 *   cbgmres_start    computes the initial residual and the first basis vector (Fig. 1 step 1);
 *   cbgmres_advance  runs up to max_steps further Arnoldi steps, restarts included, and reports
 *                    in *done whether the solve has finished (converged, failed or out of steps);
 *                    a context whose cycles run on chip (cbgmres_cycle_cluster > 0) advances by
 *                    whole restart cycles whatever max_steps: a call launches the next cycle
 *                    once the previous one has finished;
 *   cbgmres_finish   fills the result and returns the solve's status.
 * b and x must stay valid from start to finish. advance never waits on the device: at the end of
 * each cycle it polls an event and returns CBG_OK with *done = 0 until the restart's residual
 * is on the host. */
int cbgmres_start(cbg_ctx* ctx, const double* d_b, double* d_x);
int cbgmres_advance(cbg_ctx* ctx, int32_t max_steps, int32_t* done);
int cbgmres_finish(cbg_ctx* ctx, cbg_result* result);

/* ---- Serving runtime: continuous batching of many solves on one GPU -------------------------
 *
 * A server owns one block of device memory (the HBM budget), one CUDA stream per slot and the
 * pinned control blocks of its slots. Requests are queued by cbg_server_submit without GPU work.
 * Every cbg_server_poll is one scheduling turn:
 *   1. each admitted solve is advanced by up to steps_per_turn Arnoldi steps on its own stream
 *      (cbgmres_advance; a solve whose cycles run on chip advances by one whole restart cycle;
 *      at most one earlier turn's work may still be in flight per slot, so the host never runs
 *      far ahead of the device and never blocks on a full launch queue);
 *   2. finished solves release their slot and their workspace, and are reported as completions;
 *   3. queued requests are admitted in arrival order while a slot is free and their workspace
 *      (cbgmres_workspace_bytes) fits in the free budget. A request that does not fit is
 *      passed by later ones until it has been passed max_bypass times; then admission stops
 *      until it fits, so a large request is never starved.
 * Admission clears the workspace and validates the matrix on the slot's stream; the solve starts
 * on a later turn, once that validation has run (a bad matrix completes with
 * CBG_ERR_BAD_MATRIX and no SpMV ever reads it). Solves of different slots overlap on the
 * device. A solve's arithmetic is the same as cbgmres_solve's: the result does not depend on
 * the other requests in flight.
 *
 * Nothing in a turn waits on the device, allocates or frees device memory, or synchronises
 * the device. A server is not thread-safe: call it from one thread at a time, with the device it
 * was created on current. The matrix, b and x of a request are caller-owned device memory that must stay
 * valid until its completion is returned; x holds x0 on entry and the solution on completion. */
typedef struct cbg_server cbg_server;

typedef struct {
  uint64_t tag;                 /* caller's identifier, returned in the completion */
  int32_t n;
  int64_t nnz;
  const int32_t* d_row_ptr;     /* CSR, as for cbgmres_create */
  const int32_t* d_col;
  const double* d_vals;
  const double* d_b;
  double* d_x;                  /* in: x0, out: solution */
  cbg_opts opts;
} cbg_request;

typedef struct {
  uint64_t tag;
  int32_t status;               /* CBG_OK, CBG_ERR_NOT_CONVERGED, CBG_ERR_BAD_MATRIX, ... */
  cbg_result result;            /* valid when status is CBG_OK or CBG_ERR_NOT_CONVERGED */
  double t_submit;              /* seconds on the server clock (cbg_server_clock) */
  double t_admit;               /* workspace reserved and validation enqueued */
  double t_done;                /* completion observed by the server */
} cbg_completion;

/* hbm_budget: bytes of device memory the server reserves (one cudaMalloc, at create);
 * max_active: concurrent solves (slots, streams), 1..256; steps_per_turn >= 1;
 * max_bypass >= 0. Errors: CBG_ERR_INVALID_ARG, CBG_ERR_OOM, CBG_ERR_CUDA. */
int cbg_server_create(cbg_server** out, size_t hbm_budget, int32_t max_active, int32_t steps_per_turn,
                      int32_t max_bypass);

/* Queues a request (the struct is copied). CBG_ERR_INVALID_ARG for invalid options or CSR
 * arguments, CBG_ERR_OOM when its workspace alone exceeds the budget. No GPU work. */
int cbg_server_submit(cbg_server* server, const cbg_request* request);

/* One scheduling turn. Writes up to cap completions to out[0..*n_out); completions beyond cap
 * are kept for the next call. */
int cbg_server_poll(cbg_server* server, cbg_completion* out, int32_t cap, int32_t* n_out);

/* Requests admitted and not yet completed, requests queued, completions not yet returned, and
 * bytes of the budget in use. Any output pointer may be NULL. */
int cbg_server_stats(const cbg_server* server, int32_t* active, int32_t* queued, int32_t* pending,
                     size_t* bytes_in_use);

/* Seconds since the server was created (steady clock); the time base of the completions. */
double cbg_server_clock(const cbg_server* server);

/* Waits for every slot's stream and frees the server. Requests still queued or in flight are
 * dropped (their x is unspecified). Accepts NULL. */
int cbg_server_destroy(cbg_server* server);

/* Copies up to cap recorded implicit relative residuals (opts.history != 0) to h_out. */
int cbgmres_history(cbg_ctx* ctx, double* h_out, int64_t cap, int64_t* count);

/* Decodes basis vector `slot` (0 <= slot <= restart) of the context's current Krylov basis, as
 * stored in opts.fmt, into d_out (n doubles, device) on the context's stream; the call does not
 * wait. After a finished solve, slots 0 .. m-1 hold the m vectors v_1 .. v_m of the last cycle
 * (Fig. 1, decompressed as step 5 reads them). v_{m+1} of the cycle's last step is not stored,
 * because the restart never reads it, and later slots are unspecified. For inspection (value and
 * exponent distributions of the basis), not part of the solve. */
int cbgmres_basis_vector(cbg_ctx* ctx, int32_t slot, double* d_out);

/* How the context runs a restart cycle, decided at cbgmres_create from n, nnz and the options:
 * 0 for the streamed kernels (one kernel per operation, the basis in device memory), or the number
 * of CTAs (16 or 8) of the thread-block cluster that runs each whole cycle in one launch with its
 * slice of the compressed basis in each CTA's shared memory. The cluster is chosen when
 * opts.cycle is CBG_CYCLE_AUTO, the mean row length is below 12 (thread-per-row SpMV), restart +
 * 1 <= 128 and one CTA's share of the basis fits in its shared memory (with restart 50: up to
 * about 13 000 rows for FRSZ2-32, 7 000 for fp64). Returns -1 for a null context. In the
 * stepwise API, cbgmres_advance then runs whole cycles, whatever max_steps asks. */
int32_t cbgmres_cycle_cluster(const cbg_ctx* ctx);

/* Frees the context's device memory. Accepts NULL. */
int cbgmres_destroy(cbg_ctx* ctx);

/* Message of the last failed call on this thread ("" if none). cbgmres_last_error is the same
 * function under the name of the problem statement. */
const char* cbg_last_error(void);
const char* cbgmres_last_error(void);

/* Library version string. */
const char* cbg_version(void);

#ifdef __cplusplus
}
#endif
#endif
