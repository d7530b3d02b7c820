/* Plain FP64 CPU oracle for Compressed-Basis GMRES with the FRSZ2 block compressor
 * (arXiv 2409.15468, "FRSZ2 for In-Register Block Compression Inside GMRES on GPUs").
 *
 * TEST INFRASTRUCTURE ONLY. This library is the independent reference that the CUDA path is
 * checked against. Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it. It shares no code, header, table or helper with the CUDA library,
 * and the CUDA library never calls it.
 *
 * Everything here is written for a reader to check against the paper by eye: sequential
 * loops, one operation at a time, FP64 throughout, no blocking, fusion or reordering.
 *
 * Storage formats of a Krylov basis vector of n values ("encoded vector"):
 *   ORC_FP64   n x uint64 (IEEE binary64 bits)
 *   ORC_FP32   n x uint32 (IEEE binary32 bits, round-to-nearest-even from FP64)
 *   ORC_FP16   n x uint16 (IEEE binary16 bits, round-to-nearest-even from FP64)
 *   ORC_BF16   n x uint16 (bfloat16 bits, round-to-nearest-even from FP64)
 *   ORC_FRSZ2  exponents: ceil(n/32) x uint32, codes: ceil(n/32)*l x uint32 (Design section, Eq. 2-3)
 */
#ifndef CBG_ORACLE_H
#define CBG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_FP64 = 0, ORC_FP32 = 1, ORC_FP16 = 2, ORC_BF16 = 3, ORC_FRSZ2 = 4 };

/* ---- FRSZ2 codec (Design section: Eq. 2, Eq. 3, compression steps 1-6, decompression 1-4) ---- */
int64_t orc_frsz2_nblocks(int64_t n);
int64_t orc_frsz2_code_words(int64_t n, int32_t l);
int64_t orc_frsz2_bytes(int64_t n, int32_t l);
int orc_frsz2_compress(const double* x, int64_t n, int32_t l, uint32_t* exps, uint32_t* codes);
int orc_frsz2_decompress(const uint32_t* exps, const uint32_t* codes, int64_t n, int32_t l, double* out);
double orc_frsz2_decode_one(const uint32_t* exps, const uint32_t* codes, int64_t i, int32_t l);
uint32_t orc_frsz2_get_code(const uint32_t* codes, int64_t i, int32_t l);

/* ---- Cast storage formats (Compression Configuration: float64/float32/float16 storage;
 *      bfloat16 added as one more cast format) ---- */
double orc_cast_round(double x, int32_t fmt);
int orc_cast_encode(const double* x, int64_t n, int32_t fmt, void* bits);
int orc_cast_decode(const void* bits, int64_t n, int32_t fmt, double* out);

/* ---- Generic encoded-vector access (any of the five formats) ---- */
int orc_encode(const double* x, int64_t n, int32_t fmt, int32_t l, void* vals, uint32_t* exps);
int orc_decode(const void* vals, const uint32_t* exps, int64_t n, int32_t fmt, int32_t l, double* out);

/* ---- FP64 building blocks ---- */
double orc_dot(const double* a, const double* b, int64_t n);   /* sequential sum of a_k*b_k */
double orc_dot2(const double* a, const double* b, int64_t n);  /* compensated (twice-working-precision) */
double orc_nrm2(const double* a, int64_t n);
void orc_axpy(double alpha, const double* x, double* y, int64_t n); /* y += alpha x, sequential */
void orc_spmv_csr(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* vals,
                  const double* x, double* y);

/* ---- GMRES (Fig. 1, restarted, compressed basis) ---- */
typedef struct {
  int32_t restart;    /* m */
  int32_t fmt;        /* basis storage format */
  int32_t frsz2_bits; /* l in {16, 21, 32} when fmt == ORC_FRSZ2 */
  int32_t precond;    /* the M of Fig. 1 steps 3 and 17: 0 for M = I, 1 for M = diag(A) (Jacobi) */
  double tol;         /* target relative residual ||b - A x|| / ||b|| (Eq. 4) */
  int64_t max_iters;  /* cap on Arnoldi steps */
  double eta;         /* re-orthogonalization threshold of Fig. 1 step 7 */
} orc_gmres_opts;

typedef struct {
  int64_t iters;     /* Arnoldi steps (new basis vectors) */
  int64_t restarts;  /* completed restart cycles */
  int64_t reorths;   /* steps that took the second Gram-Schmidt pass */
  int32_t converged; /* explicit ||b - A x|| <= tol ||b|| reached */
  int32_t breakdowns; /* cycles that ended on the breakdown test of step 12 (R10) */
  double true_rrn;     /* last explicitly computed ||b - A x|| / ||b|| */
  double implicit_rrn; /* last |g_{j+1}| / ||b|| of the Givens recurrence */
  int32_t stagnated;   /* stopped because a cycle that ended on a breakdown (step 12) left the
                          explicit residual no smaller than at that cycle's start (R18) */
} orc_gmres_result;

/* Solves A x = b. x holds x0 on entry and the result on exit. Returns -3 when the Jacobi
 * preconditioner meets a zero, non-finite or missing diagonal entry. hist_implicit (may be NULL) gets
 * the implicit RRN after every Arnoldi step (capacity max_iters); hist_true (may be NULL) gets
 * the explicit RRN at the start of every cycle (capacity max_iters + 2). Returns 0. */
int orc_gmres(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* vals,
              const double* b, double* x, const orc_gmres_opts* opts, orc_gmres_result* res,
              double* hist_implicit, double* hist_true);

/* One Arnoldi cycle from x0, exposing its internals for the tests:
 *   V    (m+1) x n  the FP64 vectors v_1..v_{m_eff+1} (row-major, one vector per row)
 *   Vhat (m+1) x n  the same vectors as decoded from the stored basis
 *   H    (m+1) x m  the Hessenberg matrix before the Givens rotations (column-major, ld m+1)
 * Returns m_eff, the number of Arnoldi steps taken (< m on breakdown or implicit convergence),
 * or -1 when the initial residual is zero. */
int orc_arnoldi_cycle(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* vals,
                      const double* b, const double* x0, const orc_gmres_opts* opts,
                      double* V, double* Vhat, double* H, double* beta_out);

#ifdef __cplusplus
}
#endif
#endif
