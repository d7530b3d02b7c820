/* Plain FP64 CPU oracle for Compressed-Basis GMRES with the FRSZ2 block compressor
 * (arXiv 2409.15468).
 *
 * TEST INFRASTRUCTURE ONLY: the independent reference the CUDA path is checked against. Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark load it. It shares no code
 * with the CUDA library and the CUDA library never calls it.
 *
 * Pinned by the tests in tests/test_oracle_*.py against the paper's definitions, closed forms,
 * exact rational arithmetic, library routines (numpy casts, LAPACK solve) and textbook invariants
 * (Arnoldi relation, orthogonality, monotone minimal residual). Parity unpinned: the full-solve
 * behaviour of compressed bases against the paper's residual curves (the paper's figures and
 * matrices are not available), see the oracle header in the tests.
 *
 * Readings of points the paper leaves open (each cited where it is used):
 *   R1  Eq. 3's code-size term is taken as ceil(BS*l/32)*4 bytes per block (the printed
 *       ceil(BS*l/4)*4 would give 1024 bytes per block at l = 32, against the 33 bits per value
 *       stated in the synthetic-performance discussion).
 *   R2  Step 5 "cut" truncates (no rounding).
 *   R3  The stored exponent word is the raw biased IEEE exponent field of the block maximum.
 *   R4  Zero and subnormal inputs follow IEEE semantics: effective exponent 1, no hidden bit.
 *   R5  The sign bit is kept for zero and for values truncated to zero.
 *   R6  Codes form a little-endian bit stream per block: code i occupies bits [i*l, (i+1)*l),
 *       stream bit t is bit t%32 of word t/32 of the block.
 *   R7  Bit c_{l-2} is the integer bit of Eq. 2, so a code has l-2 fraction bits.
 *   R8  The last block is padded with +0.0.
 *   R9  Cast formats round to nearest even directly from FP64 (a single rounding).
 *   R10 Fig. 1 step 12: a cycle ends early when h_{j+1,j} = 0 or, after a second Gram-Schmidt
 *       pass, when h_{j+1,j} dropped below eta times its value before that pass.
 *   R11 The least-squares problem of step 17 is solved with Givens rotations; the inner loop
 *       also ends when the implicit residual |g_{j+1}| reaches tol*||b||; convergence is only
 *       declared on the explicit residual at the start of a cycle.
 *   R12 Givens rotation: r = sqrt(a*a + b*b), c = a/r, s = b/r; c = 1, s = 0 when b = 0. The
 *       length is evaluated as IEEE operations in that order (after an exact power-of-two
 *       scaling when the larger exponent field is above 1523 or below 523, i.e. outside
 *       [2^-500, 2^501)), not with a library hypot: hypot's rounding differs between C libraries,
 *       which would make the oracle's results depend on the host it runs on.
 *   R13 b = 0 gives x = 0 with RRN 0.
 *   R14 A zero diagonal entry of the rotated Hessenberg matrix truncates the least-squares
 *       solve to the leading columns before it.
 *   R18 Fig. 1 says nothing of what follows a breakdown beyond ending the Arnoldi loop: the
 *       least-squares update and the restart run as usual, and when the explicit residual at the
 *       next restart is no smaller than at the start of the cycle that broke down, the Krylov
 *       space has stopped growing; the solve then stops (stagnated) instead of repeating that
 *       cycle until max_iters.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define BS 32

static uint64_t d2u(double x) { uint64_t u; memcpy(&u, &x, 8); return u; }
static double u2d(uint64_t u) { double x; memcpy(&x, &u, 8); return x; }

/* ------------------------------------------------------------------------------------------ */
/* FRSZ2 format (Design section)                                                              */
/* ------------------------------------------------------------------------------------------ */

int64_t orc_frsz2_nblocks(int64_t n) { return (n + BS - 1) / BS; }

/* Eq. 3, compressed-values term, read as ceil(BS*l/32) 32-bit words per block (R1). */
int64_t orc_frsz2_code_words(int64_t n, int32_t l) {
  return orc_frsz2_nblocks(n) * ((BS * (int64_t)l + 31) / 32);
}

/* Eq. 3: code bytes plus one 4-byte exponent per block. */
int64_t orc_frsz2_bytes(int64_t n, int32_t l) {
  return orc_frsz2_code_words(n, l) * 4 + orc_frsz2_nblocks(n) * 4;
}

static int valid_l(int32_t l) { return l == 16 || l == 21 || l == 32; }

/* Compression of one block of BS values, the six steps of the Compression subsection. */
static void compress_block(const double x[BS], int32_t l, uint32_t* e_store, uint32_t* words) {
  uint32_t e[BS];
  uint32_t c[BS];
  /* Step 1: extract every exponent e and find the block maximum e_max. */
  uint32_t e_max = 0;
  for (int i = 0; i < BS; ++i) {
    e[i] = (uint32_t)((d2u(x[i]) >> 52) & 0x7FF);
    if (e[i] > e_max) e_max = e[i];
  }
  /* IEEE effective exponents: a zero or subnormal field stands for exponent 1 (R4). */
  uint32_t ebar = e_max > 1 ? e_max : 1;
  for (int i = 0; i < BS; ++i) {
    uint64_t u = d2u(x[i]);
    /* Step 2: sign s and significand with the usually implicit leading 1 made explicit. */
    uint32_t s = (uint32_t)(u >> 63);
    uint64_t sig = u & ((1ull << 52) - 1);
    if (e[i] != 0) sig |= 1ull << 52; /* 53-bit significand; subnormals have no hidden 1 (R4) */
    uint32_t ei = e[i] > 1 ? e[i] : 1;
    /* Step 3: normalise to e_max by prefixing k = e_max - e zero bits. */
    uint32_t k = ebar - ei;
    /* Steps 4 and 5: the sign bit goes left of the normalised significand, and the string
     * (sign, k zeros, 53 significand bits) is cut to its first l bits (R2: truncation). */
    uint32_t code = s;
    for (int t = 0; t < l - 1; ++t) {
      uint32_t bit = 0;
      if ((uint32_t)t >= k) {
        int pos = 52 - (int)((uint32_t)t - k); /* position in the 53-bit significand */
        if (pos >= 0) bit = (uint32_t)((sig >> pos) & 1);
      }
      code = (code << 1) | bit;
    }
    c[i] = code;
  }
  /* Step 6: store e_max (R3) and all codes, packed as a little-endian bit stream (R6). */
  int nw = (BS * l + 31) / 32;
  for (int w = 0; w < nw; ++w) words[w] = 0;
  for (int i = 0; i < BS; ++i) {
    for (int b = 0; b < l; ++b) {
      if ((c[i] >> b) & 1u) {
        int t = i * l + b;
        words[t / 32] |= 1u << (t % 32);
      }
    }
  }
  *e_store = e_max;
}

int orc_frsz2_compress(const double* x, int64_t n, int32_t l, uint32_t* exps, uint32_t* codes) {
  if (!valid_l(l) || n < 0) return -1;
  int64_t nb = orc_frsz2_nblocks(n);
  int nw = (BS * l + 31) / 32;
  for (int64_t b = 0; b < nb; ++b) {
    double blk[BS];
    for (int i = 0; i < BS; ++i) {
      int64_t k = b * BS + i;
      blk[i] = k < n ? x[k] : 0.0; /* R8 */
    }
    compress_block(blk, l, &exps[b], &codes[b * nw]);
  }
  return 0;
}

/* Reads code i (within its block) from the block's bit stream (R6). */
static uint32_t read_code(const uint32_t* words, int i, int32_t l) {
  uint32_t c = 0;
  for (int b = 0; b < l; ++b) {
    int t = i * l + b;
    c |= ((words[t / 32] >> (t % 32)) & 1u) << b;
  }
  return c;
}

uint32_t orc_frsz2_get_code(const uint32_t* codes, int64_t i, int32_t l) {
  int nw = (BS * l + 31) / 32;
  return read_code(&codes[(i / BS) * nw], (int)(i % BS), l);
}

/* Decompression of the value at index i, the four steps of the Decompression subsection. */
double orc_frsz2_decode_one(const uint32_t* exps, const uint32_t* codes, int64_t i, int32_t l) {
  int nw = (BS * l + 31) / 32;
  /* Step 1: read e_max of the block and the code c at index i. */
  uint32_t e_max = exps[i / BS];
  uint32_t c = read_code(&codes[(i / BS) * nw], (int)(i % BS), l);
  /* Step 2: separate the sign bit from the significand; count the inserted zeros k. */
  uint64_t s = c >> (l - 1);
  uint32_t sig = c & ((1u << (l - 1)) - 1);
  if (sig == 0) return u2d(s << 63); /* +-0 (R5) */
  int k = 0;
  while (((sig >> (l - 2 - k)) & 1u) == 0) ++k;
  /* Step 3: drop the k zeros and the explicit leading 1; actual exponent e = e_max - k. */
  int32_t ebar = e_max > 1 ? (int32_t)e_max : 1;
  int p = l - 2 - k;                               /* position of the leading 1 (R7) */
  uint64_t frac = sig & ((1ull << p) - 1);         /* the p bits after it */
  int32_t e = ebar - k;
  /* Step 4: merge s, e and the significand back into an IEEE double. */
  if (e >= 1) return u2d((s << 63) | ((uint64_t)e << 52) | (frac << (52 - p)));
  /* Below the normal range the value sig * 2^(ebar-1023-(l-2)) is an IEEE subnormal (R4). */
  return u2d((s << 63) | ((uint64_t)sig << (ebar + 53 - l)));
}

int orc_frsz2_decompress(const uint32_t* exps, const uint32_t* codes, int64_t n, int32_t l, double* out) {
  if (!valid_l(l) || n < 0) return -1;
  for (int64_t i = 0; i < n; ++i) out[i] = orc_frsz2_decode_one(exps, codes, i, l);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Cast formats (Compression Configuration; R9)                                               */
/* ------------------------------------------------------------------------------------------ */

/* Round x to the nearest value with p significand bits and minimum normal exponent emin
 * (gradual underflow below it), ties to even; values at or beyond 2^(emax+1) after rounding
 * become infinity. nearbyint in the default rounding mode is the ties-to-even step. */
static double round_rne(double x, int p, int emin, int emax) {
  if (x == 0.0 || isnan(x) || isinf(x)) return x;
  double a = fabs(x);
  int E;
  frexp(a, &E);                /* a = f * 2^E, f in [0.5, 1) */
  int e = E - 1;               /* a in [2^e, 2^(e+1)) */
  if (e < emin) e = emin;      /* subnormal spacing below the normal range */
  double quantum = ldexp(1.0, e - (p - 1));
  double r = nearbyint(a / quantum) * quantum; /* exact scaling by a power of two */
  if (r >= ldexp(1.0, emax + 1)) r = INFINITY;
  return copysign(r, x);
}

double orc_cast_round(double x, int32_t fmt) {
  switch (fmt) {
    case ORC_FP64: return x;
    case ORC_FP32: return round_rne(x, 24, -126, 127);
    case ORC_FP16: return round_rne(x, 11, -14, 15);
    case ORC_BF16: return round_rne(x, 8, -126, 127);
    default: return NAN;
  }
}

static uint16_t fp16_bits_of(double r) { /* r is already a binary16 value */
  uint16_t s = signbit(r) ? 0x8000 : 0;
  double a = fabs(r);
  if (a == 0.0) return s;
  if (isinf(a)) return s | 0x7C00;
  if (isnan(a)) return 0x7E00;
  if (a < ldexp(1.0, -14)) return s | (uint16_t)(a / ldexp(1.0, -24)); /* subnormal */
  int E;
  double f = frexp(a, &E);                    /* a = f 2^E, f in [0.5,1) */
  int e = E - 1;                              /* a = (2f) 2^e */
  uint16_t mant = (uint16_t)((2.0 * f - 1.0) * 1024.0);
  return s | (uint16_t)((e + 15) << 10) | mant;
}

static double fp16_value_of(uint16_t h) {
  double sgn = (h & 0x8000) ? -1.0 : 1.0;
  int e = (h >> 10) & 0x1F;
  int m = h & 0x3FF;
  if (e == 0) return sgn * ldexp((double)m, -24);
  if (e == 31) return m ? NAN : sgn * INFINITY;
  return sgn * ldexp((double)(1024 + m), e - 25);
}

int orc_cast_encode(const double* x, int64_t n, int32_t fmt, void* bits) {
  for (int64_t i = 0; i < n; ++i) {
    double r = orc_cast_round(x[i], fmt);
    if (fmt == ORC_FP64) {
      uint64_t u = d2u(r);
      memcpy((char*)bits + 8 * i, &u, 8);
    } else if (fmt == ORC_FP32) {
      float f = (float)r; /* exact: r is a binary32 value */
      memcpy((char*)bits + 4 * i, &f, 4);
    } else if (fmt == ORC_BF16) {
      float f = (float)r; /* exact: a bfloat16 value is a binary32 value with 16 zero low bits */
      uint32_t u;
      memcpy(&u, &f, 4);
      uint16_t h = (uint16_t)(u >> 16);
      memcpy((char*)bits + 2 * i, &h, 2);
    } else if (fmt == ORC_FP16) {
      uint16_t h = fp16_bits_of(r);
      memcpy((char*)bits + 2 * i, &h, 2);
    } else {
      return -1;
    }
  }
  return 0;
}

int orc_cast_decode(const void* bits, int64_t n, int32_t fmt, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    if (fmt == ORC_FP64) {
      uint64_t u;
      memcpy(&u, (const char*)bits + 8 * i, 8);
      out[i] = u2d(u);
    } else if (fmt == ORC_FP32) {
      float f;
      memcpy(&f, (const char*)bits + 4 * i, 4);
      out[i] = (double)f;
    } else if (fmt == ORC_BF16) {
      uint16_t h;
      memcpy(&h, (const char*)bits + 2 * i, 2);
      uint32_t u = (uint32_t)h << 16;
      float f;
      memcpy(&f, &u, 4);
      out[i] = (double)f;
    } else if (fmt == ORC_FP16) {
      uint16_t h;
      memcpy(&h, (const char*)bits + 2 * i, 2);
      out[i] = fp16_value_of(h);
    } else {
      return -1;
    }
  }
  return 0;
}

int orc_encode(const double* x, int64_t n, int32_t fmt, int32_t l, void* vals, uint32_t* exps) {
  if (fmt == ORC_FRSZ2) return orc_frsz2_compress(x, n, l, exps, (uint32_t*)vals);
  return orc_cast_encode(x, n, fmt, vals);
}

int orc_decode(const void* vals, const uint32_t* exps, int64_t n, int32_t fmt, int32_t l, double* out) {
  if (fmt == ORC_FRSZ2) return orc_frsz2_decompress(exps, (const uint32_t*)vals, n, l, out);
  return orc_cast_decode(vals, n, fmt, out);
}

static int64_t encoded_val_bytes(int64_t n, int32_t fmt, int32_t l) {
  switch (fmt) {
    case ORC_FP64: return 8 * n;
    case ORC_FP32: return 4 * n;
    case ORC_FP16:
    case ORC_BF16: return 2 * n;
    case ORC_FRSZ2: return 4 * orc_frsz2_code_words(n, l);
    default: return -1;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* FP64 building blocks                                                                       */
/* ------------------------------------------------------------------------------------------ */

double orc_dot(const double* a, const double* b, int64_t n) {
  double s = 0.0;
  for (int64_t k = 0; k < n; ++k) s += a[k] * b[k];
  return s;
}

/* Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 2005):
 * TwoProduct via fma and TwoSum, result as accurate as if computed in twice the precision. */
double orc_dot2(const double* a, const double* b, int64_t n) {
  double s = 0.0, c = 0.0;
  for (int64_t k = 0; k < n; ++k) {
    double p = a[k] * b[k];
    double pe = fma(a[k], b[k], -p);    /* a*b = p + pe exactly */
    double t = s + p;
    double z = t - s;
    double se = (s - (t - z)) + (p - z); /* s + p = t + se exactly */
    s = t;
    c += pe + se;
  }
  return s + c;
}

double orc_nrm2(const double* a, int64_t n) { return sqrt(orc_dot(a, a, n)); }

void orc_axpy(double alpha, const double* x, double* y, int64_t n) {
  for (int64_t k = 0; k < n; ++k) y[k] += alpha * x[k];
}

void orc_spmv_csr(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* vals,
                  const double* x, double* y) {
  for (int32_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) s += vals[p] * x[col[p]];
    y[i] = s;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Restarted CB-GMRES (Fig. 1)                                                                */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
  int32_t n, m, fmt, l;
  const int32_t *row_ptr, *col;
  const double* vals;
  double eta, tol, bnorm;
  int64_t max_iters;
  int64_t val_bytes;
  unsigned char* store; /* (m+1) encoded value arrays */
  uint32_t* store_exp;  /* (m+1) FRSZ2 exponent arrays */
  double* vhat;         /* (m+1) x n decoded copies of the stored basis */
  double *v, *w, *h, *u, *H, *R, *cs, *sn, *g, *y;
  double *dinv, *t; /* Jacobi: 1 / diag(A) and a scratch vector; NULL for M = I */
} cycle_ws;

/* Append v as basis vector `slot`: store it in the chosen format (Fig. 1 steps 1 and 14,
 * highlighted) and keep the decoded copy that every later read of the basis sees. */
static void store_basis(cycle_ws* ws, int slot, const double* v) {
  int64_t nb = orc_frsz2_nblocks(ws->n);
  void* vals = ws->store + (size_t)slot * ws->val_bytes;
  uint32_t* ex = ws->store_exp + (size_t)slot * nb;
  orc_encode(v, ws->n, ws->fmt, ws->l, vals, ex);
  orc_decode(vals, ex, ws->n, ws->fmt, ws->l, ws->vhat + (size_t)slot * ws->n);
}

/* The length of (a, b) for the Givens rotation (R12). */
static double givens_radius(double a, double b) {
  int ea = (int)((d2u(a) >> 52) & 0x7FF), eb = (int)((d2u(b) >> 52) & 0x7FF);
  int e = ea > eb ? ea : eb;
  double scale = 1.0;
  if (e > 1523) scale = 0x1p-600;
  else if (e < 523) scale = 0x1p600;
  double as = a * scale, bs = b * scale;
  return sqrt(as * as + bs * bs) / scale;
}

/* One cycle from the residual r with norm beta (Fig. 1 steps 1-17). Updates x in place.
 * Optional outputs for the tests: V (fp64 vectors), Vh (decoded), Hout (before rotations). */
static int run_cycle(cycle_ws* ws, const double* r, double beta, double* x, int64_t* iters,
                     int64_t* reorths, int32_t* breakdowns, double* implicit_rrn, double* hist_implicit,
                     double* V, double* Vh, double* Hout) {
  const int32_t n = ws->n, m = ws->m;
  const int ld = m + 1;
  /* Step 1: v := r0 / beta, V_1 = [v] (compressed). */
  for (int32_t k = 0; k < n; ++k) ws->v[k] = r[k] / beta;
  store_basis(ws, 0, ws->v);
  if (V) memcpy(V, ws->v, sizeof(double) * n);
  if (Vh) memcpy(Vh, ws->vhat, sizeof(double) * n);
  for (int i = 0; i <= m; ++i) ws->g[i] = 0.0;
  ws->g[0] = beta;
  int m_eff = 0;
  for (int j = 0; j < m; ++j) {
    /* Step 3: w := A (M^{-1} v); v is the FP64 vector (the SpMV is not highlighted). */
    if (ws->dinv) {
      for (int32_t k = 0; k < n; ++k) ws->t[k] = ws->v[k] * ws->dinv[k];
      orc_spmv_csr(n, ws->row_ptr, ws->col, ws->vals, ws->t, ws->w);
    } else {
      orc_spmv_csr(n, ws->row_ptr, ws->col, ws->vals, ws->v, ws->w);
    }
    /* Step 4: omega := ||w||. */
    double omega = orc_nrm2(ws->w, n);
    /* Step 5: classical Gram-Schmidt against the stored (decoded) basis:
     * h_{1:j} := V_j^T w, then w := w - V_j h_{1:j}. */
    for (int i = 0; i <= j; ++i) ws->h[i] = orc_dot(ws->vhat + (size_t)i * n, ws->w, n);
    for (int i = 0; i <= j; ++i) {
      const double* vi = ws->vhat + (size_t)i * n;
      for (int32_t k = 0; k < n; ++k) ws->w[k] -= vi[k] * ws->h[i];
    }
    /* Step 6: h_{j+1,j} := ||w||. */
    double hn = orc_nrm2(ws->w, n);
    int did_reorth = 0;
    double h_before = hn;
    /* Steps 7-11: one more Gram-Schmidt pass when the norm dropped below eta * omega. */
    if (hn < ws->eta * omega) {
      for (int i = 0; i <= j; ++i) ws->u[i] = orc_dot(ws->vhat + (size_t)i * n, ws->w, n);
      for (int i = 0; i <= j; ++i) {
        const double* vi = ws->vhat + (size_t)i * n;
        for (int32_t k = 0; k < n; ++k) ws->w[k] -= vi[k] * ws->u[i];
      }
      for (int i = 0; i <= j; ++i) ws->h[i] += ws->u[i];
      hn = orc_nrm2(ws->w, n);
      did_reorth = 1;
      ++*reorths;
    }
    /* Column j of the Hessenberg matrix (step 16). */
    for (int i = 0; i <= j; ++i) ws->H[(size_t)j * ld + i] = ws->h[i];
    ws->H[(size_t)j * ld + j + 1] = hn;
    if (Hout) {
      for (int i = 0; i <= m; ++i) Hout[(size_t)j * ld + i] = i <= j + 1 ? ws->H[(size_t)j * ld + i] : 0.0;
    }
    ++*iters;
    m_eff = j + 1;
    /* Step 12 (R10). */
    int breakdown = (hn == 0.0) || (did_reorth && hn < ws->eta * h_before);
    /* Step 17's least squares, one column at a time (R11, R12): apply the previous rotations
     * to column j, form the rotation that zeroes h_{j+1,j}, and rotate the right-hand side. */
    double* Rj = ws->R + (size_t)j * ld;
    for (int i = 0; i <= j + 1; ++i) Rj[i] = ws->H[(size_t)j * ld + i];
    for (int i = 0; i < j; ++i) {
      double t = ws->cs[i] * Rj[i] + ws->sn[i] * Rj[i + 1];
      Rj[i + 1] = -ws->sn[i] * Rj[i] + ws->cs[i] * Rj[i + 1];
      Rj[i] = t;
    }
    double a = Rj[j], bb = Rj[j + 1];
    double c, s;
    if (bb == 0.0) {
      c = 1.0;
      s = 0.0;
    } else {
      double rr = givens_radius(a, bb);
      c = a / rr;
      s = bb / rr;
      Rj[j] = rr;
    }
    Rj[j + 1] = 0.0;
    ws->cs[j] = c;
    ws->sn[j] = s;
    ws->g[j + 1] = -s * ws->g[j];
    ws->g[j] = c * ws->g[j];
    *implicit_rrn = fabs(ws->g[j + 1]) / ws->bnorm;
    if (hist_implicit) hist_implicit[*iters - 1] = *implicit_rrn;
    if (breakdown) ++*breakdowns;
    if (breakdown || *implicit_rrn <= ws->tol || *iters >= ws->max_iters) break;
    /* Steps 13-14: v := w / h_{j+1,j}; V_{j+1} := [V_j, v] (compressed). */
    for (int32_t k = 0; k < n; ++k) ws->v[k] = ws->w[k] / hn;
    store_basis(ws, j + 1, ws->v);
    if (V) memcpy(V + (size_t)(j + 1) * n, ws->v, sizeof(double) * n);
    if (Vh) memcpy(Vh + (size_t)(j + 1) * n, ws->vhat + (size_t)(j + 1) * n, sizeof(double) * n);
  }
  /* Step 17: y minimises ||beta e1 - Hbar y||: back substitution on the rotated system (R14). */
  int mls = m_eff;
  for (int k = 0; k < m_eff; ++k) {
    if (ws->R[(size_t)k * ld + k] == 0.0) {
      mls = k;
      break;
    }
  }
  for (int k = mls - 1; k >= 0; --k) {
    double t = ws->g[k];
    for (int i = k + 1; i < mls; ++i) t -= ws->R[(size_t)i * ld + k] * ws->y[i];
    ws->y[k] = t / ws->R[(size_t)k * ld + k];
  }
  /* x_m := x_0 + M^{-1} (V_m y_m), reading the stored basis (highlighted). */
  if (ws->dinv) {
    for (int32_t k = 0; k < n; ++k) ws->t[k] = 0.0;
    for (int i = 0; i < mls; ++i) {
      const double* vi = ws->vhat + (size_t)i * n;
      for (int32_t k = 0; k < n; ++k) ws->t[k] += vi[k] * ws->y[i];
    }
    for (int32_t k = 0; k < n; ++k) x[k] += ws->dinv[k] * ws->t[k];
  } else {
    for (int i = 0; i < mls; ++i) {
      const double* vi = ws->vhat + (size_t)i * n;
      for (int32_t k = 0; k < n; ++k) x[k] += vi[k] * ws->y[i];
    }
  }
  return m_eff;
}

static int ws_init(cycle_ws* ws, int32_t n, const int32_t* row_ptr, const int32_t* col, const double* vals,
                   const orc_gmres_opts* o) {
  memset(ws, 0, sizeof(*ws));
  if (n < 1 || o->restart < 1 || o->tol <= 0.0) return -1;
  if (o->fmt < ORC_FP64 || o->fmt > ORC_FRSZ2) return -1;
  if (o->fmt == ORC_FRSZ2 && !valid_l(o->frsz2_bits)) return -1;
  ws->n = n;
  ws->m = o->restart;
  ws->fmt = o->fmt;
  ws->l = o->fmt == ORC_FRSZ2 ? o->frsz2_bits : 32;
  ws->row_ptr = row_ptr;
  ws->col = col;
  ws->vals = vals;
  ws->eta = o->eta;
  ws->tol = o->tol;
  ws->max_iters = o->max_iters;
  ws->val_bytes = encoded_val_bytes(n, ws->fmt, ws->l);
  size_t m1 = (size_t)ws->m + 1;
  ws->store = (unsigned char*)malloc(m1 * (size_t)ws->val_bytes);
  ws->store_exp = (uint32_t*)calloc(m1 * (size_t)orc_frsz2_nblocks(n), sizeof(uint32_t));
  ws->vhat = (double*)malloc(m1 * (size_t)n * sizeof(double));
  ws->v = (double*)malloc((size_t)n * sizeof(double));
  ws->w = (double*)malloc((size_t)n * sizeof(double));
  ws->h = (double*)calloc(m1, sizeof(double));
  ws->u = (double*)calloc(m1, sizeof(double));
  ws->H = (double*)calloc(m1 * ws->m, sizeof(double));
  ws->R = (double*)calloc(m1 * ws->m, sizeof(double));
  ws->cs = (double*)calloc(m1, sizeof(double));
  ws->sn = (double*)calloc(m1, sizeof(double));
  ws->g = (double*)calloc(m1, sizeof(double));
  ws->y = (double*)calloc(m1, sizeof(double));
  if (!ws->store || !ws->store_exp || !ws->vhat || !ws->v || !ws->w || !ws->h || !ws->u || !ws->H || !ws->R ||
      !ws->cs || !ws->sn || !ws->g || !ws->y)
    return -2;
  if (o->precond == 1) {
    /* Jacobi: M = diag(A), entries of row i in column i summed; M^{-1} stored as 1 / a_ii. */
    ws->dinv = (double*)malloc((size_t)n * sizeof(double));
    ws->t = (double*)malloc((size_t)n * sizeof(double));
    if (!ws->dinv || !ws->t) return -2;
    for (int32_t i = 0; i < n; ++i) {
      double d = 0.0;
      for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
        if (col[p] == i) d += vals[p];
      if (d == 0.0 || !isfinite(d)) return -3;
      ws->dinv[i] = 1.0 / d;
    }
  } else if (o->precond != 0) {
    return -1;
  }
  return 0;
}

static void ws_free(cycle_ws* ws) {
  free(ws->store);
  free(ws->store_exp);
  free(ws->vhat);
  free(ws->v);
  free(ws->w);
  free(ws->h);
  free(ws->u);
  free(ws->H);
  free(ws->R);
  free(ws->cs);
  free(ws->sn);
  free(ws->g);
  free(ws->y);
  free(ws->dinv);
  free(ws->t);
}

/* r := b - A x (Fig. 1 step 1). */
static void residual(const cycle_ws* ws, const double* b, const double* x, double* r) {
  orc_spmv_csr(ws->n, ws->row_ptr, ws->col, ws->vals, x, r);
  for (int32_t k = 0; k < ws->n; ++k) r[k] = b[k] - r[k];
}

int orc_gmres(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* vals, const double* b,
              double* x, const orc_gmres_opts* opts, orc_gmres_result* res, double* hist_implicit,
              double* hist_true) {
  memset(res, 0, sizeof(*res));
  cycle_ws ws;
  int st = ws_init(&ws, n, row_ptr, col, vals, opts);
  if (st != 0) {
    ws_free(&ws);
    return st;
  }
  ws.bnorm = orc_nrm2(b, n);
  if (ws.bnorm == 0.0) { /* R13 */
    for (int32_t k = 0; k < n; ++k) x[k] = 0.0;
    res->converged = 1;
    if (hist_true) hist_true[0] = 0.0;
    ws_free(&ws);
    return 0;
  }
  double* r = (double*)malloc((size_t)n * sizeof(double));
  int64_t iters = 0, reorths = 0;
  int32_t breakdowns = 0;
  double implicit = 0.0;
  double cycle_start_rrn = 0.0;
  int broke_down = 0; /* the last cycle ended on the breakdown test */
  for (;;) {
    /* Step 1 (and the stopping test of step 18, Eq. 4): explicit residual. */
    residual(&ws, b, x, r);
    double beta = orc_nrm2(r, n);
    res->true_rrn = beta / ws.bnorm;
    if (hist_true) hist_true[res->restarts] = res->true_rrn;
    if (res->true_rrn <= ws.tol) {
      res->converged = 1;
      break;
    }
    if (broke_down && res->true_rrn >= cycle_start_rrn) { /* R18 */
      res->stagnated = 1;
      break;
    }
    if (iters >= ws.max_iters) break;
    cycle_start_rrn = res->true_rrn;
    int32_t breakdowns_before = breakdowns;
    run_cycle(&ws, r, beta, x, &iters, &reorths, &breakdowns, &implicit, hist_implicit, NULL, NULL, NULL);
    broke_down = breakdowns > breakdowns_before;
    res->restarts += 1;
  }
  res->iters = iters;
  res->reorths = reorths;
  res->breakdowns = breakdowns;
  res->implicit_rrn = implicit;
  free(r);
  ws_free(&ws);
  return 0;
}

int orc_arnoldi_cycle(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* vals, const double* b,
                      const double* x0, const orc_gmres_opts* opts, double* V, double* Vhat, double* H,
                      double* beta_out) {
  cycle_ws ws;
  int st = ws_init(&ws, n, row_ptr, col, vals, opts);
  if (st != 0) {
    ws_free(&ws);
    return -2;
  }
  ws.bnorm = orc_nrm2(b, n);
  double* r = (double*)malloc((size_t)n * sizeof(double));
  double* x = (double*)malloc((size_t)n * sizeof(double));
  memcpy(x, x0, sizeof(double) * n);
  residual(&ws, b, x, r);
  double beta = orc_nrm2(r, n);
  *beta_out = beta;
  int m_eff = -1;
  if (beta > 0.0 && ws.bnorm > 0.0) {
    int64_t iters = 0, reorths = 0;
    int32_t breakdowns = 0;
    double implicit = 0.0;
    memset(H, 0, sizeof(double) * (size_t)(ws.m + 1) * ws.m);
    m_eff = run_cycle(&ws, r, beta, x, &iters, &reorths, &breakdowns, &implicit, NULL, V, Vhat, H);
  }
  free(r);
  free(x);
  ws_free(&ws);
  return m_eff;
}
