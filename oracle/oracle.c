/*
 * CPU oracle for the BF16-split method of Henry, Tang & Heinecke,
 * "Leveraging the bfloat16 Artificial Intelligence Datatype For
 * Higher-Precision Computations" (ARITH 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or constant with the CUDA library: it is a plain, slow,
 * sequential statement of what the method computes, each function citing the
 * passage it follows.  Build flags keep C float arithmetic IEEE binary32 with
 * round-to-nearest, no contraction of a*b+c into an FMA unless fmaf() is
 * written, and gradual underflow:  gcc -O2 -ffp-contract=off -fno-fast-math.
 * OpenMP is used only to run independent outputs (rows, systems) on several
 * host threads; it never changes the order of an accumulation.
 *
 * Readings of the paper taken here (the paper is silent or garbled):
 *  R1 (B16) rounds to nearest, ties to even (Sec. II-A gives no mode; the bin
 *     bound |a1| <= 2^-8 |a0| of Sec. II-G holds for this mode).
 *  R3 a finite FP32 value whose RNE bfloat16 would overflow to infinity
 *     (|x| >= 0x7F7F8000) gets hi = x truncated toward zero; the rest of the
 *     split then proceeds as written, so the pieces still sum to x.
 *  R4 Inf/NaN: hi carries the value (NaN made quiet, sign kept), mid = lo = +0.
 *  R6 products and order: x1 = {00}; x3 = pair split, {00,01,10};
 *     x6 = {00,01,10,02,11,20}; x8 = x6 + {12,21} (the "Z3" sum of
 *     Sec. II-D); x9 = all nine; level sums and the smallest-first
 *     combination exactly as written in Sec. II-D.
 *  R25 the asymmetric split of Sec. II-G: x5 = A in two pieces, B in three,
 *     the five products {00,01,10,02,11} (the 2^-16 bin without a2 b0,
 *     since A has no a2); combined as x6 with Z2 = Z02 + Z11.
 *  R9 refinement: r = b - A x (the paper's sign slip in Sec. III corrected),
 *     residual, correction solve and update all in FP64 with the low-precision
 *     factors (Sec. III: "do the solve in a higher precision like FP64").
 *  R12 the "combined type" LU (Sec. IV-A) uses bf16xN only in the products
 *     of the trailing matrix update; pivot search, swaps and the division by
 *     the pivot are plain FP32.  Of record: orc_lu_plain (unblocked, each
 *     update product the mode's product).  orc_lu restates the device's
 *     blocked schedule as a regression mirror only.
 *  R13 GEMM result form C = alpha*Z + beta*C: t = fl32(alpha*Z), then
 *     fmaf(beta, C, t); beta == 0 does not read C.
 *  R26 the single-type LU of the Sec. IV-B plain IR table ("FP32", "BF16",
 *     "FP16" rows): A rounded to the type, then the unblocked right-looking
 *     LU with partial pivoting in which every operation (division by the
 *     pivot, product, difference) is done in FP32 and rounded to the type
 *     (round to nearest even); the refinement of R9 then uses those factors
 *     with no stall rule, converged when a correction is below the
 *     tolerance within max_iter corrections.
 *  R18 "GMRES with the LU as preconditioner" (Sec. III remark, Sec. IV-B):
 *     left-preconditioned GMRES in FP64 solves each refinement step's
 *     correction equation; restarts recompute r = b - A x in FP64.
 *  R27 the preconditioner of R18 applied through explicit inverses: the
 *     paper fixes M = P^T L U (the low-precision factors) and FP64 for
 *     GMRES, not how M^-1 v is evaluated.  With the inverses X_L = L^-1 and
 *     X_U = U^-1 of the FP32 factors formed once in FP64 (column c by
 *     substitution on the unit vector e_c), M^-1 v = X_U (X_L (P v)), two
 *     matrix-vector products; this is the same operator up to FP64
 *     rounding.  orc_gmres takes the inverses as an option; the starting
 *     x0 = M^-1 b keeps the substitution.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* bit views                                                            */
/* ------------------------------------------------------------------ */
static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float f32_from_bits(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
/* (F32) of a bfloat16 bit pattern: exact widening (Sec. I: BF16 is the top
 * 16 bits of an FP32 word). */
static float bf16_to_f32(uint16_t h) { return f32_from_bits((uint32_t)h << 16); }

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* O1  (B16): FP32 -> bfloat16, round to nearest, ties to even (R1).    */
/* bfloat16 keeps sign, the full 8-bit exponent and the top 7 stored    */
/* mantissa bits of FP32 (Sec. I).  The two bfloat16 neighbours of x    */
/* that bracket it toward and away from zero are the truncation t and   */
/* t + 1 ulp; the dropped 16 bits decide which one is nearer.           */
/* ------------------------------------------------------------------ */
uint16_t orc_bf16_rne(float x) {
  uint32_t u = f32_bits(x);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu) != 0u)
    return (uint16_t)((u >> 16) | 0x0040u); /* NaN: quiet, sign kept (R4) */
  uint16_t toward_zero = (uint16_t)(u >> 16);
  uint32_t dropped = u & 0xFFFFu;   /* distance to toward_zero, in 2^-16 ulp */
  int away;
  if (dropped > 0x8000u) away = 1;                 /* nearer the far neighbour */
  else if (dropped < 0x8000u) away = 0;            /* nearer the truncation    */
  else away = (toward_zero & 1u) ? 1 : 0;          /* tie: pick the even one   */
  /* one ulp away from zero; a carry out of the mantissa moves to the next
   * binade and past the largest finite value to infinity, as IEEE requires */
  return (uint16_t)(toward_zero + (away ? 1u : 0u));
}

void orc_bf16_rne_array(int64_t n, const float* x, uint16_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_bf16_rne(x[i]);
}

/* IEEE binary16 (1 sign, 5 exponent bits biased by 15, 10 fraction bits;
 * normal binades 2^-14 .. 2^15, subnormals in steps of 2^-24) of an FP32
 * value, rounded to nearest, ties to even, straight from the definition:
 * |x| = m 2^e with m the 24-bit significand; the quantum of x's binade in
 * binary16 is 2^(E-10) (E = floor(log2 |x|) >= -14) or 2^-24 below; m is
 * shifted to that quantum with round-to-nearest-even; a carry into the next
 * binade (and past 65504 into infinity) follows from the encoding.  NaN
 * gives a quiet NaN with the sign kept. */
uint16_t orc_f16_rne(float x) {
  const uint32_t u = f32_bits(x);
  const uint16_t sign = (uint16_t)((u >> 16) & 0x8000u);
  const uint32_t ex = (u >> 23) & 0xFFu, fr = u & 0x7FFFFFu;
  if (ex == 0xFFu) return (uint16_t)(sign | (fr ? 0x7E00u : 0x7C00u));
  if (ex == 0u && fr == 0u) return sign;
  uint32_t m;
  int e, E;
  if (ex == 0u) { /* FP32 subnormal: far below binary16's smallest step */
    m = fr;
    e = -149;
    E = -127;
  } else {
    m = fr | 0x800000u;
    e = (int)ex - 150;
    E = (int)ex - 127;
  }
  const int Q = (E >= -14) ? E - 10 : -24; /* exponent of the quantum */
  const int shift = Q - e;                 /* >= 0: binary16 has fewer bits */
  uint32_t r;
  if (shift >= 26) {
    r = 0u; /* below half the smallest step */
  } else if (shift > 0) {
    const uint32_t rem = m & ((1u << shift) - 1u), half = 1u << (shift - 1);
    r = m >> shift;
    if (rem > half || (rem == half && (r & 1u))) ++r;
  } else {
    r = m << (-shift);
  }
  if (Q == -24) return (uint16_t)(sign | r); /* subnormal; r = 1024 is 2^-14 */
  /* normal: r in [1024, 2048]; 2048 carries into the next binade */
  const uint32_t bits = ((uint32_t)(E + 15) << 10) + (r - 1024u);
  if (bits >= 0x7C00u) return (uint16_t)(sign | 0x7C00u);
  return (uint16_t)(sign | bits);
}

/* (F32) of a binary16 bit pattern (exact). */
static float f16_to_f32(uint16_t h) {
  const uint32_t sign = (uint32_t)(h & 0x8000u) << 16;
  const uint32_t ex = (h >> 10) & 0x1Fu, fr = h & 0x3FFu;
  if (ex == 0x1Fu) return f32_from_bits(sign | 0x7F800000u | (fr << 13));
  if (ex == 0u) { /* zero or subnormal: fr 2^-24 */
    const float v = (float)fr * 0x1p-24f;
    return sign ? -v : v;
  }
  return f32_from_bits(sign | ((ex + 112u) << 23) | (fr << 13));
}

void orc_f16_rne_array(int64_t n, const float* x, uint16_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_f16_rne(x[i]);
}

/* v rounded to the single type of R26: 0 FP32 (as is), 1 bfloat16,
 * 2 binary16. */
static float round_to_type(int type, float v) {
  if (type == 1) return bf16_to_f32(orc_bf16_rne(v));
  if (type == 2) return f16_to_f32(orc_f16_rne(v));
  return v;
}

/* ------------------------------------------------------------------ */
/* O2  the decomposition of Sec. II-A:                                   */
/*   b0 = (B16) a                                                        */
/*   b1 = (B16)((F32)(a - (F32)b0))                                      */
/*   b2 = (B16)((F32)(a - (F32)b0 - (F32)b1))   (left to right)          */
/* npieces = 1, 2 or 3 writes b0 / b0,b1 / b0,b1,b2.  The pair split of  */
/* Sec. I/II-G is the first two pieces of the triple split.             */
/* ------------------------------------------------------------------ */
static void split_one(float a, uint16_t* b0, uint16_t* b1, uint16_t* b2) {
  uint32_t u = f32_bits(a);
  if ((u & 0x7F800000u) == 0x7F800000u) {          /* Inf or NaN (R4) */
    if ((u & 0x007FFFFFu) != 0u)
      *b0 = (uint16_t)((u >> 16) | 0x0040u);       /* NaN, made quiet */
    else
      *b0 = (uint16_t)(u >> 16);                   /* +-Inf */
    *b1 = 0; *b2 = 0;
    return;
  }
  if ((u & 0x7FFFFFFFu) >= 0x7F7F8000u)            /* RNE would overflow (R3) */
    *b0 = (uint16_t)(u >> 16);
  else
    *b0 = orc_bf16_rne(a);
  float r1 = a - bf16_to_f32(*b0);                 /* (F32)(a - (F32)b0) */
  *b1 = orc_bf16_rne(r1);
  float r2 = (a - bf16_to_f32(*b0)) - bf16_to_f32(*b1);
  *b2 = orc_bf16_rne(r2);
}

void orc_split(int64_t n, const float* x, int npieces, uint16_t* b0, uint16_t* b1,
               uint16_t* b2) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    uint16_t p0, p1, p2;
    split_one(x[i], &p0, &p1, &p2);
    b0[i] = p0;
    if (npieces >= 2) b1[i] = p1;
    if (npieces >= 3) b2[i] = p2;
  }
}

/* Split of every FP32 bit pattern in [start, start+count): used to compare
 * against the device split over the whole 2^32 input space chunk by chunk. */
void orc_split_bits_range(uint64_t start, int64_t count, int npieces, uint16_t* b0,
                          uint16_t* b1, uint16_t* b2) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) {
    uint16_t p0, p1, p2;
    split_one(f32_from_bits((uint32_t)(start + (uint64_t)i)), &p0, &p1, &p2);
    b0[i] = p0;
    if (npieces >= 2) b1[i] = p1;
    if (npieces >= 3) b2[i] = p2;
  }
}

/* ------------------------------------------------------------------ */
/* O4  products of Sec. II-D in the paper's FP32-FMA model.              */
/* For each used piece pair (i,j):                                      */
/*   Z^(i,j) <- 0;  for l: Z^(i,j) <- FMA(x_l^(i), y_l^(j), Z^(i,j))     */
/* then the level sums, in FP32:                                        */
/*   Z0 = Z00;  Z1 = Z01 + Z10;  Z2 = Z02 + (Z11 + Z20);                 */
/*   Z3 = Z12 + Z21;  Z4 = Z22                                           */
/* and the combination, smallest first:                                  */
/*   x1: Z0;  x3: Z0 + Z1;  x6 (= Z_2 of Sec. II-D): Z0 + (Z1 + Z2);     */
/*   x9: Z0 + (Z1 + (Z2 + (Z3 + Z4)))                                    */
/* sum64 != 0 is the "d" variant of Sec. IV-A: level sums and the final   */
/* combination in FP64, one rounding to FP32 at the end.                 */
/* mode 0 is the plain FP32 reference of Sec. II-C: Z <- FMA(x_l, y_l, Z) */
/* Matrices are row-major: A is m x k (lda), B is k x n (ldb), C m x n.   */
/* ------------------------------------------------------------------ */
static int mode_pieces(int mode) {
  switch (mode) {
    case 1: return 1;
    case 3: return 2;
    case 5: return 3; /* B's pieces; A has two (mode_pieces_a) */
    case 6: return 3;
    case 8: return 3;
    case 9: return 3;
    default: return 0;
  }
}

/* pieces of the left operand A (R25: x5 splits A in two) */
static int mode_pieces_a(int mode) { return mode == 5 ? 2 : mode_pieces(mode); }

/* is product (i,j) used by the mode (R6, R25) */
static int mode_uses(int mode, int i, int j) {
  switch (mode) {
    case 1: return i == 0 && j == 0;
    case 3: return i + j <= 1;
    case 5: return i <= 1 && i + j <= 2;
    case 6: return i + j <= 2;
    case 8: return i + j <= 3;
    case 9: return 1;
    default: return 0;
  }
}

/* Level sums and the smallest-first combination of Sec. II-D in FP32 from
 * the partial products Z[i][j] (those the mode does not use are zero):
 *   Z1 = Z01 + Z10,  Z2 = Z02 + (Z11 + Z20),  Z3 = Z12 + Z21,  Z4 = Z22;
 *   x1 = Z0;  x3 = Z0 + Z1;  x6 = Z0 + (Z1 + Z2);  x8 = Z0 + (Z1 + (Z2 + Z3));
 *   x9 = Z0 + (Z1 + (Z2 + (Z3 + Z4)));  x5 (R25) = Z0 + (Z1 + (Z02 + Z11)). */
static float combine_levels32(int mode, float Z[3][3]) {
  float Z0 = Z[0][0];
  float Z1 = Z[0][1] + Z[1][0];
  float Z2 = Z[0][2] + (Z[1][1] + Z[2][0]);
  float Z3 = Z[1][2] + Z[2][1];
  float Z4 = Z[2][2];
  switch (mode) {
    case 1: return Z0;
    case 3: return Z0 + Z1;
    case 5: return Z0 + (Z1 + (Z[0][2] + Z[1][1]));
    case 6: return Z0 + (Z1 + Z2);
    case 8: return Z0 + (Z1 + (Z2 + Z3));
    default: return Z0 + (Z1 + (Z2 + (Z3 + Z4)));
  }
}

/* Shared body: when Cd != NULL the "d" combination is written to Cd in FP64
 * without a final rounding (alpha, beta ignored); otherwise C (FP32) gets
 * alpha*z + beta*C (R13). */
static int gemm_body(int mode, int sum64, int64_t m, int64_t n, int64_t k, float alpha,
                     const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                     float* C, int64_t ldc, double* Cd, int64_t ldcd) {
  if (m < 0 || n < 0 || k < 0) return 1;
  if (m == 0 || n == 0) return 0;
  if (mode == 0) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) {
        float Z = 0.0f;
        for (int64_t l = 0; l < k; ++l) Z = fmaf(A[i * lda + l], B[l * ldb + j], Z);
        if (Cd) { Cd[i * ldcd + j] = Z; continue; }
        float t = alpha * Z;
        C[i * ldc + j] = (beta == 0.0f) ? t : fmaf(beta, C[i * ldc + j], t);
      }
    return 0;
  }
  int np = mode_pieces(mode), npa = mode_pieces_a(mode);
  if (np == 0) return 1;
  /* pieces, widened to FP32 (exact) */
  float* Ap = (float*)malloc(sizeof(float) * 3 * (size_t)(m * k + 1));
  float* Bp = (float*)malloc(sizeof(float) * 3 * (size_t)(k * n + 1));
  if (!Ap || !Bp) { free(Ap); free(Bp); return 2; }
  for (int64_t i = 0; i < m; ++i)
    for (int64_t l = 0; l < k; ++l) {
      uint16_t p[3];
      split_one(A[i * lda + l], &p[0], &p[1], &p[2]);
      for (int q = 0; q < 3; ++q)
        Ap[(size_t)q * m * k + i * k + l] = (q < npa) ? bf16_to_f32(p[q]) : 0.0f;
    }
  for (int64_t l = 0; l < k; ++l)
    for (int64_t j = 0; j < n; ++j) {
      uint16_t p[3];
      split_one(B[l * ldb + j], &p[0], &p[1], &p[2]);
      for (int q = 0; q < 3; ++q)
        Bp[(size_t)q * k * n + l * n + j] = (q < np) ? bf16_to_f32(p[q]) : 0.0f;
    }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      float Z[3][3] = {{0}};
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          if (!mode_uses(mode, a, b)) continue;
          const float* xa = Ap + (size_t)a * m * k + i * k;
          const float* yb = Bp + (size_t)b * k * n + j;
          float z = 0.0f;
          for (int64_t l = 0; l < k; ++l) z = fmaf(xa[l], yb[l * n], z);
          Z[a][b] = z;
        }
      if (!sum64) {
        float zr = combine_levels32(mode, Z);
        if (Cd) { Cd[i * ldcd + j] = zr; continue; }
        float t = alpha * zr;
        C[i * ldc + j] = (beta == 0.0f) ? t : fmaf(beta, C[i * ldc + j], t);
      } else {
        double Z0 = Z[0][0];
        double Z1 = (double)Z[0][1] + (double)Z[1][0];
        double Z2 = (double)Z[0][2] + ((double)Z[1][1] + (double)Z[2][0]);
        double Z3 = (double)Z[1][2] + (double)Z[2][1];
        double Z4 = Z[2][2];
        double zd;
        switch (mode) {
          case 1: zd = Z0; break;
          case 3: zd = Z0 + Z1; break;
          case 5: zd = Z0 + (Z1 + ((double)Z[0][2] + (double)Z[1][1])); break;
          case 6: zd = Z0 + (Z1 + Z2); break;
          case 8: zd = Z0 + (Z1 + (Z2 + Z3)); break;
          default: zd = Z0 + (Z1 + (Z2 + (Z3 + Z4))); break;
        }
        if (Cd) { Cd[i * ldcd + j] = zd; continue; }
        float t = alpha * (float)zd;
        C[i * ldc + j] = (beta == 0.0f) ? t : fmaf(beta, C[i * ldc + j], t);
      }
    }
  free(Ap);
  free(Bp);
  return 0;
}

int orc_gemm(int mode, int sum64, int64_t m, int64_t n, int64_t k, float alpha,
             const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
             float* C, int64_t ldc) {
  return gemm_body(mode, sum64, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, NULL, 0);
}

/* The "d" variant of Sec. IV-A with the final answer kept in FP64:
 * Cd = combination of the FP32 partial products, summed in FP64 when sum64. */
int orc_gemm_f64out(int mode, int sum64, int64_t m, int64_t n, int64_t k, const float* A,
                    int64_t lda, const float* B, int64_t ldb, double* Cd, int64_t ldcd) {
  return gemm_body(mode, sum64, m, n, k, 1.0f, A, lda, B, ldb, 0.0f, NULL, 0, Cd, ldcd);
}

/* The nine partial inner products Z^(i,j) of Sec. II-D for one pair of
 * vectors (x, y of length n), FP32 FMA accumulation, written to Z[3*i+j]. */
void orc_dot_partials(int64_t n, const float* x, const float* y, float* Z) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      float z = 0.0f;
      for (int64_t l = 0; l < n; ++l) {
        uint16_t px[3], py[3];
        split_one(x[l], &px[0], &px[1], &px[2]);
        split_one(y[l], &py[0], &py[1], &py[2]);
        z = fmaf(bf16_to_f32(px[a]), bf16_to_f32(py[b]), z);
      }
      Z[3 * a + b] = z;
    }
}

/* inner product x^T y by the mode's products (Sec. II-B..II-D); mode 0 is
 * the plain FP32 FMA loop of Sec. II-C. */
float orc_dot(int mode, int sum64, int64_t n, const float* x, const float* y) {
  float out = 0.0f;
  orc_gemm(mode, sum64, 1, 1, n, 1.0f, x, n, y, 1, 0.0f, &out, 1);
  return out;
}

/* ------------------------------------------------------------------ */
/* O5  FP64 reference product and |A||B| for selected rows of C.         */
/* C64[r, j] = sum_l A[i_r, l] B[l, j], Cabs = sum_l |A||B|, in FP64.     */
/* ------------------------------------------------------------------ */
void orc_dgemm_rows(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                    const float* A, int64_t lda, const float* B, int64_t ldb,
                    double* C64, double* Cabs) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r) {
    const float* a = A + rows[r] * lda;
    double* c = C64 + r * n;
    double* ca = Cabs + r * n;
    for (int64_t j = 0; j < n; ++j) { c[j] = 0.0; ca[j] = 0.0; }
    for (int64_t l = 0; l < k; ++l) {
      double al = a[l];
      const float* b = B + l * ldb;
      for (int64_t j = 0; j < n; ++j) {
        double bj = b[j];
        c[j] += al * bj;
        ca[j] += fabs(al * bj);
      }
    }
  }
}

/* ------------------------------------------------------------------ */
/* O6  LU with partial pivoting (the factorisation of LAPACK xGETRF).    */
/* Row-major A (n x n, lda).  ipiv[j] = 0-based row swapped with row j.  */
/* Pivot = first row index of the largest |a_ij| in the column.  The     */
/* return value is LAPACK's info: 0, or the 1-based index of the first   */
/* exactly zero pivot (the elimination still completes).                 */
/* ------------------------------------------------------------------ */
int orc_dgetrf(int64_t n, double* A, int64_t lda, int32_t* ipiv) {
  int info = 0;
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = j;
    double best = fabs(A[j * lda + j]);
    for (int64_t i = j + 1; i < n; ++i) {
      double v = fabs(A[i * lda + j]);
      if (v > best) { best = v; p = i; }
    }
    ipiv[j] = (int32_t)p;
    if (p != j)
      for (int64_t c = 0; c < n; ++c) {
        double t = A[j * lda + c]; A[j * lda + c] = A[p * lda + c]; A[p * lda + c] = t;
      }
    double piv = A[j * lda + j];
    if (piv == 0.0) { if (info == 0) info = (int)(j + 1); continue; }
    for (int64_t i = j + 1; i < n; ++i) A[i * lda + j] /= piv;
#pragma omp parallel for schedule(static) if (n - j > 256)
    for (int64_t i = j + 1; i < n; ++i) {
      double l = A[i * lda + j];
      if (l == 0.0) continue;
      for (int64_t c = j + 1; c < n; ++c) A[i * lda + c] -= l * A[j * lda + c];
    }
  }
  return info;
}

/* Solve with FP64 factors: x <- U^-1 L^-1 P b, nrhs columns, row-major b (ldb). */
void orc_dgetrs(int64_t n, int64_t nrhs, const double* LU, int64_t lda, const int32_t* ipiv,
                double* b, int64_t ldb) {
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = ipiv[j];
    if (p != j)
      for (int64_t c = 0; c < nrhs; ++c) {
        double t = b[j * ldb + c]; b[j * ldb + c] = b[p * ldb + c]; b[p * ldb + c] = t;
      }
  }
  for (int64_t c = 0; c < nrhs; ++c) {
    for (int64_t i = 0; i < n; ++i) {           /* L y = P b, L unit lower */
      double s = b[i * ldb + c];
      for (int64_t l = 0; l < i; ++l) s -= LU[i * lda + l] * b[l * ldb + c];
      b[i * ldb + c] = s;
    }
    for (int64_t i = n - 1; i >= 0; --i) {      /* U x = y */
      double s = b[i * ldb + c];
      for (int64_t l = i + 1; l < n; ++l) s -= LU[i * lda + l] * b[l * ldb + c];
      b[i * ldb + c] = s / LU[i * lda + i];
    }
  }
}

/* The LU of record for Sec. IV-A's "SGETRF based on triplets" (R12): the
 * plain unblocked right-looking LU with partial pivoting of an FP32 matrix,
 * in which every product of the trailing update is the mode's product.
 * Column j: the pivot is the first row of the largest |a_ij|, i >= j; the
 * whole rows j and p are swapped (ipiv[j] = p, 0-based); an exactly zero
 * pivot records info = j + 1 (the first one) and the column is skipped;
 * otherwise each multiplier is l_i = a_ij / a_jj (an IEEE FP32 division) and
 * every a_ic, i, c > j, becomes
 *   mode 0:   fmaf(-l_i, a_jc, a_ic)      (the FP32 FMA of Sec. II-C)
 *   mode N:   a_ic - z,  z = the mode's product of l_i and a_jc (one term of
 *             Sec. II-D: both factors split, the kept piece products, which
 *             are exact, summed by level and combined smallest first), the
 *             subtraction in FP32 (C = alpha Z + beta C with alpha = -1,
 *             beta = 1, reading R13).
 * No blocking, no reciprocal: the definition, not an implementation's
 * schedule.  Returns info, or -1 for an unknown mode. */
int orc_lu_plain(int mode, int64_t n, float* A, int64_t lda, int32_t* ipiv) {
  if (mode != 0 && mode_pieces(mode) == 0) return -1;
  const int npa = mode ? mode_pieces_a(mode) : 0, npb = mode ? mode_pieces(mode) : 0;
  float* lp = (float*)malloc(sizeof(float) * 3 * (size_t)(n + 1));
  float* up = (float*)malloc(sizeof(float) * 3 * (size_t)(n + 1));
  if (!lp || !up) { free(lp); free(up); return -1; }
  int info = 0;
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = j;
    float best = fabsf(A[j * lda + j]);
    for (int64_t i = j + 1; i < n; ++i) {
      float v = fabsf(A[i * lda + j]);
      if (v > best) { best = v; p = i; }
    }
    ipiv[j] = (int32_t)p;
    if (p != j)
      for (int64_t c = 0; c < n; ++c) {
        float t = A[j * lda + c]; A[j * lda + c] = A[p * lda + c]; A[p * lda + c] = t;
      }
    const float piv = A[j * lda + j];
    if (piv == 0.0f) { if (info == 0) info = (int)(j + 1); continue; }
    for (int64_t i = j + 1; i < n; ++i) A[i * lda + j] = A[i * lda + j] / piv;
    if (mode != 0) {
      /* pieces of the multipliers (left factor) and of row j (right factor) */
      for (int64_t i = j + 1; i < n; ++i) {
        uint16_t q[3];
        split_one(A[i * lda + j], &q[0], &q[1], &q[2]);
        for (int t = 0; t < 3; ++t) lp[3 * i + t] = (t < npa) ? bf16_to_f32(q[t]) : 0.0f;
      }
      for (int64_t c = j + 1; c < n; ++c) {
        uint16_t q[3];
        split_one(A[j * lda + c], &q[0], &q[1], &q[2]);
        for (int t = 0; t < 3; ++t) up[3 * c + t] = (t < npb) ? bf16_to_f32(q[t]) : 0.0f;
      }
    }
#pragma omp parallel for schedule(static) if (n - j > 128)
    for (int64_t i = j + 1; i < n; ++i) {
      const float l = A[i * lda + j];
      for (int64_t c = j + 1; c < n; ++c) {
        if (mode == 0) {
          A[i * lda + c] = fmaf(-l, A[j * lda + c], A[i * lda + c]);
          continue;
        }
        float Z[3][3] = {{0}};
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            if (mode_uses(mode, a, b)) Z[a][b] = lp[3 * i + a] * up[3 * c + b]; /* exact */
        A[i * lda + c] = A[i * lda + c] - combine_levels32(mode, Z);
      }
    }
  }
  free(lp);
  free(up);
  return info;
}

/* REGRESSION MIRROR, not the oracle of record: the blocked schedule the
 * device LU runs (tiles of 8 panel columns, multipliers by division,
 * rank-nb trailing updates), restated here so that a change of the
 * device's FP32 arithmetic shows up bit for bit.  Agreement with it says the
 * device still runs this schedule; agreement with the method is checked
 * against orc_lu_plain and orc_dgetrf. */
/* LU of an FP32 matrix with the combined type of Sec. IV-A (R12), blocked
 * like LAPACK's xGETRF (the routine the paper compares with): block columns
 * of width nb; inside a block column, the panel is itself blocked in tiles of
 * w columns (w = 8):
 *   tile    unblocked LU of the tile columns, partial pivoting (first row of
 *           the largest |a|), the whole row swapped, division by the pivot,
 *           FMA rank-1 updates of the remaining tile columns;
 *   rest of the block column: U rows of the tile by forward substitution with
 *           the tile's unit lower triangle, then the rows below updated by
 *           a <- fma(-l_rk, u_kc, a) for k over the tile columns in order;
 * then U12 = L11^-1 A12 (unit lower, FP32 FMA, row by row) and the trailing
 * update A22 <- A22 - L21 U12 as the mode's product (mode 0: the plain FP32
 * FMA product of Sec. II-C) with alpha = -1, beta = 1. */
int orc_lu(int mode, int64_t n, int64_t nb, float* A, int64_t lda, int32_t* ipiv) {
  const int64_t w = 8;
  if (nb <= 0) nb = 64;
  int info = 0;
  for (int64_t J0 = 0; J0 < n; J0 += nb) {
    int64_t JB = (n - J0 < nb) ? n - J0 : nb;
    for (int64_t j0 = J0; j0 < J0 + JB; j0 += w) {
      int64_t jw = (J0 + JB - j0 < w) ? J0 + JB - j0 : w;
      for (int64_t j = j0; j < j0 + jw; ++j) {
        int64_t p = j;
        float best = fabsf(A[j * lda + j]);
        for (int64_t i = j + 1; i < n; ++i) {
          float v = fabsf(A[i * lda + j]);
          if (v > best) { best = v; p = i; }
        }
        ipiv[j] = (int32_t)p;
        if (p != j)   /* whole row: the same as swapping panel, left and right parts */
          for (int64_t c = 0; c < n; ++c) {
            float t = A[j * lda + c]; A[j * lda + c] = A[p * lda + c]; A[p * lda + c] = t;
          }
        float piv = A[j * lda + j];
        if (piv == 0.0f) { if (info == 0) info = (int)(j + 1); continue; }
        for (int64_t i = j + 1; i < n; ++i) A[i * lda + j] = A[i * lda + j] / piv;
        for (int64_t i = j + 1; i < n; ++i) {
          float l = A[i * lda + j];
          for (int64_t c = j + 1; c < j0 + jw; ++c)
            A[i * lda + c] = fmaf(-l, A[j * lda + c], A[i * lda + c]);
        }
      }
      /* rest of the block column: tile rows by forward substitution ... */
      for (int64_t i = j0 + 1; i < j0 + jw; ++i)
        for (int64_t l = j0; l < i; ++l)
          for (int64_t c = j0 + jw; c < J0 + JB; ++c)
            A[i * lda + c] = fmaf(-A[i * lda + l], A[l * lda + c], A[i * lda + c]);
      /* ... and the rows below by the tile's rank-jw update */
      for (int64_t r = j0 + jw; r < n; ++r)
        for (int64_t c = j0 + jw; c < J0 + JB; ++c) {
          float a = A[r * lda + c];
          for (int64_t l = j0; l < j0 + jw; ++l) a = fmaf(-A[r * lda + l], A[l * lda + c], a);
          A[r * lda + c] = a;
        }
    }
    int64_t nr = n - J0 - JB;
    if (nr <= 0) continue;
    /* U12 = L11^-1 A12 (unit lower, forward substitution row by row) */
    for (int64_t i = J0 + 1; i < J0 + JB; ++i)
      for (int64_t l = J0; l < i; ++l) {
        float lil = A[i * lda + l];
        for (int64_t c = J0 + JB; c < n; ++c)
          A[i * lda + c] = fmaf(-lil, A[l * lda + c], A[i * lda + c]);
      }
    /* A22 <- A22 - L21 U12 */
    int rc = orc_gemm(mode, 0, nr, nr, JB, -1.0f, A + (J0 + JB) * lda + J0, lda,
                      A + J0 * lda + J0 + JB, lda, 1.0f, A + (J0 + JB) * lda + J0 + JB, lda);
    if (rc) return -rc;
  }
  return info;
}

/* Single-type LU (reading R26; the Sec. IV-B plain IR table): A (n x n,
 * row-major, lda) is overwritten by its factors, every stored value a value
 * of the type.  Column by column: the pivot is the first row of the largest
 * |a| at or below the diagonal; the whole rows are swapped; each multiplier
 * is a / pivot and each update a - l u, every operation in FP32 and rounded
 * to the type.  An exactly zero pivot column records info = k + 1 (the
 * first one) and is skipped, as LAPACK's xGETF2 does.  ipiv[k] = the row
 * swapped with row k (0-based).  Returns info. */
int orc_lu_lowp(int type, int64_t n, float* A, int64_t lda, int32_t* ipiv) {
  int info = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) A[i * lda + j] = round_to_type(type, A[i * lda + j]);
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = k;
    float amax = fabsf(A[k * lda + k]);
    for (int64_t i = k + 1; i < n; ++i)
      if (fabsf(A[i * lda + k]) > amax) {
        amax = fabsf(A[i * lda + k]);
        p = i;
      }
    ipiv[k] = (int32_t)p;
    if (amax == 0.0f) {
      if (!info) info = (int)(k + 1);
      continue;
    }
    if (p != k)
      for (int64_t j = 0; j < n; ++j) {
        float t = A[k * lda + j];
        A[k * lda + j] = A[p * lda + j];
        A[p * lda + j] = t;
      }
    const float piv = A[k * lda + k];
    for (int64_t i = k + 1; i < n; ++i) {
      const float l = round_to_type(type, A[i * lda + k] / piv);
      A[i * lda + k] = l;
      for (int64_t j = k + 1; j < n; ++j)
        A[i * lda + j] = round_to_type(type, A[i * lda + j] - round_to_type(type, l * A[k * lda + j]));
    }
  }
  return info;
}

/* ------------------------------------------------------------------ */
/* O7  residual-form iterative refinement (Sec. III, reading R9).        */
/* A32 (n x n, FP32, the problem matrix), b (n x nrhs, FP64), x (out).    */
/* LU (FP32 factors from orc_lu) and ipiv are given.  For each column:   */
/*   x <- LU^-1 b            (FP64 arithmetic with the FP32 factors)     */
/*   repeat: r = b - A x (FP64); d = LU^-1 r (FP64); x += d (FP64)        */
/*     stop, converged, when |d|_inf <= tol |x|_inf;                      */
/*     stop when |d| >= stall * |d_prev| (no more progress: the limiting  */
/*     accuracy is reached, or the factors are too inaccurate);           */
/*     stop after max_iter corrections.                                   */
/*   Finally r = b - A x; berr = |r|_inf / (|A|_inf |x|_inf + |b|_inf);    */
/*   converged also when the last stop was a stall with berr <= tol_b.    */
/* iters[c] = corrections applied after the first solve; conv[c] = 1/0.  */
/* ------------------------------------------------------------------ */
static void lu32_solve64(int64_t n, const float* LU, int64_t lda, const int32_t* ipiv,
                         double* v) {
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = ipiv[j];
    if (p != j) { double t = v[j]; v[j] = v[p]; v[p] = t; }
  }
  for (int64_t i = 0; i < n; ++i) {
    double s = v[i];
    for (int64_t l = 0; l < i; ++l) s -= (double)LU[i * lda + l] * v[l];
    v[i] = s;
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = v[i];
    for (int64_t l = i + 1; l < n; ++l) s -= (double)LU[i * lda + l] * v[l];
    v[i] = s / (double)LU[i * lda + i];
  }
}

/* R27: X = L^-1 (lower != 0: the unit lower factor) or X = U^-1 (the      */
/* upper factor) of the packed FP32 factors LU, FP64, n x n row-major with */
/* zeros outside the triangle.  Column c solves T x = e_c by substitution: */
/* forward x_i = [i == c] - sum_{l < i} L_il x_l, backward                 */
/* x_i = ([i == c] - sum_{l > i} U_il x_l) / U_ii, l in increasing order.   */
void orc_tri_inverse(int64_t n, const float* LU, int64_t lda, int lower, double* X) {
  double* x = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t c = 0; c < n; ++c) {
    if (lower) {
      for (int64_t i = 0; i < n; ++i) {
        double s = (i == c) ? 1.0 : 0.0;
        for (int64_t l = 0; l < i; ++l) s -= (double)LU[i * lda + l] * x[l];
        x[i] = s;
      }
    } else {
      for (int64_t i = n - 1; i >= 0; --i) {
        double s = (i == c) ? 1.0 : 0.0;
        for (int64_t l = i + 1; l < n; ++l) s -= (double)LU[i * lda + l] * x[l];
        x[i] = s / (double)LU[i * lda + i];
      }
    }
    for (int64_t i = 0; i < n; ++i) X[i * n + c] = x[i];
  }
  free(x);
}

/* M^-1 v through the inverses (R27): v <- X_U (X_L (P v)) */
static void inv_solve64(int64_t n, const double* XL, const double* XU, const int32_t* ipiv,
                        double* v) {
  double* t = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = ipiv[j];
    if (p != j) { double u = v[j]; v[j] = v[p]; v[p] = u; }
  }
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t l = 0; l <= i; ++l) s += XL[i * n + l] * v[l];
    t[i] = s;
  }
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t l = i; l < n; ++l) s += XU[i * n + l] * t[l];
    v[i] = s;
  }
  free(t);
}

void orc_solve_ir(int64_t n, int64_t nrhs, const float* A32, int64_t lda, const float* LU,
                  int64_t ldlu, const int32_t* ipiv, const double* b, int64_t ldb,
                  double* x, int64_t ldx, int max_iter, double tol, double tol_b, double stall,
                  int32_t* iters, int32_t* conv, double* berr_out) {
  double anorm = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t l = 0; l < n; ++l) s += fabs((double)A32[i * lda + l]);
    if (s > anorm) anorm = s;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < nrhs; ++c) {
    double* xv = (double*)malloc(sizeof(double) * (size_t)n);
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double bnorm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      xv[i] = b[i * ldb + c];
      if (fabs(b[i * ldb + c]) > bnorm) bnorm = fabs(b[i * ldb + c]);
    }
    lu32_solve64(n, LU, ldlu, ipiv, xv);
    double dprev = 0.0;
    for (int64_t i = 0; i < n; ++i) if (fabs(xv[i]) > dprev) dprev = fabs(xv[i]);
    int it = 0, ok = 0, stalled = 0;
    while (it < max_iter) {
      for (int64_t i = 0; i < n; ++i) {
        double s = b[i * ldb + c];
        for (int64_t l = 0; l < n; ++l) s -= (double)A32[i * lda + l] * xv[l];
        r[i] = s;
      }
      lu32_solve64(n, LU, ldlu, ipiv, r);
      double dn = 0.0, xn = 0.0;
      int bad = 0; /* a NaN or Inf entry: the max below would skip a NaN */
      for (int64_t i = 0; i < n; ++i) {
        xv[i] += r[i];
        if (!isfinite(r[i]) || !isfinite(xv[i])) bad = 1;
        if (fabs(r[i]) > dn) dn = fabs(r[i]);
        if (fabs(xv[i]) > xn) xn = fabs(xv[i]);
      }
      ++it;
      if (bad) break; /* diverged */
      if (dn <= tol * xn) { ok = 1; break; }
      if (dn >= stall * dprev) { stalled = 1; break; }
      dprev = dn;
    }
    double rn = 0.0, xn = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double s = b[i * ldb + c];
      for (int64_t l = 0; l < n; ++l) s -= (double)A32[i * lda + l] * xv[l];
      if (fabs(s) > rn) rn = fabs(s);
      if (fabs(xv[i]) > xn) xn = fabs(xv[i]);
    }
    double den = anorm * xn + bnorm;
    double berr = (den > 0.0) ? rn / den : 0.0;
    if (!(berr == berr)) berr = INFINITY;
    if (!ok && stalled && berr <= tol_b) ok = 1;
    for (int64_t i = 0; i < n; ++i) x[i * ldx + c] = xv[i];
    iters[c] = it;
    conv[c] = ok;
    if (berr_out) berr_out[c] = berr;
    free(xv);
    free(r);
  }
}

/* ------------------------------------------------------------------ */
/* O8  GMRES with the low-precision LU as preconditioner (Sec. III, the   */
/* GMRES remark, and the diagonally dominant table of Sec. IV-B).         */
/* Reading R18: the correction equation A d = r of each refinement step   */
/* is solved by left-preconditioned GMRES, M^-1 A d = M^-1 r with         */
/* M = P^T L U (the FP32 factors applied in FP64), zero first guess.      */
/* Arnoldi by modified Gram-Schmidt; the least-squares problem is         */
/* reduced by Givens rotations (the textbook GMRES).  A refinement step   */
/* with FP64 residual is a restart, so the whole is restarted GMRES(m)    */
/* with the residual recomputed from x at every restart.                  */
/* ------------------------------------------------------------------ */

/* d = (M^-1 A)^-1 M^-1 rhs approximately; returns k, the Arnoldi steps    */
/* taken.  M^-1 by substitution with the factors, or through the explicit  */
/* inverses XL, XU when XL != NULL (R27).                                   */
/* taken.  Stops when the residual estimate |g_k| <= tau * beta, after m  */
/* steps, or at breakdown (h_{k+1,k} = 0: the Krylov space is invariant   */
/* and the solution in it exact).  hist[j] = |g_{j+1}| if hist != NULL.   */
int orc_gmres(int64_t n, const float* A32, int64_t lda, const float* LU, int64_t ldlu,
              const int32_t* ipiv, const double* XL, const double* XU, const double* rhs, int m,
              double tau, double* d, double* hist) {
  double* V = (double*)calloc((size_t)(m + 1) * (size_t)n, sizeof(double));
  double* H = (double*)calloc((size_t)(m + 1) * (size_t)m, sizeof(double)); /* H[i*m+j] */
  double* cs = (double*)calloc((size_t)m + 1, sizeof(double));
  double* sn = (double*)calloc((size_t)m + 1, sizeof(double));
  double* g = (double*)calloc((size_t)m + 1, sizeof(double));
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) d[i] = 0.0;
  /* r0 = M^-1 rhs, beta = |r0|_2, v0 = r0 / beta */
  for (int64_t i = 0; i < n; ++i) w[i] = rhs[i];
  if (XL) inv_solve64(n, XL, XU, ipiv, w); else lu32_solve64(n, LU, ldlu, ipiv, w);
  double beta = 0.0;
  for (int64_t i = 0; i < n; ++i) beta += w[i] * w[i];
  beta = sqrt(beta);
  int k = 0;
  if (beta > 0.0 && beta == beta) {
    for (int64_t i = 0; i < n; ++i) V[i] = w[i] / beta;
    g[0] = beta;
    for (int j = 0; j < m; ++j) {
      /* w = M^-1 A v_j */
      const double* vj = V + (size_t)j * (size_t)n;
      for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t l = 0; l < n; ++l) s += (double)A32[i * lda + l] * vj[l];
        w[i] = s;
      }
      if (XL) inv_solve64(n, XL, XU, ipiv, w); else lu32_solve64(n, LU, ldlu, ipiv, w);
      /* modified Gram-Schmidt against v_0 .. v_j */
      for (int i = 0; i <= j; ++i) {
        const double* vi = V + (size_t)i * (size_t)n;
        double h = 0.0;
        for (int64_t l = 0; l < n; ++l) h += w[l] * vi[l];
        H[i * m + j] = h;
        for (int64_t l = 0; l < n; ++l) w[l] -= h * vi[l];
      }
      double hn = 0.0;
      for (int64_t l = 0; l < n; ++l) hn += w[l] * w[l];
      hn = sqrt(hn);
      H[(j + 1) * m + j] = hn;
      if (hn > 0.0)
        for (int64_t l = 0; l < n; ++l) V[(size_t)(j + 1) * (size_t)n + l] = w[l] / hn;
      /* earlier rotations on column j, then the one that zeroes h_{j+1,j} */
      for (int i = 0; i < j; ++i) {
        const double a = H[i * m + j], b = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * b;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
      }
      {
        const double a = H[j * m + j], b = H[(j + 1) * m + j];
        const double rho = hypot(a, b);
        cs[j] = (rho > 0.0) ? a / rho : 1.0;
        sn[j] = (rho > 0.0) ? b / rho : 0.0;
        H[j * m + j] = rho;
        H[(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
      }
      k = j + 1;
      if (hist) hist[j] = fabs(g[j + 1]);
      if (fabs(g[j + 1]) <= tau * beta || hn == 0.0 || !(hn == hn)) break;
    }
    /* y = R_k^-1 g_k (back substitution), d = V_k y */
    double* y = (double*)calloc((size_t)k + 1, sizeof(double));
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int l = i + 1; l < k; ++l) s -= H[i * m + l] * y[l];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i < k; ++i)
      for (int64_t l = 0; l < n; ++l) d[l] += y[i] * V[(size_t)i * (size_t)n + l];
    free(y);
  }
  free(V); free(H); free(cs); free(sn); free(g); free(w);
  return k;
}

/* GMRES-IR: x0 = M^-1 b, then refinement steps r = b - A x (FP64),        */
/* d = GMRES(m, tau) on M^-1 A d = M^-1 r, x += d, with the stop rules of  */
/* O7 (tol on |d|/|x|, the stall ratio, max_iter, the backward-error test), */
/* except that the first correction is not tested for a stall.              */
/* iters[c] = refinement steps; inner[c] = Arnoldi steps summed over them. */
void orc_solve_gmres_ir(int64_t n, int64_t nrhs, const float* A32, int64_t lda, const float* LU,
                        int64_t ldlu, const int32_t* ipiv, const double* b, int64_t ldb,
                        double* x, int64_t ldx, int max_iter, double tol, double tol_b,
                        double stall, int m, double tau, int explicit_inv, int32_t* iters,
                        int32_t* inner, int32_t* conv, double* berr_out) {
  double *XL = NULL, *XU = NULL;
  if (explicit_inv) { /* R27: the GMRES preconditioner through the inverses */
    XL = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n * n : 1));
    XU = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n * n : 1));
    orc_tri_inverse(n, LU, ldlu, 1, XL);
    orc_tri_inverse(n, LU, ldlu, 0, XU);
  }
  double anorm = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t l = 0; l < n; ++l) s += fabs((double)A32[i * lda + l]);
    if (s > anorm) anorm = s;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < nrhs; ++c) {
    double* xv = (double*)malloc(sizeof(double) * (size_t)n);
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* d = (double*)malloc(sizeof(double) * (size_t)n);
    double bnorm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      xv[i] = b[i * ldb + c];
      if (fabs(b[i * ldb + c]) > bnorm) bnorm = fabs(b[i * ldb + c]);
    }
    lu32_solve64(n, LU, ldlu, ipiv, xv);
    /* no stall test on the first correction: with poor factors x0 may be far */
    /* off, and the first GMRES correction is then as large as x0 itself      */
    double dprev = INFINITY;
    int it = 0, ok = 0, stalled = 0, kin = 0;
    while (it < max_iter) {
      for (int64_t i = 0; i < n; ++i) {
        double s = b[i * ldb + c];
        for (int64_t l = 0; l < n; ++l) s -= (double)A32[i * lda + l] * xv[l];
        r[i] = s;
      }
      kin += orc_gmres(n, A32, lda, LU, ldlu, ipiv, XL, XU, r, m, tau, d, NULL);
      double dn = 0.0, xn = 0.0;
      int bad = 0; /* a NaN or Inf entry: the max below would skip a NaN */
      for (int64_t i = 0; i < n; ++i) {
        xv[i] += d[i];
        if (!isfinite(d[i]) || !isfinite(xv[i])) bad = 1;
        if (fabs(d[i]) > dn) dn = fabs(d[i]);
        if (fabs(xv[i]) > xn) xn = fabs(xv[i]);
      }
      ++it;
      if (bad) break; /* diverged */
      if (dn <= tol * xn) { ok = 1; break; }
      if (dn >= stall * dprev) { stalled = 1; break; }
      dprev = dn;
    }
    double rn = 0.0, xn = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double s = b[i * ldb + c];
      for (int64_t l = 0; l < n; ++l) s -= (double)A32[i * lda + l] * xv[l];
      if (fabs(s) > rn) rn = fabs(s);
      if (fabs(xv[i]) > xn) xn = fabs(xv[i]);
    }
    double den = anorm * xn + bnorm;
    double berr = (den > 0.0) ? rn / den : 0.0;
    if (!(berr == berr)) berr = INFINITY;
    if (!ok && stalled && berr <= tol_b) ok = 1;
    for (int64_t i = 0; i < n; ++i) x[i * ldx + c] = xv[i];
    iters[c] = it;
    inner[c] = kin;
    conv[c] = ok;
    if (berr_out) berr_out[c] = berr;
    free(xv); free(r); free(d);
  }
  free(XL);
  free(XU);
}
