/*
 * bfx: FP32-accurate linear algebra assembled from bfloat16 pieces on the
 * B300 (sm_103a) tensor cores, after Henry, Tang & Heinecke, "Leveraging the
 * bfloat16 Artificial Intelligence Datatype For Higher-Precision
 * Computations" (ARITH 2019).
 *
 * C ABI.  Every pointer argument named d_* is a device pointer on the current
 * CUDA device; h_* pointers are host memory.  The caller owns every buffer:
 * the library never frees caller memory.  The compute calls (split, GEMM,
 * dot, LU, solves) allocate no device memory: their scratch space is a
 * caller-provided workspace whose size a *_workspace_size query returns.  Two
 * host-thread resources are created once and kept until the thread ends:
 * the LU's auxiliary stream and two events (on the thread's first LU call on
 * a device) and, for the GMRES phase of bfx_solve_ir, a small pinned,
 * device-mapped host ring of flags with its events.  The batch, autotune and server calls allocate as
 * each says.  Matrices are row-major with a leading dimension (elements
 * between the starts of consecutive rows).  bfloat16 values travel as their
 * 16-bit patterns in uint16_t.
 *
 * Calls are asynchronous on the given stream (a cudaStream_t passed as
 * bfx_stream; NULL is the legacy default stream), except where a call says
 * it is synchronous (bfx_solve_ir, which decides escalation and GMRES-IR on
 * the host; bfx_device_error; the autotuner; the server's wait).  For the
 * asynchronous calls the returned status only reports what is known at
 * launch: invalid arguments (BFX_EINVAL), a shape or device the kernels do
 * not support (BFX_EUNSUPPORTED), a workspace that is too small (BFX_ENOMEM)
 * or a CUDA launch error (BFX_ECUDA).  Outcomes computed on the device (a
 * zero pivot, non-convergence, a device-side wait that expired) are written
 * to device memory the caller reads after synchronising.
 *
 * There is no CPU fallback: every entry point runs its work in the library's
 * own sm_103a kernels.
 */
#ifndef BFX_H
#define BFX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define BFX_API __attribute__((visibility("default")))
#else
#define BFX_API
#endif

typedef void* bfx_stream; /* cudaStream_t */

typedef enum bfx_status {
  BFX_OK = 0,
  BFX_EINVAL = 1,         /* invalid argument (negative size, null pointer, ld too small) */
  BFX_ENOMEM = 2,         /* caller workspace too small */
  BFX_ECUDA = 3,          /* CUDA runtime / launch error */
  BFX_EUNSUPPORTED = 4,   /* valid but unsupported (alignment, device not sm_103) */
  BFX_SINGULAR = 5,       /* an exactly zero pivot (reported on the device via info) */
  BFX_NOT_CONVERGED = 6,  /* refinement stopped without converging (device-side result) */
  BFX_TIMEOUT = 7         /* a bounded device-side wait expired (device error word) */
} bfx_status;

/* Which products assemble a result (Sec. II-D, II-G of the paper):
 *   BFX_FP32 : no split; plain FP32 FMA accumulation (Sec. II-C), SIMT cores
 *   BFX_X1   : hi*hi                                    (one bfloat16 piece)
 *   BFX_X3   : + hi*mid + mid*hi                        (pair split, "bx2_3")
 *   BFX_X6   : + hi*lo + mid*mid + lo*hi                (triple split, "bx3_6")
 *   BFX_X8   : + mid*lo + lo*mid, the 2^-24 bin Z3      (triple split; Sec. II-D's
 *              Z0 + (Z1 + (Z2 + Z3)), "might offer higher accuracy than FP32")
 *   BFX_X9   : all nine products                       (triple split)
 *   BFX_X5   : A split in two pieces, B in three: hi*hi, hi*mid, mid*hi,
 *              hi*lo, mid*mid (Sec. II-G's asymmetric case).  GEMM entry
 *              points only (bfx_gemm_bf16xN, bfx_gemm_presplit,
 *              bfx_gemm_bf16xN_f64, bfx_gemm_bf16xN_noalloc); the others
 *              return BFX_EINVAL.  Its
 *              accuracy is bounded by A's dropped third piece (~2^-16 |a|),
 *              as for X3, unless A has at most 16 significant bits.
 * The mode's value is the number of bfloat16 products per scalar product. */
typedef enum bfx_mode {
  BFX_FP32 = 0,
  BFX_X1 = 1,
  BFX_X3 = 3,
  BFX_X5 = 5,
  BFX_X6 = 6,
  BFX_X8 = 8,
  BFX_X9 = 9
} bfx_mode;

/* Library version (major*10000 + minor*100 + patch). */
BFX_API int bfx_version(void);

/* Static text for a status code; never NULL. */
BFX_API const char* bfx_status_string(bfx_status s);

/* Number of SMs of the current device, or -1 on error. */
BFX_API int bfx_num_sms(void);

/* Read and clear the device error word of the current device.  Kernels whose
 * waits are bounded (tensor-core GEMM pipeline barriers, the refinement's
 * triangular solves waiting on earlier row blocks, the LU panel's pivot
 * exchange between the CTAs of a cluster, the batched GMRES-IR's exchanges
 * between the two CTAs of a hard system) set it instead of hanging: 0 = no
 * error, otherwise a code naming the wait that expired (1-5 GEMM pipeline,
 * 6 triangular solve, 7 LU panel, 8 batched GMRES-IR).
 * Synchronises `stream`.  h_code: host int (output). */
BFX_API bfx_status bfx_device_error(int* h_code, bfx_stream stream);

/* ---------------------------------------------------------------------------
 * Split (Sec. II-A).  For each FP32 element a of the rows x cols matrix d_x:
 *   hi  = (B16) a
 *   mid = (B16)((F32)(a - hi))
 *   lo  = (B16)((F32)(a - hi - mid))
 * with (B16) round-to-nearest-even.  For every finite |a| >= 2^-110 (and 0)
 * the pieces sum exactly to a (Sec. II-F).  Edge readings: a finite value whose
 * rounding would overflow to infinity gets hi = a truncated toward zero;
 * Inf/NaN go to hi (NaN made quiet, sign kept) with mid = lo = +0.
 * npieces: 1 (hi), 2 (hi, mid) or 3 (hi, mid, lo); unused piece pointers may
 * be NULL.  Output planes share the leading dimension ldp (>= cols).
 * Errors: BFX_EINVAL for rows/cols < 0, npieces outside 1..3, ld too small or
 * a required pointer NULL. */
BFX_API bfx_status bfx_split(int64_t rows, int64_t cols, const float* d_x, int64_t ldx, int npieces,
                             uint16_t* d_hi, uint16_t* d_mid, uint16_t* d_lo, int64_t ldp,
                             bfx_stream stream);

/* Same split, written transposed: piece planes are cols x rows with leading
 * dimension ldp (>= rows).  Lays a row-major right-hand operand out with its
 * contraction index contiguous.  Errors as bfx_split. */
BFX_API bfx_status bfx_split_transpose(int64_t rows, int64_t cols, const float* d_x, int64_t ldx,
                                       int npieces, uint16_t* d_hi, uint16_t* d_mid,
                                       uint16_t* d_lo, int64_t ldp, bfx_stream stream);

/* Both operands of a product C = A B in one launch: A (rows_a x cols_a, lda)
 * split as bfx_split into planes a0..a2 (leading dimension ldpa), B (rows_b x
 * cols_b, ldb) split as bfx_split_transpose into planes b0..b2 (ldpb).  The
 * same pieces as the two calls; one kernel when A's rows are contiguous
 * (lda == ldpa == cols_a, cols_a a multiple of 8, 16-byte aligned) and B's
 * planes are 16-byte aligned with ldpb a multiple of 8, so the two passes
 * overlap; otherwise the two kernels in turn.  Errors as bfx_split. */
BFX_API bfx_status bfx_split_pair(int64_t rows_a, int64_t cols_a, const float* d_a, int64_t lda,
                                  int npa, uint16_t* d_a0, uint16_t* d_a1, uint16_t* d_a2,
                                  int64_t ldpa, int64_t rows_b, int64_t cols_b, const float* d_b,
                                  int64_t ldb, int npb, uint16_t* d_b0, uint16_t* d_b1,
                                  uint16_t* d_b2, int64_t ldpb, bfx_stream stream);

/* ---------------------------------------------------------------------------
 * GEMM C = alpha * (A B) + beta * C from FP32 A (m x k, lda) and B (k x n, ldb)
 * by the mode's bfloat16 products (Sec. II-D, II-G; Sec. IV-A: a GEMM that
 * starts from FP32 data and converts it to one to three bfloat16 matrices
 * behind the scenes).  The products run on the tcgen05 tensor cores with FP32
 * accumulation in tensor memory; the hi*hi product is accumulated apart from
 * the correction products, which are issued smallest bin first, and the two
 * are added in FP32 in the epilogue (for X6, X8 and X9 with k > 512 the
 * hi*hi accumulator restarts every 256 of k and its chunk sums are added in
 * FP32 registers with round-to-nearest adds).  Then t = alpha * Z and
 * C = beta == 0 ? t : fma(beta, C, t) (C is not read when beta == 0).
 * mode BFX_FP32 runs the plain FP32 SIMT GEMM instead (no workspace).
 * Workspace: d_ws of ws_bytes >= bfx_gemm_workspace_size(mode, m, n, k), 256-
 * byte aligned; it holds the pieces.  Errors: BFX_EINVAL (sizes, ld, pointers,
 * mode), BFX_ENOMEM (workspace too small), BFX_EUNSUPPORTED (device not sm_103,
 * or a dimension >= 2^31). */
BFX_API size_t bfx_gemm_workspace_size(bfx_mode mode, int64_t m, int64_t n, int64_t k);
BFX_API bfx_status bfx_gemm_bf16xN(bfx_mode mode, int64_t m, int64_t n, int64_t k, float alpha,
                                   const float* d_A, int64_t lda, const float* d_B, int64_t ldb,
                                   float beta, float* d_C, int64_t ldc, void* d_ws,
                                   size_t ws_bytes, bfx_stream stream);

/* The same GEMM with the split fused into the kernel (Sec. V: the conversion
 * "can be hidden"): the FP32 tiles of A and B are loaded by TMA and split in
 * registers into the bfloat16 pieces the tensor cores read, so no workspace is
 * needed and no pieces go through global memory.  Same result as
 * bfx_gemm_bf16xN bit for bit (same pieces, same products in the same order)
 * for k <= 512 and for modes X1, X3 and X5; for X6, X8 and X9 beyond k = 512
 * it keeps one hi*hi accumulator over all of k and meets the same bound.
 * Requirements of the TMA descriptors: lda and ldb multiples of 4, d_A and
 * d_B 16-byte aligned; otherwise BFX_EUNSUPPORTED.  mode must be X1..X9
 * (BFX_EINVAL).  Other errors as bfx_gemm_bf16xN. */
BFX_API bfx_status bfx_gemm_bf16xN_fused(bfx_mode mode, int64_t m, int64_t n, int64_t k,
                                         float alpha, const float* d_A, int64_t lda,
                                         const float* d_B, int64_t ldb, float beta, float* d_C,
                                         int64_t ldc, bfx_stream stream);

/* GEMM from pieces already split.  d_Ap: npieces(mode) planes of m x k
 * bfloat16 (row-major, leading dimension lda_p, plane p at d_Ap + p*a_plane),
 * d_Btp: npieces planes of the TRANSPOSED right operand, n x k (leading
 * dimension ldb_p, plane stride b_plane), e.g. from bfx_split /
 * bfx_split_transpose.  npieces(mode) = 1, 2, 3, 3, 3 for X1, X3, X6, X8, X9;
 * X5 reads 2 planes of A and 3 of B.
 * Requirements of the tensor-memory-access (TMA) descriptors: lda_p, ldb_p,
 * a_plane and b_plane multiples of 8 elements, both base pointers 16-byte
 * aligned; otherwise BFX_EUNSUPPORTED.  mode must be X1..X9 (BFX_EINVAL). */
BFX_API bfx_status bfx_gemm_presplit(bfx_mode mode, int64_t m, int64_t n, int64_t k, float alpha,
                                     const uint16_t* d_Ap, int64_t lda_p, int64_t a_plane,
                                     const uint16_t* d_Btp, int64_t ldb_p, int64_t b_plane,
                                     float beta, float* d_C, int64_t ldc, bfx_stream stream);

/* The "d" variant of Sec. IV-A: the same bfloat16 products, each accumulated
 * in FP32 in its own tensor-memory accumulator, then added together in FP64
 * in Sec. II-D's order, smallest level first (Z1 = Z01 + Z10,
 * Z2 = Z02 + (Z11 + Z20), Z3 = Z12 + Z21, Z4 = Z22,
 * C = Z0 + (Z1 + (Z2 + (Z3 + Z4))), the levels the mode has), and stored in
 * FP64 without a final rounding to FP32: C = A B (no alpha, beta).
 * d_C: m x n FP64, row-major, leading dimension ldc (>= n).  mode: X1, X3,
 * X5, X6, X8, X9 (else BFX_EINVAL; FP32 has no pieces).  k must be >= 1.
 * Workspace as bfx_gemm_bf16xN (bfx_gemm_workspace_size).  Errors as
 * bfx_gemm_bf16xN. */
BFX_API bfx_status bfx_gemm_bf16xN_f64(bfx_mode mode, int64_t m, int64_t n, int64_t k,
                                       const float* d_A, int64_t lda, const float* d_B,
                                       int64_t ldb, double* d_C, int64_t ldc, void* d_ws,
                                       size_t ws_bytes, bfx_stream stream);

/* ---------------------------------------------------------------------------
 * Single-type LU with refinement (the plain IR table of Sec. IV-B: FP32
 * factors against factors computed entirely in one bfloat16 or one binary16
 * type), for `count` independent n x n systems, one warp each.
 * LU: A rounded to the type; unblocked right-looking LU with partial
 * pivoting (first row of the largest |a|, whole rows swapped); every
 * division, product and difference done in FP32 (IEEE, no contraction) and
 * rounded to the type (round to nearest even); an exactly zero pivot column
 * sets info to its 1-based index (the first one) and is skipped.
 * Refinement (Sec. III, FP64): x = (LU)^-1 P b, then up to max_iter times
 * r = b - A x, d = (LU)^-1 P r, x += d; converged when |d|_inf <= tol[s]
 * |x|_inf (the paper's "residual tolerance of cond(A)*eps": pass cond(A)
 * 2^-53); stopped unconverged at the first NaN or Inf entry.  All sums run
 * in a fixed sequential order, so results are reproducible bit for bit.
 * d_A: count x n x n FP32, row-major, systems back to back; d_b, d_x: count
 * x n FP64; d_tol: count FP64.  Outputs (device, caller-owned): d_x, d_iters
 * (corrections applied after the first solve), d_conv (1/0), d_info; d_LU
 * (count x n x n FP32 words holding the type's values) and d_ipiv (count x n,
 * 0-based, row swapped with row k) may be NULL.  1 <= n <= 128 (else
 * BFX_EUNSUPPORTED), count >= 0, max_iter >= 0 (BFX_EINVAL). */
typedef enum bfx_lowp {
  BFX_LOWP_FP32 = 0,
  BFX_LOWP_BF16 = 1,
  BFX_LOWP_FP16 = 2
} bfx_lowp;
BFX_API bfx_status bfx_lowp_lu_ir_batched(bfx_lowp type, int count, int n, const float* d_A,
                                          const double* d_b, const double* d_tol, int max_iter,
                                          double* d_x, float* d_LU, int32_t* d_ipiv,
                                          int32_t* d_iters, int32_t* d_conv, int32_t* d_info,
                                          bfx_stream stream);

/* Workspace-free variant of bfx_gemm_bf16xN (same arguments minus the
 * workspace, same result).  The paper has no counterpart: this exists for
 * callers that cannot allocate device memory, e.g. a plugin inside a host
 * application that owns all device memory through its own pool and forbids
 * libraries from calling cudaMalloc, or a latency-critical loop where an
 * allocation is not acceptable.  The bfloat16 pieces go to a fixed 32 MiB
 * device array inside the library; the call allocates nothing.  The array is
 * reserved on a device when the library's module is loaded there (with lazy
 * module loading, at the first launch of any of the library's kernels on
 * that device), so every process using the library holds 32 MiB on each
 * device it uses until it exits.  Limit: the pieces need
 * 2 * (npa * round_up(m*kp,128) + npb * round_up(n*kp,128)) bytes, kp = k
 * rounded up to 8, with (npa, npb) = (1, 1) for X1, (2, 2) for X3, (2, 3)
 * for X5 and (3, 3) for X6, X8, X9 (e.g. x6 fits m = n = k = 1536); larger
 * problems return BFX_ENOMEM before anything is launched.  Accepted modes:
 * X1, X3, X5, X6, X8, X9; BFX_FP32 (which bfx_gemm_bf16xN sends to the SIMT
 * GEMM) and any other value return BFX_EINVAL.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the one
 * array: calls whose work overlaps on the GPU (other streams, other host
 * threads on the same device) race on it and must be serialised.  Other
 * errors as bfx_gemm_bf16xN. */
BFX_API bfx_status bfx_gemm_bf16xN_noalloc(bfx_mode mode, int64_t m, int64_t n, int64_t k,
                                           float alpha, const float* d_A, int64_t lda,
                                           const float* d_B, int64_t ldb, float beta, float* d_C,
                                           int64_t ldc, bfx_stream stream);

/* Measured arithmetic peak of the CUDA cores: a kernel of independent FMA
 * chains (8 a thread, a full wave of CTAs on every SM), timed with CUDA
 * events on `stream`; fp64 = 0 FFMA (FP32), 1 DFMA (FP64).  The FP32 figure
 * is the roofline denominator of the FP32 SIMT baseline.  *h_tflops
 * receives TFLOP/s (2 per FMA).  Synchronous.  Errors: BFX_EINVAL (h_tflops
 * NULL), BFX_ECUDA. */
BFX_API bfx_status bfx_measure_fma_peak(int fp64, double* h_tflops, bfx_stream stream);

/* Plain FP32 SIMT GEMM (the Sec. II-C reference computation on CUDA cores;
 * the same-GPU baseline).  Each C element is accumulated with one FMA per k
 * in increasing k, then t = alpha*Z, C = beta == 0 ? t : fma(beta, C, t).
 * Errors: BFX_EINVAL (sizes, ld, pointers). */
BFX_API bfx_status bfx_sgemm_simt(int64_t m, int64_t n, int64_t k, float alpha, const float* d_A,
                                  int64_t lda, const float* d_B, int64_t ldb, float beta,
                                  float* d_C, int64_t ldc, bfx_stream stream);

/* ---------------------------------------------------------------------------
 * Inner product x^T y of two FP32 vectors of length n (contiguous) by the
 * mode's bfloat16 products (Sec. II-B..II-G): each element pair is split,
 * every kept product is accumulated with FMA into the FP32 accumulator of its
 * level i+j, levels are reduced in a fixed tree and combined smallest first.
 * BFX_FP32 accumulates plain FMAs (Sec. II-C).  The FP32 result goes to
 * device memory d_result.  Workspace: d_ws (16-byte aligned) of at least
 * bfx_dot_workspace_size() bytes (per-block partial sums; depends on the
 * current device's SM count).  Errors: BFX_EINVAL, BFX_ENOMEM. */
BFX_API size_t bfx_dot_workspace_size(void);
BFX_API bfx_status bfx_dot_bf16xN(bfx_mode mode, int64_t n, const float* d_x, const float* d_y,
                                  float* d_result, void* d_ws, size_t ws_bytes, bfx_stream stream);

/* ---------------------------------------------------------------------------
 * LU with partial pivoting (LAPACK xGETRF semantics) of the n x n FP32 matrix
 * d_A (row-major, lda), in place: unit-lower L below the diagonal, U on and
 * above it.  Blocked right-looking with block width nb (0 = 64, at most 128):
 * the panel (warp-shuffle argmax pivot search, first row on ties), the row
 * swaps and the unit-lower block solve are FP32; the trailing update
 * A22 <- A22 - L21 U12 is the mode's bf16xN product on the tensor cores
 * (Sec. IV-A, "SGETRF based on triplets"), or the FP32 SIMT GEMM for
 * BFX_FP32.  d_ipiv[j] (int32, 0-based) is the row swapped with row j at
 * step j.  d_info (device int32) receives 0 or the 1-based index of the first
 * exactly zero pivot; the factorisation completes either way.  Workspace:
 * bfx_lu_workspace_size(mode, n, nb) bytes, 256-byte aligned (the bfloat16
 * pieces of the trailing update for X1..X9; 0 bytes for BFX_FP32, when d_ws
 * may be NULL).  Errors: BFX_EINVAL, BFX_ENOMEM, BFX_EUNSUPPORTED. */
BFX_API size_t bfx_lu_workspace_size(bfx_mode mode, int64_t n, int nb);
BFX_API bfx_status bfx_lu_bf16xN(bfx_mode mode, int64_t n, int nb, float* d_A, int64_t lda,
                                 int32_t* d_ipiv, int32_t* d_info, void* d_ws, size_t ws_bytes,
                                 bfx_stream stream);

/* ---------------------------------------------------------------------------
 * Solve A x = b by residual-form iterative refinement (Sec. III): A32 is
 * factored by bfx_lu_bf16xN (FP32 factors, bf16xN trailing updates); then
 * r = b - A32 x in FP64, d = U^-1 L^-1 P r in FP64 arithmetic with the FP32
 * factors, x += d in FP64.  A column converges when |d|_inf <= tol |x|_inf,
 * or when its corrections stop shrinking (|d_i| >= stall |d_{i-1}|) with
 * normwise backward error |r|_inf/(|A|_inf |x|_inf + |b|_inf) <= tol_b.
 * With escalate != 0, columns that stop unconverged are refined further after
 * refactoring with more products (x1 -> x3 -> x6).
 * GMRES-IR (the GMRES remark of Sec. III, the GMRES table of Sec. IV-B): with
 * gmres != 0 the correction of a refinement step is instead computed by
 * left-preconditioned GMRES in FP64, M^-1 A d = M^-1 r with M = P^T L U from
 * the FP32 factors, zero first guess, at most gmres_m Arnoldi steps, ending
 * early when the preconditioned residual has fallen by gmres_tol.  gmres = 1:
 * after plain refinement has stopped unconverged at the final mode (after any
 * escalation), the unconverged columns continue from their current x by
 * GMRES-IR; gmres = 2: GMRES-IR from the first correction.  The first GMRES
 * correction is not tested for a stall.  The same stop rules apply otherwise.
 * d_A: n x n FP32 (lda); d_b: n x nrhs FP64 (ldb); d_x: n x nrhs FP64 (ldx,
 * output).  h_params may be NULL (max_iter 50, tol 2^-53, tol_b sqrt(n) 2^-53,
 * stall 0.5, escalate 1, nb 64, gmres 1, gmres_m 0, gmres_tol 1e-10,
 * gmres_inverses 1); a
 * zero gmres_m means min(n, BFX_GMRES_MAX_M) (full GMRES up to that size:
 * factors of FP32 precision leave about as many poorly approximated
 * directions as A has singular values below ~2^-24 |A|, and a restart before
 * they are all captured stagnates), a gmres_tol <= 0 means 1e-10; max_iter bounds the
 * refinement steps of each phase (each factorisation, then GMRES-IR).
 * The call is synchronous: it returns after the refinement has finished and
 * fills *h_result (host).  Returns BFX_OK when every column converged,
 * BFX_NOT_CONVERGED otherwise (x holds the last iterate), BFX_SINGULAR on an
 * exactly zero pivot (h_result->info > 0), BFX_EINVAL for gmres outside 0..2
 * or gmres_m outside 0..BFX_GMRES_MAX_M, and the usual argument / workspace
 * errors.  Workspace: bfx_solve_ir_workspace_size(mode, n, nrhs, h_params)
 * bytes (h_params NULL: the defaults), 256-byte aligned; with gmres != 0 it
 * includes the Krylov basis, (gmres_m + 1) n nrhs doubles, the
 * Hessenberg matrices, nrhs (gmres_m + 1) gmres_m doubles, and the prepared
 * preconditioner, about n^2 doubles (both triangles; built once per
 * factorisation when the GMRES phase starts).  The preconditioner is the
 * same operator in both forms, up to FP64 rounding: gmres_inverses = 1 forms
 * L^-1 and U^-1 of the FP32 factors in FP64 (n^3/3 FP64 FMAs) so that each
 * application is two matrix-vector products (the fastest single solve when
 * the GMRES phase runs hundreds of Arnoldi steps or more); gmres_inverses = 0
 * folds each diagonal block's inverse into the factor blocks (about n^3/64
 * FMAs) and solves by row blocks in solve order (slower per application,
 * but the least FP64 work: the choice for many concurrent solves). */
#define BFX_GMRES_MAX_M 4096
typedef struct bfx_ir_params {
  int max_iter;
  double tol;
  double tol_b;   /* < 0: sqrt(n) * 2^-53 */
  double stall;
  int escalate;
  int nb;
  int gmres;        /* 0 off, 1 after plain refinement stalls, 2 always */
  int gmres_m;      /* Arnoldi steps per refinement step (0: min(n, BFX_GMRES_MAX_M)) */
  double gmres_tol; /* relative residual reduction ending a GMRES cycle (<= 0: 1e-10) */
  int gmres_inverses; /* M^-1 in GMRES: 1 explicit FP64 inverses of the factors, 0 row-sliced
                         block substitution (see below) */
} bfx_ir_params;
typedef struct bfx_ir_result {
  int32_t info;             /* first zero pivot (1-based) or 0 */
  int32_t mode_used;        /* mode of the final factorisation */
  int32_t converged;        /* 1 if every column converged */
  int32_t iters;            /* most corrections applied to any column */
  int32_t refactorizations; /* escalations performed */
  double berr;              /* largest normwise backward error over the columns */
  int32_t gmres_steps;      /* refinement steps whose correction came from GMRES */
  int32_t arnoldi;          /* Arnoldi steps run, summed over those refinement steps */
} bfx_ir_result;
BFX_API size_t bfx_solve_ir_workspace_size(bfx_mode mode, int64_t n, int64_t nrhs,
                                           const bfx_ir_params* h_params);
BFX_API bfx_status bfx_solve_ir(bfx_mode mode, int64_t n, int64_t nrhs, const float* d_A,
                                int64_t lda, const double* d_b, int64_t ldb, double* d_x,
                                int64_t ldx, const bfx_ir_params* h_params,
                                bfx_ir_result* h_result, void* d_ws, size_t ws_bytes,
                                bfx_stream stream);

/* The same solve, asynchronous: every step is enqueued on `stream` and the
 * result goes to device memory, so solves can be chained on a stream (or
 * captured) without the host reading anything back.  It runs the plain
 * refinement of bfx_solve_ir with the given mode, the same kernels in the
 * same order, and makes the stop decisions on the device: x and the result
 * equal bfx_solve_ir's with escalate = 0 and gmres = 0.  Exactly max_iter
 * refinement steps are enqueued; once every column has stopped, the later
 * ones return at once.  h_params as bfx_solve_ir, except that escalate and
 * gmres must be 0 (BFX_EINVAL otherwise: both need host decisions); NULL
 * means the defaults with escalate = gmres = 0.  d_result (device,
 * caller-owned) receives the bfx_ir_result when the stream reaches the end
 * of the solve: info > 0 is an exactly zero pivot (x is then not written),
 * converged = 0 a solve that did not converge (x holds the last iterate).
 * Workspace: bfx_solve_ir_workspace_size(mode, n, nrhs, params) with the
 * same params.  Returns only launch-time errors (BFX_EINVAL, BFX_ENOMEM,
 * BFX_EUNSUPPORTED, BFX_ECUDA); n and nrhs must be >= 1. */
BFX_API bfx_status bfx_solve_ir_async(bfx_mode mode, int64_t n, int64_t nrhs, const float* d_A,
                                      int64_t lda, const double* d_b, int64_t ldb, double* d_x,
                                      int64_t ldx, const bfx_ir_params* h_params,
                                      bfx_ir_result* d_result, void* d_ws, size_t ws_bytes,
                                      bfx_stream stream);

/* ---------------------------------------------------------------------------
 * Batched solves: many independent systems A_s x_s = b_s of uneven sizes
 * (1 <= n_s <= 1024, the same nrhs <= 16 for all), each by the bf16xN-update
 * LU and residual-form refinement of bfx_solve_ir, all systems together: every
 * block-column step of every system's LU runs in one launch per kernel
 * (panel tiles, row swaps and block solves one CTA per system; the trailing
 * updates of all systems in one grouped tcgen05 GEMM), then the refinement
 * runs with per-system stop decisions made on the device.  The whole sequence
 * is captured once into a CUDA graph per set of buffers and replayed.
 * Packed layout, systems in the caller's order: A at offset sum_{t<s} n_t^2
 * (n_s x n_s row-major, FP32); b and x at offset sum_{t<s} n_t nrhs (n_s x
 * nrhs row-major, FP64).
 * bfx_batch_create plans the batch (host memory only); params may be NULL
 * (as bfx_solve_ir; escalate is ignored: a batch keeps its mode).  With
 * gmres != 0 (the default) systems whose plain refinement stops unconverged
 * continue by GMRES-IR, each in one CTA of a persistent grid that takes them
 * from a queue: restarted GMRES(min(n, 256)), at most 20 refinement steps,
 * inner tolerance 1e-10 (d_status.gmres_steps counts its steps).
 * bfx_batch_solve enqueues the graph on `stream` and returns without
 * waiting; d_status (device, one entry per system, caller order) is written
 * at the end: converged, corrections applied, LAPACK info, backward error.
 * The first call with a new set of buffers captures and instantiates the
 * graph (do not call it while `stream` is being captured).
 * Workspace: bfx_batch_workspace_size(plan) bytes, 256-byte aligned.
 * Errors: BFX_EINVAL (sizes, mode FP32, pointers), BFX_ENOMEM,
 * BFX_EUNSUPPORTED (device), BFX_ECUDA. */
typedef struct bfx_batch_status {
  int32_t converged;
  int32_t iters;       /* refinement steps, plain and GMRES-IR */
  int32_t info;
  int32_t gmres_steps; /* of which GMRES-IR refinement steps */
  double berr;
} bfx_batch_status;
typedef struct bfx_batch_plan* bfx_batch;
BFX_API bfx_status bfx_batch_create(bfx_batch* out, bfx_mode mode, int count, const int32_t* h_n,
                                    int nrhs, const bfx_ir_params* params);
/* Tile shapes of a batch: nb = block-column width of the LU (32, 64 or 128;
 * also the K of every grouped trailing update), gemm_bn = N width of the
 * grouped tensor-core tiles (64, 128 or 256); 0 = default (64, 256).
 * bfx_batch_create is bfx_batch_create_config with config NULL.  The shape
 * changes the blocking (so the rounding) of the factorisation, not the
 * method.  BFX_EINVAL for other values. */
typedef struct bfx_batch_config {
  int nb;
  int gemm_bn;
} bfx_batch_config;
BFX_API bfx_status bfx_batch_create_config(bfx_batch* out, bfx_mode mode, int count,
                                           const int32_t* h_n, int nrhs,
                                           const bfx_ir_params* params,
                                           const bfx_batch_config* config);
BFX_API bfx_status bfx_batch_get_config(bfx_batch plan, bfx_batch_config* out);
/* Autotuner: solves the caller's batch (packed d_A, d_b as for
 * bfx_batch_solve) under each of the 9 shapes nb x gemm_bn, each as the
 * captured graph the batch replays: one untimed solve, then `reps` timed with
 * CUDA events on `stream` (median).  Workspaces are allocated with cudaMalloc
 * and freed per shape; a shape whose workspace does not fit is skipped
 * (BFX_ENOMEM in its table entry).  d_x and d_status are overwritten.
 * Returns the fastest shape in *h_best (and its median ms in *h_best_ms if
 * not NULL); if h_table_len is not NULL, up to *h_table_len entries (one per
 * shape: shape, median ms or -1, status) go to h_table and *h_table_len is
 * set to the number of shapes tried.  The result is also remembered for the
 * process under a coarse signature of the batch (mode, nrhs, max_iter,
 * count to two digits, the size histogram in bins of 128 to 1/20), which
 * bfx_batch_tuned_config looks up (BFX_EINVAL if absent).  Synchronous.
 * Errors: BFX_EINVAL (arguments, or the batch itself), BFX_ENOMEM (no shape
 * fits), BFX_ECUDA. */
typedef struct bfx_tune_entry {
  bfx_batch_config config;
  float ms;
  int32_t status;
} bfx_tune_entry;
BFX_API bfx_status bfx_batch_autotune(bfx_mode mode, int count, const int32_t* h_n, int nrhs,
                                      const bfx_ir_params* params, const float* d_A,
                                      const double* d_b, double* d_x,
                                      bfx_batch_status* d_status, int reps, bfx_stream stream,
                                      bfx_batch_config* h_best, float* h_best_ms,
                                      bfx_tune_entry* h_table, int* h_table_len);
BFX_API bfx_status bfx_batch_tuned_config(bfx_mode mode, int count, const int32_t* h_n, int nrhs,
                                          const bfx_ir_params* params, bfx_batch_config* out);
BFX_API size_t bfx_batch_workspace_size(bfx_batch plan);
BFX_API bfx_status bfx_batch_solve(bfx_batch plan, const float* d_A, const double* d_b,
                                   double* d_x, bfx_batch_status* d_status, void* d_ws,
                                   size_t ws_bytes, bfx_stream stream);
BFX_API void bfx_batch_destroy(bfx_batch plan);

/* ---------------------------------------------------------------------------
 * Serving: continuous admission of solve requests (A x = b, FP32 A, FP64 b,
 * any n and nrhs) into a fixed device-memory budget.  A server allocates its
 * pool (budget_bytes) once at creation and starts max_inflight worker threads,
 * each with its own CUDA stream.  Requests wait in FIFO order and are admitted
 * when a worker is free and the pool can hold the request's buffers (A, b, x
 * and the bfx_solve_ir workspace); admitted requests run concurrently and
 * their kernels overlap on the device.  Each request is solved exactly as
 * bfx_solve_ir would solve it alone (same kernels, same order of operations),
 * with params {50, 2^-53, sqrt(n) 2^-53, 0.5, escalate, nb, gmres,
 * min(n, 1024), 1e-10} (the Krylov length capped so that one large request's
 * reservation does not crowd the pool).
 * Continuous batching (batch_max_n > 0): a free worker whose next request
 * is small (n <= batch_max_n, nrhs <= 16) takes every small request with the
 * same nrhs that is waiting, in arrival order (up to batch_max, as far as the
 * pool has room), and solves them together with the batched path of
 * bfx_batch_solve (mode as configured, fixed tile shape nb 32, gemm_bn 64,
 * GMRES-IR for the systems plain refinement leaves unconverged, max_iter
 * 20); a small request's result is the same whichever requests share its
 * batch (every kernel of the batched path works on one system at a time), so
 * it equals the result of that request alone through the server.  Large
 * requests are solved one per worker as above.  A batched request reports
 * mode_used = the configured mode, refactorizations = 0 and arnoldi = 0.
 * The caller's host buffers h_A (n x n), h_b (n x nrhs) must stay valid and
 * h_x (n x nrhs, output) writable until the request completes.
 * submit: BFX_ENOMEM if the request can never fit the budget; never blocks.
 * wait: blocks until done (timeout_s < 0: no limit) and returns its result,
 * releasing the ticket; BFX_TIMEOUT if still pending after timeout_s.
 * destroy: running requests finish; queued ones are dropped. */
typedef struct bfx_server_config {
  size_t budget_bytes;
  int max_inflight;
  bfx_mode mode;
  int nb;       /* LU block width (0 = 64) */
  int escalate; /* refactor with more products when refinement stalls */
  int gmres;    /* bfx_ir_params.gmres of every request (0, 1 or 2) */
  int batch_max_n; /* continuous batching: requests with n <= batch_max_n (<= 1024) and
                      nrhs <= 16 waiting together are solved as one batch (0 = off) */
  int batch_max;   /* most requests in one batch (0 = 64) */
} bfx_server_config;
typedef struct bfx_request_result {
  int32_t status;           /* bfx_status of the solve */
  int32_t converged;
  int32_t iters;
  int32_t info;
  int32_t mode_used;
  int32_t refactorizations;
  double berr;
  double latency_s;         /* submission to completion */
  double queue_s;           /* submission to admission */
  int32_t gmres_steps;      /* as bfx_ir_result */
  int32_t arnoldi;
} bfx_request_result;
typedef struct bfx_server_stats_t {
  int32_t queued, running, peak_running;
  int32_t batches; /* batches of small requests run so far */
  size_t pool_bytes, used_bytes, peak_used_bytes;
} bfx_server_stats_t;
typedef struct bfx_server_impl* bfx_server;
BFX_API bfx_status bfx_server_create(bfx_server* out, const bfx_server_config* cfg);
BFX_API bfx_status bfx_server_submit(bfx_server server, int64_t n, int64_t nrhs, const float* h_A,
                                     const double* h_b, double* h_x, int64_t* ticket);
BFX_API bfx_status bfx_server_wait(bfx_server server, int64_t ticket, bfx_request_result* out,
                                   double timeout_s);
BFX_API bfx_status bfx_server_stats(bfx_server server, bfx_server_stats_t* out);
BFX_API void bfx_server_destroy(bfx_server server);

#ifdef __cplusplus
}
#endif

#endif /* BFX_H */
