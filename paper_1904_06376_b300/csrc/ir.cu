// Residual-form iterative refinement (Sec. III of the paper).
//
//   factor   A32 = P L U with the bf16xN-update LU (lu.cu), FP32 factors;
//   x0       = U^-1 L^-1 P b
//   repeat   r = b - A32 x          (FP64, A32 widened exactly)
//            d = U^-1 L^-1 P r      (FP64 arithmetic with the FP32 factors:
//                                    "do the solve in a higher precision")
//            x = x + d              (FP64)
// The paper's r = A x - b with x + y is read as r = b - A x, x + d.  A column
// stops converged when |d|_inf <= tol |x|_inf; it stops when the corrections no
// longer shrink (|d_i| >= stall |d_{i-1}|) and then counts as converged if the
// normwise backward error |r|_inf / (|A|_inf |x|_inf + |b|_inf) <= tol_b.
// Escalation (an addition of this library): columns that stop without
// converging are refined again after refactoring with more products
// (x1 -> x3 -> x6), continuing from the current x.
//
// Everything runs in this library's kernels; the host only loops over
// iterations and reads the per-column norms (a few doubles) to decide.
// Triangular solves: row blocks of 64 whose diagonal blocks are inverted once
// per factorisation (FP64); one launch a triangle, CTAs taking row blocks from
// an atomic ticket in solve order and publishing their results by value
// (ir_trsv_kernel).  In a GMRES phase, which applies M^-1 thousands of times
// with one set of factors, L^-1 and U^-1 are formed once in FP64 and each
// application is a row gather and two triangular matrix-vector products
// (ir_xmv_kernel), with no dependent chain of row blocks.
// GMRES-IR (Sec. III remark, Sec. IV-B): when plain refinement and the
// escalations stall, each refinement step solves its correction equation by
// left-preconditioned GMRES in FP64 (gm_* kernels, gmres_cycle).
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "bfx_internal.cuh"

namespace bfx {

// perm (optional): receives P of P A = L U as a row list (perm[i] = the
// original row at row i), built from the same swap sets as the row swaps
bfx_status lu_factor(bfx_mode mode, int64_t n, int nb, float* A, int64_t lda, int32_t* ipiv,
                     int32_t* info, void* ws, size_t ws_bytes, cudaStream_t s, int32_t* perm);
size_t lu_workspace_bytes(bfx_mode mode, int64_t n, int nb);

namespace {

constexpr int TB = 64;         // triangular-solve row block
constexpr int MAXR = 16;       // right-hand sides handled per pass

// Programmatic dependent launch for the chain of short kernels of a GMRES
// step: a kernel launched with launch_pdl may start while its predecessor in
// the stream finishes; pdl_begin (first statement of every such kernel)
// waits until the predecessor has completed and its writes are visible,
// then lets the next kernel start launching.  Launched without the
// attribute, the wait returns at once.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns (NaN sorts above Inf)
  atomicMax(reinterpret_cast<unsigned long long*>(addr), __double_as_longlong(v));
}

// out[c] = max_i |M[i, c]| for c < ncols (out must start at 0).
__global__ void ir_colmax_kernel(const double* __restrict__ M, int64_t ld, int64_t n, int ncols,
                                 double* __restrict__ out) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n * ncols;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / ncols;
    const int c = static_cast<int>(e - i * ncols);
    atomic_max_nonneg(&out[c], fabs(M[i * ld + c]));
  }
}

// out[0] = |A|_inf = max_i sum_l |A[i, l]|, FP64 (out must start at 0).  Warp a row.
__global__ void ir_anorm_kernel(const float* __restrict__ A, int64_t lda, int n,
                                double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  if (row >= n) return;
  const float* a = A + row * lda;
  double s = 0.0;
  for (int l = lane; l < n; l += 32) s += fabs(widen(a[l]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) atomic_max_nonneg(out, s);
}

// r = b - A x (FP64; r = A x when b is null) for columns c0 .. c0+NC.  Four
// warps a row (RES_WPR), two rows a CTA: warp q of a row takes the 32-element
// pieces q, q + 4, q + 8, ... (coalesced 128-byte loads, four of them in
// flight a lane), the four partial sums meet in shared memory and are added
// in warp order (deterministic).  NC is a compile-time column count so no
// predicated-off FP64 work is issued.  With one warp a row the GPU held only
// 28 warps an SM at n = 4096 and the kernel waited on load latency (43 % of
// the FP64 pipe, long-scoreboard stalls).
// If rn != nullptr, rn[c] = max |r[:, c]| (must start at 0).
constexpr int RES_WPR = 4;
constexpr int RES_ROWS = 256 / (32 * RES_WPR);  // rows a 256-thread CTA
template <int NC>
__global__ void __launch_bounds__(256)
    ir_residual_kernel(const float* __restrict__ A, int64_t lda, int n,
                       const double* __restrict__ b, int64_t ldb,
                       const double* __restrict__ x, int64_t ldx, double* __restrict__ r,
                       int64_t ldr, int c0, double* __restrict__ rn,
                       const int32_t* __restrict__ gate) {
  pdl_begin();
  if (gate && *gate == 0) return;  // asynchronous solve: every column has stopped
  __shared__ double part[RES_ROWS][RES_WPR][NC];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int lr = wid / RES_WPR, q = wid - lr * RES_WPR;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * RES_ROWS + lr;
  double acc[4][NC];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[u][c] = 0.0;
  if (row < n) {
    const float* a = A + row * lda;
    constexpr int S = 32 * RES_WPR;  // stride between a warp's pieces
    int l = q * 32 + lane;
    for (; l + 3 * S < n; l += 4 * S) {
      float av[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) av[u] = __ldg(a + l + S * u);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double al = widen(av[u]);
        const double* xl = x + static_cast<int64_t>(l + S * u) * ldx + c0;
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[u][c] = fma(al, xl[c], acc[u][c]);
      }
    }
    for (; l < n; l += S) {
      const double al = widen(a[l]);
      const double* xl = x + static_cast<int64_t>(l) * ldx + c0;
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[0][c] = fma(al, xl[c], acc[0][c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double v = (acc[0][c] + acc[1][c]) + (acc[2][c] + acc[3][c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) part[lr][q][c] = v;
  }
  __syncthreads();
  if (q == 0 && lane < NC && row < n) {
    const int c = lane;
    double v = part[lr][0][c];
#pragma unroll
    for (int k = 1; k < RES_WPR; ++k) v += part[lr][k][c];
    const double rv = b ? b[row * ldb + c0 + c] - v : v;  // no b: the product A x
    r[row * ldr + c0 + c] = rv;
    if (rn) atomic_max_nonneg(&rn[c0 + c], fabs(rv));
  }
}

// The triangular solve's "not yet published" marker: a signalling NaN with a
// payload bit set.  FP64 arithmetic only ever returns quiet NaNs, so no
// computed value has this bit pattern.
constexpr unsigned long long kTrsvSentinel = 0xFFF4000000000001ull;

// d[i, c] = r[perm[i], c]; when fill (fill2) != null, also fill[] (fill2[]) =
// the triangular solve's sentinel (n x nrhs), the same for fill3 (2 n x
// nrhs), and tickets[0..1] = 0.
__global__ void ir_gather_kernel(const double* __restrict__ r, int64_t ldr,
                                 const int32_t* __restrict__ perm, int64_t n, int nrhs,
                                 double* __restrict__ d, int64_t ldd, double* __restrict__ fill,
                                 double* __restrict__ fill2, double* __restrict__ fill3,
                                 int* __restrict__ tickets, const int32_t* __restrict__ gate) {
  pdl_begin();
  if (gate && *gate == 0) return;
  if (tickets && blockIdx.x == 0 && threadIdx.x < 2) tickets[threadIdx.x] = 0;
  const double sent = __longlong_as_double(static_cast<long long>(kTrsvSentinel));
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n * nrhs;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / nrhs;
    const int c = static_cast<int>(e - i * nrhs);
    d[i * ldd + c] = r[static_cast<int64_t>(perm[i]) * ldr + c];
    if (fill) fill[e] = sent;
    if (fill2) fill2[e] = sent;
    if (fill3) {
      fill3[e] = sent;
      fill3[e + n * nrhs] = sent;
    }
  }
}

// Inverses of the diagonal blocks of L (unit lower) and U (upper), FP64,
// once per factorisation.  CTA b inverts block b: thread k solves
// T x = e_k by column-oriented substitution in registers.  x stays zero
// above row k (L) or below it (U), so a warp skips the steps whose pivot
// column is zero in all its lanes' x; U's diagonal enters through its
// reciprocals (one division a thread).
// T, rdiag: the caller's shared memory ([TB][TB + 1] and [TB] doubles), one
// pair a kernel whichever triangle its CTA inverts
template <bool LOWER>
__device__ __forceinline__ void diag_inverse_body(const float* __restrict__ F, int64_t ldf, int n,
                                                  int blk, double* __restrict__ D,
                                                  double (*T)[TB + 1], double* rdiag) {
  const int b0 = blk * TB, bs = min(TB, n - b0), k = threadIdx.x;
  for (int e = k; e < TB * TB; e += TB) {
    const int i = e / TB, l = e % TB;
    T[i][l] = (i < bs && l < bs) ? static_cast<double>(F[static_cast<int64_t>(b0 + i) * ldf + b0 + l])
                                 : (i == l ? 1.0 : 0.0);
  }
  __syncthreads();
  if (!LOWER) rdiag[k] = 1.0 / T[k][k];
  __syncthreads();
  const int w0 = k & ~31;  // the warp's first column
  double x[TB];
#pragma unroll
  for (int i = 0; i < TB; ++i) x[i] = (i == k) ? 1.0 : 0.0;
  if (LOWER) {
#pragma unroll
    for (int l = 0; l < TB - 1; ++l) {
      if (l < w0) continue;  // x[l] == 0 in every lane of the warp
#pragma unroll
      for (int i = l + 1; i < TB; ++i) x[i] = fma(-T[i][l], x[l], x[i]);
    }
  } else {
#pragma unroll
    for (int l = TB - 1; l >= 0; --l) {
      if (l > w0 + 31) continue;
      x[l] *= rdiag[l];
#pragma unroll
      for (int i = 0; i < l; ++i) x[i] = fma(-T[i][l], x[l], x[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < TB; ++i) D[i * TB + k] = x[i];  // column k of the inverse
}

// Both factors' diagonal-block inverses in one launch: CTAs [0, nblk) for L,
// [nblk, 2 nblk) for U.
__global__ void __launch_bounds__(TB) ir_diag_inverse_kernel(const float* __restrict__ F,
                                                             int64_t ldf, int n,
                                                             double* __restrict__ Linv,
                                                             double* __restrict__ Uinv) {
  __shared__ double T[TB][TB + 1];
  __shared__ double rdiag[TB];
  const int nblk = (n + TB - 1) / TB, bx = static_cast<int>(blockIdx.x);
  if (bx < nblk)
    diag_inverse_body<true>(F, ldf, n, bx, Linv + static_cast<int64_t>(bx) * TB * TB, T, rdiag);
  else
    diag_inverse_body<false>(F, ldf, n, bx - nblk, Uinv + static_cast<int64_t>(bx - nblk) * TB * TB,
                             T, rdiag);
}

// Chain matrices, FP64, once per factorisation: G_b = Dinv_b F[b, p] and
// G2_b = Dinv_b F[b, q] for every row block b with a predecessor p (and q)
// one (two) steps back in solve order (p = b - 1, q = b - 2 forward; b + 1,
// b + 2 backward), stored at block b (G) and nblk + b (G2).  The triangular
// solve then needs only the products G2_b y_q and G_b y_p between those
// blocks' arrivals and the publication of y_b.  One launch for both factors:
// CTA (b', h, d) with b' < nblk - 1 for L, else U, h the half of the rows it
// computes and d + 1 the distance; a warp's 32 outputs share a row i, so the
// product runs only over Dinv_b's nonzero columns (l <= i for L, l >= i for U).
constexpr int CHAIN_HALF = TB / 2;
__global__ void __launch_bounds__(256)
    ir_chain_kernel(const float* __restrict__ F, int64_t ldf, int n,
                    const double* __restrict__ Linv, const double* __restrict__ Uinv,
                    double* __restrict__ Lg, double* __restrict__ Ug) {
  __shared__ double Ds[CHAIN_HALF][TB];  // rows read by broadcast, Fs rows by consecutive lanes:
  __shared__ float Fs[TB][TB];           // no padding needed (32 KB in all)
  const int nblk = (n + TB - 1) / TB;
  const bool lower = static_cast<int>(blockIdx.x) < nblk - 1;
  const int bi = lower ? blockIdx.x : blockIdx.x - (nblk - 1);
  const int dist = 1 + static_cast<int>(blockIdx.z);
  const int b = lower ? bi + 1 : bi;  // blocks with a predecessor
  const int p = lower ? b - dist : b + dist;
  if (p < 0 || p >= nblk) return;
  const int h0 = blockIdx.y * CHAIN_HALF;  // first row of G_b here
  const int b0 = b * TB, bs = min(TB, n - b0), p0 = p * TB, ps = min(TB, n - p0);
  const double* D = (lower ? Linv : Uinv) + static_cast<int64_t>(b) * TB * TB;
  for (int e = threadIdx.x; e < CHAIN_HALF * TB; e += 256)
    Ds[e / TB][e % TB] = D[h0 * TB + e];
  for (int e = threadIdx.x; e < TB * TB; e += 256) {
    const int i = e / TB, l = e % TB;
    Fs[i][l] = (i < bs && l < ps) ? F[static_cast<int64_t>(b0 + i) * ldf + p0 + l] : 0.0f;
  }
  __syncthreads();
  double* g = (lower ? Lg : Ug) + (static_cast<int64_t>(dist - 1) * nblk + b) * TB * TB;
  for (int e = threadIdx.x; e < CHAIN_HALF * TB; e += 256) {
    const int ii = e / TB, i = h0 + ii, j = e % TB;
    const int la = lower ? 0 : i, lb = lower ? i + 1 : TB;  // Dinv_b's nonzero columns of row i
    double s0 = 0.0;
    for (int l = la; l < lb; ++l) s0 = fma(Ds[ii][l], widen(Fs[l][j]), s0);
    g[static_cast<int64_t>(i) * TB + j] = s0;
  }
}

// Triangular solve L y = v (unit lower, forward) or U y = v (upper, backward)
// with the FP32 factors in FP64 arithmetic, in one launch without a grid-wide
// barrier.  Row blocks of 64, each computed by TRSV_SLICES CTAs of 32 rows;
// right-hand sides in groups of up to 4 columns.  A CTA takes a (row block,
// column group, slice) from an atomic ticket in solve order, so every block
// it waits on belongs to CTAs that started earlier and are running: the
// waits always end (and are bounded in time regardless).
// CTA for block b, group g, rows S of the block; p and q the blocks one and
// two steps back in solve order:
//   acc_S = v_b[S] - sum over the earlier blocks k but p and q of
//           F[b, k][S, :] y_k   (each y_k polled as it is published);
//   the other slice's acc rows through an exchange buffer (the inverse of
//   the triangular diagonal block needs them on one side only: the slice
//   whose rows come first in solve order publishes, the other reads);
//   z = (Dinv_b acc)[S] - (G2_b y_q)[S];   y_b[S] = z - (G_b y_p)[S];  publish.
// One SM's FP64 rate bounds the products (a 32 x 64 tile takes about 1.3 us
// with the pipeline's fill and drain), so the slices halve each step's tile,
// and the chain matrices G_b = Dinv_b F[b, p], G2_b = Dinv_b F[b, q] leave
// only G2_b y_q and G_b y_p between the arrivals of y_q, y_p and the
// publication of y_b.  The tile of F is fetched before the wait, so it
// overlaps the wait; the sums run in a fixed order (deterministic).  A
// block's result is published by storing it into y, which holds a sentinel (a
// signalling-NaN pattern no arithmetic produces) until then: consumers poll
// the values themselves, so there is no flag and no fence between the
// product and the next block; the exchange works the same way.  y and the
// exchange buffer xch (n x R) must be all sentinel at launch (the row gather
// fills them); v is only read.  out (optional) gets a plain copy of y.
// ticket: zero at launch.
constexpr int TRSV_THREADS = 256;
constexpr int TRSV_CG = 4;  // right-hand sides a CTA
constexpr int TRSV_SLICES = 2;               // CTAs a row block
constexpr int TRSV_RS = TB / TRSV_SLICES;    // rows a CTA publishes

__device__ __forceinline__ bool is_trsv_sentinel(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) == kTrsvSentinel;
}
// relaxed (morally strong, single-copy atomic) 8-byte accesses at GPU scope:
// the published values and the polls on them never form a data race
__device__ __forceinline__ double ld_relaxed_gpu(const double* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return __longlong_as_double(static_cast<long long>(v));
}
__device__ __forceinline__ void st_relaxed_gpu(double* p, double x) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p),
               "l"(static_cast<unsigned long long>(__double_as_longlong(x)))
               : "memory");
}


// A published value of the triangular solve: *src once it is no longer the
// sentinel.  The wait is bounded (4 s of %globaltimer); on expiry the error
// word gets kErrWaitBlock, *fail is set (later polls of the CTA skip their
// wait) and the sentinel is returned.
__device__ __forceinline__ double poll_published(const double* src, volatile int* fail,
                                                 int* err) {
  double val = ld_relaxed_gpu(src);
  if (is_trsv_sentinel(val) && !*fail) {
    const uint64_t t0 = global_ns();
    while (is_trsv_sentinel(val = ld_relaxed_gpu(src))) {
      if (global_ns() - t0 > 4000000000ull) {
        atomicExch(err, kErrWaitBlock);
        *fail = 1;
        break;
      }
    }
  }
  return val;
}

// out[i][c] (+)= sign * sum_l T[i][l] x[l][c], i < ROWS, c < cg; Q threads a
// product (the largest of 8, 4, 2, 1 with ROWS cg Q <= 256), their partial
// sums added by shuffle.
template <typename T, int LDT, int ROWS>
__device__ __forceinline__ void trsv_tile_product(const T* Tm, const double (*x)[TRSV_CG + 1],
                                                  double (*out)[TRSV_CG + 1], int cg, bool sub) {
  const int t = threadIdx.x;
  const int rc = ROWS * cg;
  const int Q = 8 * rc <= TRSV_THREADS ? 8 : (4 * rc <= TRSV_THREADS ? 4 : (2 * rc <= TRSV_THREADS ? 2 : 1));
  const int items = rc * Q;  // a multiple of 32: whole warps take part or leave
  if (t >= items) return;
  const int o = t / Q, q = t - o * Q;
  const int i = o / cg, c = o - i * cg;
  const int len = TB / Q, l0 = q * len;
  const T* row = Tm + i * LDT + l0;
  double s0 = 0.0, s1 = 0.0;
#pragma unroll 4
  for (int l = 0; l < len; l += 2) {
    s0 = fma(widen(row[l]), x[l0 + l][c], s0);
    s1 = fma(widen(row[l + 1]), x[l0 + l + 1][c], s1);
  }
  double sum = s0 + s1;
  if (Q >= 2) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, 1);
  if (Q >= 4) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, 2);
  if (Q >= 8) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, 4);
  if (q == 0) out[i][c] = sub ? out[i][c] - sum : sum;
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, bool valid) {
  // 4-byte asynchronous copy; an invalid element is zero-filled (source size 0)
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(smem)), "l"(gmem),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <bool LOWER>
__global__ void __launch_bounds__(TRSV_THREADS)
    ir_trsv_kernel(const float* __restrict__ F, int64_t ldf, int n,
                   const double* __restrict__ Dinv, const double* __restrict__ Gm,
                   const double* __restrict__ v, double* __restrict__ y, double* __restrict__ out,
                   double* __restrict__ xch, int R, int* __restrict__ ticket, int* __restrict__ err,
                   const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;  // every CTA leaves: no block is waited on
  constexpr int RS = TRSV_RS, LD = TB + 1;
  extern __shared__ __align__(16) uint8_t trsv_smem[];
  double* Ds = reinterpret_cast<double*>(trsv_smem);              // [RS][LD]: rows S of Dinv_b
  double* Gs = Ds + RS * LD;                                       // [RS][LD]: rows S of G_b
  double* G2s = Gs + RS * LD;                                      // [RS][LD]: rows S of G2_b
  float* Fs = reinterpret_cast<float*>(G2s + RS * LD);            // 2 x [RS][LD]
  auto acc = reinterpret_cast<double (*)[TRSV_CG + 1]>(Fs + 2 * RS * LD);  // [TB][CG + 1]
  auto xs = acc + TB;                                              // [TB][CG + 1]
  auto zs = xs + TB;                                               // [RS][CG + 1]
  __shared__ int s_ticket, s_fail;
  const int t = threadIdx.x;
  const int nblk = (n + TB - 1) / TB;
  const int G = (R + TRSV_CG - 1) / TRSV_CG;
  if (t == 0) {
    s_ticket = atomicAdd(ticket, 1);
    s_fail = 0;
  }
  __syncthreads();
  // the slice whose rows come first in solve order takes the earlier ticket
  const int sk = s_ticket % TRSV_SLICES, unit = s_ticket / TRSV_SLICES;
  const int slice = LOWER ? sk : TRSV_SLICES - 1 - sk;
  const int step = unit / G, grp = unit - step * G;
  const int b = LOWER ? step : nblk - 1 - step;
  const int b0 = b * TB, bs = min(TB, n - b0);
  const int r0 = slice * RS;  // the slice's first row in the block
  const bool first = sk == 0;  // its acc rows feed the other slice's rows of Dinv_b acc
  const int c0 = grp * TRSV_CG, cg = min(TRSV_CG, R - c0);
  // rows S of F[b, k_s] -> Fs buffer (s & 1), asynchronously; rows >= bs /
  // columns >= ks zero
  auto prefetch = [&](int s) {
    const int k = LOWER ? s : nblk - 1 - s;
    const int k0 = k * TB, ks = min(TB, n - k0);
    float* dst = Fs + (s & 1) * RS * LD;
    for (int e = t; e < RS * TB; e += TRSV_THREADS) {
      const int i = e / TB, l = e % TB;
      const bool ok = r0 + i < bs && l < ks;
      cp_async4(dst + i * LD + l, ok ? F + static_cast<int64_t>(b0 + r0 + i) * ldf + k0 + l : F, ok);
    }
  };
  // tiles of all predecessors but the last two (those go through G2_b, G_b)
  const int ntile = step > 2 ? step - 2 : 0;
  if (ntile > 0) prefetch(0);
  cp_async_commit();
  // the slice's rows of the block's inverse and chain matrices
  const double* D = Dinv + (static_cast<int64_t>(b) * TB + r0) * TB;
  const double* Gb = Gm + (static_cast<int64_t>(b) * TB + r0) * TB;
  const double* G2b = Gm + (static_cast<int64_t>(nblk + b) * TB + r0) * TB;
  for (int e = t; e < RS * TB; e += TRSV_THREADS) {
    const int i = e / TB, l = e % TB;
    Ds[i * LD + l] = D[e];
    if (step > 0) Gs[i * LD + l] = Gb[e];
    if (step > 1) G2s[i * LD + l] = G2b[e];
  }
  // acc = v_b on rows S, 0 elsewhere (the other rows come from the exchange)
  for (int e = t; e < TB * cg; e += TRSV_THREADS) {
    const int i = e / cg, c = e - i * cg;
    const bool own = i >= r0 && i < r0 + RS && i < bs;
    acc[i][c] = own ? v[static_cast<int64_t>(b0 + i) * R + c0 + c] : 0.0;
  }
  __syncthreads();  // acc rows are read and written by other threads below
  // fetch y_k into xs, each thread polling one value until it is not the
  // sentinel (an 8-byte aligned store is seen whole or not at all); with a
  // warp polling two values a lane, the second poll cost a round trip more
  // after the first value arrived
  volatile int* fail = &s_fail;
  auto fetch = [&](int k) {
    const int k0 = k * TB, ks = min(TB, n - k0);
    for (int e = t; e < TB * cg; e += TRSV_THREADS) {  // one value a thread: all polled at once
      const int i = e / cg, c = e - i * cg;
      double val = 0.0;
      if (i < ks) val = poll_published(y + static_cast<int64_t>(k0 + i) * R + c0 + c, fail, err);
      xs[i][c] = val;
    }
  };
  for (int s = 0; s < ntile; ++s) {
    if (s + 1 < ntile) prefetch(s + 1);
    cp_async_commit();
    fetch(LOWER ? s : nblk - 1 - s);
    cp_async_wait1();  // this thread's copies of tile s have landed
    __syncthreads();
    trsv_tile_product<float, LD, RS>(Fs + (s & 1) * RS * LD, xs, acc + r0, cg, true);
    __syncthreads();
  }
  // the exchange of acc rows between the slices
  if (first) {
    for (int e = t; e < RS * cg; e += TRSV_THREADS) {
      const int i = e / cg, c = e - i * cg;
      if (r0 + i < bs)
        st_relaxed_gpu(xch + static_cast<int64_t>(b0 + r0 + i) * R + c0 + c, acc[r0 + i][c]);
    }
  } else {
    const int o0 = LOWER ? r0 - RS : r0 + RS;  // the other slice's rows
    for (int e = t; e < RS * cg; e += TRSV_THREADS) {
      const int i = e / cg, c = e - i * cg;
      if (o0 + i < bs)
        acc[o0 + i][c] = poll_published(xch + static_cast<int64_t>(b0 + o0 + i) * R + c0 + c, fail, err);
    }
  }
  // z = rows S of Dinv_b acc (rows past a partial block come out 0: acc and
  // the inverse's padding are zero / identity there)
  __syncthreads();
  trsv_tile_product<double, LD, RS>(Ds, acc, zs, cg, false);
  __syncthreads();
  if (step > 1) {  // z -= G2_b y_q
    fetch(LOWER ? b - 2 : b + 2);
    __syncthreads();
    trsv_tile_product<double, LD, RS>(G2s, xs, zs, cg, true);
    __syncthreads();
  }
  if (step > 0) {  // y_b = z - G_b y_p
    fetch(LOWER ? b - 1 : b + 1);
    __syncthreads();
    trsv_tile_product<double, LD, RS>(Gs, xs, zs, cg, true);
    __syncthreads();
  }
  // publish: the values themselves are the signal (no flag, no fence)
  for (int e = t; e < RS * cg; e += TRSV_THREADS) {
    const int i = e / cg, c = e - i * cg;
    if (r0 + i >= bs) continue;
    const int64_t o = static_cast<int64_t>(b0 + r0 + i) * R + c0 + c;
    st_relaxed_gpu(y + o, zs[i][c]);
    if (out) out[o] = zs[i][c];
  }
}

// ------------------------------------------------------- row-sliced solve
// For the many solves of a GMRES phase with one set of factors (the
// substitution form of its preconditioner, GmPrec::kRowSliced), the block
// inverse is folded into the factor once: H[b][s] = Dinv_b F[b, k_s] for
// every block b and its s-th predecessor k_s in solve order (FP64, blocks of
// block b stored consecutively, block b at step st starting at block
// st (st - 1) / 2).  Then y_b = Dinv_b v_b - sum_s H[b][s] y_{k_s} separates
// by rows, and each block's rows are split over TRSV_S CTAs: the 64 x 64
// FP64 product that follows each arrival, bounded by one SM's FP64 rate
// (about 1.5 us), becomes TRSV_S products of 16 rows.
constexpr int TRSV_S = 4;
constexpr int TRSV_SR = TB / TRSV_S;  // rows a slice

template <bool LOWER>
__global__ void __launch_bounds__(256)
    ir_hmat_kernel(const float* __restrict__ F, int64_t ldf, int n,
                   const double* __restrict__ Dinv, double* __restrict__ H) {
  __shared__ double Ds[TB][TB];
  __shared__ float Fs[TB][TB];
  const int nblk = (n + TB - 1) / TB;
  const int st = blockIdx.x, sp = blockIdx.y;  // step of the block, index of the predecessor
  if (sp >= st || st >= nblk) return;
  const int b = LOWER ? st : nblk - 1 - st;
  const int k = LOWER ? sp : nblk - 1 - sp;
  const int b0 = b * TB, bs = min(TB, n - b0), k0 = k * TB, ks = min(TB, n - k0);
  const double* D = Dinv + static_cast<int64_t>(b) * TB * TB;
  for (int e = threadIdx.x; e < TB * TB; e += 256) {
    const int i = e / TB, l = e % TB;
    Ds[i][l] = D[e];
    Fs[i][l] = (i < bs && l < ks) ? F[static_cast<int64_t>(b0 + i) * ldf + k0 + l] : 0.0f;
  }
  __syncthreads();
  double* h = H + (static_cast<int64_t>(st) * (st - 1) / 2 + sp) * TB * TB;
  for (int e = threadIdx.x; e < TB * TB; e += 256) {
    const int i = e / TB, j = e % TB;
    double s0 = 0.0, s1 = 0.0;
    for (int l = 0; l < TB; l += 2) {
      s0 = fma(Ds[i][l], static_cast<double>(Fs[l][j]), s0);
      s1 = fma(Ds[i][l + 1], static_cast<double>(Fs[l + 1][j]), s1);
    }
    h[e] = s0 + s1;
  }
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem)), "l"(gmem)
               : "memory");
}

// out[i][c] (+)= sign * sum_l T[i][l] x[l][c] for the TRSV_SR rows of a slice;
// Q threads per output (8, 4, 2, 2 for cg = 1 .. 4) take l = q, q + Q, ...
// and add their partial sums by shuffle (a fixed order: deterministic).  On
// B300 the shuffle-adds run on the FP64 pipe like the FMAs (2 a clock per
// SM), so fewer threads per output with longer chains finish sooner: at
// cg = 1, 8 threads per output leave 4 warps of 8 FMAs + 3 adds.
__device__ __forceinline__ void slice_product(const double* Tm, const double (*x)[TRSV_CG + 1],
                                              double (*out)[TRSV_CG + 1], int cg, bool sub) {
  const int t = threadIdx.x;
  const int Q = cg == 1 ? 8 : (cg == 2 ? 4 : 2);
  const int o = t / Q, q = t - o * Q;
  const bool act = o < TRSV_SR * cg;
  const int i = act ? o / cg : 0, c = act ? o - i * cg : 0;
  double sum = 0.0;
  if (act) {
    const double* row = Tm + i * (TB + 1);
    for (int l = q; l < TB; l += Q) sum = fma(row[l], x[l][c], sum);
  }
  for (int off = Q / 2; off > 0; off >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, off);
  if (act && q == 0) out[i][c] = sub ? out[i][c] - sum : sum;
}

// One launch a triangle, CTAs on (row block, column group, slice) tickets in
// solve order, results published by value as in ir_trsv_kernel (y all
// sentinel at launch).  v is only read (several slices read each row); with
// dout the rows are also stored there (plain stores: nothing polls dout).
template <bool LOWER>
__global__ void __launch_bounds__(TRSV_THREADS)
    ir_trsv_h_kernel(const double* __restrict__ H, const double* __restrict__ Dinv, int n,
                     const double* __restrict__ v, double* __restrict__ y,
                     double* __restrict__ dout, int R, int* __restrict__ ticket,
                     int* __restrict__ err) {
  __shared__ __align__(16) double Hs[2][TRSV_SR][TB + 1];
  __shared__ double Ds[TRSV_SR][TB + 1];
  __shared__ double xs[TB][TRSV_CG + 1];
  __shared__ double acc[TRSV_SR][TRSV_CG + 1];
  __shared__ int s_ticket, s_fail;
  const int t = threadIdx.x;
  const int nblk = (n + TB - 1) / TB;
  const int G = (R + TRSV_CG - 1) / TRSV_CG;
  if (t == 0) {
    s_ticket = atomicAdd(ticket, 1);
    s_fail = 0;
  }
  __syncthreads();
  const int step = s_ticket / (G * TRSV_S);
  const int rem = s_ticket - step * (G * TRSV_S);
  const int grp = rem / TRSV_S, sl = rem - grp * TRSV_S;
  const int b = LOWER ? step : nblk - 1 - step;
  const int b0 = b * TB, bs = min(TB, n - b0);
  const int r0 = sl * TRSV_SR;
  const int c0 = grp * TRSV_CG, cg = min(TRSV_CG, R - c0);
  const double* Hb = H + static_cast<int64_t>(step) * (step - 1) / 2 * TB * TB;
  // rows r0 .. r0 + 15 of H[b][s] -> Hs[s & 1], asynchronously
  auto prefetch = [&](int s) {
    const double* src = Hb + static_cast<int64_t>(s) * TB * TB + r0 * TB;
    for (int e = t; e < TRSV_SR * TB; e += TRSV_THREADS) {
      const int i = e / TB, l = e - i * TB;
      cp_async8(&Hs[s & 1][i][l], src + i * TB + l);
    }
  };
  if (step > 0) prefetch(0);
  cp_async_commit();
  // acc = (Dinv_b v_b) on this slice's rows
  const double* D = Dinv + static_cast<int64_t>(b) * TB * TB + r0 * TB;
  for (int e = t; e < TRSV_SR * TB; e += TRSV_THREADS) Ds[e / TB][e % TB] = D[e];
  for (int e = t; e < TB * cg; e += TRSV_THREADS) {
    const int i = e / cg, c = e - i * cg;
    xs[i][c] = i < bs ? v[static_cast<int64_t>(b0 + i) * R + c0 + c] : 0.0;
  }
  __syncthreads();
  slice_product(&Ds[0][0], xs, acc, cg, false);
  __syncthreads();
  volatile int* fail = &s_fail;
  for (int s = 0; s < step; ++s) {
    if (s + 1 < step) prefetch(s + 1);
    cp_async_commit();
    const int k = LOWER ? s : nblk - 1 - s;
    const int k0 = k * TB, ks = min(TB, n - k0);
    {  // y_k into xs, one value a thread: every value is polled at once
      for (int e = t; e < TB * cg; e += TRSV_THREADS) {
        const int i = e / cg, c = e - i * cg;
        double val = 0.0;
        if (i < ks) val = poll_published(y + static_cast<int64_t>(k0 + i) * R + c0 + c, fail, err);
        xs[i][c] = val;
      }
    }
    cp_async_wait1();  // this thread's copies of H[b][s] have landed
    __syncthreads();
    slice_product(&Hs[s & 1][0][0], xs, acc, cg, true);
    __syncthreads();
  }
  for (int e = t; e < TRSV_SR * cg; e += TRSV_THREADS) {
    const int i = e / cg, c = e - i * cg;
    if (r0 + i >= bs) continue;
    const int64_t at = static_cast<int64_t>(b0 + r0 + i) * R + c0 + c;
    st_relaxed_gpu(y + at, acc[i][c]);
    if (dout) dout[at] = acc[i][c];
  }
}

// ------------------------------------------------------- explicit inverses
// For the many preconditioner applications of a GMRES phase, the inverses
// of the FP32 factors are formed once per factorisation in FP64: X = L^-1
// (unit lower) and X = U^-1 (upper), so each application of M^-1 = U^-1 L^-1
// P is a row gather and two triangular matrix-vector products, with no
// dependent chain of row blocks.  X is kept in 64 x 64 blocks in solve
// order: block (st, sk), sk <= st, holds rows of natural block b(st) and
// columns of natural block b(sk) (b(s) = s for L, nblk - 1 - s for U), at
// offset (st (st + 1) / 2 + sk) TB^2, row-major.  In those coordinates both
// triangles follow one recurrence:
//   X[st][st] = Dinv_b(st)  (the diagonal block's inverse),
//   X[st][sk] = -Dinv_b(st) sum_{ss = sk}^{st - 1} F[b(st)][b(ss)] X[ss][sk].
// It runs right-looking by the distance t = st - sk: once X[sk + t][sk] is
// final, its products F[b(st)][b(sk + t)] X[sk + t][sk] are added into the
// accumulators X[st][sk] of every st > sk + t (one launch, a CTA a block),
// in the order of ss (deterministic); then X[sk + t + 1][sk] = -Dinv times
// its accumulator (one launch).  n^3 / 6 FP64 FMAs a triangle.
__host__ __device__ __forceinline__ int64_t xblk(int st, int sk) {
  return (static_cast<int64_t>(st) * (st + 1) / 2 + sk) * TB * TB;
}
constexpr int XB_THREADS = 256;
constexpr size_t kXbSmem = 2 * sizeof(double) * TB * (TB + 1);  // two padded FP64 tiles

// out (+)= sign * A B for 64 x 64 FP64 tiles in shared memory (rows TB + 1
// apart); thread (ty, tx) of 16 x 16 owns rows ty + 16 r and columns
// tx + 16 c; l in order (deterministic).
__device__ __forceinline__ void xb_product(const double (*As)[TB + 1], const double (*Bs)[TB + 1],
                                           double (&acc)[4][4]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int l = 0; l < TB; ++l) {
    double a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = As[ty + 16 * r][l];
#pragma unroll
    for (int c = 0; c < 4; ++c) b[c] = Bs[l][tx + 16 * c];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
  }
}

// X[st][st] = Dinv_b(st); X[st][sk] = 0 below it (the accumulators).  A CTA a block.
template <bool LOWER>
__global__ void __launch_bounds__(XB_THREADS)
    ir_xinit_kernel(const double* __restrict__ Dinv, int nblk, double* __restrict__ X) {
  const int64_t e0 = static_cast<int64_t>(blockIdx.x) * TB * TB;
  int st = 0;
  while (xblk(st + 1, 0) <= e0) ++st;
  const int sk = static_cast<int>(e0 / (TB * TB) - static_cast<int64_t>(st) * (st + 1) / 2);
  const int b = LOWER ? st : nblk - 1 - st;
  const double* D = Dinv + static_cast<int64_t>(b) * TB * TB;
  double* out = X + e0;
  for (int e = threadIdx.x; e < TB * TB; e += XB_THREADS) out[e] = sk == st ? D[e] : 0.0;
}

// Distance t: X[st][sk] += F[b(st)][b(ss)] X[ss][sk] with ss = sk + t, for
// every st > ss.  grid (nblk - t - 1, nblk - t - 1): x = sk, y = st - ss - 1.
template <bool LOWER>
__global__ void __launch_bounds__(XB_THREADS)
    ir_xupd_kernel(const float* __restrict__ F, int64_t ldf, int n, int nblk, int t,
                   double* __restrict__ X) {
  extern __shared__ double xsm[];
  double (*Fs)[TB + 1] = reinterpret_cast<double (*)[TB + 1]>(xsm);
  double (*Ys)[TB + 1] = reinterpret_cast<double (*)[TB + 1]>(xsm + TB * (TB + 1));
  const int sk = blockIdx.x, ss = sk + t, st = ss + 1 + static_cast<int>(blockIdx.y);
  if (st >= nblk) return;
  const int b = LOWER ? st : nblk - 1 - st, bs_ = LOWER ? ss : nblk - 1 - ss;
  const int r0 = b * TB, c0 = bs_ * TB;
  const double* Y = X + xblk(ss, sk);
  for (int e = threadIdx.x; e < TB * TB; e += XB_THREADS) {
    const int i = e / TB, l = e % TB;
    Fs[i][l] = (r0 + i < n && c0 + l < n)
                   ? static_cast<double>(F[static_cast<int64_t>(r0 + i) * ldf + c0 + l])
                   : 0.0;
    Ys[i][l] = Y[e];
  }
  __syncthreads();
  double* out = X + xblk(st, sk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = out[(ty + 16 * r) * TB + tx + 16 * c];
  xb_product(Fs, Ys, acc);
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) out[(ty + 16 * r) * TB + tx + 16 * c] = acc[r][c];
}

// Distance t >= 1: X[st][st - t] = -Dinv_b(st) X[st][st - t] (the accumulator
// is complete).  A CTA per st = t + blockIdx.x.
template <bool LOWER>
__global__ void __launch_bounds__(XB_THREADS)
    ir_xfin_kernel(const double* __restrict__ Dinv, int nblk, int t, double* __restrict__ X) {
  extern __shared__ double xsm[];
  double (*Ds)[TB + 1] = reinterpret_cast<double (*)[TB + 1]>(xsm);
  double (*As)[TB + 1] = reinterpret_cast<double (*)[TB + 1]>(xsm + TB * (TB + 1));
  const int st = t + static_cast<int>(blockIdx.x), sk = st - t;
  const int b = LOWER ? st : nblk - 1 - st;
  const double* D = Dinv + static_cast<int64_t>(b) * TB * TB;
  double* io = X + xblk(st, sk);
  for (int e = threadIdx.x; e < TB * TB; e += XB_THREADS) {
    Ds[e / TB][e % TB] = D[e];
    As[e / TB][e % TB] = io[e];
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  xb_product(Ds, As, acc);
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) io[(ty + 16 * r) * TB + tx + 16 * c] = -acc[r][c];
}

// y = X v for columns c0 .. c0 + CG of v, y (row-major, ld R); a warp per
// pair of rows i and n - 1 - i, so every warp reads about the same number of
// blocks (a row of natural block b reads b + 1 blocks of L^-1, nblk - b of
// U^-1).  The product is bound by its loads' latency, so a lane loads the
// row pieces and v entries of XMV_U(CG) blocks before their FMAs (eight
// blocks for one column; measured 1.5x the rate of one block at a time),
// into XMV_U running sums per column added in a fixed order, then across
// the lanes by an xor tree: deterministic.  Two warps a CTA spread the
// warps evenly over the SMs.
__host__ __device__ constexpr int xmv_u(int cg) { return cg == 1 ? 8 : 2; }
constexpr int XMV_THREADS = 64;
template <bool LOWER, int CG>
__global__ void __launch_bounds__(XMV_THREADS)
    ir_xmv_kernel(const double* __restrict__ X, int n, int nblk, const double* __restrict__ v,
                  double* __restrict__ y, int R, int c0) {
  pdl_begin();
  constexpr int U = xmv_u(CG);
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int half = (n + 1) / 2;
  if (w >= half) return;
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const int i = pass == 0 ? w : n - 1 - w;
    if (pass == 1 && i == w) break;  // the middle row of an odd n
    const int b = i / TB, r = i - b * TB;
    const int st = LOWER ? b : nblk - 1 - b;
    const double* base = X + xblk(st, 0) + static_cast<int64_t>(r) * TB;  // block sk at + sk TB^2
    double acc[U][CG];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int c = 0; c < CG; ++c) acc[u][c] = 0.0;
    for (int sk0 = 0; sk0 <= st; sk0 += U) {
      double a[U][2], vv[U][2][CG];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int sk = sk0 + u;
        const int k = LOWER ? sk : nblk - 1 - sk;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int l = lane + 32 * h, col = k * TB + l;
          const bool ok = sk <= st && col < n;
          a[u][h] = ok ? __ldg(base + static_cast<int64_t>(sk) * TB * TB + l) : 0.0;
#pragma unroll
          for (int c = 0; c < CG; ++c)
            vv[u][h][c] = ok ? __ldg(v + static_cast<int64_t>(col) * R + c0 + c) : 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < CG; ++c) {
          acc[u][c] = fma(a[u][0], vv[u][0][c], acc[u][c]);
          acc[u][c] = fma(a[u][1], vv[u][1][c], acc[u][c]);
        }
    }
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      double sum = 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u) sum += acc[u][c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
      acc[0][c] = sum;
    }
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < CG; ++c) y[static_cast<int64_t>(i) * R + c0 + c] = acc[0][c];
    }
  }
}

constexpr size_t kTrsvSmemUsed = 3 * sizeof(double) * TRSV_RS * (TB + 1) +
                                 2 * sizeof(float) * TRSV_RS * (TB + 1) +
                                 sizeof(double) * (2 * TB + TRSV_RS) * (TRSV_CG + 1);
// launched with more than half an SM's shared memory, so no two CTAs of a
// triangular solve share an SM: every CTA runs a 64 x 64 FP64 tile product
// for each block that arrives, and two on one SM's FP64 pipe stretch every
// step of the chain
constexpr size_t kTrsvSmem = kTrsvSmemUsed > 120 * 1024 ? kTrsvSmemUsed : 120 * 1024;

// x += d on active columns; dn[c] = max|d|, xn[c] = max|x| (must start at 0).
__global__ void ir_update_kernel(double* __restrict__ x, int64_t ldx, const double* __restrict__ d,
                                 int64_t ldd, int64_t n, int nrhs, const int32_t* __restrict__ active,
                                 double* __restrict__ dn, double* __restrict__ xn,
                                 const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n * nrhs;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / nrhs;
    const int c = static_cast<int>(e - i * nrhs);
    if (!active[c]) continue;
    const double dv = d[i * ldd + c];
    const double xv = x[i * ldx + c] + dv;
    x[i * ldx + c] = xv;
    atomic_max_nonneg(&dn[c], fabs(dv));
    atomic_max_nonneg(&xn[c], fabs(xv));
  }
}

// ------------------------------------------------------------- GMRES-IR
// The correction equation of a refinement step, A d = r, solved by GMRES on
// M^-1 A d = M^-1 r (M = P^T L U, the FP32 factors applied in FP64), zero
// first guess, all right-hand sides together, each with its own Krylov basis
// (GMRES remark of Sec. III; Sec. IV-B).  Vectors are n x R row-major like x,
// so the basis V is (m+1) blocks of n x R.  Arnoldi orthogonalises by two
// passes of classical Gram-Schmidt (each a dot-product launch and an update
// launch, so the FP64 work is spread over the SMs instead of j dependent
// launches); the Hessenberg column is reduced by Givens rotations as it is
// formed, one thread per right-hand side.  Dot products are split into
// chunks of rows; each chunk's partial sums go to `part` and every consumer
// adds them in chunk order, so results do not depend on scheduling.
constexpr int GM_THREADS = 256;
constexpr int GM_ELEMS = 1024;  // vector elements one CTA covers in a dot product
constexpr int GM_MAXCH = 64;    // most chunks a dot product is split into
constexpr int GM_WHOLE = 64;    // from this many vectors, a Gram-Schmidt dot takes whole vectors

// part[(i * nchunk + ch) * R + c] = sum over the chunk's rows of V_i[r, c] w[r, c].
// Threads own one column each and step through rows, so a warp reads
// consecutive addresses; partial sums are combined in a fixed order.
__global__ void __launch_bounds__(GM_THREADS)
    gm_dot_kernel(const double* __restrict__ V, int64_t vstride, const double* __restrict__ w,
                  int n, int R, int rows_per_chunk, int nchunk, double* __restrict__ part) {
  pdl_begin();
  __shared__ double acc[GM_THREADS];
  __shared__ double red[8 * MAXR];
  const int i = blockIdx.x, ch = blockIdx.y, t = threadIdx.x;
  const int tpc = GM_THREADS / R;  // rows a pass
  const double* v = V + static_cast<int64_t>(i) * vstride;
  const int r_begin = ch * rows_per_chunk, r_end = min(n, r_begin + rows_per_chunk);
  double sum = 0.0;
  if (t < tpc * R) {
    const int c = t % R;
    for (int r = r_begin + t / R; r < r_end; r += tpc) {
      const int64_t e = static_cast<int64_t>(r) * R + c;
      sum = fma(v[e], w[e], sum);
    }
  }
  acc[t] = t < tpc * R ? sum : 0.0;
  __syncthreads();
  if (t < 8 * R) {  // acc[r0 * R + c]: eight strided partial sums per column
    const int c = t % R, q = t / R;
    double u = 0.0;
    for (int r0 = q; r0 < tpc; r0 += 8) u += acc[r0 * R + c];
    red[t] = u;
  }
  __syncthreads();
  if (t < R) {
    double u = 0.0;
    for (int q = 0; q < 8; ++q) u += red[q * R + t];
    part[(static_cast<int64_t>(i) * nchunk + ch) * R + t] = u;
  }
}

// h_i[c] = sum of the chunk partials of <V_i, w> (chunk order), i < nv, into
// hb[i * R + c]; on Arnoldi-active columns also written (accumulate = 0) or
// added (accumulate = 1) into column j of H.
__global__ void gm_reduce_h_kernel(const double* __restrict__ part, int nchunk, int nv, int R,
                                   double* __restrict__ hb, double* __restrict__ H, int m, int j,
                                   int accumulate, const int32_t* __restrict__ act) {
  pdl_begin();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nv * R) return;
  const int i = e / R, c = e % R;
  double u = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) u += part[(static_cast<int64_t>(i) * nchunk + ch) * R + c];
  hb[e] = u;
  if (act[c]) {
    double* hp = H + (static_cast<int64_t>(c) * m + j) * (m + 1) + i;
    *hp = accumulate ? *hp + u : u;
  }
}

// One classical Gram-Schmidt update: w -= sum_i h_i V_i (i < nv, in order)
// on Arnoldi-active columns.
__global__ void __launch_bounds__(GM_THREADS)
    gm_orth_kernel(const double* __restrict__ V, int64_t vstride, int nv, double* __restrict__ w,
                   int n, int R, const double* __restrict__ hb, const int32_t* __restrict__ act) {
  pdl_begin();
  __shared__ int32_t a[MAXR];
  if (threadIdx.x < R) a[threadIdx.x] = act[threadIdx.x];
  __syncthreads();
  const int64_t total = static_cast<int64_t>(n) * R;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(GM_THREADS) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * GM_THREADS) {
    const int c = static_cast<int>(e % R);
    if (!a[c]) continue;
    double u = w[e];
    for (int i = 0; i < nv; ++i) u = fma(-__ldg(hb + i * R + c), V[i * vstride + e], u);
    w[e] = u;
  }
}

// The same update when there are many vectors: gm_orth_kernel's grid covers
// only the n R elements (16 CTAs at n = 4096, R = 1), so its (j + 1) n FP64
// FMAs ran on 16 SMs (133 us at j = 2000).  Here CTA (x, y) sums the vectors
// of chunk y (GM_KC of them, in order) for its elements into part2[y], and
// gm_orth_finish_kernel subtracts the chunk sums from w in chunk order: the
// work spreads over every SM and the order stays fixed (deterministic).
constexpr int GM_KC = 64;
constexpr int GM_PT = 128;  // threads of a chunk-sum CTA (more CTAs over the elements)
__global__ void __launch_bounds__(GM_PT)
    gm_orth_part_kernel(const double* __restrict__ V, int64_t vstride, int nv, int n, int R,
                        const double* __restrict__ hb, const int32_t* __restrict__ act,
                        double* __restrict__ part2) {
  pdl_begin();
  __shared__ int32_t a[MAXR];
  if (threadIdx.x < R) a[threadIdx.x] = act[threadIdx.x];
  __syncthreads();
  const int64_t total = static_cast<int64_t>(n) * R;
  const int i0 = blockIdx.y * GM_KC, i1 = min(nv, i0 + GM_KC);
  for (int64_t e = blockIdx.x * static_cast<int64_t>(GM_PT) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * GM_PT) {
    const int c = static_cast<int>(e % R);
    if (!a[c]) continue;
    double u = 0.0;
    for (int i = i0; i < i1; ++i) u = fma(__ldg(hb + i * R + c), V[i * vstride + e], u);
    part2[blockIdx.y * total + e] = u;
  }
}
__global__ void __launch_bounds__(GM_THREADS)
    gm_orth_finish_kernel(double* __restrict__ w, int n, int R, const int32_t* __restrict__ act,
                          const double* __restrict__ part2, int nkc) {
  pdl_begin();
  __shared__ int32_t a[MAXR];
  if (threadIdx.x < R) a[threadIdx.x] = act[threadIdx.x];
  __syncthreads();
  const int64_t total = static_cast<int64_t>(n) * R;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(GM_THREADS) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * GM_THREADS) {
    const int c = static_cast<int>(e % R);
    if (!a[c]) continue;
    double u = w[e];
    for (int y = 0; y < nkc; ++y) u -= part2[y * total + e];
    w[e] = u;
  }
}

// Start of a cycle: w = M^-1 r; beta = |w|_2 (from the partials of <w, w>),
// V_0 = w / beta, g = beta e_1; a column takes part when it is refinement-
// active and beta is positive and finite.
__global__ void __launch_bounds__(GM_THREADS)
    gm_start_kernel(double* __restrict__ V, const double* __restrict__ w, int n, int R,
                    const double* __restrict__ part, int nchunk, double* __restrict__ g,
                    double* __restrict__ beta, int m, const int32_t* __restrict__ active,
                    int32_t* __restrict__ act_out, int32_t* __restrict__ kdone) {
  pdl_begin();
  __shared__ double bs[MAXR];
  __shared__ int32_t a[MAXR];
  if (threadIdx.x < R) {
    double u = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) u += part[static_cast<int64_t>(ch) * R + threadIdx.x];
    const double b = sqrt(u);
    bs[threadIdx.x] = b;
    a[threadIdx.x] = active[threadIdx.x] && b > 0.0 && b <= 1.7976931348623157e308;
  }
  __syncthreads();
  const int64_t total = static_cast<int64_t>(n) * R;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(GM_THREADS) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * GM_THREADS) {
    const int c = static_cast<int>(e % R);
    if (a[c]) V[e] = w[e] / bs[c];
  }
  if (blockIdx.x == 0 && threadIdx.x < R) {
    const int c = threadIdx.x;
    beta[c] = bs[c];
    double* gc = g + static_cast<int64_t>(c) * (m + 1);
    for (int i = 0; i <= m; ++i) gc[i] = 0.0;
    gc[0] = bs[c];
    kdone[c] = 0;
    act_out[c] = a[c];
  }
}

// End of Arnoldi step j, part 1: h_{j+1,j} = |w|_2 (partials of <w, w>),
// V_{j+1} = w / h_{j+1,j} for the Arnoldi-active columns.
__global__ void __launch_bounds__(GM_THREADS)
    gm_next_kernel(double* __restrict__ V, int64_t vstride, int j, const double* __restrict__ w,
                   int n, int R, const double* __restrict__ part, int nchunk,
                   const int32_t* __restrict__ act_in) {
  pdl_begin();
  __shared__ double hn[MAXR];
  __shared__ int32_t a[MAXR];
  if (threadIdx.x < R) {
    double u = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) u += part[static_cast<int64_t>(ch) * R + threadIdx.x];
    hn[threadIdx.x] = sqrt(u);
    a[threadIdx.x] = act_in[threadIdx.x];
  }
  __syncthreads();
  double* vn = V + static_cast<int64_t>(j + 1) * vstride;
  const int64_t total = static_cast<int64_t>(n) * R;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(GM_THREADS) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * GM_THREADS) {
    const int c = static_cast<int>(e % R);
    if (a[c] && hn[c] > 0.0) vn[e] = w[e] / hn[c];
  }
}

// End of Arnoldi step j, part 2, CTA c for column c: the earlier rotations
// applied to column j of H, the rotation that zeroes h_{j+1,j}, g updated;
// the column stays Arnoldi-active unless |g_{j+1}| <= tau beta, the space
// became invariant (h_{j+1,j} = 0), m steps are done, or a NaN appeared.
// Applying rotation i carries the rotated lower entry p to the next one:
// p_{i+1} = -s_i p_i + c_i h_{i+1}, an affine recurrence, so instead of j
// dependent steps on one thread (each waiting on a load: a millisecond at
// j ~ 2000) the CTA composes the maps x -> a x + b with a prefix scan over
// its threads (fixed thread order: deterministic), then every thread
// finishes its own rows h_i = c_i p_i + s_i h_{i+1}.
constexpr int GIV_THREADS = 1024;
constexpr int GIV_E = (BFX_GMRES_MAX_M + GIV_THREADS - 1) / GIV_THREADS;  // rows a thread

// The earlier rotations (csc, snc, i < j) applied to Hessenberg column hcol
// (rows 0..j) by all NT threads of the CTA (called by every thread): the
// carried lower entry follows the affine recurrence p_{i+1} = -s_i p_i +
// c_i h_{i+1}; each thread composes the maps of its E consecutive rows, an
// exclusive prefix scan over the threads (warp shuffles, then the 32 warp
// totals; fixed order) gives its starting p, and it finishes its own rows.
// Returns p_j, the entry the new rotation must zero against h_{j+1,j}, in
// every thread.  wA, wB: NT / 32 doubles of shared memory; sp: one.
template <int NT, int MAXE>
__device__ double givens_apply_scan(double* hcol, const double* csc, const double* snc, int j,
                                    double* wA, double* wB, double* sp) {
  static_assert(NT % 32 == 0 && NT / 32 <= 32, "CTA of whole warps, at most 32");
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int E = (j + NT - 1) / NT;  // <= MAXE
  const int i0 = t * E;
  double cv[MAXE], sv[MAXE], qv[MAXE];
  double A = 1.0, B = 0.0;  // composition of this thread's maps, in order
#pragma unroll
  for (int e = 0; e < MAXE; ++e) {
    const int i = i0 + e;
    cv[e] = sv[e] = qv[e] = 0.0;
    if (e < E && i < j) {
      cv[e] = csc[i];
      sv[e] = snc[i];
      qv[e] = hcol[i + 1];
      const double a = -sv[e], b = cv[e] * qv[e];
      B = a * B + b;
      A = a * A;
    }
  }
  const double p0 = hcol[0];
  double pA = A, pB = B;  // inclusive scan within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double oA = __shfl_up_sync(0xFFFFFFFFu, pA, o);
    const double oB = __shfl_up_sync(0xFFFFFFFFu, pB, o);
    if (lane >= o) {  // this (later) map after the earlier ones
      pB = pA * oB + pB;
      pA = pA * oA;
    }
  }
  if (lane == 31) {
    wA[wid] = pA;
    wB[wid] = pB;
  }
  __syncthreads();
  if (wid == 0) {  // inclusive scan of the warp totals
    double xA = lane < NT / 32 ? wA[lane] : 1.0, xB = lane < NT / 32 ? wB[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double oA = __shfl_up_sync(0xFFFFFFFFu, xA, o);
      const double oB = __shfl_up_sync(0xFFFFFFFFu, xB, o);
      if (lane >= o) {
        xB = xA * oB + xB;
        xA = xA * oA;
      }
    }
    if (lane < NT / 32) {
      wA[lane] = xA;
      wB[lane] = xB;
    }
  }
  __syncthreads();
  double eA = 1.0, eB = 0.0;  // exclusive prefix: earlier warps, then earlier lanes
  if (wid > 0) {
    eA = wA[wid - 1];
    eB = wB[wid - 1];
  }
  {
    const double lA = __shfl_up_sync(0xFFFFFFFFu, pA, 1), lB = __shfl_up_sync(0xFFFFFFFFu, pB, 1);
    if (lane > 0) {
      eB = lA * eB + lB;
      eA = lA * eA;
    }
  }
  double p = eA * p0 + eB;  // p_{i0}
#pragma unroll
  for (int e = 0; e < MAXE; ++e) {
    const int i = i0 + e;
    if (e < E && i < j) {
      hcol[i] = cv[e] * p + sv[e] * qv[e];
      p = -sv[e] * p + cv[e] * qv[e];
      if (i == j - 1) *sp = p;  // p_j
    }
  }
  if (j == 0 && t == 0) *sp = p0;
  __syncthreads();
  const double pj = *sp;
  __syncthreads();  // sp and the warp totals may be reused by the caller
  return pj;
}

__global__ void __launch_bounds__(GIV_THREADS)
    gm_givens_kernel(int j, int R, const double* __restrict__ part, int nchunk,
                     double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                     double* __restrict__ g, const double* __restrict__ beta, int m, double tau,
                     const int32_t* __restrict__ act_in, int32_t* __restrict__ act_out,
                     int32_t* __restrict__ kdone, int32_t* __restrict__ host_flags) {
  pdl_begin();
  __shared__ double wA[GIV_THREADS / 32], wB[GIV_THREADS / 32];
  __shared__ double s_p;
  const int c = blockIdx.x, t = threadIdx.x;
  if (!act_in[c]) {
    if (t == 0) {
      act_out[c] = 0;
      host_flags[c] = 0;
    }
    return;
  }
  double* hcol = H + (static_cast<int64_t>(c) * m + j) * (m + 1);  // column j, rows 0..j+1
  const double pj = givens_apply_scan<GIV_THREADS, GIV_E>(hcol, cs + static_cast<int64_t>(c) * m,
                                                          sn + static_cast<int64_t>(c) * m, j, wA,
                                                          wB, &s_p);
  if (t == 0) {
    double u = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) u += part[static_cast<int64_t>(ch) * R + c];
    const double hj = sqrt(u);  // as part 1 computed it
    double* gc = g + static_cast<int64_t>(c) * (m + 1);
    const double rho = hypot(pj, hj);
    const double cj = rho > 0.0 ? pj / rho : 1.0, sj = rho > 0.0 ? hj / rho : 0.0;
    cs[static_cast<int64_t>(c) * m + j] = cj;
    sn[static_cast<int64_t>(c) * m + j] = sj;
    hcol[j] = rho;
    hcol[j + 1] = 0.0;
    gc[j + 1] = -sj * gc[j];
    gc[j] = cj * gc[j];
    kdone[c] = j + 1;
    const double res = fabs(gc[j + 1]);
    int keep = 1;
    if (res <= tau * beta[c] || !(hj > 0.0) || j + 1 >= m || !(res == res)) keep = 0;
    act_out[c] = keep;
    host_flags[c] = keep;  // mapped pinned memory: the host reads it after an event
  }
}

// y = R_k^-1 g_k for each refinement-active column (k = kdone[c]): CTA c,
// one warp, back substitution with the lanes splitting each row's sum.
__global__ void __launch_bounds__(32)
    gm_solve_y_kernel(const double* __restrict__ H, const double* __restrict__ g,
                      const int32_t* __restrict__ kdone, const int32_t* __restrict__ active, int m,
                      double* __restrict__ y) {
  extern __shared__ double ys[];  // m doubles
  const int c = blockIdx.x, lane = threadIdx.x;
  if (!active[c]) return;
  const int k = kdone[c];
  const double* Hc = H + static_cast<int64_t>(c) * m * (m + 1);  // H(i, l) at Hc[l (m+1) + i]
  const double* gc = g + static_cast<int64_t>(c) * (m + 1);
  for (int i = k - 1; i >= 0; --i) {
    double u = 0.0;
    for (int l = i + 1 + lane; l < k; l += 32)
      u = fma(Hc[static_cast<int64_t>(l) * (m + 1) + i], ys[l], u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xFFFFFFFFu, u, o);
    if (lane == 0) ys[i] = (gc[i] - u) / Hc[static_cast<int64_t>(i) * (m + 1) + i];
    __syncwarp();
  }
  for (int i = lane; i < k; i += 32) y[static_cast<int64_t>(c) * m + i] = ys[i];
}

// d[:, c] = sum_{i < kdone[c]} y[c][i] V_i[:, c] on refinement-active columns, 0 elsewhere.
__global__ void __launch_bounds__(GM_THREADS)
    gm_combine_kernel(const double* __restrict__ V, int64_t vstride, const double* __restrict__ y,
                      const int32_t* __restrict__ kdone, const int32_t* __restrict__ active, int n,
                      int R, int m, double* __restrict__ d) {
  __shared__ int32_t ks[MAXR];
  if (threadIdx.x < R) ks[threadIdx.x] = active[threadIdx.x] ? kdone[threadIdx.x] : 0;
  __syncthreads();
  const int64_t total = static_cast<int64_t>(n) * R;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(GM_THREADS) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * GM_THREADS) {
    const int c = static_cast<int>(e % R);
    const double* yc = y + static_cast<int64_t>(c) * m;
    double u = 0.0;
    for (int i = 0; i < ks[c]; ++i) u = fma(__ldg(yc + i), V[i * vstride + e], u);
    d[e] = u;
  }
}

// ------------------------------------------------------------- batched forms
constexpr int BIR_THREADS = 512;
// the batched GMRES-IR runs each hard system in one CTA of BGM_THREADS
// threads: its FP64 work is latency-bound on one SM, and 1024 threads keep
// more FMA chains in flight than 512 (a 2000-system batch 57.2 -> 54.8 ms)
constexpr int BGM_THREADS = 1024;
constexpr int BGM_GIV_E = 4;  // Krylov length of the batched GMRES at most 4 x BGM_THREADS

__device__ __forceinline__ double block_max(double v, double* red) {
  // max over the CTA of non-negative values (NaN propagates: compared as bits)
  unsigned long long u = __double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xFFFFFFFFu, u, o);
    u = w > u ? w : u;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = __longlong_as_double(u);
  __syncthreads();
  unsigned long long m = 0;
  for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) {
    const unsigned long long w = __double_as_longlong(red[i]);
    m = w > m ? w : m;
  }
  return __longlong_as_double(m);
}

// |A|_inf, |b|_inf, state reset.
__global__ void __launch_bounds__(BIR_THREADS) bir_prepare_kernel(const BatchIr* __restrict__ sys) {
  __shared__ double red[BIR_THREADS / 32];
  const BatchIr q = sys[blockIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double am = 0.0;
  for (int i = wid; i < q.n; i += BIR_THREADS / 32) {
    double sum = 0.0;
    for (int l = lane; l < q.n; l += 32) sum += fabs(widen(q.A[static_cast<int64_t>(i) * q.n + l]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    am = fmax(am, sum);
  }
  double bm = 0.0;
  for (int e = threadIdx.x; e < q.n * q.nrhs; e += BIR_THREADS) bm = fmax(bm, fabs(q.b[e]));
  const double an = block_max(am, red);
  const double bn = block_max(bm, red);
  if (threadIdx.x == 0) {
    BatchIrState st{};
    st.active = 1;
    st.anorm = an;
    st.bnorm = bn;
    st.dprev = INFINITY;
    st.berr = INFINITY;
    *q.st = st;
  }
}

// After the factorisation: a zero pivot stops the system; permutation from the
// pivots; inverses of the diagonal blocks (grid: blocks x systems).
constexpr int BIR_MAXN = 1024;
__global__ void __launch_bounds__(TB) bir_post_lu_kernel(const BatchIr* __restrict__ sys) {
  // one shared buffer: the permutation's staging first (CTA 0), then the
  // inverse's triangle (every CTA holds one block: 34 KB, six CTAs an SM)
  __shared__ double T[TB][TB + 1];
  __shared__ double rdiag[TB];
  static_assert(2 * BIR_MAXN * sizeof(int32_t) <= sizeof(T), "the staging fits the triangle");
  int32_t* sp = reinterpret_cast<int32_t*>(&T[0][0]);
  const BatchIr q = sys[blockIdx.y];
  const int nblk = (q.n + TB - 1) / TB;
  if (blockIdx.x == 0) {  // the permutation, staged in shared memory
    for (int i = threadIdx.x; i < q.n; i += TB) {
      sp[i] = i;
      sp[BIR_MAXN + i] = q.ipiv[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (*q.info != 0) q.st->active = 0;
      for (int j = 0; j < q.n; ++j) {
        const int r = sp[BIR_MAXN + j];
        if (r != j) {
          const int32_t t = sp[j];
          sp[j] = sp[r];
          sp[r] = t;
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < q.n; i += TB) q.perm[i] = sp[i];
    __syncthreads();  // the staging is read before the triangle overwrites it
  }
  if (static_cast<int>(blockIdx.x) >= 2 * nblk) return;
  const bool lower = static_cast<int>(blockIdx.x) < nblk;
  const int blk = lower ? blockIdx.x : blockIdx.x - nblk;
  if (lower)
    diag_inverse_body<true>(q.LU, q.n, q.n, blk, q.Linv + static_cast<int64_t>(blk) * TB * TB, T,
                            rdiag);
  else
    diag_inverse_body<false>(q.LU, q.n, q.n, blk, q.Uinv + static_cast<int64_t>(blk) * TB * TB, T,
                             rdiag);
}

// d[i] -= F[i, b0 .. b0+bs) y for rows rs <= i < re (F the system's FP32
// factors): eight lanes a row, four rows a warp at a time, each lane eight
// consecutive columns (the eight lanes read the row's 256 bytes together),
// the eight partial sums added by three shuffles.  A warp a row would add
// five shuffle levels of FP64 adds to the row's two FMAs a lane, a thread a
// row would read the factor column-wise.
__device__ __forceinline__ void block_row_update(const BatchIr& q, const double (*y)[MAXR + 1],
                                                 int b0, int bs, int rs, int re) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = q.n, R = q.nrhs;
  const int g = lane >> 3, c0 = (lane & 7) * 8;  // row slot in the warp, first column
  for (int c = 0; c < R; ++c) {
    double yv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) yv[k] = c0 + k < bs ? y[c0 + k][c] : 0.0;
    for (int i0 = rs + wid * 4; i0 < re; i0 += nw * 4) {
      const int i = i0 + g;
      const bool ok = i < re;
      const float* fr = q.LU + static_cast<int64_t>(ok ? i : i0) * n + b0 + c0;
      double s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        if (ok && c0 + k < bs) s0 = fma(widen(fr[k]), yv[k], s0);
        if (ok && c0 + k + 1 < bs) s1 = fma(widen(fr[k + 1]), yv[k + 1], s1);
      }
      double sum = s0 + s1;
      sum += __shfl_xor_sync(0xFFFFFFFFu, sum, 4);
      sum += __shfl_xor_sync(0xFFFFFFFFu, sum, 2);
      sum += __shfl_xor_sync(0xFFFFFFFFu, sum, 1);
      if (ok && (lane & 7) == 0) q.d[static_cast<int64_t>(i) * R + c] -= sum;
    }
  }
}

// d <- U^-1 L^-1 P r for one system in one CTA: blocks in sequence, each
// block's inverse applied (Q threads an output, their partial sums added by
// shuffle), then the rows still to solve updated (a thread a row and column,
// four independent partial sums: with many systems resident an SM this
// beats the coalesced warp-a-row form of block_row_update).
template <bool WARPROW = false>
__device__ void bir_solve_body(const BatchIr& q) {
  __shared__ double y[TB][MAXR + 1];
  const int n = q.n, R = q.nrhs, t = threadIdx.x, NT = blockDim.x;
  for (int e = t; e < n * R; e += NT) {
    const int i = e / R, c = e % R;
    q.d[e] = q.r[static_cast<int64_t>(q.perm[i]) * R + c];
  }
  __syncthreads();
  const int nblk = (n + TB - 1) / TB;
  // the largest power of two Q <= 8 with TB R Q <= BIR_THREADS: TB R Q is a
  // multiple of 64, so whole warps take part in the shuffles or leave
  int Q = 8;
  while (Q > 1 && TB * R * Q > NT) Q >>= 1;
  const int len = TB / Q;
  for (int pass = 0; pass < 2; ++pass) {
    const bool lower = pass == 0;
    for (int bb = 0; bb < nblk; ++bb) {
      const int blk = lower ? bb : nblk - 1 - bb;
      const int b0 = blk * TB, bs = min(TB, n - b0);
      const double* D = (lower ? q.Linv : q.Uinv) + static_cast<int64_t>(blk) * TB * TB;
      for (int e = t; e < TB * R * Q; e += NT) {  // one pass when TB R <= BIR_THREADS
        const int o = e / Q, qq = e - o * Q;
        const int i = o / R, c = o - i * R;
        const int l0 = qq * len, l1 = min(l0 + len, bs);
        double s0 = 0.0, s1 = 0.0;
        int l = l0;
        for (; l + 1 < l1; l += 2) {
          s0 = fma(D[i * TB + l], q.d[static_cast<int64_t>(b0 + l) * R + c], s0);
          s1 = fma(D[i * TB + l + 1], q.d[static_cast<int64_t>(b0 + l + 1) * R + c], s1);
        }
        if (l < l1) s0 = fma(D[i * TB + l], q.d[static_cast<int64_t>(b0 + l) * R + c], s0);
        double sum = s0 + s1;
        for (int o2 = 1; o2 < Q; o2 <<= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o2);
        if (qq == 0 && i < bs) y[i][c] = sum;
      }
      __syncthreads();
      for (int e = t; e < bs * R; e += NT) {
        const int i = e / R, c = e % R;
        q.d[static_cast<int64_t>(b0 + i) * R + c] = y[i][c];
      }
      const int rs = lower ? b0 + bs : 0, re = lower ? n : b0;
      if (WARPROW) {
        block_row_update(q, y, b0, bs, rs, re);
      } else {
        for (int e = t; e < (re - rs) * R; e += NT) {
        const int i = rs + e / R, c = e % R;
        const float* fr = q.LU + static_cast<int64_t>(i) * n + b0;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int l = 0;
        for (; l + 3 < bs; l += 4) {
          s0 = fma(widen(fr[l]), y[l][c], s0);
          s1 = fma(widen(fr[l + 1]), y[l + 1][c], s1);
          s2 = fma(widen(fr[l + 2]), y[l + 2][c], s2);
          s3 = fma(widen(fr[l + 3]), y[l + 3][c], s3);
        }
        for (; l < bs; ++l) s0 = fma(widen(fr[l]), y[l][c], s0);
        q.d[static_cast<int64_t>(i) * R + c] -= (s0 + s1) + (s2 + s3);
        }
      }
      __syncthreads();
    }
  }
}

// x0 = LU^-1 b
__global__ void __launch_bounds__(BIR_THREADS) bir_first_solve_kernel(const BatchIr* __restrict__ sys) {
  __shared__ double red[BIR_THREADS / 32];
  const BatchIr q = sys[blockIdx.x];
  if (!q.st->active) return;
  for (int e = threadIdx.x; e < q.n * q.nrhs; e += BIR_THREADS) q.r[e] = q.b[e];
  __syncthreads();
  bir_solve_body(q);
  double xm = 0.0;
  for (int e = threadIdx.x; e < q.n * q.nrhs; e += BIR_THREADS) {
    q.x[e] = q.d[e];
    xm = fmax(xm, fabs(q.d[e]));
  }
  const double xn = block_max(xm, red);
  if (threadIdx.x == 0) q.st->dprev = xn;
}

// out = b - A x (b null: out = A x) for one system, n x R columns (FP64;
// warp a row).  Returns max |out| when asked.
__device__ double bir_matvec(const float* __restrict__ A, int n, int R, const double* x,
                             const double* __restrict__ b, double* out, double* red,
                             bool want_max) {
  // eight lanes a row, four rows a warp at a time: each lane takes every
  // eighth column (two independent partial sums), three shuffle levels add
  // the eight lanes' sums (a warp a row spent five levels of FP64 adds on
  // each row's sixteen FMAs a lane at n = 512)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = lane >> 3, sub = lane & 7;
  double rm = 0.0;
  for (int i0 = wid * 4; i0 < n; i0 += nw * 4) {
    const int i = i0 + g;
    const bool ok = i < n;
    const float* a = A + static_cast<int64_t>(ok ? i : i0) * n;
    for (int c = 0; c < R; ++c) {
      double s0 = 0.0, s1 = 0.0;
      int l = sub;
      for (; l + 8 < n; l += 16) {
        s0 = fma(widen(a[l]), x[static_cast<int64_t>(l) * R + c], s0);
        s1 = fma(widen(a[l + 8]), x[static_cast<int64_t>(l + 8) * R + c], s1);
      }
      if (l < n) s0 = fma(widen(a[l]), x[static_cast<int64_t>(l) * R + c], s0);
      double sum = s0 + s1;
      sum += __shfl_xor_sync(0xFFFFFFFFu, sum, 4);
      sum += __shfl_xor_sync(0xFFFFFFFFu, sum, 2);
      sum += __shfl_xor_sync(0xFFFFFFFFu, sum, 1);
      if (ok && sub == 0) {
        const double v = b ? b[static_cast<int64_t>(i) * R + c] - sum : sum;
        out[static_cast<int64_t>(i) * R + c] = v;
        rm = fmax(rm, fabs(v));
      }
    }
  }
  return want_max ? block_max(rm, red) : 0.0;
}

// r = b - A x for one system.  Returns max |r| when asked.
__device__ double bir_residual_body(const BatchIr& q, double* red, bool want_max) {
  return bir_matvec(q.A, q.n, q.nrhs, q.x, q.b, q.r, red, want_max);
}

// One refinement step of every active system: r = b - A x, d = LU^-1 P r,
// x += d, and the stop decision (converged / stalled) on the device.
// LAT: the form for the later steps, when few systems are still active
// and a step's time is the latency of the slowest: BIR_LAT_THREADS threads
// and the coalesced warp-a-row block updates (with many systems resident an
// SM, the default form's thread-a-row updates and three CTAs an SM win).
constexpr int BIR_LAT_THREADS = 1024;
template <bool LAT>
__global__ void __launch_bounds__(LAT ? BIR_LAT_THREADS : BIR_THREADS)
    bir_step_kernel(const BatchIr* __restrict__ sys, BatchIrParams p) {
  __shared__ double red[BIR_LAT_THREADS / 32];
  const BatchIr q = sys[blockIdx.x];
  if (!q.st->active) return;
  bir_residual_body(q, red, false);
  __syncthreads();
  bir_solve_body<LAT>(q);
  double dm = 0.0, xm = 0.0;
  for (int e = threadIdx.x; e < q.n * q.nrhs; e += static_cast<int>(blockDim.x)) {
    const double xv = q.x[e] + q.d[e];
    q.x[e] = xv;
    dm = fmax(dm, fabs(q.d[e]));
    xm = fmax(xm, fabs(xv));
  }
  const double dn = block_max(dm, red);
  const double xn = block_max(xm, red);
  if (threadIdx.x == 0) {
    BatchIrState* st = q.st;
    st->iters += 1;
    if (!(dn == dn) || !(xn == xn)) {
      st->active = 0;
    } else if (dn <= p.tol * xn) {
      st->active = 0;
      st->conv = 1;
    } else if (dn >= p.stall * st->dprev) {
      st->active = 0;
      st->stalled = 1;
    } else {
      st->dprev = dn;
    }
  }
}

// Backward error of every system; stalled systems within tol_b count as converged.
__global__ void __launch_bounds__(BIR_THREADS) bir_finish_kernel(const BatchIr* __restrict__ sys,
                                                                BatchIrParams p) {
  __shared__ double red[BIR_THREADS / 32];
  const BatchIr q = sys[blockIdx.x];
  if (*q.info != 0) {
    if (threadIdx.x == 0) {
      q.out->converged = 0;
      q.out->iters = 0;
      q.out->info = *q.info;
      q.out->gmres_steps = 0;
      q.out->berr = INFINITY;
    }
    return;
  }
  const double rn = bir_residual_body(q, red, true);
  double xm = 0.0;
  for (int e = threadIdx.x; e < q.n * q.nrhs; e += BIR_THREADS) xm = fmax(xm, fabs(q.x[e]));
  const double xn = block_max(xm, red);
  if (threadIdx.x == 0) {
    BatchIrState* st = q.st;
    const double den = st->anorm * xn + st->bnorm;
    double be = den > 0.0 ? rn / den : 0.0;
    if (!(be == be)) be = INFINITY;
    st->berr = be;
    if (!st->conv && st->stalled && be <= p.tol_b) st->conv = 1;
    st->active = 0;
    q.out->converged = st->conv;
    q.out->iters = st->iters;
    q.out->info = 0;
    q.out->gmres_steps = 0;
    q.out->berr = be;
  }
}

int grid_elems(int64_t work) {
  const int sms = current_num_sms() > 0 ? current_num_sms() : 148;
  const int64_t g = ceil_div(work, 256);
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, 8LL * sms)));
}

// Per-column stop state of the asynchronous solve (bfx_solve_ir_async).
struct IraState {
  int32_t conv, stalled, iters, pad;
  double dprev;
};

struct IrWs {
  float* LU;
  int32_t* ipiv;
  int32_t* perm;
  int32_t* info;
  int32_t* active;
  double* r;
  double* d;
  double* norms;  // [0] anorm, then per column: bn, dn, xn, rn
  double* Linv;   // inverses of the 64 x 64 diagonal blocks of L, then of U
  double* Uinv;
  double* Lg;     // chain matrices Linv_b L[b, b-1] (block b), Linv_b L[b, b-2] (nblk + b)
  double* Ug;     // the same for U with U[b, b+1], U[b, b+2]
  double* xch;    // triangular solves' exchange of row-slice sums (2 n x nrhs)
  double* y1;     // forward-solve result (sentinel-filled between solves)
  double* XL;     // L^-1 and U^-1 in FP64 (GMRES only), 64 x 64 blocks in solve order
  double* XU;
  double* Hl;     // inverse-scaled blocks Linv_b L[b, k] (GMRES only, in place of XL)
  double* Hu;     // the same for U (in place of XU)
  double* y2;     // backward-solve output of the triangular solves (published values)
  int32_t* tsync; // triangular-solve tickets, one per triangle
  int32_t* live;  // asynchronous solve: columns still refining (0: later steps skip)
  IraState* ira;  // asynchronous solve: per-column stop state
  void* luws;
  size_t luws_bytes;
  // GMRES-IR (gm_m > 0 only)
  int gm_m, gm_nchunk, gm_rows;
  double* V;      // (m+1) blocks of n x R
  double* H;      // R x m columns of m+1 (column j of column c's matrix contiguous)
  double* cs;     // R x m
  double* sn;     // R x m
  double* g;      // R x (m+1)
  double* y;      // R x m
  double* beta;   // R
  double* hb;     // (m+1) x R, one Gram-Schmidt pass's coefficients
  double* part;   // (m+1) x nchunk x R
  double* part2;  // ceil((m+1) / GM_KC) x n x R, the chunk sums of a long Gram-Schmidt update
  int32_t* flags; // 2 x R (Arnoldi-active, alternating between steps)
  int32_t* kdone; // R
  size_t total;
};

IrWs carve(void* base, bfx_mode mode, int64_t n, int64_t nrhs, int nb, int gm_m) {
  IrWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return static_cast<char*>(base) + o;
  };
  w.LU = reinterpret_cast<float*>(take(sizeof(float) * n * n));
  w.ipiv = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
  w.perm = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
  w.info = reinterpret_cast<int32_t*>(take(sizeof(int32_t)));
  w.active = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * nrhs));
  w.r = reinterpret_cast<double*>(take(sizeof(double) * n * nrhs));
  w.d = reinterpret_cast<double*>(take(sizeof(double) * n * nrhs));
  w.norms = reinterpret_cast<double*>(take(sizeof(double) * (1 + 4 * nrhs)));
  const int64_t nblk = (n + TB - 1) / TB;
  w.Linv = reinterpret_cast<double*>(take(sizeof(double) * nblk * TB * TB));
  w.Uinv = reinterpret_cast<double*>(take(sizeof(double) * nblk * TB * TB));
  w.Lg = reinterpret_cast<double*>(take(sizeof(double) * 2 * nblk * TB * TB));
  w.Ug = reinterpret_cast<double*>(take(sizeof(double) * 2 * nblk * TB * TB));
  w.y1 = reinterpret_cast<double*>(take(sizeof(double) * n * nrhs));
  w.y2 = reinterpret_cast<double*>(take(sizeof(double) * n * nrhs));
  w.xch = reinterpret_cast<double*>(take(sizeof(double) * 2 * n * nrhs));
  w.tsync = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 2));
  w.live = reinterpret_cast<int32_t*>(take(sizeof(int32_t)));
  w.ira = reinterpret_cast<IraState*>(take(sizeof(IraState) * nrhs));
  size_t lub = 0;
  for (bfx_mode m : {BFX_X1, BFX_X3, BFX_X6, BFX_X8, BFX_X9})
    if (static_cast<int>(m) >= static_cast<int>(mode)) lub = std::max(lub, lu_workspace_bytes(m, n, nb));
  w.luws_bytes = lub;
  w.luws = lub ? take(lub) : nullptr;
  w.gm_m = gm_m;
  if (gm_m > 0) {
    const int64_t R = nrhs, m = gm_m;
    const int64_t xblocks = nblk * (nblk + 1) / 2;  // the row-sliced blocks need nblk fewer
    w.XL = reinterpret_cast<double*>(take(sizeof(double) * xblocks * TB * TB));
    w.XU = reinterpret_cast<double*>(take(sizeof(double) * xblocks * TB * TB));
    w.Hl = w.XL;  // a GMRES phase uses one preconditioner form
    w.Hu = w.XU;
    int64_t rows = std::max<int64_t>(1, GM_ELEMS / R);
    int64_t nch = ceil_div(n, rows);
    if (nch > GM_MAXCH) {
      rows = ceil_div(n, GM_MAXCH);
      nch = ceil_div(n, rows);
    }
    w.gm_rows = static_cast<int>(rows);
    w.gm_nchunk = static_cast<int>(nch);
    w.V = reinterpret_cast<double*>(take(sizeof(double) * (m + 1) * n * R));
    w.H = reinterpret_cast<double*>(take(sizeof(double) * R * (m + 1) * m));
    w.cs = reinterpret_cast<double*>(take(sizeof(double) * R * m));
    w.sn = reinterpret_cast<double*>(take(sizeof(double) * R * m));
    w.g = reinterpret_cast<double*>(take(sizeof(double) * R * (m + 1)));
    w.y = reinterpret_cast<double*>(take(sizeof(double) * R * m));
    w.beta = reinterpret_cast<double*>(take(sizeof(double) * R));
    w.hb = reinterpret_cast<double*>(take(sizeof(double) * (m + 1) * R));
    w.part = reinterpret_cast<double*>(take(sizeof(double) * (m + 1) * nch * R));
    w.part2 = reinterpret_cast<double*>(take(sizeof(double) * ceil_div(m + 1, GM_KC) * n * R));
    w.flags = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 2 * R));
    w.kdone = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * R));
  }
  w.total = off;
  return w;
}

// y = X v (all nrhs columns) with X an explicit inverse (ir_xmv_kernel)
template <bool LOWER>
void inverse_mv(const double* X, int64_t n, int nrhs, const double* v, double* y, cudaStream_t s) {
  const int N = static_cast<int>(n), nblk = static_cast<int>(ceil_div(n, TB));
  const unsigned grid = static_cast<unsigned>(ceil_div((n + 1) / 2, XMV_THREADS / 32));
  int c0 = 0;
  for (; c0 + 4 <= nrhs; c0 += 4)
    launch_pdl(ir_xmv_kernel<LOWER, 4>, grid, XMV_THREADS, 0, s, X, N, nblk, v, y, nrhs, c0);
  for (; c0 + 2 <= nrhs; c0 += 2)
    launch_pdl(ir_xmv_kernel<LOWER, 2>, grid, XMV_THREADS, 0, s, X, N, nblk, v, y, nrhs, c0);
  for (; c0 < nrhs; ++c0)
    launch_pdl(ir_xmv_kernel<LOWER, 1>, grid, XMV_THREADS, 0, s, X, N, nblk, v, y, nrhs, c0);
}

// How M^-1 = U^-1 L^-1 P is applied: the chained block solve (every solve
// outside a GMRES phase), the row-sliced solve with the inverse-scaled
// blocks Hl, Hu, or the explicit inverses XL, XU (both prepared once per
// factorisation for a GMRES phase).
enum class GmPrec { kChain, kRowSliced, kInverse };

// d <- U^-1 L^-1 P r (all columns; r is left as it is).  d = P r (gathered),
// the forward solve reads d and writes y1, the backward solve reads y1 and
// writes d.  The gather also fills y1 with the sentinel and zeroes both
// tickets; the forward solve leaves d all sentinel for the backward one.
// kRowSliced: the row-sliced solves instead; the backward one publishes
// through y2 (also sentinel-filled by the gather) and writes its result to d.
// kInverse: d = P r, y1 = L^-1 d, d = U^-1 y1 by two matrix-vector products.
bfx_status lu_solve64(const IrWs& w, int64_t n, int nrhs, cudaStream_t s,
                      GmPrec prec = GmPrec::kChain, const int32_t* gate = nullptr) {
  static const bool attr_ok = [] {
    return cudaFuncSetAttribute(ir_trsv_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kTrsvSmem)) == cudaSuccess &&
           cudaFuncSetAttribute(ir_trsv_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kTrsvSmem)) == cudaSuccess;
  }();
  if (!attr_ok) return BFX_ECUDA;
  int* err = device_error_word();
  if (!err) return BFX_ECUDA;
  const int N = static_cast<int>(n);
  const int nblk = static_cast<int>(ceil_div(n, TB));
  if (prec == GmPrec::kInverse) {  // launched as dependents of their predecessors
    launch_pdl(ir_gather_kernel, dim3(static_cast<unsigned>(grid_elems(n * nrhs))), 256, 0, s,
               static_cast<const double*>(w.r), static_cast<int64_t>(nrhs),
               static_cast<const int32_t*>(w.perm), n, nrhs, w.d, static_cast<int64_t>(nrhs),
               static_cast<double*>(nullptr), static_cast<double*>(nullptr),
               static_cast<double*>(nullptr), static_cast<int*>(nullptr),
               gate);
    inverse_mv<true>(w.XL, n, nrhs, w.d, w.y1, s);
    inverse_mv<false>(w.XU, n, nrhs, w.y1, w.d, s);
    return last_launch_status();
  }
  if (prec == GmPrec::kRowSliced) {
    const int G = static_cast<int>(ceil_div(nrhs, TRSV_CG));
    const unsigned hgrid = static_cast<unsigned>(nblk * G * TRSV_S);
    ir_gather_kernel<<<grid_elems(n * nrhs), 256, 0, s>>>(w.r, nrhs, w.perm, n, nrhs, w.d, nrhs,
                                                          w.y1, w.y2, nullptr, w.tsync, gate);
    ir_trsv_h_kernel<true><<<hgrid, TRSV_THREADS, 0, s>>>(w.Hl, w.Linv, N, w.d, w.y1, nullptr,
                                                          nrhs, w.tsync, err);
    ir_trsv_h_kernel<false><<<hgrid, TRSV_THREADS, 0, s>>>(w.Hu, w.Uinv, N, w.y1, w.y2, w.d,
                                                           nrhs, w.tsync + 1, err);
    return last_launch_status();
  }
  const int G = static_cast<int>(ceil_div(nrhs, TRSV_CG));
  const unsigned grid = static_cast<unsigned>(nblk * G * TRSV_SLICES);
  // d = P r; both triangles' outputs set to the sentinel; L y1 = d; U y2 = y1
  // with the result also copied into d
  ir_gather_kernel<<<grid_elems(n * nrhs), 256, 0, s>>>(w.r, nrhs, w.perm, n, nrhs, w.d, nrhs,
                                                        w.y1, w.y2, w.xch, w.tsync, gate);
  ir_trsv_kernel<true><<<grid, TRSV_THREADS, kTrsvSmem, s>>>(
      w.LU, n, N, w.Linv, w.Lg, w.d, w.y1, nullptr, w.xch, nrhs, w.tsync, err, gate);
  ir_trsv_kernel<false><<<grid, TRSV_THREADS, kTrsvSmem, s>>>(
      w.LU, n, N, w.Uinv, w.Ug, w.y1, w.y2, w.d, w.xch + n * nrhs, nrhs, w.tsync + 1, err, gate);
  return last_launch_status();
}

// L^-1 and U^-1 of the FP32 factors in w.LU (FP64, into w.XL and w.XU), from
// the diagonal blocks' inverses w.Linv, w.Uinv; once per factorisation.
bfx_status form_inverses(const IrWs& w, int64_t n, cudaStream_t s) {
  static const bool attr_ok = [] {
    const int b = static_cast<int>(kXbSmem);
    return cudaFuncSetAttribute(ir_xupd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b) ==
               cudaSuccess &&
           cudaFuncSetAttribute(ir_xupd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b) ==
               cudaSuccess &&
           cudaFuncSetAttribute(ir_xfin_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b) ==
               cudaSuccess &&
           cudaFuncSetAttribute(ir_xfin_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b) ==
               cudaSuccess;
  }();
  if (!attr_ok) return BFX_ECUDA;
  const int N = static_cast<int>(n), nblk = static_cast<int>(ceil_div(n, TB));
  const unsigned nx = static_cast<unsigned>(nblk * (nblk + 1) / 2);
  ir_xinit_kernel<true><<<nx, XB_THREADS, 0, s>>>(w.Linv, nblk, w.XL);
  ir_xinit_kernel<false><<<nx, XB_THREADS, 0, s>>>(w.Uinv, nblk, w.XU);
  for (int t = 0; t + 1 < nblk; ++t) {
    const unsigned M = static_cast<unsigned>(nblk - 1 - t);
    ir_xupd_kernel<true><<<dim3(M, M), XB_THREADS, kXbSmem, s>>>(w.LU, n, N, nblk, t, w.XL);
    ir_xupd_kernel<false><<<dim3(M, M), XB_THREADS, kXbSmem, s>>>(w.LU, n, N, nblk, t, w.XU);
    ir_xfin_kernel<true><<<M, XB_THREADS, kXbSmem, s>>>(w.Linv, nblk, t + 1, w.XL);
    ir_xfin_kernel<false><<<M, XB_THREADS, kXbSmem, s>>>(w.Uinv, nblk, t + 1, w.XU);
  }
  return last_launch_status();
}

// pdl: launched as a dependent of its predecessor (inside a GMRES step)
bfx_status residual(const IrWs& w, const float* A, int64_t lda, int64_t n, int nrhs,
                    const double* b, int64_t ldb, const double* x, int64_t ldx, double* rn,
                    cudaStream_t s, const int32_t* gate = nullptr, bool pdl = false) {
  const unsigned blocks = static_cast<unsigned>(ceil_div(n, RES_ROWS));
  const int N = static_cast<int>(n);
  auto go = [&](auto kernel, int c0) {
    if (pdl)
      launch_pdl(kernel, dim3(blocks), 256, 0, s, A, lda, N, b, ldb, x, ldx, w.r,
                 static_cast<int64_t>(nrhs), c0, rn, gate);
    else
      kernel<<<blocks, 256, 0, s>>>(A, lda, N, b, ldb, x, ldx, w.r, nrhs, c0, rn, gate);
  };
  int c0 = 0;
  for (; c0 + 8 <= nrhs; c0 += 8) go(ir_residual_kernel<8>, c0);
  for (; c0 + 4 <= nrhs; c0 += 4) go(ir_residual_kernel<4>, c0);
  for (; c0 + 2 <= nrhs; c0 += 2) go(ir_residual_kernel<2>, c0);
  for (; c0 < nrhs; ++c0) go(ir_residual_kernel<1>, c0);
  return last_launch_status();
}

// Pinned, device-mapped host slots and events through which the GMRES loop
// reads the Arnoldi-active flags without stalling the stream: the Givens
// kernel writes each step's flags into a slot directly (no copy in the
// stream), and the host reads the slot after the event recorded behind it
// (one set per host thread and device, released when the thread ends).
constexpr int GM_LAG = 2;               // steps launched ahead of the flags read
constexpr int GM_RING = GM_LAG + 2;
struct GmFlagRing {
  int dev = -1;
  int32_t* h = nullptr;   // GM_RING x MAXR
  int32_t* hd = nullptr;  // the same memory, device address
  cudaEvent_t ev[GM_RING] = {};
  ~GmFlagRing() { release(); }
  void release() {
    if (h) cudaFreeHost(h);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    h = hd = nullptr;
    for (auto& e : ev) e = nullptr;
    dev = -1;
  }
  bool ready() {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) return false;
    if (d == dev && h) return true;
    release();
    if (cudaHostAlloc(reinterpret_cast<void**>(&h), sizeof(int32_t) * GM_RING * MAXR,
                      cudaHostAllocMapped) != cudaSuccess) {
      h = nullptr;
      return false;
    }
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&hd), h, 0) != cudaSuccess) {
      release();
      return false;
    }
    for (auto& e : ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        release();
        return false;
      }
    dev = d;
    return true;
  }
};

// One GMRES cycle for every refinement-active column.  On entry w.r holds
// r = b - A x (consumed); on exit w.d holds the correction (0 in the other
// columns).  *steps = Arnoldi steps run (the most over the columns).  After
// each step the R Arnoldi-active flags are copied to pinned host memory; the
// host reads the copy GM_LAG + 1 steps later (long complete by then), so the
// stream never drains, and stops launching once no column is active.  Up to
// GM_LAG + 1 steps launched past the last active one find every column
// inactive and leave the state alone (the kernels skip inactive columns).
bfx_status gmres_cycle(const IrWs& w, const float* A, int64_t lda, int64_t n, int R, double tau,
                       cudaStream_t s, int* steps, GmPrec prec) {
  thread_local GmFlagRing ring;
  if (!ring.ready()) return BFX_ECUDA;
  const int N = static_cast<int>(n), m = w.gm_m, nch = w.gm_nchunk;
  const int64_t vstride = n * R;
  const int grid = grid_elems(n * R);
  bfx_status st;
  *steps = 0;
  if ((st = lu_solve64(w, n, R, s, prec)) != BFX_OK) return st;  // w.d = M^-1 r
  gm_dot_kernel<<<dim3(1, nch), GM_THREADS, 0, s>>>(w.d, 0, w.d, N, R, w.gm_rows, nch, w.part);
  gm_start_kernel<<<grid, GM_THREADS, 0, s>>>(w.V, w.d, N, R, w.part, nch, w.g, w.beta, m, w.active,
                                              w.flags, w.kdone);
  {  // the flags after the start ("step -1") into ring slot GM_RING - 1, by a copy
    const int slot = GM_RING - 1;
    if (cudaMemcpyAsync(ring.h + slot * MAXR, w.flags, sizeof(int32_t) * R, cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaEventRecord(ring.ev[slot], s) != cudaSuccess)
      return BFX_ECUDA;
  }
  int j = 0;
  for (; j < m; ++j) {
    const int look = j - 1 - GM_LAG;  // the step whose output flags decide (-1: the start)
    if (look >= -1) {
      const int slot = (look + GM_RING) % GM_RING;
      if (cudaEventSynchronize(ring.ev[slot]) != cudaSuccess) return BFX_ECUDA;
      bool any = false;
      for (int c = 0; c < R; ++c) any = any || ring.h[slot * MAXR + c];
      if (!any) break;
    }
    int32_t* ain = w.flags + (j & 1) * R;
    int32_t* aout = w.flags + ((j + 1) & 1) * R;
    const double* vj = w.V + static_cast<int64_t>(j) * vstride;
    // w.d = M^-1 A v_j; every kernel of the step launched as a dependent of
    // the one before it (programmatic dependent launch)
    if ((st = residual(w, A, lda, n, R, nullptr, 0, vj, R, nullptr, s, nullptr, true)) != BFX_OK)
      return st;
    if ((st = lu_solve64(w, n, R, s, prec)) != BFX_OK) return st;
    const int64_t r64 = R;
    const unsigned g1 = static_cast<unsigned>(grid);
    // with many vectors, each CTA of a Gram-Schmidt dot product takes a whole
    // vector (its fixed costs outweighed the 1024 FMAs of a chunk)
    const int pch = j + 1 >= GM_WHOLE ? 1 : nch;
    const int prows = pch == 1 ? N : w.gm_rows;
    for (int pass = 0; pass < 2; ++pass) {
      launch_pdl(gm_dot_kernel, dim3(static_cast<unsigned>(j + 1), pch), GM_THREADS, 0, s,
                 static_cast<const double*>(w.V), vstride, static_cast<const double*>(w.d), N, R,
                 prows, pch, w.part);
      launch_pdl(gm_reduce_h_kernel, dim3(static_cast<unsigned>(ceil_div((j + 1) * r64, 256))), 256, 0,
                 s, static_cast<const double*>(w.part), pch, j + 1, R, w.hb, w.H, m, j, pass,
                 static_cast<const int32_t*>(ain));
      if (j + 1 > GM_KC) {
        const int nkc = static_cast<int>(ceil_div(j + 1, GM_KC));
        const unsigned eb = static_cast<unsigned>(ceil_div(n * R, GM_PT));
        launch_pdl(gm_orth_part_kernel, dim3(eb, nkc), GM_PT, 0, s, static_cast<const double*>(w.V),
                   vstride, j + 1, N, R, static_cast<const double*>(w.hb),
                   static_cast<const int32_t*>(ain), w.part2);
        launch_pdl(gm_orth_finish_kernel, dim3(g1), GM_THREADS, 0, s, w.d, N, R,
                   static_cast<const int32_t*>(ain), static_cast<const double*>(w.part2), nkc);
      } else {
        launch_pdl(gm_orth_kernel, dim3(g1), GM_THREADS, 0, s, static_cast<const double*>(w.V),
                   vstride, j + 1, w.d, N, R, static_cast<const double*>(w.hb),
                   static_cast<const int32_t*>(ain));
      }
    }
    launch_pdl(gm_dot_kernel, dim3(1, nch), GM_THREADS, 0, s, static_cast<const double*>(w.d),
               static_cast<int64_t>(0), static_cast<const double*>(w.d), N, R, w.gm_rows, nch, w.part);
    launch_pdl(gm_next_kernel, dim3(g1), GM_THREADS, 0, s, w.V, vstride, j,
               static_cast<const double*>(w.d), N, R, static_cast<const double*>(w.part), nch,
               static_cast<const int32_t*>(ain));
    const int slot = (j + GM_RING) % GM_RING;
    launch_pdl(gm_givens_kernel, dim3(static_cast<unsigned>(R)), GIV_THREADS, 0, s, j, R,
               static_cast<const double*>(w.part), nch, w.H, w.cs, w.sn, w.g,
               static_cast<const double*>(w.beta), m, tau, static_cast<const int32_t*>(ain), aout,
               w.kdone, ring.hd + slot * MAXR);
    if (cudaGetLastError() != cudaSuccess) return BFX_ECUDA;
    if (cudaEventRecord(ring.ev[slot], s) != cudaSuccess) return BFX_ECUDA;
  }
  // steps taken: the most over the columns
  std::vector<int32_t> kd(R);
  if (cudaMemcpyAsync(kd.data(), w.kdone, sizeof(int32_t) * R, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BFX_ECUDA;
  for (int c = 0; c < R; ++c) *steps = std::max(*steps, static_cast<int>(kd[c]));
  gm_solve_y_kernel<<<R, 32, sizeof(double) * m, s>>>(w.H, w.g, w.kdone, w.active, m, w.y);
  gm_combine_kernel<<<grid, GM_THREADS, 0, s>>>(w.V, vstride, w.y, w.kdone, w.active, N, R, m, w.d);
  return last_launch_status();
}

// ------------------------------------------------------------- batched GMRES-IR
// Systems whose plain refinement stopped unconverged (and whose factors are
// regular) continue by GMRES-IR, as bfx_solve_ir does with gmres = 1:
// restarted GMRES(min(n, m)) in FP64 preconditioned by the system's FP32
// factors, each right-hand side with its own Krylov basis, the first
// correction exempt from the stall test.  A persistent grid of CTAs takes
// systems from an atomic queue, one CTA a system, all of its work inside the
// CTA; each CTA owns one slot of Krylov memory (basis, Hessenberg columns,
// rotations) sized for the largest system.  Orthogonalisation: two classical
// Gram-Schmidt passes, each coefficient a warp dot product with a fixed
// reduction order (deterministic).
struct BgmSlot {
  double *V, *H, *hc, *g, *cs, *sn, *y;
};
__device__ __forceinline__ BgmSlot bgm_carve(double* base, int mm, int n, int R) {
  BgmSlot sl;
  sl.V = base;                                        // (mm + 1) x n x R
  sl.H = sl.V + static_cast<int64_t>(mm + 1) * n * R;  // R x mm columns of mm + 1
  sl.hc = sl.H + static_cast<int64_t>(R) * mm * (mm + 1);  // (mm + 1) x R, one pass
  sl.g = sl.hc + static_cast<int64_t>(mm + 1) * R;     // R x (mm + 1)
  sl.cs = sl.g + static_cast<int64_t>(R) * (mm + 1);   // R x mm
  sl.sn = sl.cs + static_cast<int64_t>(R) * mm;
  sl.y = sl.sn + static_cast<int64_t>(R) * mm;
  return sl;
}

// ---- groups of CTAs on one hard system (batched GMRES-IR)
// BGM_GROUP CTAs share a system: CTA rank r owns whole 64-row blocks
// [r nbr, (r+1) nbr) (nbr = ceil(nblk / BGM_GROUP)), computes matrix-vector
// products, dot products and updates on those rows only, and the group
// combines its partial sums through a mailbox in global memory: each CTA
// writes its values, then publishes an exchange number with a release
// store; its partners wait (bounded) for that number with acquire loads and
// read the values from L2.  Every CTA of a group runs the same control flow
// on the same combined values (sums taken in rank order), so their decisions
// agree.  Mailbox slots alternate by exchange parity: a CTA writes slot
// e & 1 again only at exchange e + 2, which it reaches after its partners
// have finished reading exchange e.  Three CTAs a system measured best on
// a batch of 2000 systems up to n = 512 whose 56 hard systems then hold 147
// of the 148 SMs (2: 43.1 ms, 3: 41.6 ms, 4: 42.9 ms a batch).
constexpr int BGM_GROUP = 3;
constexpr int kErrWaitGroup = 8;  // device error word: a group exchange expired

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

struct BgmBox {
  double* data;               // [BGM_GROUP][2][xmax]: exchanged values
  unsigned long long* seq;    // [BGM_GROUP]: the last exchange each rank published
  double* ybox;               // [2][nbmax][TB * MAXR]: block results of the triangular solves
  unsigned long long* yseq;   // [2][nbmax]: the solve each block result belongs to
  int xmax, nbmax;
};
__host__ __device__ inline int64_t bgm_box_doubles(int xmax, int nbmax) {
  return static_cast<int64_t>(BGM_GROUP) * 2 * xmax + BGM_GROUP +
         static_cast<int64_t>(2) * nbmax * TB * MAXR + 2 * static_cast<int64_t>(nbmax);
}
__device__ __forceinline__ BgmBox bgm_box(double* base, int xmax, int nbmax) {
  BgmBox b;
  b.data = base;
  b.seq = reinterpret_cast<unsigned long long*>(base + static_cast<int64_t>(BGM_GROUP) * 2 * xmax);
  b.ybox = base + static_cast<int64_t>(BGM_GROUP) * 2 * xmax + BGM_GROUP;
  b.yseq = reinterpret_cast<unsigned long long*>(b.ybox + static_cast<int64_t>(2) * nbmax * TB * MAXR);
  b.xmax = xmax;
  b.nbmax = nbmax;
  return b;
}
// thread 0: wait until *p >= want (4 s of %globaltimer at most)
__device__ __forceinline__ bool group_wait(const unsigned long long* p, unsigned long long want,
                                           int* err) {
  if (ld_acquire_u64(p) >= want) return true;
  const uint64_t t0 = global_ns();
  while (ld_acquire_u64(p) < want) {
    if (global_ns() - t0 > 4000000000ull) {
      atomicExch(err, kErrWaitGroup);
      return false;
    }
  }
  return true;
}
// res[i] = sum (OP 0) or max of non-negative values (OP 1) over the group's
// vals[i], i < cnt <= xmax, in rank order; res may alias vals.  All threads
// call it; false: a wait expired (*fail set, the group leaves).
template <int OP>
__device__ bool group_reduce(const BgmBox& bx, int rank, unsigned long long& ex, const double* vals,
                             double* res, int cnt, int* err, volatile int* fail) {
  const int t = threadIdx.x, NT = blockDim.x;
  if (BGM_GROUP == 1) {
    if (res != vals)
      for (int i = t; i < cnt; i += NT) res[i] = vals[i];
    __syncthreads();
    return true;
  }
  const unsigned long long e = ++ex;
  double* mine = bx.data + (static_cast<int64_t>(rank) * 2 + (e & 1)) * bx.xmax;
  for (int i = t; i < cnt; i += NT) mine[i] = vals[i];
  __syncthreads();
  if (t == 0) {
    __threadfence();
    st_release_u64(&bx.seq[rank], e);
    for (int r = 0; r < BGM_GROUP && !*fail; ++r)
      if (r != rank && !group_wait(&bx.seq[r], e, err)) *fail = 1;
  }
  __syncthreads();
  if (*fail) return false;
  for (int i = t; i < cnt; i += NT) {
    double a = 0.0;
    for (int r = 0; r < BGM_GROUP; ++r) {
      const double v =
          r == rank ? vals[i] : __ldcg(bx.data + (static_cast<int64_t>(r) * 2 + (e & 1)) * bx.xmax + i);
      if (r == 0 || OP == 0) {
        a = r == 0 ? v : a + v;
      } else {  // non-negative doubles order like their bits (NaN above Inf)
        a = __longlong_as_double(max(static_cast<unsigned long long>(__double_as_longlong(a)),
                                     static_cast<unsigned long long>(__double_as_longlong(v))));
      }
    }
    res[i] = a;
  }
  __syncthreads();
  return true;
}
// the group waits until every rank has reached this point (its earlier
// global writes visible to the others)
__device__ __forceinline__ bool group_sync(const BgmBox& bx, int rank, unsigned long long& ex,
                                           int* err, volatile int* fail) {
  return group_reduce<0>(bx, rank, ex, nullptr, nullptr, 0, err, fail);
}

// out = b - A x (b null: out = A x) on rows [lo, hi) of one system (warp a
// row, four independent partial sums a lane); x is read from L2 (its rows
// come from the whole group).  Returns the CTA's max |out|.
__device__ __forceinline__ double bgm_matvec_rows(const float* __restrict__ A, int n, int R,
                                                  const double* x, const double* __restrict__ b,
                                                  double* out, int lo, int hi) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double rm = 0.0;
  for (int i = lo + wid; i < hi; i += nw) {
    const float* a = A + static_cast<int64_t>(i) * n;
    for (int c = 0; c < R; ++c) {
      double sum = 0.0;
      for (int l = lane; l < n; l += 32) sum = fma(widen(a[l]), __ldcg(x + static_cast<int64_t>(l) * R + c), sum);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
      const double v = b ? b[static_cast<int64_t>(i) * R + c] - sum : sum;
      if (lane == 0) out[static_cast<int64_t>(i) * R + c] = v;
      rm = fmax(rm, fabs(v));
    }
  }
  return rm;
}

// y = D_blk d[block blk] (the block's inverse, Q threads an output) into ys,
// written back into d; published in the mailbox for the other ranks when
// the group has more than one CTA.  All threads call it.
__device__ __forceinline__ void bgm_block_inverse(const BatchIr& q, const BgmBox& bx, int pass,
                                                  int blk, unsigned long long tok,
                                                  double (*ys)[MAXR + 1]) {
  const int n = q.n, R = q.nrhs, t = threadIdx.x, NT = blockDim.x;
  const int b0 = blk * TB, bs = min(TB, n - b0);
  int Q = 8;  // as in bir_solve_body
  while (Q > 1 && TB * R * Q > NT) Q >>= 1;
  const int len = TB / Q;
  const double* D = (pass == 0 ? q.Linv : q.Uinv) + static_cast<int64_t>(blk) * TB * TB;
  for (int e = t; e < TB * R * Q; e += NT) {
    const int o = e / Q, qq = e - o * Q;
    const int i = o / R, c = o - i * R;
    const int l0 = qq * len, l1 = min(l0 + len, bs);
    double s0 = 0.0, s1 = 0.0;
    int l = l0;
    for (; l + 1 < l1; l += 2) {
      s0 = fma(D[i * TB + l], q.d[static_cast<int64_t>(b0 + l) * R + c], s0);
      s1 = fma(D[i * TB + l + 1], q.d[static_cast<int64_t>(b0 + l + 1) * R + c], s1);
    }
    if (l < l1) s0 = fma(D[i * TB + l], q.d[static_cast<int64_t>(b0 + l) * R + c], s0);
    double sum = s0 + s1;
    for (int o2 = 1; o2 < Q; o2 <<= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o2);
    if (qq == 0 && i < bs) ys[i][c] = sum;
  }
  __syncthreads();
  double* box = bx.ybox + (static_cast<int64_t>(pass) * bx.nbmax + blk) * TB * MAXR;
  for (int e = t; e < bs * R; e += NT) {
    const int i = e / R, c = e % R;
    q.d[static_cast<int64_t>(b0 + i) * R + c] = ys[i][c];
    if (BGM_GROUP > 1) box[e] = ys[i][c];
  }
  if (BGM_GROUP > 1) {
    __syncthreads();
    if (t == 0) {
      __threadfence();
      st_release_u64(bx.yseq + pass * bx.nbmax + blk, tok);
    }
  }
  __syncthreads();
}

// d <- U^-1 L^-1 P r on rows [lo, hi) of one system, shared by the group:
// the owner of each 64-row block applies its inverse and hands the block's
// result to the others through the mailbox (tagged with the solve number
// sv); every rank updates its own rows below (L) or above (U) the block.
// One block of look-ahead: a rank that owns the next block in solve order
// first updates that block's rows, applies its inverse and publishes it,
// and only then updates its other rows, so the chain from one block's
// result to the next block's result holds one 64-row update, not all of
// them.  r is read from L2 (its rows come from the whole group).
__device__ bool bgm_solve(const BatchIr& q, const BgmBox& bx, int rank, int nbr, int lo, int hi,
                          unsigned long long& sv, int* err, volatile int* fail) {
  __shared__ double ybuf[2][TB][MAXR + 1];
  const int n = q.n, R = q.nrhs, t = threadIdx.x, NT = blockDim.x;
  for (int e = t; e < (hi - lo) * R; e += NT) {
    const int i = lo + e / R, c = e % R;
    q.d[static_cast<int64_t>(i) * R + c] = __ldcg(q.r + static_cast<int64_t>(q.perm[i]) * R + c);
  }
  __syncthreads();
  const unsigned long long tok = ++sv;
  const int nblk = (n + TB - 1) / TB;
  auto owner_of = [&](int blk) { return min(BGM_GROUP - 1, blk / nbr); };
  for (int pass = 0; pass < 2; ++pass) {
    const bool lower = pass == 0;
    int cur = 0;  // ybuf[cur] holds the current block's result once known here
    const int first = lower ? 0 : nblk - 1;
    if (owner_of(first) == rank) bgm_block_inverse(q, bx, pass, first, tok, ybuf[cur]);
    for (int bb = 0; bb < nblk; ++bb) {
      const int blk = lower ? bb : nblk - 1 - bb;
      const int b0 = blk * TB, bs = min(TB, n - b0);
      if (owner_of(blk) != rank) {  // the block's result from its owner
        if (t == 0 && !*fail && !group_wait(bx.yseq + pass * bx.nbmax + blk, tok, err)) *fail = 1;
        __syncthreads();
        if (*fail) return false;
        const double* box = bx.ybox + (static_cast<int64_t>(pass) * bx.nbmax + blk) * TB * MAXR;
        for (int e = t; e < bs * R; e += NT) ybuf[cur][e / R][e % R] = __ldcg(box + e);
        __syncthreads();
      }
      const double (*y)[MAXR + 1] = ybuf[cur];
      // rows this rank still updates with this block: below (L) or above (U)
      int rs = max(lower ? b0 + bs : 0, lo), re = min(lower ? n : b0, hi);
      const int nxt = lower ? blk + 1 : blk - 1;
      if (nxt >= 0 && nxt < nblk && owner_of(nxt) == rank) {  // look-ahead
        const int n0 = nxt * TB, ns = min(TB, n - n0);
        block_row_update(q, y, b0, bs, n0, n0 + ns);
        __syncthreads();
        bgm_block_inverse(q, bx, pass, nxt, tok, ybuf[cur ^ 1]);
        if (lower)
          rs = max(rs, n0 + ns);
        else
          re = min(re, n0);
      }
      block_row_update(q, y, b0, bs, rs, re);
      __syncthreads();
      cur ^= 1;
    }
  }
  return true;
}

// per-column sum of squares of v (n x R) -> out[c] (warp c, c + 8, ...)
__device__ __forceinline__ void bgm_colnorm(const double* v, int n, int R, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = wid; c < R; c += static_cast<int>(blockDim.x >> 5)) {
    double s2 = 0.0;
    for (int i = lane; i < n; i += 32) {
      const double a = v[static_cast<int64_t>(i) * R + c];
      s2 = fma(a, a, s2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, o);
    if (lane == 0) out[c] = s2;
  }
}

__global__ void __launch_bounds__(BGM_THREADS)
    bgm_kernel(const BatchIr* __restrict__ sys, int S, int* __restrict__ queue,
               double* __restrict__ slots, int64_t slot_doubles, double* __restrict__ boxes,
               int xmax, int nbmax, int m, BatchIrParams p, int max_outer, double tau,
               int* __restrict__ err) {
  __shared__ double s_beta[MAXR], s_tmp[MAXR], s_dprev[MAXR], s_dn[MAXR], s_xn[MAXR];
  __shared__ int s_act[MAXR], s_arn[MAXR], s_k[MAXR], s_conv[MAXR], s_stall[MAXR];
  __shared__ int s_sys, s_any, s_steps, s_fail;
  __shared__ double s_gA[BGM_THREADS / 32], s_gB[BGM_THREADS / 32], s_gp;  // Givens scan
  __shared__ double s_x[2];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  constexpr int NW = BGM_THREADS / 32;
  const int rank = static_cast<int>(blockIdx.x) % BGM_GROUP, grp = blockIdx.x / BGM_GROUP;
  // the group's shared Krylov basis, this rank's Hessenberg data, the mailbox
  double* base = slots + static_cast<int64_t>(grp) * slot_doubles;
  const BgmBox bx = bgm_box(boxes + static_cast<int64_t>(grp) * bgm_box_doubles(xmax, nbmax), xmax, nbmax);
  unsigned long long ex = 0, sv = 0;
  volatile int* fail = &s_fail;
  if (t == 0) s_fail = 0;
  __syncthreads();
  for (;;) {
    // rank 0 takes the next system from the queue and hands it to the group
    if (t == 0) s_x[0] = rank == 0 ? static_cast<double>(atomicAdd(queue, 1)) : 0.0;
    __syncthreads();
    if (!group_reduce<0>(bx, rank, ex, s_x, s_x, 1, err, fail)) return;
    const int k = static_cast<int>(s_x[0]);
    if (k >= S) break;
    const BatchIr q = sys[k];
    if (*q.info != 0 || q.st->conv) continue;
    const int n = q.n, R = q.nrhs, mm = min(m, n);
    const int nblk = (n + TB - 1) / TB, nbr = (nblk + BGM_GROUP - 1) / BGM_GROUP;
    const int lo = min(n, rank * nbr * TB), hi = min(n, (rank + 1) * nbr * TB);
    BgmSlot sl = bgm_carve(base, mm, n, R);
    {  // this rank's own copy of the small arrays (after the shared basis)
      const int64_t small = static_cast<int64_t>(R) * mm * (mm + 1) + (mm + 1) * R + R * (mm + 1) + 3 * R * mm;
      const int64_t shift = static_cast<int64_t>(rank) * small;
      sl.H += shift;
      sl.hc += shift;
      sl.g += shift;
      sl.cs += shift;
      sl.sn += shift;
      sl.y += shift;
    }
    const int64_t vs = static_cast<int64_t>(n) * R;  // one basis vector
    const int64_t e_lo = static_cast<int64_t>(lo) * R, e_hi = static_cast<int64_t>(hi) * R;
    if (t < R) {
      s_act[t] = 1;
      s_conv[t] = 0;
      s_stall[t] = 0;
      s_dprev[t] = INFINITY;
    }
    if (t == 0) s_steps = 0;
    __syncthreads();
    for (int outer = 0; outer < max_outer; ++outer) {
      if (t == 0) {
        int a = 0;
        for (int c = 0; c < R; ++c) a |= s_act[c];
        s_any = a;
      }
      __syncthreads();
      if (!s_any) break;
      // ---- r = b - A x, w = M^-1 r, beta = |w|_2, V_0 = w / beta, g = beta e_1
      bgm_matvec_rows(q.A, n, R, q.x, q.b, q.r, lo, hi);
      __syncthreads();
      if (!group_sync(bx, rank, ex, err, fail)) return;
      if (!bgm_solve(q, bx, rank, nbr, lo, hi, sv, err, fail)) return;
      bgm_colnorm(q.d + e_lo, hi - lo, R, s_tmp);
      __syncthreads();
      if (!group_reduce<0>(bx, rank, ex, s_tmp, s_tmp, R, err, fail)) return;
      if (t < R) {
        const double b = sqrt(s_tmp[t]);
        s_beta[t] = b;
        s_arn[t] = s_act[t] && b > 0.0 && b <= 1.7976931348623157e308;
        s_k[t] = 0;
        double* gc = sl.g + static_cast<int64_t>(t) * (mm + 1);
        for (int i = 0; i <= mm; ++i) gc[i] = 0.0;
        gc[0] = b;
      }
      __syncthreads();
      for (int64_t e = e_lo + t; e < e_hi; e += BGM_THREADS) {
        const int c = static_cast<int>(e % R);
        if (s_arn[c]) sl.V[e] = q.d[e] / s_beta[c];
      }
      __syncthreads();
      if (!group_sync(bx, rank, ex, err, fail)) return;
      // ---- Arnoldi
      for (int j = 0; j < mm; ++j) {
        if (t == 0) {
          int a = 0;
          for (int c = 0; c < R; ++c) a |= s_arn[c];
          s_any = a;
        }
        __syncthreads();
        if (!s_any) break;
        // w = M^-1 A v_j
        bgm_matvec_rows(q.A, n, R, sl.V + j * vs, nullptr, q.r, lo, hi);
        __syncthreads();
        if (!group_sync(bx, rank, ex, err, fail)) return;
        if (!bgm_solve(q, bx, rank, nbr, lo, hi, sv, err, fail)) return;
        for (int pass = 0; pass < 2; ++pass) {
          // hc[i][c] = <V_i, w> on this rank's rows (warp i mod NW), summed
          // over the group, then H(:, j) += hc
          for (int i = wid; i <= j; i += NW) {
            const double* vi = sl.V + i * vs;
            for (int c = 0; c < R; ++c) {
              double sum = 0.0;
              if (s_arn[c])
                for (int r = lo + lane; r < hi; r += 32)
                  sum = fma(vi[static_cast<int64_t>(r) * R + c], q.d[static_cast<int64_t>(r) * R + c], sum);
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
              if (lane == 0) sl.hc[static_cast<int64_t>(i) * R + c] = sum;
            }
          }
          __syncthreads();
          if (!group_reduce<0>(bx, rank, ex, sl.hc, sl.hc, (j + 1) * R, err, fail)) return;
          for (int e = t; e < (j + 1) * R; e += BGM_THREADS) {
            const int i = e / R, c = e % R;
            double* hp = sl.H + (static_cast<int64_t>(c) * mm + j) * (mm + 1) + i;
            *hp = pass ? *hp + sl.hc[e] : sl.hc[e];
          }
          for (int64_t e = e_lo + t; e < e_hi; e += BGM_THREADS) {
            const int c = static_cast<int>(e % R);
            if (!s_arn[c]) continue;
            // four partial sums over i mod 4 (independent chains), then w -= their sum
            double u0 = 0.0, u1 = 0.0, u2 = 0.0, u3 = 0.0;
            int i = 0;
            for (; i + 3 <= j; i += 4) {
              u0 = fma(sl.hc[static_cast<int64_t>(i) * R + c], sl.V[i * vs + e], u0);
              u1 = fma(sl.hc[static_cast<int64_t>(i + 1) * R + c], sl.V[(i + 1) * vs + e], u1);
              u2 = fma(sl.hc[static_cast<int64_t>(i + 2) * R + c], sl.V[(i + 2) * vs + e], u2);
              u3 = fma(sl.hc[static_cast<int64_t>(i + 3) * R + c], sl.V[(i + 3) * vs + e], u3);
            }
            for (; i <= j; ++i) u0 = fma(sl.hc[static_cast<int64_t>(i) * R + c], sl.V[i * vs + e], u0);
            q.d[e] -= (u0 + u1) + (u2 + u3);
          }
          __syncthreads();
        }
        // h_{j+1,j} = |w|_2, V_{j+1} = w / h, Givens (thread c)
        bgm_colnorm(q.d + e_lo, hi - lo, R, s_tmp);
        __syncthreads();
        if (!group_reduce<0>(bx, rank, ex, s_tmp, s_tmp, R, err, fail)) return;
        if (t < R) s_tmp[t] = sqrt(s_tmp[t]);
        __syncthreads();
        for (int64_t e = e_lo + t; e < e_hi; e += BGM_THREADS) {
          const int c = static_cast<int>(e % R);
          if (s_arn[c] && s_tmp[c] > 0.0) sl.V[(j + 1) * vs + e] = q.d[e] / s_tmp[c];
        }
        __syncthreads();
        for (int c = 0; c < R; ++c) {
          if (!s_arn[c]) continue;  // uniform over the CTA
          double* hcol = sl.H + (static_cast<int64_t>(c) * mm + j) * (mm + 1);
          double* csc = sl.cs + static_cast<int64_t>(c) * mm;
          double* snc = sl.sn + static_cast<int64_t>(c) * mm;
          const double pv = givens_apply_scan<BGM_THREADS, BGM_GIV_E>(hcol, csc, snc, j, s_gA, s_gB,
                                                                      &s_gp);
          if (t != 0) continue;
          double* gc = sl.g + static_cast<int64_t>(c) * (mm + 1);
          const double hj = s_tmp[c];
          const double rho = hypot(pv, hj);
          const double cj = rho > 0.0 ? pv / rho : 1.0, sj = rho > 0.0 ? hj / rho : 0.0;
          csc[j] = cj;
          snc[j] = sj;
          hcol[j] = rho;
          hcol[j + 1] = 0.0;
          gc[j + 1] = -sj * gc[j];
          gc[j] = cj * gc[j];
          s_k[c] = j + 1;
          const double res = fabs(gc[j + 1]);
          if (res <= tau * s_beta[c] || !(hj > 0.0) || j + 1 >= mm || !(res == res)) s_arn[c] = 0;
        }
        __syncthreads();
        if (!group_sync(bx, rank, ex, err, fail)) return;  // V_{j+1} whole before the next product
      }
      // ---- y = R_k^-1 g_k (warp per column, lanes split each row's sum)
      for (int c = wid; c < R; c += NW) {
        if (!s_act[c]) continue;
        const int kk = s_k[c];
        const double* Hc = sl.H + static_cast<int64_t>(c) * mm * (mm + 1);
        const double* gc = sl.g + static_cast<int64_t>(c) * (mm + 1);
        double* yc = sl.y + static_cast<int64_t>(c) * mm;
        for (int i = kk - 1; i >= 0; --i) {
          double u = 0.0;
          for (int l = i + 1 + lane; l < kk; l += 32)
            u = fma(Hc[static_cast<int64_t>(l) * (mm + 1) + i], yc[l], u);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xFFFFFFFFu, u, o);
          if (lane == 0) yc[i] = (gc[i] - u) / Hc[static_cast<int64_t>(i) * (mm + 1) + i];
          __syncwarp();
        }
      }
      __syncthreads();
      // ---- x += V y on refinement-active columns; |d|, |x| per column
      if (t < R) {
        s_dn[t] = 0.0;
        s_xn[t] = 0.0;
      }
      __syncthreads();
      for (int64_t e = e_lo + t; e < e_hi; e += BGM_THREADS) {
        const int c = static_cast<int>(e % R);
        if (!s_act[c]) continue;
        const double* yc = sl.y + static_cast<int64_t>(c) * mm;
        double u = 0.0;
        for (int i = 0; i < s_k[c]; ++i) u = fma(yc[i], sl.V[i * vs + e], u);
        const double xv = q.x[e] + u;
        q.x[e] = xv;
        atomic_max_nonneg(&s_dn[c], fabs(u));
        atomic_max_nonneg(&s_xn[c], fabs(xv));
      }
      __syncthreads();
      if (!group_reduce<1>(bx, rank, ex, s_dn, s_dn, R, err, fail)) return;
      if (!group_reduce<1>(bx, rank, ex, s_xn, s_xn, R, err, fail)) return;
      if (t < R && s_act[t]) {
        const double dn = s_dn[t], xn = s_xn[t];
        if (!(dn == dn) || !(xn == xn)) {
          s_act[t] = 0;
        } else if (dn <= p.tol * xn) {
          s_act[t] = 0;
          s_conv[t] = 1;
        } else if (dn >= p.stall * s_dprev[t]) {
          s_act[t] = 0;
          s_stall[t] = 1;
        } else {
          s_dprev[t] = dn;
        }
      }
      if (t == 0) s_steps += 1;
      __syncthreads();
    }
    // ---- backward error as bir_finish_kernel; converged if every column is
    if (t < 2) s_x[t] = 0.0;
    __syncthreads();
    {
      const double rm = bgm_matvec_rows(q.A, n, R, q.x, q.b, q.r, lo, hi);
      double xm = 0.0;
      for (int64_t e = e_lo + t; e < e_hi; e += BGM_THREADS) xm = fmax(xm, fabs(q.x[e]));
      atomic_max_nonneg(&s_x[0], rm);
      atomic_max_nonneg(&s_x[1], xm);
    }
    __syncthreads();
    if (!group_reduce<1>(bx, rank, ex, s_x, s_x, 2, err, fail)) return;
    const double rn = s_x[0], xn = s_x[1];
    if (t == 0 && rank == 0) {
      BatchIrState* st = q.st;
      const double den = st->anorm * xn + st->bnorm;
      double be = den > 0.0 ? rn / den : 0.0;
      if (!(be == be)) be = INFINITY;
      int all = 1;
      for (int c = 0; c < R; ++c) all &= (s_conv[c] || (s_stall[c] && be <= p.tol_b));
      st->conv = all;
      st->berr = be;
      st->iters += s_steps;
      q.out->converged = all;
      q.out->iters = st->iters;
      q.out->gmres_steps = s_steps;
      q.out->berr = be;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- asynchronous solve
// The stop decisions of bfx_solve_ir, made on the device so that a whole
// solve is enqueued without the host reading anything back.  *live counts
// the columns still refining; once it is 0 the gated kernels of the later
// steps return at once.

// after the factorisation: a zero pivot stops the solve before it starts
__global__ void ira_start_kernel(const int32_t* __restrict__ info, int R,
                                 int32_t* __restrict__ active, int32_t* __restrict__ live,
                                 IraState* __restrict__ st) {
  const bool ok = *info == 0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < R; c += gridDim.x * blockDim.x) {
    active[c] = ok ? 1 : 0;
    st[c] = IraState{0, 0, 0, 0, 0.0};
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *live = ok ? R : 0;
}

// x <- d (x0 of the asynchronous solve; nothing is written after a zero pivot)
__global__ void ira_copy_kernel(double* __restrict__ x, int64_t ldx, const double* __restrict__ d,
                                int64_t n, int R, const int32_t* __restrict__ gate) {
  if (*gate == 0) return;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n * R;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / R;
    const int c = static_cast<int>(e - i * R);
    x[i * ldx + c] = d[e];
  }
}

// after x0 = LU^-1 P b: the first correction is tested for a stall against |x0|
__global__ void ira_x0_kernel(const double* __restrict__ xn, int R, IraState* __restrict__ st) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < R; c += gridDim.x * blockDim.x)
    st[c].dprev = xn[c];
}

// after x += d: bfx_solve_ir's tests for every active column (one CTA)
__global__ void __launch_bounds__(256)
    ira_decide_kernel(const double* __restrict__ dn, const double* __restrict__ xn, int R,
                      double tol, double stall, int32_t* __restrict__ active,
                      IraState* __restrict__ st, int32_t* __restrict__ live) {
  __shared__ int count;
  if (*live == 0) return;  // this step ran nothing
  if (threadIdx.x == 0) count = 0;
  __syncthreads();
  int mine = 0;
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    if (!active[c]) continue;
    const double d = dn[c], x = xn[c];
    IraState q = st[c];
    ++q.iters;
    int act = 1;
    if (!(d == d) || !(x == x)) {  // NaN: diverged
      act = 0;
    } else if (d <= tol * x) {
      act = 0;
      q.conv = 1;
    } else if (d >= stall * q.dprev) {
      act = 0;
      q.stalled = 1;
    } else {
      q.dprev = d;
    }
    st[c] = q;
    active[c] = act;
    mine += act;
  }
  if (mine) atomicAdd(&count, mine);
  __syncthreads();
  if (threadIdx.x == 0) *live = count;
}

// after |x| (xn) and |b - A x| (rn) of every column: backward errors, the
// stalled columns whose backward error is small enough count as converged,
// and the result (one CTA)
__global__ void __launch_bounds__(256)
    ira_finish_kernel(const double* __restrict__ norms, int R, const IraState* __restrict__ st,
                      double tol_b, const int32_t* __restrict__ info, int mode,
                      bfx_ir_result* __restrict__ res) {
  __shared__ double s_berr[256];
  __shared__ int s_all[256], s_it[256];
  const double anorm = norms[0];
  const double* bn = norms + 1;
  const double* xn = bn + 2 * R;
  const double* rn = bn + 3 * R;
  double berr = 0.0;
  int all = 1, itmax = 0;
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    const double den = anorm * xn[c] + bn[c];
    double be = den > 0 ? rn[c] / den : 0.0;
    if (!(be == be)) be = INFINITY;
    const int conv = st[c].conv || (st[c].stalled && be <= tol_b);
    berr = fmax(berr, be);
    all = all && conv;
    itmax = max(itmax, st[c].iters);
  }
  s_berr[threadIdx.x] = berr;
  s_all[threadIdx.x] = all;
  s_it[threadIdx.x] = itmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < blockDim.x; ++k) {  // fixed order
      berr = fmax(berr, s_berr[k]);
      all = all && s_all[k];
      itmax = max(itmax, s_it[k]);
    }
    bfx_ir_result r{};
    r.info = *info;
    r.mode_used = mode;
    r.converged = (r.info == 0 && all) ? 1 : 0;
    r.iters = r.info == 0 ? itmax : 0;
    r.refactorizations = 0;
    r.berr = r.info == 0 ? berr : INFINITY;
    r.gmres_steps = 0;
    r.arnoldi = 0;
    *res = r;
  }
}

}  // namespace

// mailbox sizes of a group: any nrhs <= MAXR, any n <= BIR_MAXN
int bgm_xmax(int m) { return std::max(2, (m + 1) * MAXR); }
constexpr int kBgmNbMax = (BIR_MAXN + TB - 1) / TB;

// nslots slots of slot_doubles each (batched_gmres_slot_doubles): the groups'
// mailboxes first (cleared here, so every launch starts its exchange
// numbers from zero), then each group's Krylov basis and its ranks' small
// arrays.  One group of BGM_GROUP CTAs a slot, at most one CTA an SM.
bfx_status ir_batched_gmres(const BatchIr* d_ir, int S, int* d_queue, double* d_slots,
                            int64_t slot_doubles, int nslots, int m, BatchIrParams p,
                            int max_outer, double tau, cudaStream_t s) {
  if (S <= 0 || nslots <= 0) return BFX_OK;
  if (m > BGM_GIV_E * BGM_THREADS) return BFX_EINVAL;  // the Givens scan's rows per thread
  int* err = device_error_word();
  if (!err) return BFX_ECUDA;
  const int sms = current_num_sms() > 0 ? current_num_sms() : 148;
  const int groups = std::max(1, std::min(nslots, sms / BGM_GROUP));
  const int xmax = bgm_xmax(m);
  const int64_t box = bgm_box_doubles(xmax, kBgmNbMax);
  if (cudaMemsetAsync(d_queue, 0, sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(d_slots, 0, sizeof(double) * box * nslots, s) != cudaSuccess)
    return BFX_ECUDA;
  bgm_kernel<<<groups * BGM_GROUP, BGM_THREADS, 0, s>>>(
      d_ir, S, d_queue, d_slots + box * nslots, slot_doubles - box, d_slots, xmax, kBgmNbMax, m, p,
      max_outer, tau, err);
  return last_launch_status();
}

int64_t batched_gmres_slot_doubles(int m, int nmax, int R) {
  const int64_t mm = std::min(m, nmax);
  const int64_t small = R * mm * (mm + 1) + (mm + 1) * R + R * (mm + 1) + 3 * R * mm;
  return (mm + 1) * nmax * R + BGM_GROUP * small + bgm_box_doubles(bgm_xmax(m), kBgmNbMax);
}

bfx_status ir_batched_prepare(const BatchIr* d_ir, int S, int nmax, cudaStream_t s) {
  (void)nmax;
  if (S <= 0) return BFX_OK;
  bir_prepare_kernel<<<S, BIR_THREADS, 0, s>>>(d_ir);
  return last_launch_status();
}
bfx_status ir_batched_post_lu(const BatchIr* d_ir, int S, int nmax, cudaStream_t s) {
  if (S <= 0) return BFX_OK;
  const unsigned nblk = static_cast<unsigned>(ceil_div(nmax, TB));
  bir_post_lu_kernel<<<dim3(2 * nblk, S), TB, 0, s>>>(d_ir);
  return last_launch_status();
}
bfx_status ir_batched_first_solve(const BatchIr* d_ir, int S, cudaStream_t s) {
  if (S <= 0) return BFX_OK;
  bir_first_solve_kernel<<<S, BIR_THREADS, 0, s>>>(d_ir);
  return last_launch_status();
}
bfx_status ir_batched_step(const BatchIr* d_ir, int S, BatchIrParams p, cudaStream_t s) {
  if (S <= 0) return BFX_OK;
  bir_step_kernel<false><<<S, BIR_THREADS, 0, s>>>(d_ir, p);
  return last_launch_status();
}
// the same step in the latency form (later steps of a batch)
bfx_status ir_batched_step_latency(const BatchIr* d_ir, int S, BatchIrParams p, cudaStream_t s) {
  if (S <= 0) return BFX_OK;
  bir_step_kernel<true><<<S, BIR_LAT_THREADS, 0, s>>>(d_ir, p);
  return last_launch_status();
}
bfx_status ir_batched_finish(const BatchIr* d_ir, int S, BatchIrParams p, cudaStream_t s) {
  if (S <= 0) return BFX_OK;
  bir_finish_kernel<<<S, BIR_THREADS, 0, s>>>(d_ir, p);
  return last_launch_status();
}

}  // namespace bfx

using namespace bfx;

extern "C" {

namespace {

bfx_ir_params ir_defaults() {
  bfx_ir_params p{};
  p.max_iter = 50;
  p.tol = 1.1102230246251565e-16;
  p.tol_b = -1.0;
  p.stall = 0.5;
  p.escalate = 1;
  p.nb = 64;
  p.gmres = 1;
  p.gmres_m = 0;
  p.gmres_tol = 1e-10;
  p.gmres_inverses = 1;
  return p;
}

// Fills the defaults of zero / negative fields; false if a field is out of range.
bool ir_resolve(const bfx_ir_params* h, int64_t n, bfx_ir_params* out) {
  bfx_ir_params p = h ? *h : ir_defaults();
  if (p.nb <= 0) p.nb = 64;
  if (p.gmres_m == 0) p.gmres_m = static_cast<int>(std::min<int64_t>(n, BFX_GMRES_MAX_M));
  if (!(p.gmres_tol > 0.0)) p.gmres_tol = 1e-10;
  if (p.tol_b < 0) p.tol_b = 1.1102230246251565e-16 * std::sqrt(static_cast<double>(n));
  if (p.nb > 128 || p.max_iter < 0 || p.gmres < 0 || p.gmres > 2 || p.gmres_m < 0 ||
      p.gmres_m > BFX_GMRES_MAX_M || p.gmres_inverses < 0 || p.gmres_inverses > 1)
    return false;
  *out = p;
  return true;
}

}  // namespace

BFX_API size_t bfx_solve_ir_workspace_size(bfx_mode mode, int64_t n, int64_t nrhs,
                                           const bfx_ir_params* h_params) {
  if (n <= 0 || nrhs <= 0) return 0;
  bfx_ir_params p;
  if (!ir_resolve(h_params, n, &p)) return 0;
  return carve(nullptr, mode, n, nrhs, p.nb, p.gmres ? p.gmres_m : 0).total;
}

BFX_API bfx_status bfx_solve_ir(bfx_mode mode, int64_t n, int64_t nrhs, const float* d_A,
                                int64_t lda, const double* d_b, int64_t ldb, double* d_x,
                                int64_t ldx, const bfx_ir_params* h_params,
                                bfx_ir_result* h_result, void* d_ws, size_t ws_bytes,
                                bfx_stream stream) {
  if (mode != BFX_FP32 && mode_pieces(mode) == 0) return BFX_EINVAL;
  if (n < 0 || nrhs < 0 || !h_result) return BFX_EINVAL;
  bfx_ir_result res{};
  res.mode_used = mode;
  *h_result = res;
  if (n == 0 || nrhs == 0) {
    h_result->converged = 1;
    return BFX_OK;
  }
  if (!d_A || !d_b || !d_x || lda < n || ldb < nrhs || ldx < nrhs) return BFX_EINVAL;
  if (n >= (1 << 30) || nrhs > (1 << 20)) return BFX_EUNSUPPORTED;
  bfx_ir_params p;
  if (!ir_resolve(h_params, n, &p)) return BFX_EINVAL;
  if (p.gmres && nrhs > MAXR) return BFX_EUNSUPPORTED;  // one Krylov basis a column, <= 16
  if (mode != BFX_FP32 && !is_sm103()) return BFX_EUNSUPPORTED;
  IrWs w = carve(d_ws, mode, n, nrhs, p.nb, p.gmres ? p.gmres_m : 0);
  if (!d_ws || ws_bytes < w.total || !aligned(d_ws, 256)) return BFX_ENOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int R = static_cast<int>(nrhs);
  const int N = static_cast<int>(n);
  double* anorm = w.norms;
  double* bn = w.norms + 1;
  double* dn = bn + R;
  double* xn = dn + R;
  double* rn = xn + R;
  std::vector<double> h(1 + 4 * static_cast<size_t>(R));
  std::vector<int32_t> act(R, 1), conv(R, 0), iters(R, 0), stalled(R, 0);
  std::vector<double> dprev(R, 0.0);

  // |A|_inf and |b|_inf once
  if (cudaMemsetAsync(w.norms, 0, sizeof(double) * (1 + 4 * R), s) != cudaSuccess) return BFX_ECUDA;
  ir_anorm_kernel<<<static_cast<unsigned>(ceil_div(n * 32, 256)), 256, 0, s>>>(d_A, lda, N, anorm);
  // b may have ldb > nrhs: column max over the first nrhs columns
  ir_colmax_kernel<<<grid_elems(n * R), 256, 0, s>>>(d_b, ldb, n, R, bn);

  bfx_mode cur = mode;
  bool first = true, refactor = true, use_gmres = p.gmres == 2, x_ready = false;
  bfx_status st = BFX_OK;
  for (;;) {
    if (refactor) {
      // ---- factor (again, after an escalation)
      if (cudaMemcpy2DAsync(w.LU, sizeof(float) * n, d_A, sizeof(float) * lda, sizeof(float) * n,
                            n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return BFX_ECUDA;
      st = lu_factor(cur, n, p.nb, w.LU, n, w.ipiv, w.info, w.luws, w.luws_bytes, s, w.perm);
      if (st != BFX_OK) return st;
      int32_t info = 0;
      if (cudaMemcpyAsync(&info, w.info, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
              cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return BFX_ECUDA;
      h_result->info = info;
      if (info != 0) return BFX_SINGULAR;
      const unsigned nblk = static_cast<unsigned>(ceil_div(n, TB));
      ir_diag_inverse_kernel<<<2 * nblk, TB, 0, s>>>(w.LU, n, N, w.Linv, w.Uinv);
      if (nblk > 1)
        ir_chain_kernel<<<dim3(2 * (nblk - 1), TB / CHAIN_HALF, 2), 256, 0, s>>>(w.LU, n, N, w.Linv,
                                                                            w.Uinv, w.Lg, w.Ug);
      x_ready = false;
    }
    if (cudaMemcpyAsync(w.active, act.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return BFX_ECUDA;
    if (first) {
      // x0 = LU^-1 b: r <- b, solve, x <- d
      if (cudaMemcpy2DAsync(w.r, sizeof(double) * R, d_b, sizeof(double) * ldb, sizeof(double) * R,
                            n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return BFX_ECUDA;
      if ((st = lu_solve64(w, n, R, s)) != BFX_OK) return st;
      if (cudaMemcpy2DAsync(d_x, sizeof(double) * ldx, w.d, sizeof(double) * R, sizeof(double) * R,
                            n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return BFX_ECUDA;
      if (cudaMemsetAsync(xn, 0, sizeof(double) * R, s) != cudaSuccess) return BFX_ECUDA;
      ir_colmax_kernel<<<grid_elems(n * R), 256, 0, s>>>(d_x, ldx, n, R, xn);
      if (cudaMemcpyAsync(h.data(), w.norms, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                          s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return BFX_ECUDA;
      for (int c = 0; c < R; ++c) dprev[c] = use_gmres ? INFINITY : h[1 + 2 * R + c];  // |x0|
      first = false;
    } else {
      // fresh factors, or the switch to GMRES: no stall test on the first correction
      for (int c = 0; c < R; ++c) dprev[c] = INFINITY;
    }
    // ---- refinement loop
    for (int it = 0; it < p.max_iter; ++it) {
      bool any = false;
      for (int c = 0; c < R; ++c) any = any || act[c];
      if (!any) break;
      if ((st = residual(w, d_A, lda, n, R, d_b, ldb, d_x, ldx, nullptr, s)) != BFX_OK) return st;
      if (use_gmres) {
        const GmPrec prec = p.gmres_inverses ? GmPrec::kInverse : GmPrec::kRowSliced;
        if (!x_ready) {  // once per factorisation: the preconditioner's prepared form
          if (prec == GmPrec::kInverse) {
            if ((st = form_inverses(w, n, s)) != BFX_OK) return st;
          } else {
            const unsigned nblk = static_cast<unsigned>(ceil_div(n, TB));
            if (nblk > 1) {
              ir_hmat_kernel<true><<<dim3(nblk, nblk), 256, 0, s>>>(w.LU, n, N, w.Linv, w.Hl);
              ir_hmat_kernel<false><<<dim3(nblk, nblk), 256, 0, s>>>(w.LU, n, N, w.Uinv, w.Hu);
            }
          }
          x_ready = true;
        }
        int k = 0;
        if ((st = gmres_cycle(w, d_A, lda, n, R, p.gmres_tol, s, &k, prec)) != BFX_OK) return st;
        h_result->gmres_steps += 1;
        h_result->arnoldi += k;
      } else if ((st = lu_solve64(w, n, R, s)) != BFX_OK) {
        return st;
      }
      if (cudaMemsetAsync(dn, 0, sizeof(double) * 2 * R, s) != cudaSuccess) return BFX_ECUDA;
      ir_update_kernel<<<grid_elems(n * R), 256, 0, s>>>(d_x, ldx, w.d, R, n, R, w.active, dn, xn,
                                                         nullptr);
      if (cudaMemcpyAsync(h.data(), w.norms, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                          s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return BFX_ECUDA;
      bool changed = false;
      for (int c = 0; c < R; ++c) {
        if (!act[c]) continue;
        const double d_c = h[1 + R + c], x_c = h[1 + 2 * R + c];
        ++iters[c];
        if (!(d_c == d_c) || !(x_c == x_c)) {  // NaN: diverged
          act[c] = 0;
          changed = true;
        } else if (d_c <= p.tol * x_c) {
          act[c] = 0;
          conv[c] = 1;
          changed = true;
        } else if (d_c >= p.stall * dprev[c]) {
          act[c] = 0;
          stalled[c] = 1;
          changed = true;
        } else {
          dprev[c] = d_c;
        }
      }
      if (changed &&
          cudaMemcpyAsync(w.active, act.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice, s) !=
              cudaSuccess)
        return BFX_ECUDA;
    }
    // ---- backward error of every column
    if (cudaMemsetAsync(xn, 0, sizeof(double) * 2 * R, s) != cudaSuccess) return BFX_ECUDA;
    ir_colmax_kernel<<<grid_elems(n * R), 256, 0, s>>>(d_x, ldx, n, R, xn);
    if ((st = residual(w, d_A, lda, n, R, d_b, ldb, d_x, ldx, rn, s)) != BFX_OK) return st;
    if (cudaMemcpyAsync(h.data(), w.norms, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return BFX_ECUDA;
    double berr_max = 0.0;
    bool all = true;
    for (int c = 0; c < R; ++c) {
      const double den = h[0] * h[1 + 2 * R + c] + h[1 + c];
      double be = den > 0 ? h[1 + 3 * R + c] / den : 0.0;
      if (!(be == be)) be = INFINITY;
      if (!conv[c] && stalled[c] && be <= p.tol_b) conv[c] = 1;
      berr_max = std::max(berr_max, be);
      all = all && conv[c];
    }
    h_result->berr = berr_max;
    int itmax = 0;
    for (int c = 0; c < R; ++c) itmax = std::max(itmax, iters[c]);
    h_result->iters = itmax;
    h_result->converged = all ? 1 : 0;
    h_result->mode_used = cur;
    if (all) return BFX_OK;
    // ---- next phase: refactor with more products, else GMRES-IR on these factors
    bfx_mode next = cur;
    if (cur == BFX_X1) next = BFX_X3;
    else if (cur == BFX_X3) next = BFX_X6;
    if (!use_gmres && p.escalate && next != cur) {
      cur = next;
      refactor = true;
      h_result->refactorizations += 1;
    } else if (!use_gmres && p.gmres) {
      use_gmres = true;
      refactor = false;
    } else {
      return BFX_NOT_CONVERGED;
    }
    for (int c = 0; c < R; ++c) {
      act[c] = conv[c] ? 0 : 1;
      stalled[c] = 0;
    }
  }
}

BFX_API bfx_status bfx_solve_ir_async(bfx_mode mode, int64_t n, int64_t nrhs, const float* d_A,
                                      int64_t lda, const double* d_b, int64_t ldb, double* d_x,
                                      int64_t ldx, const bfx_ir_params* h_params,
                                      bfx_ir_result* d_result, void* d_ws, size_t ws_bytes,
                                      bfx_stream stream) {
  if (mode != BFX_FP32 && mode_pieces(mode) == 0) return BFX_EINVAL;
  if (n <= 0 || nrhs <= 0 || !d_result) return BFX_EINVAL;
  if (!d_A || !d_b || !d_x || lda < n || ldb < nrhs || ldx < nrhs) return BFX_EINVAL;
  if (n >= (1 << 30) || nrhs > (1 << 20)) return BFX_EUNSUPPORTED;
  bfx_ir_params p = ir_defaults();
  p.escalate = 0;
  p.gmres = 0;
  if (h_params) p = *h_params;
  if (p.escalate != 0 || p.gmres != 0) return BFX_EINVAL;  // both need host decisions
  if (!ir_resolve(&p, n, &p)) return BFX_EINVAL;
  if (mode != BFX_FP32 && !is_sm103()) return BFX_EUNSUPPORTED;
  IrWs w = carve(d_ws, mode, n, nrhs, p.nb, 0);
  if (!d_ws || ws_bytes < w.total || !aligned(d_ws, 256)) return BFX_ENOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int R = static_cast<int>(nrhs);
  const int N = static_cast<int>(n);
  double* anorm = w.norms;
  double* bn = w.norms + 1;
  double* dn = bn + R;
  double* xn = dn + R;
  double* rn = xn + R;
  const unsigned cgrid = static_cast<unsigned>(std::min<int64_t>(ceil_div(R, 256), 1024));
  bfx_status st;
  if (cudaMemsetAsync(w.norms, 0, sizeof(double) * (1 + 4 * R), s) != cudaSuccess) return BFX_ECUDA;
  ir_anorm_kernel<<<static_cast<unsigned>(ceil_div(n * 32, 256)), 256, 0, s>>>(d_A, lda, N, anorm);
  ir_colmax_kernel<<<grid_elems(n * R), 256, 0, s>>>(d_b, ldb, n, R, bn);
  // ---- factor; a zero pivot leaves *live = 0 and every gated kernel idle
  if (cudaMemcpy2DAsync(w.LU, sizeof(float) * n, d_A, sizeof(float) * lda, sizeof(float) * n, n,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return BFX_ECUDA;
  if ((st = lu_factor(mode, n, p.nb, w.LU, n, w.ipiv, w.info, w.luws, w.luws_bytes, s, w.perm)) !=
      BFX_OK)
    return st;
  ira_start_kernel<<<cgrid, 256, 0, s>>>(w.info, R, w.active, w.live, w.ira);
  const unsigned nblk = static_cast<unsigned>(ceil_div(n, TB));
  ir_diag_inverse_kernel<<<2 * nblk, TB, 0, s>>>(w.LU, n, N, w.Linv, w.Uinv);
  if (nblk > 1)
    ir_chain_kernel<<<dim3(2 * (nblk - 1), TB / CHAIN_HALF, 2), 256, 0, s>>>(w.LU, n, N, w.Linv, w.Uinv,
                                                                        w.Lg, w.Ug);
  // ---- x0 = LU^-1 P b
  if (cudaMemcpy2DAsync(w.r, sizeof(double) * R, d_b, sizeof(double) * ldb, sizeof(double) * R, n,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return BFX_ECUDA;
  if ((st = lu_solve64(w, n, R, s, GmPrec::kChain, w.live)) != BFX_OK) return st;
  ira_copy_kernel<<<grid_elems(n * R), 256, 0, s>>>(d_x, ldx, w.d, n, R, w.live);
  ir_colmax_kernel<<<grid_elems(n * R), 256, 0, s>>>(d_x, ldx, n, R, xn);
  ira_x0_kernel<<<cgrid, 256, 0, s>>>(xn, R, w.ira);
  // ---- max_iter refinement steps, each skipped once every column stopped
  for (int it = 0; it < p.max_iter; ++it) {
    if ((st = residual(w, d_A, lda, n, R, d_b, ldb, d_x, ldx, nullptr, s, w.live)) != BFX_OK)
      return st;
    if ((st = lu_solve64(w, n, R, s, GmPrec::kChain, w.live)) != BFX_OK) return st;
    if (cudaMemsetAsync(dn, 0, sizeof(double) * 2 * R, s) != cudaSuccess) return BFX_ECUDA;
    ir_update_kernel<<<grid_elems(n * R), 256, 0, s>>>(d_x, ldx, w.d, R, n, R, w.active, dn, xn,
                                                       w.live);
    ira_decide_kernel<<<1, 256, 0, s>>>(dn, xn, R, p.tol, p.stall, w.active, w.ira, w.live);
  }
  // ---- backward errors and the result
  if (cudaMemsetAsync(xn, 0, sizeof(double) * 2 * R, s) != cudaSuccess) return BFX_ECUDA;
  ir_colmax_kernel<<<grid_elems(n * R), 256, 0, s>>>(d_x, ldx, n, R, xn);
  if ((st = residual(w, d_A, lda, n, R, d_b, ldb, d_x, ldx, rn, s)) != BFX_OK) return st;
  ira_finish_kernel<<<1, 256, 0, s>>>(w.norms, R, w.ira, p.tol_b, w.info, static_cast<int>(mode),
                                      d_result);
  return last_launch_status();
}

}  // extern "C"
