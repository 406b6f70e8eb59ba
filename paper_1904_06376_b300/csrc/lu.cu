// Blocked right-looking LU with partial pivoting whose trailing update is the
// bf16xN product (Sec. IV-A of the paper: "SGETRF based on triplets of BF16s
// and six products"; Sec. III: the cubic work in low precision).
//
// For each block column j0 (width jb <= nb):
//   panel   : unblocked FP32 LU of A[j0:n, j0:j0+jb] - pivot = first row of the
//             largest |a| (warp-shuffle argmax), row swap inside the panel,
//             division by the pivot, FMA rank-1 updates of the panel;
//   laswp   : the panel's row swaps applied to the columns left and right of it;
//   trsm    : U12 = L11^-1 A12 (unit lower, FP32 FMA, one thread a column);
//   update  : A22 <- A22 - L21 U12 by the mode's bfloat16 products on the
//             tensor cores (split of L21, transposed split of U12, tcgen05
//             GEMM with alpha = -1, beta = 1), or the FP32 SIMT GEMM.
// Pivots: ipiv[j] (0-based) is the row swapped with row j at step j.  info is
// LAPACK's: 0, or the 1-based index of the first exactly zero pivot (the
// factorisation still completes).
#include "bfx_internal.cuh"

namespace bfx {
namespace {

constexpr int PANEL_THREADS = 1024;

struct ArgMax {
  float v;
  int i;
};

__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b) {
  // larger value wins; equal values: the smaller row index (LAPACK i?amax)
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}

// One CTA factors the panel A[j0:n, j0:j0+jb] in place.  Thread t owns rows
// j0 + t, j0 + t + 1024, ...; rows above the current column are finished.
__global__ void __launch_bounds__(PANEL_THREADS) lu_panel_kernel(float* __restrict__ A, int64_t lda,
                                                               int n, int j0, int jb,
                                                               int32_t* __restrict__ ipiv,
                                                               int32_t* __restrict__ info) {
  __shared__ ArgMax warp_best[PANEL_THREADS / 32];
  __shared__ int s_piv;
  __shared__ float s_row[256];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  for (int j = j0; j < j0 + jb; ++j) {
    // ---- pivot search over rows j..n-1 of column j
    ArgMax best{-1.0f, n};
    for (int r = j + t; r < n; r += PANEL_THREADS) {
      float v = fabsf(A[static_cast<int64_t>(r) * lda + j]);
      if (v != v) v = -1.0f;  // NaN below the diagonal is never chosen
      best = better(best, ArgMax{v, r});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ArgMax other{__shfl_xor_sync(0xFFFFFFFFu, best.v, o), __shfl_xor_sync(0xFFFFFFFFu, best.i, o)};
      best = better(best, other);
    }
    if (lane == 0) warp_best[wid] = best;
    __syncthreads();
    if (wid == 0) {
      best = warp_best[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ArgMax other{__shfl_xor_sync(0xFFFFFFFFu, best.v, o), __shfl_xor_sync(0xFFFFFFFFu, best.i, o)};
        best = better(best, other);
      }
      if (lane == 0) {
        const float d = A[static_cast<int64_t>(j) * lda + j];
        // a NaN on the diagonal stays (nothing compares greater than it)
        s_piv = (d != d || best.i >= n) ? j : best.i;
        ipiv[j] = s_piv;
      }
    }
    __syncthreads();
    const int p = s_piv;
    // ---- swap rows j and p inside the panel; keep the pivot row in shared memory
    for (int c = t; c < jb; c += PANEL_THREADS) {
      float* rj = A + static_cast<int64_t>(j) * lda + j0 + c;
      float* rp = A + static_cast<int64_t>(p) * lda + j0 + c;
      const float a = *rj, b = *rp;
      if (p != j) {
        *rj = b;
        *rp = a;
      }
      s_row[c] = (p != j) ? b : a;
    }
    __syncthreads();
    const float piv = s_row[j - j0];
    if (piv == 0.0f) {
      if (t == 0 && *info == 0) *info = j + 1;
      __syncthreads();
      continue;
    }
    // ---- scale the column and update the rest of the panel
    for (int r = j + 1 + t; r < n; r += PANEL_THREADS) {
      float* row = A + static_cast<int64_t>(r) * lda + j0;
      const float l = __fdiv_rn(row[j - j0], piv);
      row[j - j0] = l;
      for (int c = j - j0 + 1; c < jb; ++c) row[c] = fmaf(-l, s_row[c], row[c]);
    }
    __syncthreads();
  }
}

// Apply the swaps ipiv[j0 .. j0+jb) to every column outside [j0, j0+jb).
__global__ void lu_laswp_kernel(float* __restrict__ A, int64_t lda, int n, int j0, int jb,
                                const int32_t* __restrict__ ipiv) {
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t ncols = n - jb;
  if (idx >= ncols) return;
  const int c = static_cast<int>(idx < j0 ? idx : idx + jb);
  for (int j = j0; j < j0 + jb; ++j) {
    const int p = ipiv[j];
    if (p != j) {
      float* a = A + static_cast<int64_t>(j) * lda + c;
      float* b = A + static_cast<int64_t>(p) * lda + c;
      const float tmp = *a;
      *a = *b;
      *b = tmp;
    }
  }
}

// U12 = L11^-1 A12: forward substitution with the unit lower triangle L11,
// one thread a column of A12, accumulation order l = 0 .. i-1.
__global__ void lu_trsm_kernel(float* __restrict__ A, int64_t lda, int n, int j0, int jb) {
  extern __shared__ float L11[];  // jb x jb
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x)
    L11[e] = A[static_cast<int64_t>(j0 + e / jb) * lda + j0 + e % jb];
  __syncthreads();
  const int64_t c = j0 + jb + blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (c >= n) return;
  float* col = A + static_cast<int64_t>(j0) * lda + c;
  for (int i = 1; i < jb; ++i) {
    float acc = col[static_cast<int64_t>(i) * lda];
    for (int l = 0; l < i; ++l) acc = fmaf(-L11[i * jb + l], col[static_cast<int64_t>(l) * lda], acc);
    col[static_cast<int64_t>(i) * lda] = acc;
  }
}

struct LuWs {
  int64_t kp, ap, bp;
  size_t bytes;
};

LuWs lu_ws(int np, int64_t n, int nb) {
  LuWs w;
  w.kp = round_up(nb, 8);
  w.ap = round_up(n * w.kp, 128);
  w.bp = w.ap;
  w.bytes = static_cast<size_t>(np) * static_cast<size_t>(w.ap + w.bp) * 2;
  return w;
}

}  // namespace

bfx_status lu_factor(bfx_mode mode, int64_t n, int nb, float* A, int64_t lda, int32_t* ipiv,
                     int32_t* info, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (nb <= 0) nb = 64;
  if (nb > 128) return BFX_EINVAL;
  if (cudaMemsetAsync(info, 0, sizeof(int32_t), s) != cudaSuccess) return BFX_ECUDA;
  if (n == 0) return BFX_OK;
  const int np = mode_pieces(mode);
  LuWs w = lu_ws(np > 0 ? np : 1, n, nb);
  if (np > 0 && (!ws || ws_bytes < w.bytes || !aligned(ws, 256))) return BFX_ENOMEM;
  const size_t trsm_smem = static_cast<size_t>(nb) * nb * sizeof(float);
  if (trsm_smem > 48 * 1024 &&
      cudaFuncSetAttribute(lu_trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(trsm_smem)) != cudaSuccess)
    return BFX_ECUDA;
  uint16_t* Lp = static_cast<uint16_t*>(ws);
  uint16_t* Up = Lp ? Lp + np * w.ap : nullptr;
  const int N = static_cast<int>(n);
  for (int j0 = 0; j0 < N; j0 += nb) {
    const int jb = (N - j0 < nb) ? N - j0 : nb;
    lu_panel_kernel<<<1, PANEL_THREADS, 0, s>>>(A, lda, N, j0, jb, ipiv, info);
    if (N - jb > 0) {
      const int64_t cols = N - jb;
      lu_laswp_kernel<<<static_cast<unsigned>(ceil_div(cols, 256)), 256, 0, s>>>(A, lda, N, j0, jb,
                                                                              ipiv);
    }
    const int nr = N - j0 - jb;
    if (nr <= 0) continue;
    lu_trsm_kernel<<<static_cast<unsigned>(ceil_div(nr, 128)), 128, trsm_smem, s>>>(A, lda, N, j0,
                                                                                jb);
    float* L21 = A + static_cast<int64_t>(j0 + jb) * lda + j0;
    float* U12 = A + static_cast<int64_t>(j0) * lda + j0 + jb;
    float* A22 = A + static_cast<int64_t>(j0 + jb) * lda + j0 + jb;
    bfx_status st;
    if (np == 0) {
      st = launch_sgemm_simt(nr, nr, jb, -1.0f, L21, lda, U12, lda, 1.0f, A22, lda, s);
    } else {
      st = launch_split(nr, jb, L21, lda, np, Lp, np > 1 ? Lp + w.ap : nullptr,
                        np > 2 ? Lp + 2 * w.ap : nullptr, w.kp, s);
      if (st != BFX_OK) return st;
      st = launch_split_transpose(jb, nr, U12, lda, np, Up, np > 1 ? Up + w.bp : nullptr,
                                  np > 2 ? Up + 2 * w.bp : nullptr, w.kp, s);
      if (st != BFX_OK) return st;
      st = launch_gemm_presplit(mode, nr, nr, jb, -1.0f, Lp, w.kp, w.ap, Up, w.kp, w.bp, 1.0f,
                                A22, lda, s);
    }
    if (st != BFX_OK) return st;
  }
  return last_launch_status();
}

size_t lu_workspace_bytes(bfx_mode mode, int64_t n, int nb) {
  const int np = mode_pieces(mode);
  if (np == 0 || n <= 0) return 0;
  if (nb <= 0) nb = 64;
  return lu_ws(np, n, nb).bytes;
}

}  // namespace bfx

using namespace bfx;

extern "C" {

BFX_API size_t bfx_lu_workspace_size(bfx_mode mode, int64_t n, int nb) {
  return lu_workspace_bytes(mode, n, nb);
}

BFX_API bfx_status bfx_lu_bf16xN(bfx_mode mode, int64_t n, int nb, float* d_A, int64_t lda,
                                 int32_t* d_ipiv, int32_t* d_info, void* d_ws, size_t ws_bytes,
                                 bfx_stream stream) {
  if (mode != BFX_FP32 && mode_pieces(mode) == 0) return BFX_EINVAL;
  if (n < 0 || !d_info || (n > 0 && (!d_A || !d_ipiv || lda < n))) return BFX_EINVAL;
  if (nb < 0 || nb > 128) return BFX_EINVAL;
  if (n >= INT32_MAX) return BFX_EUNSUPPORTED;
  if (mode != BFX_FP32 && !is_sm103()) return BFX_EUNSUPPORTED;
  return lu_factor(mode, n, nb, d_A, lda, d_ipiv, d_info, d_ws, ws_bytes,
                   static_cast<cudaStream_t>(stream));
}

}  // extern "C"
