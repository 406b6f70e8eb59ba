// Blocked right-looking LU with partial pivoting whose trailing update is the
// bf16xN product (Sec. IV-A of the paper: "SGETRF based on triplets of BF16s
// and six products"; Sec. III: the cubic work in low precision).
//
// For each block column j0 (width jb <= nb):
//   panel   : FP32 LU of A[j0:n, j0:j0+jb] (pivot = first row of the largest
//             |a|, found by warp-shuffle argmaxes; whole block-column rows
//             swapped; multipliers by IEEE division by the pivot; FMA rank-1
//             updates in column order).  Up to 8 x 512 rows and jb <= 64:
//             one thread-block cluster holds the whole block column in
//             registers and exchanges the pivot candidates through
//             distributed shared memory (one cluster barrier a column).
//             Otherwise in tiles of 8 columns, one CTA each (registers or
//             shared memory), the tile's rows of the block columns right of
//             it forward-substituted and the rows below given the tile's
//             rank-8 update: for every element the same operations in the
//             same order;
//   laswp   : the panel's row swaps applied to the columns left and right of it
//             (each CTA forms their net effect on the touched rows itself);
//   trsm    : U12 = L11^-1 A12 (unit lower, FP32 FMA, one warp a column);
//   update  : A22 <- A22 - L21 U12 by the mode's bfloat16 products on the
//             tensor cores (split of L21, transposed split of U12, tcgen05
//             GEMM with alpha = -1, beta = 1), or the FP32 SIMT GEMM.
// Pivots: ipiv[j] (0-based) is the row swapped with row j at step j.  info is
// LAPACK's: 0, or the 1-based index of the first exactly zero pivot (the
// factorisation still completes).
#include <algorithm>

#include "bfx_internal.cuh"

namespace bfx {
namespace {

constexpr int PANEL_THREADS = 512;
static_assert(PANEL_THREADS % 32 == 0 && PANEL_THREADS <= 1024, "panel CTA size");

struct ArgMax {
  float v;
  int i;
};

__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b) {
  // larger value wins; equal values: the smaller row index (LAPACK i?amax)
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}

constexpr int TILE_W = 8;                      // panel tile width
constexpr size_t TILE_SMEM_MAX = 200 * 1024;   // tile rows kept in shared memory up to this

// One CTA factors the tile A[j0:n, j0:j0+jw] (jw <= 8) of the block column
// [J0, J0+JB), keeping the tile in shared memory when it fits:
//   for each tile column j: pivot = first row of the largest |a| (warp-shuffle
//   argmax), rows j and p swapped across the whole block column, division by
//   the pivot, FMA rank-1 update of the remaining tile columns;
// then the tile rows of the block columns right of the tile are solved with
// the tile's unit lower triangle (forward substitution, FMA, l in order).
template <bool use_smem>
__device__ __forceinline__ void tile_body(float* __restrict__ A, int64_t lda, int n, int J0,
                                          int JB, int j0, int jw, int32_t* __restrict__ ipiv,
                                          int32_t* __restrict__ info) {
  extern __shared__ float tile[];  // (n - j0) x TILE_W when use_smem
  __shared__ ArgMax warp_best[PANEL_THREADS / 32];
  __shared__ int s_piv;
  __shared__ float s_row[TILE_W];
  __shared__ int s_pivs[TILE_W];
  __shared__ int s_rows[2 * TILE_W], s_src[2 * TILE_W], s_ns;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int rows = n - j0;
  auto T = [&](int r, int c) -> float& {
    return use_smem ? tile[static_cast<int64_t>(r - j0) * TILE_W + c]
                    : A[static_cast<int64_t>(r) * lda + j0 + c];
  };
  if (use_smem) {
    // a row's tile values go through registers, all loads of a thread first
    for (int r0 = j0 + t; r0 < n; r0 += 4 * PANEL_THREADS) {
      float v[4][TILE_W];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = r0 + q * PANEL_THREADS;
#pragma unroll
        for (int c = 0; c < TILE_W; ++c)
          v[q][c] = (r < n && c < jw) ? A[static_cast<int64_t>(r) * lda + j0 + c] : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = r0 + q * PANEL_THREADS;
        if (r < n) {
#pragma unroll
          for (int c = 0; c < TILE_W; ++c) tile[static_cast<int64_t>(r - j0) * TILE_W + c] = v[q][c];
        }
      }
    }
    __syncthreads();
  }
  const int nout = JB - jw;  // block-column columns outside the tile
  for (int jj = 0; jj < jw; ++jj) {
    const int j = j0 + jj;
    // ---- pivot search over rows j..n-1
    ArgMax best{-1.0f, n};
    for (int r = j + t; r < n; r += PANEL_THREADS) {
      float v = fabsf(T(r, jj));
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
      best = lane < PANEL_THREADS / 32 ? warp_best[lane] : ArgMax{-1.0f, n};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ArgMax other{__shfl_xor_sync(0xFFFFFFFFu, best.v, o), __shfl_xor_sync(0xFFFFFFFFu, best.i, o)};
        best = better(best, other);
      }
      if (lane == 0) {
        const float d = T(j, jj);
        // a NaN on the diagonal stays (nothing compares greater than it)
        s_piv = (d != d || best.i >= n) ? j : best.i;
        ipiv[j] = s_piv;
      }
    }
    __syncthreads();
    const int p = s_piv;
    // ---- swap rows j and p: tile part, then the rest of the block column
    if (t < jw) {
      const float a = T(j, t), b = T(p, t);
      if (p != j) {
        T(j, t) = b;
        T(p, t) = a;
      }
      s_row[t] = (p != j) ? b : a;
    }
    if (t == 0) s_pivs[jj] = p;
    __syncthreads();
    const float piv = s_row[jj];
    if (piv == 0.0f) {
      if (t == 0 && *info == 0) *info = j + 1;
      __syncthreads();
      continue;
    }
    // ---- multipliers (IEEE division by the pivot), rank-1 update of the rest of the tile
    for (int r = j + 1 + t; r < n; r += PANEL_THREADS) {
      const float l = __fdiv_rn(T(r, jj), piv);
      T(r, jj) = l;
      for (int c = jj + 1; c < jw; ++c) T(r, c) = fmaf(-l, s_row[c], T(r, c));
    }
    __syncthreads();
  }
  if (use_smem) {
    for (int e = t; e < rows * jw; e += PANEL_THREADS) {
      const int r = j0 + e / jw, c = e % jw;
      A[static_cast<int64_t>(r) * lda + j0 + c] = tile[static_cast<int64_t>(r - j0) * TILE_W + c];
    }
  }
  // ---- the tile's row swaps, applied once to the block-column columns outside
  // the tile: net effect of the (at most 8) sequential swaps on the (at most
  // 16) rows they touch, all loads of a column before its stores
  if (t == 0) {
    int ns = 0;
    for (int jj = 0; jj < jw; ++jj) {
      const int rr[2] = {j0 + jj, s_pivs[jj]};
      for (int q = 0; q < 2; ++q) {
        bool seen = false;
        for (int k = 0; k < ns; ++k) seen = seen || s_rows[k] == rr[q];
        if (!seen) {
          s_rows[ns] = rr[q];
          s_src[ns] = rr[q];
          ++ns;
        }
      }
      int a = 0, b = 0;
      for (int k = 0; k < ns; ++k) {
        if (s_rows[k] == j0 + jj) a = k;
        if (s_rows[k] == s_pivs[jj]) b = k;
      }
      const int tmp = s_src[a];
      s_src[a] = s_src[b];
      s_src[b] = tmp;
    }
    s_ns = ns;
  }
  __syncthreads();
  if (nout > 0) {
    const int ns = s_ns;
    for (int k = t; k < nout; k += PANEL_THREADS) {
      const int c = (J0 + k < j0) ? J0 + k : J0 + k + jw;
      float v[2 * TILE_W];
#pragma unroll
      for (int q = 0; q < 2 * TILE_W; ++q)
        v[q] = q < ns ? A[static_cast<int64_t>(s_src[q]) * lda + c] : 0.0f;
#pragma unroll
      for (int q = 0; q < 2 * TILE_W; ++q)
        if (q < ns) A[static_cast<int64_t>(s_rows[q]) * lda + c] = v[q];
    }
    __syncthreads();
  }
  // ---- tile rows of the block columns right of the tile: forward substitution
  for (int c = j0 + jw + t; c < J0 + JB; c += PANEL_THREADS) {
    float* col = A + static_cast<int64_t>(j0) * lda + c;
    float x[TILE_W];
#pragma unroll
    for (int i = 0; i < TILE_W; ++i) x[i] = i < jw ? col[static_cast<int64_t>(i) * lda] : 0.0f;
#pragma unroll
    for (int i = 1; i < TILE_W; ++i) {
      if (i >= jw) break;
      float acc = x[i];
#pragma unroll
      for (int l = 0; l < i; ++l) acc = fmaf(-T(j0 + i, l), x[l], acc);
      x[i] = acc;
      col[static_cast<int64_t>(i) * lda] = acc;
    }
  }
}

// The same tile factorisation with the tile in registers, for tiles of at
// most PANEL_THREADS * RPT rows: thread t holds rows j0 + t + q*PANEL_THREADS
// (q < RPT), all 8 columns.  One barrier per column: every warp posts its
// best candidate together with that row's values, then every warp reduces
// the posted candidates itself (same data, same order: the same pivot), so
// the pivot row is known without a second barrier.  The shared rows
// alternate between two buffers by column parity, so a warp still using
// column jj's data never sees column jj+1's.  Every element sees the same
// operations as in tile_body (same pivot rule, scaling, fmaf order).
template <int RPT>
__device__ __forceinline__ void tile_body_regs(float* __restrict__ A, int64_t lda, int n, int J0,
                                               int JB, int j0, int jw,
                                               int32_t* __restrict__ ipiv,
                                               int32_t* __restrict__ info) {
  constexpr int NW = PANEL_THREADS / 32;
  __shared__ ArgMax wbest[2][NW];
  __shared__ float wrow[2][NW][TILE_W];   // each warp's candidate row
  __shared__ float rowj[2][TILE_W];       // row j before the swap
  __shared__ int s_pivs[TILE_W];
  __shared__ int s_rows[2 * TILE_W], s_src[2 * TILE_W], s_ns;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  // rows as two 16-byte words when the tile is full and aligned
  const bool vec = jw == TILE_W && (lda % 4) == 0 && (j0 % 4) == 0 &&
                   (reinterpret_cast<uintptr_t>(A) % 16) == 0;
  float v[RPT][TILE_W];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int r = j0 + t + q * PANEL_THREADS;
    const float* src = A + static_cast<int64_t>(r < n ? r : j0) * lda + j0;
    if (vec) {
      const float4 x0 = *reinterpret_cast<const float4*>(src);
      const float4 x1 = *reinterpret_cast<const float4*>(src + 4);
      v[q][0] = x0.x; v[q][1] = x0.y; v[q][2] = x0.z; v[q][3] = x0.w;
      v[q][4] = x1.x; v[q][5] = x1.y; v[q][6] = x1.z; v[q][7] = x1.w;
    } else {
#pragma unroll
      for (int c = 0; c < TILE_W; ++c) v[q][c] = c < jw ? src[c] : 0.0f;
    }
    if (r >= n) {
#pragma unroll
      for (int c = 0; c < TILE_W; ++c) v[q][c] = 0.0f;
    }
  }
  // Column jj of the tile is always register column 0: after each pivot
  // column the registers rotate left by one (column 0 moves to the back), so
  // the loop body is the same for every column and need not be unrolled;
  // after TILE_W rotations the columns are back in place.
  for (int jj = 0; jj < TILE_W; ++jj) {
    if (jj < jw) {
      const int j = j0 + jj, bf = jj & 1;
      const int rem = jw - jj;  // tile columns from the current one on
      // ---- pivot search over rows j..n-1; row j's owner posts row j
      // (row r lives in thread (r - j0) % PANEL_THREADS, slot (r - j0) / PANEL_THREADS:
      // only the owner runs the copies, its slot picked by a compare chain)
      const int tj = (j - j0) % PANEL_THREADS, qj = (j - j0) / PANEL_THREADS;
      if (t == tj) {
#pragma unroll
        for (int q = 0; q < RPT; ++q)
          if (q == qj) {
#pragma unroll
            for (int c = 0; c < TILE_W; ++c) rowj[bf][c] = v[q][c];
          }
      }
      ArgMax best{-1.0f, n};
      int bq = -1;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = j0 + t + q * PANEL_THREADS;
        if (r >= j && r < n) {
          float a = fabsf(v[q][0]);
          if (a != a) a = -1.0f;  // NaN below the diagonal is never chosen
          const ArgMax cand{a, r};
          const ArgMax nb = better(best, cand);
          if (nb.i != best.i) bq = q;
          best = nb;
        }
      }
      const int own = best.i;  // this thread's candidate row
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ArgMax other{__shfl_xor_sync(0xFFFFFFFFu, best.v, o), __shfl_xor_sync(0xFFFFFFFFu, best.i, o)};
        best = better(best, other);
      }
      if (lane == 0) wbest[bf][wid] = best;
      if (bq >= 0 && own == best.i) {  // the lane holding the warp's winner posts its row
        const int qw = (own - j0) / PANEL_THREADS;
#pragma unroll
        for (int q = 0; q < RPT; ++q)
          if (q == qw) {
#pragma unroll
            for (int c = 0; c < TILE_W; ++c) wrow[bf][wid][c] = v[q][c];
          }
      }
      __syncthreads();  // the column's only barrier: every warp decides the pivot itself
      ArgMax b = lane < NW ? wbest[bf][lane] : ArgMax{-1.0f, n};
      int w = lane;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ArgMax other{__shfl_xor_sync(0xFFFFFFFFu, b.v, o), __shfl_xor_sync(0xFFFFFFFFu, b.i, o)};
        const int ow = __shfl_xor_sync(0xFFFFFFFFu, w, o);
        const ArgMax nb = better(b, other);
        if (nb.i != b.i) w = ow;
        b = nb;
      }
      const float d = rowj[bf][0];
      const bool keep = (d != d || b.i >= n);  // a NaN on the diagonal stays
      const int p = keep ? j : b.i;
      if (t == 0) {
        s_pivs[jj] = p;
        ipiv[j] = p;
      }
      const float* prow = keep ? rowj[bf] : wrow[bf][w];  // the pivot row = row j after the swap
      // ---- swap rows j and p (tile part): only their owners
      if (p != j) {
        const int tp = (p - j0) % PANEL_THREADS, qp = (p - j0) / PANEL_THREADS;
        if (t == tj) {
#pragma unroll
          for (int q = 0; q < RPT; ++q)
            if (q == qj) {
#pragma unroll
              for (int c = 0; c < TILE_W; ++c) v[q][c] = prow[c];
            }
        }
        if (t == tp) {
#pragma unroll
          for (int q = 0; q < RPT; ++q)
            if (q == qp) {
#pragma unroll
              for (int c = 0; c < TILE_W; ++c) v[q][c] = rowj[bf][c];
            }
        }
      }
      const float piv = prow[0];
      if (piv == 0.0f) {
        if (t == 0 && *info == 0) *info = j + 1;
      } else {
        // ---- multipliers (IEEE division by the pivot), rank-1 update of
        // the rest of the tile
        float u[TILE_W];
#pragma unroll
        for (int c = 1; c < TILE_W; ++c) u[c] = prow[c];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          const int r = j0 + t + q * PANEL_THREADS;
          if (r > j && r < n) {
            const float l = __fdiv_rn(v[q][0], piv);
            v[q][0] = l;
#pragma unroll
            for (int c = 1; c < TILE_W; ++c)
              if (c < rem) v[q][c] = fmaf(-l, u[c], v[q][c]);
          }
        }
      }
    }
    // ---- rotate the columns left by one
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const float c0 = v[q][0];
#pragma unroll
      for (int c = 0; c < TILE_W - 1; ++c) v[q][c] = v[q][c + 1];
      v[q][TILE_W - 1] = c0;
    }
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int r = j0 + t + q * PANEL_THREADS;
    if (r < n) {
      float* dst = A + static_cast<int64_t>(r) * lda + j0;
      if (vec) {
        *reinterpret_cast<float4*>(dst) = make_float4(v[q][0], v[q][1], v[q][2], v[q][3]);
        *reinterpret_cast<float4*>(dst + 4) = make_float4(v[q][4], v[q][5], v[q][6], v[q][7]);
      } else {
#pragma unroll
        for (int c = 0; c < TILE_W; ++c)
          if (c < jw) dst[c] = v[q][c];
      }
    }
  }
  // ---- the tile's row swaps on the block-column columns outside the tile
  // (net effect of the sequential swaps, as in tile_body)
  __syncthreads();
  if (t == 0) {
    int ns = 0;
    for (int jj = 0; jj < jw; ++jj) {
      const int rr[2] = {j0 + jj, s_pivs[jj]};
      for (int q = 0; q < 2; ++q) {
        bool seen = false;
        for (int k = 0; k < ns; ++k) seen = seen || s_rows[k] == rr[q];
        if (!seen) {
          s_rows[ns] = rr[q];
          s_src[ns] = rr[q];
          ++ns;
        }
      }
      int a = 0, b = 0;
      for (int k = 0; k < ns; ++k) {
        if (s_rows[k] == j0 + jj) a = k;
        if (s_rows[k] == s_pivs[jj]) b = k;
      }
      const int tmp = s_src[a];
      s_src[a] = s_src[b];
      s_src[b] = tmp;
    }
    s_ns = ns;
  }
  __syncthreads();
  const int nout = JB - jw;
  if (nout > 0) {
    const int ns = s_ns;
    for (int k = t; k < nout; k += PANEL_THREADS) {
      const int c = (J0 + k < j0) ? J0 + k : J0 + k + jw;
      float w[2 * TILE_W];
#pragma unroll
      for (int q = 0; q < 2 * TILE_W; ++q)
        w[q] = q < ns ? A[static_cast<int64_t>(s_src[q]) * lda + c] : 0.0f;
#pragma unroll
      for (int q = 0; q < 2 * TILE_W; ++q)
        if (q < ns) A[static_cast<int64_t>(s_rows[q]) * lda + c] = w[q];
    }
    __syncthreads();
  }
  // ---- tile rows of the block columns right of the tile: forward substitution
  for (int c = j0 + jw + t; c < J0 + JB; c += PANEL_THREADS) {
    float* col = A + static_cast<int64_t>(j0) * lda + c;
    float x[TILE_W];
#pragma unroll
    for (int i = 0; i < TILE_W; ++i) x[i] = i < jw ? col[static_cast<int64_t>(i) * lda] : 0.0f;
#pragma unroll
    for (int i = 1; i < TILE_W; ++i) {
      if (i >= jw) break;
      float acc = x[i];
#pragma unroll
      for (int l = 0; l < i; ++l)
        acc = fmaf(-A[static_cast<int64_t>(j0 + i) * lda + j0 + l], x[l], acc);
      x[i] = acc;
      col[static_cast<int64_t>(i) * lda] = acc;
    }
  }
}

template <bool use_smem>
__global__ void __launch_bounds__(PANEL_THREADS)
    lu_tile_kernel(float* __restrict__ A, int64_t lda, int n, int J0, int JB, int j0, int jw,
                   int32_t* __restrict__ ipiv, int32_t* __restrict__ info) {
  tile_body<use_smem>(A, lda, n, J0, JB, j0, jw, ipiv, info);
}

template <int RPT>
__global__ void __launch_bounds__(PANEL_THREADS)
    lu_tile_regs_kernel(float* __restrict__ A, int64_t lda, int n, int J0, int JB, int j0, int jw,
                        int32_t* __restrict__ ipiv, int32_t* __restrict__ info) {
  tile_body_regs<RPT>(A, lda, n, J0, JB, j0, jw, ipiv, info);
}

// Rows below the tile, block columns right of it: a <- fma(-l_rk, u_kc, a)
// for the jw tile columns k in order.  Grid-stride with block `bid` of `nbk`.
__device__ __forceinline__ void tile_update_body(float* __restrict__ A, int64_t lda, int n, int J0,
                                                 int JB, int j0, int jw, int bid, int nbk) {
  const int cs = j0 + jw, ncol = J0 + JB - cs;
  if (ncol <= 0) return;
  const int64_t total = static_cast<int64_t>(n - cs) * ncol;
  for (int64_t e = bid * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(nbk) * blockDim.x) {
    const int r = cs + static_cast<int>(e / ncol);
    const int c = cs + static_cast<int>(e % ncol);
    const float* lr = A + static_cast<int64_t>(r) * lda + j0;
    float a = A[static_cast<int64_t>(r) * lda + c];
    for (int l = 0; l < jw; ++l) a = fmaf(-lr[l], A[static_cast<int64_t>(j0 + l) * lda + c], a);
    A[static_cast<int64_t>(r) * lda + c] = a;
  }
}

__global__ void lu_tile_update_kernel(float* __restrict__ A, int64_t lda, int n, int J0, int JB,
                                      int j0, int jw) {
  tile_update_body(A, lda, n, J0, JB, j0, jw, blockIdx.x, gridDim.x);
}

// Apply the swaps ipiv[j0 .. j0+jb) to columns outside [j0, j0+jb).
// Every CTA first turns the sequential swaps into their net effect on the at
// most 2 jb rows they touch (slot k ends up holding the original row
// cont[k]), then moves those rows of its LASWP_COLS columns: warp w loads
// slots w, w + LASWP_WARPS, ... of its lane's column into registers, and
// after a CTA barrier (which orders every load of the column before every
// store) writes them to their new rows.
constexpr int LASWP_COLS = 32;     // columns a CTA, one a lane
constexpr int LASWP_WARPS = 8;     // warps a CTA
constexpr int LASWP_THREADS = LASWP_COLS * LASWP_WARPS;
constexpr int LASWP_SLOTS = 256;   // 2 x the largest block width
constexpr int LASWP_PER_WARP = LASWP_SLOTS / LASWP_WARPS;
struct SwapSet {
  int rowid[LASWP_SLOTS];  // the touched rows
  int cont[LASWP_SLOTS];   // row rowid[k] receives the original row cont[k]
  int nslots;
};

// One warp (all lanes) turns piv[0 .. jb) (absolute rows, piv[j] >= j0 + j;
// shared memory, 16-byte aligned, jb <= 128) into *ss (shared memory).
// Slot k < jb is row j0 + k; each row p >= j0 + jb that a swap names gets
// the next slot in the order of its first appearance.  Swap j exchanges
// slots j and sp[j] >= j, so slot j is final once swap j is done; one lane
// replays the swaps on the slot contents.
__device__ __forceinline__ void swapset_warp(const int* __restrict__ piv, int j0, int jb,
                                             SwapSet* ss, int* sp) {
  const int lane = threadIdx.x & 31;
  constexpr int G = 4;  // groups of 32 swaps
  uint32_t fresh[G];    // swaps that name a row outside the block for the first time
  int first[G];         // the first swap naming the same outside row (-1: inside)
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = 32 * g + lane;
    const int p = j < jb ? piv[j] : -1;
    int f = -1;
    if (p >= j0 + jb) {
      f = j;
      for (int q0 = 0; q0 < j && f == j; q0 += 4) {
        const int4 x = *reinterpret_cast<const int4*>(piv + q0);
        if (x.x == p) f = q0;
        else if (q0 + 1 < j && x.y == p) f = q0 + 1;
        else if (q0 + 2 < j && x.z == p) f = q0 + 2;
        else if (q0 + 3 < j && x.w == p) f = q0 + 3;
      }
    }
    first[g] = f;
    fresh[g] = __ballot_sync(0xFFFFFFFFu, f >= 0 && f == j);
  }
  int nfresh = 0;
#pragma unroll
  for (int g = 0; g < G; ++g) nfresh += __popc(fresh[g]);
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = 32 * g + lane;
    if (j < jb) {
      const int f = first[g];
      int s = piv[j] - j0;
      if (f >= 0) {
        int below = 0;  // first appearances before swap f
#pragma unroll
        for (int h = 0; h < G; ++h) {
          if (h < (f >> 5)) below += __popc(fresh[h]);
          else if (h == (f >> 5)) below += __popc(fresh[h] & ((1u << (f & 31)) - 1u));
        }
        s = jb + below;
        if (f == j) ss->rowid[s] = piv[j];
      }
      sp[j] = s;
      ss->rowid[j] = j0 + j;
    }
  }
  const int ns = jb + nfresh;
  __syncwarp();
  for (int k = lane; k < ns; k += 32) ss->cont[k] = ss->rowid[k];
  __syncwarp();
  if (lane == 0) {
    for (int j = 0; j < jb; ++j) {
      const int s = sp[j];
      if (s != j) {
        const int a = ss->cont[j];
        ss->cont[j] = ss->cont[s];
        ss->cont[s] = a;
      }
    }
    ss->nslots = ns;
  }
  __syncwarp();
}

// Moves the touched rows of column blocks cb0, cb0 + cstep, ...: column
// index idx = cb * LASWP_COLS + lane of the list [c0, c0 + n0) ++
// [c1, c1 + n1).  Builds the swap set of ipiv[j0 .. j0+jb) once itself
// (blockDim = LASWP_THREADS).
__device__ __forceinline__ void laswp_body(float* __restrict__ A, int64_t lda, int j0, int jb,
                                           const int32_t* __restrict__ ipiv, int c0, int n0,
                                           int c1, int n1, int cb0, int cstep, SwapSet* ssp) {
  SwapSet& ss = *ssp;
  __shared__ __align__(16) int piv[128];
  __shared__ int sp[128];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int j = t; j < jb; j += blockDim.x) piv[j] = ipiv[j0 + j];
  __syncthreads();
  if (w == 0) swapset_warp(piv, j0, jb, &ss, sp);
  __syncthreads();
  const int ns = ss.nslots;
  for (int cb = cb0; cb * LASWP_COLS < n0 + n1; cb += cstep) {  // the same for the whole CTA
    const int idx = cb * LASWP_COLS + lane;
    const bool on = idx < n0 + n1;
    const int64_t c = idx < n0 ? c0 + idx : c1 + (idx - n0);
    float v[LASWP_PER_WARP];
#pragma unroll
    for (int q = 0; q < LASWP_PER_WARP; ++q) {
      const int k = w + LASWP_WARPS * q;
      v[q] = (on && k < ns) ? A[static_cast<int64_t>(ss.cont[k]) * lda + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < LASWP_PER_WARP; ++q) {
      const int k = w + LASWP_WARPS * q;
      if (on && k < ns) A[static_cast<int64_t>(ss.rowid[k]) * lda + c] = v[q];
    }
  }
}

// Columns [c0, c0 + n0) ++ [c1, c1 + n1) of one matrix.  perm (optional,
// n rows): the row permutation so far, perm[i] = the original row now at
// row i; CTA 0 applies the block's swaps to it as to one more column (for
// j0 == 0 it starts from the identity).  The launches for consecutive
// blocks run in order, so perm ends as P of P A = L U.
__global__ void __launch_bounds__(LASWP_THREADS)
    lu_laswp_kernel(float* __restrict__ A, int64_t lda, int j0, int jb,
                    const int32_t* __restrict__ ipiv, int c0, int n0, int c1, int n1,
                    int32_t* __restrict__ perm, int n) {
  __shared__ SwapSet ss;
  laswp_body(A, lda, j0, jb, ipiv, c0, n0, c1, n1, static_cast<int>(blockIdx.x),
             static_cast<int>(gridDim.x), &ss);
  if (!perm || blockIdx.x != 0) return;
  static_assert(LASWP_THREADS >= LASWP_SLOTS, "one slot a thread");
  const int k = threadIdx.x;
  if (j0 == 0)
    for (int i = k; i < n; i += blockDim.x) perm[i] = i;
  __syncthreads();
  const bool on = k < ss.nslots;
  const int32_t moved = on ? perm[ss.cont[k]] : 0;
  __syncthreads();
  if (on) perm[ss.rowid[k]] = moved;
}

// U12 = L11^-1 A12: forward substitution with the unit lower triangle L11,
// one warp a column of A12, lane k owning rows k, k+32, ... (registers).
// Column-oriented: x_i receives -l_il x_l for l = 0, 1, ..., i-1 in order -
// per element the same FMA sequence as row-by-row substitution - with x_l
// broadcast from its owner lane.
constexpr int TRSM_COLS = 8;  // columns (warps) a CTA
__host__ __device__ constexpr int trsm_lds(int nb) { return nb + 1; }  // row stride of L11 in shared memory
// shared bytes of the block solve's L11 for register tile nb
constexpr size_t trsm_smem_bytes(int nb) {
  return static_cast<size_t>(nb) * trsm_lds(nb) * sizeof(float);
}
// L11 of block row j0 into shared memory: NB x NB, the jb x jb triangle
// padded with zeros; rows trsm_lds(NB) apart so the lanes' rows
// i = lane + 32 q of one column l fall in distinct banks.
template <int NB>
__device__ __forceinline__ void load_l11(const float* __restrict__ A, int64_t lda, int j0, int jb,
                                         float* L11) {
  constexpr int LS = trsm_lds(NB);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, l = e % NB;
    L11[i * LS + l] = (i < jb && l < jb) ? A[static_cast<int64_t>(j0 + i) * lda + j0 + l] : 0.0f;
  }
}
// The column col[i * lda], i < jb, solved in x (lane's rows i = lane + 32 q);
// rows 1 .. jb-1 written back (row 0 is its own solution).
template <int NB>
__device__ __forceinline__ void solve_col(float* __restrict__ col, int64_t lda, int jb,
                                          const float* L11, int lane, float (&x)[NB / 32]) {
  constexpr int RPL = NB / 32;  // rows a lane
  constexpr int LS = trsm_lds(NB);
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    const int i = lane + 32 * q;
    x[q] = i < jb ? col[static_cast<int64_t>(i) * lda] : 0.0f;
  }
#pragma unroll
  for (int q0 = 0; q0 < RPL; ++q0) {
    for (int ll = 0; ll < 32; ++ll) {
      const int l = 32 * q0 + ll;
      if (l >= jb - 1) break;
      const float xl = __shfl_sync(0xFFFFFFFFu, x[q0], ll);
#pragma unroll
      for (int q = q0; q < RPL; ++q) {
        const int i = lane + 32 * q;
        if (i > l && i < jb) x[q] = fmaf(-L11[i * LS + l], xl, x[q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    const int i = lane + 32 * q;
    if (i >= 1 && i < jb) col[static_cast<int64_t>(i) * lda] = x[q];
  }
}

// Batched block solve: TRSM_WCOLS adjacent columns a warp, solved together
// (independent FMA chains, each L11 element read once for all of them; per
// element the FMA sequence of solve_col), so that a CTA stages L11 once for
// TRSM_COLS * TRSM_WCOLS columns.  Columns c_begin + (cb * TRSM_COLS + warp)
// * TRSM_WCOLS + j below c_end of the block row j0.
constexpr int TRSM_WCOLS = 4;
template <int NB>
__device__ __forceinline__ void trsm_wide_body(float* __restrict__ A, int64_t lda, int c_end,
                                               int j0, int jb, int c_begin, int cb) {
  extern __shared__ float L11[];
  constexpr int RPL = NB / 32;  // rows a lane
  constexpr int LS = trsm_lds(NB);
  load_l11<NB>(A, lda, j0, jb, L11);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t c0 = c_begin + (static_cast<int64_t>(cb) * TRSM_COLS + w) * TRSM_WCOLS;
  if (c0 >= c_end) return;
  float* col = A + static_cast<int64_t>(j0) * lda + c0;
  float x[TRSM_WCOLS][RPL];
#pragma unroll
  for (int j = 0; j < TRSM_WCOLS; ++j) {
    const bool on = c0 + j < c_end;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int i = lane + 32 * q;
      x[j][q] = (on && i < jb) ? col[static_cast<int64_t>(i) * lda + j] : 0.0f;
    }
  }
#pragma unroll
  for (int q0 = 0; q0 < RPL; ++q0) {
    for (int ll = 0; ll < 32; ++ll) {
      const int l = 32 * q0 + ll;
      if (l >= jb - 1) break;
      float xl[TRSM_WCOLS];
#pragma unroll
      for (int j = 0; j < TRSM_WCOLS; ++j) xl[j] = __shfl_sync(0xFFFFFFFFu, x[j][q0], ll);
#pragma unroll
      for (int q = q0; q < RPL; ++q) {
        const int i = lane + 32 * q;
        if (i > l && i < jb) {
          const float lil = L11[i * LS + l];
#pragma unroll
          for (int j = 0; j < TRSM_WCOLS; ++j) x[j][q] = fmaf(-lil, xl[j], x[j][q]);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < TRSM_WCOLS; ++j) {
    if (c0 + j >= c_end) break;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int i = lane + 32 * q;
      if (i >= 1 && i < jb) col[static_cast<int64_t>(i) * lda + j] = x[j][q];
    }
  }
}

// Single system: columns [c_begin, c_end) of block row j0 (one warp a
// column), each first given the block column's row swaps ipiv[j0 .. j0+jb)
// (the CTA forms their net effect; warp w's lanes move the touched rows of
// its column, all loads before a warp barrier, then the stores), then solved;
// with np > 0 the bfloat16 pieces of the solved column (U12^T row
// c - (j0 + jb)) go to planes Up, Up + bp, Up + 2 bp (row stride kp), which
// the trailing update reads.
template <int NB>
__global__ void __launch_bounds__(TRSM_COLS * 32)
    lu_solve_cols_kernel(float* __restrict__ A, int64_t lda, int j0, int jb, int c_begin, int c_end,
                         const int32_t* __restrict__ ipiv, int np, uint16_t* __restrict__ Up,
                         int64_t bp, int64_t kp) {
  extern __shared__ float L11[];
  __shared__ SwapSet ss;
  __shared__ __align__(16) int piv[128];
  __shared__ int sp[128];
  constexpr int SPL = 2 * NB / 32;  // swap slots a lane (at most 2 jb)
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  load_l11<NB>(A, lda, j0, jb, L11);
  for (int j = t; j < jb; j += blockDim.x) piv[j] = ipiv[j0 + j];
  __syncthreads();
  if (w == 0) swapset_warp(piv, j0, jb, &ss, sp);
  __syncthreads();
  const int64_t c = c_begin + static_cast<int64_t>(blockIdx.x) * TRSM_COLS + w;
  if (c >= c_end) return;
  {
    const int ns = ss.nslots;
    float sv[SPL];
#pragma unroll
    for (int q = 0; q < SPL; ++q) {
      const int k = lane + 32 * q;
      sv[q] = k < ns ? A[static_cast<int64_t>(ss.cont[k]) * lda + c] : 0.0f;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < SPL; ++q) {
      const int k = lane + 32 * q;
      if (k < ns) A[static_cast<int64_t>(ss.rowid[k]) * lda + c] = sv[q];
    }
    __syncwarp();
  }
  float x[NB / 32];
  solve_col<NB>(A + static_cast<int64_t>(j0) * lda + c, lda, jb, L11, lane, x);
  if (np > 0) {
    uint16_t* u = Up + (c - (j0 + jb)) * kp;
#pragma unroll
    for (int q = 0; q < NB / 32; ++q) {
      const int i = lane + 32 * q;
      if (i < jb) {
        uint16_t h, m, l;
        split_elem(x[q], h, m, l);
        u[i] = h;
        if (np > 1) u[bp + i] = m;
        if (np > 2) u[2 * bp + i] = l;
      }
    }
  }
}

// ------------------------------------------------------------- batched forms
// blockIdx.y (or x for the tile kernel) selects a system; systems with no
// work in the step return at once.
template <int RPT>
__global__ void __launch_bounds__(PANEL_THREADS, 1)
    lu_tile_regs_batched_kernel(const BatchLu* __restrict__ sys, int nb, int J0, int j0) {
  const BatchLu b = sys[blockIdx.x];
  const int JB = min(nb, b.n - J0);
  const int jw = min(TILE_W, J0 + JB - j0);
  if (JB <= 0 || jw <= 0) return;
  tile_body_regs<RPT>(b.A, b.n, b.n, J0, JB, j0, jw, b.ipiv, b.info);
}

__global__ void lu_tile_update_batched_kernel(const BatchLu* __restrict__ sys, int nb, int J0,
                                              int j0) {
  const BatchLu b = sys[blockIdx.y];
  const int JB = min(nb, b.n - J0);
  const int jw = min(TILE_W, J0 + JB - j0);
  if (JB <= 0 || jw <= 0) return;
  tile_update_body(b.A, b.n, b.n, J0, JB, j0, jw, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(LASWP_THREADS)
    lu_laswp_batched_kernel(const BatchLu* __restrict__ sys, int nb, int J0) {
  const BatchLu b = sys[blockIdx.y];
  const int JB = min(nb, b.n - J0);
  if (JB <= 0 || static_cast<int>(blockIdx.x) * LASWP_COLS >= b.n - JB) return;
  __shared__ SwapSet ss;
  laswp_body(b.A, b.n, J0, JB, b.ipiv, 0, J0, J0 + JB, b.n - J0 - JB, static_cast<int>(blockIdx.x),
             static_cast<int>(gridDim.x), &ss);
}

template <int NB>
__global__ void __launch_bounds__(TRSM_COLS * 32)
    lu_trsm_batched_kernel(const BatchLu* __restrict__ sys, int nb, int J0) {
  const BatchLu b = sys[blockIdx.y];
  const int JB = min(nb, b.n - J0);
  if (JB <= 0 || J0 + JB + static_cast<int>(blockIdx.x) * TRSM_COLS * TRSM_WCOLS >= b.n) return;
  trsm_wide_body<NB>(b.A, b.n, b.n, J0, JB, J0 + JB, blockIdx.x);
}

// Pieces of L21 (rows below the block, block columns) and of U12^T for the
// grouped trailing update; columns past the block width are written as zero
// so a K-slice never reads stale values.  kp = nb (32, 64 or 128).  A CTA
// takes 32 rows of L21 and the matching 32 columns of U12 at a time: L21 a
// warp a row, two columns a lane, each piece's pair stored as one 32-bit
// word; U12 through a shared-memory transpose, so that the reads along a row
// of U12 and the writes along a row of U12^T are both coalesced.  (An
// element-wise loop over the flat index, with 64-bit divisions and 2-byte
// stores 2 kp bytes apart into U12^T, ran at ~1/7 of the HBM rate.)
constexpr int SPLIT_ROWS = 32, SPLIT_KMAX = 128, SPLIT_THREADS = 256;
__global__ void __launch_bounds__(SPLIT_THREADS)
    lu_split_batched_kernel(const BatchLu* __restrict__ sys, int nb, int J0, int np,
                            uint16_t* __restrict__ packA, uint16_t* __restrict__ packB,
                            int64_t slot_rows, int64_t kp) {
  __shared__ __align__(16) uint16_t tr[3][SPLIT_ROWS][SPLIT_KMAX + 2];  // [piece][U12 column][k]
  const BatchLu b = sys[blockIdx.y];
  const int JB = min(nb, b.n - J0);
  const int M = b.n - J0 - JB;
  if (JB <= 0 || M <= 0) return;
  const int K = static_cast<int>(kp);
  const int64_t plane = slot_rows * kp;  // even: kp is
  uint16_t* pa = packA + static_cast<int64_t>(blockIdx.y) * np * plane;
  uint16_t* pb = packB + static_cast<int64_t>(blockIdx.y) * np * plane;
  const int warp = static_cast<int>(threadIdx.x) >> 5, lane = static_cast<int>(threadIdx.x) & 31;
  constexpr int WARPS = SPLIT_THREADS / 32;
  for (int r0 = static_cast<int>(blockIdx.x) * SPLIT_ROWS; r0 < M;
       r0 += static_cast<int>(gridDim.x) * SPLIT_ROWS) {
    // L21 rows r0 .. r0 + 31
    for (int rr = warp; rr < SPLIT_ROWS && r0 + rr < M; rr += WARPS) {
      const int r = r0 + rr;
      const float* src = b.A + static_cast<int64_t>(J0 + JB + r) * b.n + J0;
      for (int c = 2 * lane; c < K; c += 64) {
        uint16_t h0, m0, l0, h1, m1, l1;
        split_elem(c < JB ? src[c] : 0.0f, h0, m0, l0);
        split_elem(c + 1 < JB ? src[c + 1] : 0.0f, h1, m1, l1);
        uint32_t* d = reinterpret_cast<uint32_t*>(pa + static_cast<int64_t>(r) * K + c);
        d[0] = h0 | (static_cast<uint32_t>(h1) << 16);
        if (np > 1) d[plane / 2] = m0 | (static_cast<uint32_t>(m1) << 16);
        if (np > 2) d[plane] = l0 | (static_cast<uint32_t>(l1) << 16);
      }
    }
    // U12 columns r0 .. r0 + 31: lane = column, warp = row k of U12
    const int cp = r0 + lane;
    for (int k = warp; k < K; k += WARPS) {
      uint16_t h, m, l;
      split_elem((k < JB && cp < M) ? b.A[static_cast<int64_t>(J0 + k) * b.n + J0 + JB + cp] : 0.0f,
                 h, m, l);
      tr[0][lane][k] = h;
      tr[1][lane][k] = m;
      tr[2][lane][k] = l;
    }
    __syncthreads();
    for (int rr = warp; rr < SPLIT_ROWS && r0 + rr < M; rr += WARPS) {
      uint32_t* d = reinterpret_cast<uint32_t*>(pb + static_cast<int64_t>(r0 + rr) * K);
      for (int k = 2 * lane; k < K; k += 64) {
        d[k / 2] = *reinterpret_cast<const uint32_t*>(&tr[0][rr][k]);
        if (np > 1) d[plane / 2 + k / 2] = *reinterpret_cast<const uint32_t*>(&tr[1][rr][k]);
        if (np > 2) d[plane + k / 2] = *reinterpret_cast<const uint32_t*>(&tr[2][rr][k]);
      }
    }
    __syncthreads();  // the transpose buffer is read before the next columns overwrite it
  }
}

// ---------------------------------------------------------------------------
// Whole block column by one thread-block cluster (single-system path).
//
// The block column [J0, J0+JB) of rows J0..n-1 (JB <= NB) is spread over the
// cs CTAs of one cluster: CTA c holds rows J0 + c*CLP_THREADS + t, one row a
// thread, the row's NB values in registers (one CTA of as many threads as
// rows when they fit one CTA).  Per pivot column j:
//  1. every thread offers its row's |a_rj| (rows >= j) as a key: the value's
//     bits plus two (a NaN gets 1: never chosen over a number; no offer 0)
//     with the row index; a warp keeps the largest key and, among equal keys,
//     the lowest row (LAPACK's first row of the largest |a|) by one warp max
//     and a ballot, as rows rise with lane, warp and CTA rank;
//     each warp posts its winner's key and index to shared memory, and the
//     thread holding row j posts row j;
//  2. after a CTA barrier every warp reduces the warps' offers the same way,
//     and only the CTA's winner stores its row (every warp storing its own
//     candidate row queued some 250 single-lane stores a column ahead of
//     the reads that follow: 7 % of the n = 4096 LU, 20 % at n = 512).  In a
//     cluster, after another CTA barrier, the pushing threads store the
//     CTA's offer (key, row index, row) and, from CTA 0, row j into an
//     exchange slot of every CTA of the cluster: into the other CTAs by
//     asynchronous remote shared-memory stores that complete their bytes on
//     the receiving slot's mbarrier, into the own slot by plain stores
//     followed by an arrival on it.  A cluster of one (a compile-time form)
//     has the winner and the holder of row j store straight into its slot;
//  3. every thread waits (acquire, cluster scope) for its CTA's slot to be
//     complete - each CTA waits only for the bytes sent to it, no cluster-wide
//     barrier; every warp reduces the cs offers -> pivot row p (a NaN on the
//     diagonal stays); the holder of row j takes the pivot row, the holder of
//     row p the old row j;
//  4. rows below j: l = a_rj / a_jj (IEEE division), then a_rc <- fma(-l,
//     u_jc, a_rc) for the block column's columns c > j, in column order.
// Each element therefore sees the operations of the unblocked right-looking
// LU of the block column, in the same order as the 8-column tile path.
// The slots, the staged rows and offers alternate by column parity.  A CTA
// stores column j+2's offer into CTA b only after its own slot for column
// j+1 is complete, which needs b's column j+1 offer, which b sends only after
// a CTA barrier that all its threads pass once they have read column j's
// slot; the same barrier orders a CTA's reads of its staged rows for column j
// before their rewrite for column j+2.  Columns go in groups of 8 whose
// register indices are compile-time constants; after a group the row rotates
// left by 8, so after NB / 8 groups it is back in place.  Every wait is
// bounded: an expired wait records kErrWaitPanel in the device error word and
// the kernel runs to its end without further waits.
constexpr int CLP_THREADS = 512;  // rows a CTA holds
constexpr int CLP_MAX_CL = 16;    // exchange slots (16 would be a non-portable cluster size)
constexpr int kPanelMaxCluster = 8;  // clusters launched: the portable size, up to 4096 rows
constexpr uint64_t kPanelWaitNs = 2000000000ull;  // a column's exchange takes microseconds

template <int NB>
struct ClusterSlot {
  float row[CLP_MAX_CL][NB];  // each CTA's offered row (rotated register order)
  float rowj[NB];             // row j before the swap
  uint2 ki[CLP_MAX_CL];       // each CTA's offer: key, row index
};

template <int NB>
struct PanelShared {
  static constexpr int MW = CLP_THREADS / 32;
  ClusterSlot<NB> slot[2];  // by column parity
  float wrow[2][NB];        // the CTA's offered row, by column parity
  float rowj[2][NB];        // row j (CTA 0), by column parity
  uint32_t wkey[2][MW];
  uint32_t widx[2][MW];
  uint64_t bar[2];          // slot complete (clusters of more than one CTA)
  int piv[NB];              // the block column's pivots
  int zero;                 // 1-based row of the first zero pivot, or 0
};

// A slot of CTA cr (cs > 1) completes a phase when its bytes from the other
// CTAs have landed (their offers; row j unless cr is CTA 0) and the threads
// that fill it locally (the offer: NQ threads; row j in CTA 0: NQ more) have
// arrived after their stores, besides the arrival that sets the byte count.
template <int NB>
__device__ __forceinline__ uint32_t slot_bytes(int cs, int cr) {
  return static_cast<uint32_t>(cs - 1) * (NB * 4 + 8) + (cr == 0 ? 0u : NB * 4u);
}
template <int NB>
__device__ __forceinline__ uint32_t slot_arrivals(int cr) {
  return 1u + (cr == 0 ? 2u : 1u) * (NB / 4);
}

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_sync() {
  __syncwarp();  // the .aligned barrier wants the warp converged
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of `p` (this CTA's shared memory) in the shared window of CTA `rank`
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// shared-memory stores into another CTA of the cluster that complete their
// bytes on mbarrier `bar` (an address in the same CTA's shared window)
__device__ __forceinline__ void st_async(uint32_t addr, float4 v, uint32_t bar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];"
      ::"r"(addr), "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
      "r"(__float_as_uint(v.w)), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void st_async(uint32_t addr, uint2 v, uint32_t bar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1, %2}, [%3];"
      ::"r"(addr), "r"(v.x), "r"(v.y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the slot's phase; *expired: an earlier wait gave up (skip)
__device__ __forceinline__ void panel_wait(uint64_t* bar, uint32_t parity, int* err,
                                           bool* expired) {
  if (*expired || mbar_try_wait_cluster(bar, parity)) return;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait_cluster(bar, parity)) {
    if (global_ns() - t0 > kPanelWaitNs) {
      if (err) atomicCAS(err, 0, kErrWaitPanel);
      *expired = true;
      return;
    }
  }
}

// pivot offer of a row: larger key wins, ties to the lower row index.  A
// number's key is its |a| bits plus 2, a NaN's 1 (below any number), and a
// lane with nothing to offer passes 0.
__device__ __forceinline__ uint32_t offer_key(float a) {
  const float m = fabsf(a);
  return m == m ? __float_as_uint(m) + 2u : 1u;
}
// warp winner of (key, idx) over all 32 lanes: the largest key, then the
// lowest lane holding it.  At every level the lanes hold rows (or groups of
// rows) in increasing row order, so the lowest lane is the lowest row: one
// max reduction and a ballot instead of a second reduction over the indices.
// *lane_out = the winning lane.
__device__ __forceinline__ void warp_offer(uint32_t key, uint32_t idx, uint32_t* kout,
                                           uint32_t* iout, int* lane_out) {
  const uint32_t m = __reduce_max_sync(0xFFFFFFFFu, key);
  const int l = __ffs(__ballot_sync(0xFFFFFFFFu, key == m)) - 1;
  *kout = m;
  *iout = __shfl_sync(0xFFFFFFFFu, idx, l);
  *lane_out = l;
}

template <int NQ>
__device__ __forceinline__ void put_row(float* dst, const float* v) {
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    *reinterpret_cast<float4*>(dst + 4 * q) =
        make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
template <int NQ>
__device__ __forceinline__ void get_row(float* v, const float* src) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const float4 x = *reinterpret_cast<const float4*>(src + 4 * q);
    v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
  }
}

// One pivot column of the cluster panel; K = the column's register (the
// current rotation puts column g*8 + K there), JB the block-column width.
template <int NB, int K, bool LOCAL>
__device__ __forceinline__ void panel_column(float (&v)[NB], int jj, int JB, int n, int J0, int r,
                                             bool has, int t, int lane, int wid, int nw, int cr,
                                             int cs, PanelShared<NB>& sh, int* err,
                                             bool* expired) {
  constexpr int NQ = NB / 4;
  const int j = J0 + jj, bf = jj & 1;
  const int g8 = jj - K;  // columns rotated away so far
  constexpr bool local = LOCAL;  // one CTA (cs == 1): no cluster exchange
  ClusterSlot<NB>& sl = sh.slot[bf];
  // ---- 1. offers: every warp's winner posts its row, the holder of row j posts row j
  const bool offers = has && r >= j;
  uint32_t wk, wi;
  int wl;
  warp_offer(offers ? offer_key(v[K]) : 0u, offers ? static_cast<uint32_t>(r) : 0xFFFFFFFFu, &wk,
             &wi, &wl);
  if (lane == 0) {
    sh.wkey[bf][wid] = wk;
    sh.widx[bf][wid] = wi;
  }
  if (local) {
    // one CTA: only the CTA's winner stores its row, straight into the
    // slot, once every warp has found it; the holder of row j stores row j
    // there too
    if (cr == 0 && t == jj) put_row<NQ>(sl.rowj, v);
    __syncthreads();
    uint32_t ck, ci;
    int cw;
    warp_offer(lane < nw ? sh.wkey[bf][lane] : 0u, lane < nw ? sh.widx[bf][lane] : 0xFFFFFFFFu,
               &ck, &ci, &cw);
    if (offers && static_cast<uint32_t>(r) == ci) put_row<NQ>(sl.row[0], v);
    if (t == 0) sl.ki[0] = make_uint2(ck, ci);
  } else {
    // only the CTA's winner stores its row, once every warp has found it
    if (cr == 0 && t == jj) put_row<NQ>(sh.rowj[bf], v);  // row j: CTA 0, thread jj
    __syncthreads();
    uint32_t ck, ci;
    int cw;
    warp_offer(lane < nw ? sh.wkey[bf][lane] : 0u, lane < nw ? sh.widx[bf][lane] : 0xFFFFFFFFu,
               &ck, &ci, &cw);
    if (offers && static_cast<uint32_t>(r) == ci) put_row<NQ>(sh.wrow[bf], v);
    __syncthreads();
  }
  // ---- 2. pushes: the pushing warps reduce the warps' offers themselves
  const int npush = local ? 0 : cs * NQ;
  if (!local && t == 0) mbar_arrive_expect_tx(&sh.bar[bf], slot_bytes<NB>(cs, cr));
  if (wid * 32 < npush) {  // whole warps: the reductions need every lane
    uint32_t ck, ci;
    int cw;
    warp_offer(lane < nw ? sh.wkey[bf][lane] : 0u, lane < nw ? sh.widx[bf][lane] : 0xFFFFFFFFu,
               &ck, &ci, &cw);
    cw = min(cw, nw - 1);  // every CTA offers a row (its rows are >= j)
    if (t < npush) {
      const int dst = t / NQ, q = t % NQ;
      const float4 x = *reinterpret_cast<const float4*>(&sh.wrow[bf][4 * q]);
      float4* to = reinterpret_cast<float4*>(&sl.row[cr][4 * q]);
      if (dst == cr) {  // this CTA's own slot: plain stores, then an arrival
        *to = x;
        if (q == 0) sl.ki[cr] = make_uint2(ck, ci);
        if (!local) mbar_arrive(&sh.bar[bf]);
      } else {
        const uint32_t rb = cl_map(&sh.bar[bf], dst);
        st_async(cl_map(to, dst), x, rb);
        if (q == 0) st_async(cl_map(&sl.ki[cr], dst), make_uint2(ck, ci), rb);
      }
    }
  }
  if (cr == 0 && t >= npush && t < 2 * npush) {
    const int e = t - npush, dst = e / NQ, q = e % NQ;
    const float4 x = *reinterpret_cast<const float4*>(&sh.rowj[bf][4 * q]);
    float4* to = reinterpret_cast<float4*>(&sl.rowj[4 * q]);
    if (dst == 0) {
      *to = x;
      if (!local) mbar_arrive(&sh.bar[bf]);
    } else {
      st_async(cl_map(to, dst), x, cl_map(&sh.bar[bf], dst));
    }
  }
  if (local)
    __syncthreads();
  else
    panel_wait(&sh.bar[bf], static_cast<uint32_t>((jj >> 1) & 1), err, expired);
  // ---- 3. the pivot: every warp reduces the cs offers (same data, same result)
  uint32_t gk, gi;
  int gw;
  warp_offer(lane < cs ? sl.ki[lane].x : 0u, lane < cs ? sl.ki[lane].y : 0xFFFFFFFFu, &gk, &gi,
             &gw);
  const float d = sl.rowj[K];
  const bool keep = (d != d || gi >= static_cast<uint32_t>(n));  // a NaN on the diagonal stays
  const int p = keep ? j : static_cast<int>(gi);
  const float* prow = keep ? sl.rowj : sl.row[min(gw, cs - 1)];
  if (t == jj) sh.piv[jj] = p;  // to global memory once, at the end, by the same thread
  if (p != j && has) {
    if (r == j)
      get_row<NQ>(v, prow);
    else if (r == p)
      get_row<NQ>(v, sl.rowj);
  }
  const float piv = prow[K];
  if (piv == 0.0f) {
    if (t == 0 && sh.zero == 0) sh.zero = j + 1;  // the first zero pivot
  } else if (has && r > j) {
    // ---- 4. multiplier and rank-1 update of the row's later columns
    const float l = __fdiv_rn(v[K], piv);
    v[K] = l;
    const int lim = JB - g8;  // registers below lim hold the block column's columns
#pragma unroll
    for (int q = (K + 1) / 4; q < NQ; ++q) {
      if (4 * q >= lim) break;  // the same for every thread
      const float4 u = *reinterpret_cast<const float4*>(prow + 4 * q);
      const float uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = 4 * q + e;
        if (c > K && c < lim) v[c] = fmaf(-l, uu[e], v[c]);
      }
    }
  }
}

template <int NB, bool LOCAL>
__device__ __forceinline__ void panel_body(float* __restrict__ A, int64_t lda, int n, int J0, int JB,
                                           int32_t* __restrict__ ipiv, int32_t* __restrict__ info,
                                           int* __restrict__ err) {
  constexpr int NQ = NB / 4;  // float4 words a row
  static_assert(PanelShared<NB>::MW <= 32 && CLP_MAX_CL <= 32, "one warp reduces the offers");
  static_assert(2 * CLP_MAX_CL * NQ <= CLP_THREADS, "pushes of the offered row and of row j");
  static_assert(NB % 8 == 0, "columns go in groups of 8");
  __shared__ __align__(16) PanelShared<NB> sh;
  // launched as a programmatic dependent of the previous block column's
  // update: wait for it before reading the block column (a no-op otherwise)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
  const int cr = static_cast<int>(cl_rank()), cs = static_cast<int>(cl_size());
  const int r = J0 + cr * CLP_THREADS + t;  // this thread's row
  const bool has = r < n;
  const bool vec = JB == NB && (lda % 4) == 0 && (J0 % 4) == 0 &&
                   (reinterpret_cast<uintptr_t>(A) % 16) == 0;
  float v[NB];
  {
    const float* src = A + static_cast<int64_t>(has ? r : J0) * lda + J0;
    if (vec) {
      get_row<NQ>(v, src);
    } else {
#pragma unroll
      for (int c = 0; c < NB; ++c) v[c] = c < JB ? src[c] : 0.0f;
    }
    if (!has) {
#pragma unroll
      for (int c = 0; c < NB; ++c) v[c] = 0.0f;
    }
  }
  if (t == 0) {
    sh.zero = 0;
    if (cs > 1) {
      mbar_init(&sh.bar[0], slot_arrivals<NB>(cr));
      mbar_init(&sh.bar[1], slot_arrivals<NB>(cr));
      fence_barrier_init();
    }
  }
  cl_sync();  // the slots' mbarriers set up in every CTA before the first remote store
  bool expired = false;
  for (int g = 0; g < NB; g += 8) {
#define BFX_PANEL_COL(K)                                                                      \
  if (g + K < JB)                                                                             \
    panel_column<NB, K, LOCAL>(v, g + K, JB, n, J0, r, has, t, lane, wid, nw, cr, cs, sh, err,\
                        &expired);
    BFX_PANEL_COL(0)
    BFX_PANEL_COL(1)
    BFX_PANEL_COL(2)
    BFX_PANEL_COL(3)
    BFX_PANEL_COL(4)
    BFX_PANEL_COL(5)
    BFX_PANEL_COL(6)
    BFX_PANEL_COL(7)
#undef BFX_PANEL_COL
    float tmp[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) tmp[c] = v[c];
#pragma unroll
    for (int c = 0; c < NB - 8; ++c) v[c] = v[c + 8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[NB - 8 + c] = tmp[c];
  }
  if (has) {
    float* dst = A + static_cast<int64_t>(r) * lda + J0;
    if (vec) {
      put_row<NQ>(dst, v);
    } else {
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c < JB) dst[c] = v[c];
    }
  }
  if (cr == 0) {
    for (int c = t; c < JB; c += blockDim.x) ipiv[J0 + c] = sh.piv[c];
    if (t == 0 && sh.zero != 0 && *info == 0) *info = sh.zero;
  }
  cl_sync();  // every CTA has received all it waits for before any leaves
}

// LOCAL: launched as one CTA (a cluster of one)
template <int NB, bool LOCAL>
__global__ void __launch_bounds__(CLP_THREADS, 1)
    lu_panel_cluster_kernel(float* __restrict__ A, int64_t lda, int n, int J0, int JB,
                            int32_t* __restrict__ ipiv, int32_t* __restrict__ info,
                            int* __restrict__ err) {
  panel_body<NB, LOCAL>(A, lda, n, J0, JB, ipiv, info, err);
}

// Batched form: cluster c (of the grid's clusters) factors block column J0
// of system sys[c]; a system whose n <= J0 has no work (the whole cluster
// leaves together).
template <int NB, bool LOCAL>
__global__ void __launch_bounds__(CLP_THREADS, 1)
    lu_panel_batched_kernel(const BatchLu* __restrict__ sys, int nb, int J0, int* __restrict__ err) {
  const BatchLu b = sys[blockIdx.x / cl_size()];
  const int JB = min(nb, b.n - J0);
  if (JB <= 0) return;
  panel_body<NB, LOCAL>(b.A, b.n, b.n, J0, JB, b.ipiv, b.info, err);
}

// Launch the cluster panel for the block column [J0, J0+JB) if it fits
// (rows <= kPanelMaxCluster * CLP_THREADS, JB <= 64); returns false to fall
// back on the tiles.  A single CTA has as many threads as rows (rounded up
// to whole warps), a cluster CLP_THREADS a CTA.
bool launch_panel_cluster(float* A, int64_t lda, int n, int J0, int JB, int32_t* ipiv,
                          int32_t* info, cudaStream_t s, bfx_status* st) {
  const int rows = n - J0;
  const int cs = static_cast<int>(ceil_div(rows, CLP_THREADS));
  if (JB > 64 || cs > kPanelMaxCluster) return false;
  const int threads = cs == 1 ? static_cast<int>(round_up(rows, 32)) : CLP_THREADS;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = static_cast<unsigned>(cs);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // the kernel waits itself
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3(static_cast<unsigned>(cs), 1, 1);
  cfg.blockDim = dim3(static_cast<unsigned>(threads), 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  int* err = device_error_word();
  if (!err) {
    *st = BFX_ECUDA;
    return false;
  }
  auto kern = JB <= 32 ? (cs == 1 ? lu_panel_cluster_kernel<32, true> : lu_panel_cluster_kernel<32, false>)
                       : (cs == 1 ? lu_panel_cluster_kernel<64, true> : lu_panel_cluster_kernel<64, false>);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, A, lda, n, J0, JB, ipiv, info, err);
  if (e != cudaSuccess) {  // e.g. a cluster size the device does not offer: use the tiles
    cudaGetLastError();
    return false;
  }
  *st = BFX_OK;
  return true;
}

struct LuWs {
  int64_t kp, ap, bp;
  size_t bytes;
};

// Workspace: two sets (by block-column parity: a panel writes its L21
// pieces while the previous block's trailing update still reads the other
// set) of np planes of the L21 pieces, then np planes of the U12^T pieces.
LuWs lu_ws(int np, int64_t n, int nb) {
  LuWs w;
  w.kp = round_up(nb, 8);
  w.ap = round_up(n * w.kp, 128);
  w.bp = w.ap;
  w.bytes = static_cast<size_t>(np) * static_cast<size_t>(2 * w.ap + w.bp) * 2;
  return w;
}

}  // namespace

// split.cu: launch_split as a programmatic dependent of the previous kernel
bfx_status launch_split_pdl(int64_t rows, int64_t cols, const float* x, int64_t ldx, int npieces,
                            uint16_t* hi, uint16_t* mid, uint16_t* lo, int64_t ldp, cudaStream_t s);

bfx_status lu_factor(bfx_mode mode, int64_t n, int nb, float* A, int64_t lda, int32_t* ipiv,
                     int32_t* info, void* ws, size_t ws_bytes, cudaStream_t s, int32_t* perm) {
  if (nb <= 0) nb = 64;
  if (nb > 128) return BFX_EINVAL;
  if (cudaMemsetAsync(info, 0, sizeof(int32_t), s) != cudaSuccess) return BFX_ECUDA;
  if (n == 0) return BFX_OK;
  const int np = mode_pieces(mode);
  LuWs w = lu_ws(np, n, nb);
  if (w.bytes > 0 && (!ws || ws_bytes < w.bytes || !aligned(ws, 256))) return BFX_ENOMEM;
  if (cudaFuncSetAttribute(lu_tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(TILE_SMEM_MAX)) != cudaSuccess)
    return BFX_ECUDA;
  const int tnb = nb <= 32 ? 32 : (nb <= 64 ? 64 : 128);  // register tile of the block solve
  auto solve = tnb == 32 ? lu_solve_cols_kernel<32>
                          : (tnb == 64 ? lu_solve_cols_kernel<64> : lu_solve_cols_kernel<128>);
  const size_t trsm_smem = trsm_smem_bytes(tnb);
  if (trsm_smem > 40 * 1024 &&
      cudaFuncSetAttribute(solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(trsm_smem)) != cudaSuccess)
    return BFX_ECUDA;
  uint16_t* Lset[2] = {static_cast<uint16_t*>(ws), static_cast<uint16_t*>(ws) + np * w.ap};
  uint16_t* Up = Lset[1] + np * w.ap;
  const int N = static_cast<int>(n);
  // Look-ahead: the caller's stream s carries the panel and the next block
  // column's row swaps, solve and update; an auxiliary stream (one per host
  // thread, joined to s by events) carries the other columns' row swaps and
  // the rest of the solve and of the trailing update, so they run while the
  // next panel is factored.  The next row swaps wait for them.  Each element
  // sees the same operations as without it.
  // The auxiliary stream and its two events are created once per host thread
  // and device (on the first LU call there) and kept until the thread ends;
  // later calls create nothing.
  struct Aux {
    int dev = -1;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, rest = nullptr;
    ~Aux() { release(); }
    void release() {
      if (fork) cudaEventDestroy(fork);
      if (rest) cudaEventDestroy(rest);
      if (s) cudaStreamDestroy(s);
      fork = rest = nullptr;
      s = nullptr;
      dev = -1;
    }
    bool ready() {
      int d = -1;
      if (cudaGetDevice(&d) != cudaSuccess) return false;
      if (d == dev && s) return true;
      release();
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&rest, cudaEventDisableTiming) != cudaSuccess) {
        release();
        return false;
      }
      dev = d;
      return true;
    }
  };
  thread_local Aux aux_owner;
  if (!aux_owner.ready()) return BFX_ECUDA;
  cudaStream_t aux = aux_owner.s;
  cudaEvent_t ev_fork = aux_owner.fork, ev_rest = aux_owner.rest;
  // on every return path the caller's stream is joined to the auxiliary
  // stream's last recorded work
  struct Join {
    cudaStream_t s;
    cudaEvent_t rest;
    bool pending = false;
    ~Join() {
      if (pending) cudaStreamWaitEvent(s, rest, 0);
    }
  } join{s, ev_rest};
  bool& rest_pending = join.pending;
  // C[:, c0 .. c0+nc) -= L21 U12[:, c0 .. c0+nc) for block column j0 on stream st
  // (pieces: L21's in Lp, split after the panel; U12^T's written by the
  // block solve)
  auto update = [&](int j0, int jb, int c0, int nc, const uint16_t* Lp, cudaStream_t st,
                    bool pdl) -> bfx_status {
    const int nr = N - j0 - jb;
    float* L21 = A + static_cast<int64_t>(j0 + jb) * lda + j0;
    float* U12 = A + static_cast<int64_t>(j0) * lda + j0 + jb + c0;
    float* A22 = A + static_cast<int64_t>(j0 + jb) * lda + j0 + jb + c0;
    if (np == 0) return launch_sgemm_simt(nr, nc, jb, -1.0f, L21, lda, U12, lda, 1.0f, A22, lda, st);
    const uint16_t* Uc = Up + static_cast<int64_t>(c0) * w.kp;  // rows c0.. of the U12^T planes
    return launch_gemm_presplit(mode, nr, nc, jb, -1.0f, Lp, w.kp, w.ap, Uc, w.kp, w.bp, 1.0f, A22,
                                lda, st, pdl);
  };
  for (int j0 = 0, blk = 0; j0 < N; j0 += nb, ++blk) {
    const int jb = (N - j0 < nb) ? N - j0 : nb;
    const int nr = N - j0 - jb;
    uint16_t* Lp = Lset[blk & 1];
    bfx_status pst = BFX_OK;
    const bool clustered = launch_panel_cluster(A, lda, N, j0, jb, ipiv, info, s, &pst);
    if (pst != BFX_OK) return pst;
    for (int t0 = j0; !clustered && t0 < j0 + jb; t0 += TILE_W) {
      const int tw = std::min(TILE_W, j0 + jb - t0);
      const int rows = N - t0;
      const size_t tsm = static_cast<size_t>(rows) * TILE_W * sizeof(float);
      if (rows <= PANEL_THREADS)
        lu_tile_regs_kernel<1><<<1, PANEL_THREADS, 0, s>>>(A, lda, N, j0, jb, t0, tw, ipiv, info);
      else if (rows <= 2 * PANEL_THREADS)
        lu_tile_regs_kernel<2><<<1, PANEL_THREADS, 0, s>>>(A, lda, N, j0, jb, t0, tw, ipiv, info);
      else if (rows <= 4 * PANEL_THREADS)
        lu_tile_regs_kernel<4><<<1, PANEL_THREADS, 0, s>>>(A, lda, N, j0, jb, t0, tw, ipiv, info);
      else if (rows <= 8 * PANEL_THREADS)
        lu_tile_regs_kernel<8><<<1, PANEL_THREADS, 0, s>>>(A, lda, N, j0, jb, t0, tw, ipiv, info);
      else if (tsm <= TILE_SMEM_MAX)
        lu_tile_kernel<true><<<1, PANEL_THREADS, tsm, s>>>(A, lda, N, j0, jb, t0, tw, ipiv, info);
      else
        lu_tile_kernel<false><<<1, PANEL_THREADS, 0, s>>>(A, lda, N, j0, jb, t0, tw, ipiv, info);
      const int ncol = j0 + jb - t0 - tw;
      if (ncol > 0 && N - t0 - tw > 0) {
        const int64_t work = static_cast<int64_t>(N - t0 - tw) * ncol;
        const int g = static_cast<int>(std::min<int64_t>(ceil_div(work, 256), 8LL * 148));
        lu_tile_update_kernel<<<g, 256, 0, s>>>(A, lda, N, j0, jb, t0, tw);
      }
    }
    // the L21 pieces into this block's set (the previous block's update may
    // still read the other), before waiting for that update
    if (np > 0 && nr > 0) {
      const float* L21 = A + static_cast<int64_t>(j0 + jb) * lda + j0;
      const bfx_status e = launch_split_pdl(nr, jb, L21, lda, np, Lp, np > 1 ? Lp + w.ap : nullptr,
                                            np > 2 ? Lp + 2 * w.ap : nullptr, w.kp, s);
      if (e != BFX_OK) return e;
    }
    // the row swaps move rows of columns the previous rest update writes
    if (rest_pending && cudaStreamWaitEvent(s, ev_rest, 0) != cudaSuccess) return BFX_ECUDA;
    rest_pending = false;
    const int nc = std::min(nb, nr);  // the next block column's width (0 after the last)
    // the next block column: row swaps and solve (one kernel), update on s
    if (nc > 0) {
      solve<<<static_cast<unsigned>(ceil_div(nc, TRSM_COLS)), TRSM_COLS * 32, trsm_smem, s>>>(
          A, lda, j0, jb, j0 + jb, j0 + jb + nc, ipiv, np, Up, w.bp, w.kp);
      const bfx_status st = update(j0, jb, 0, nc, Lp, s, true);
      if (st != BFX_OK) return st;
    }
    // the rest on the auxiliary stream, after the L21 pieces: the row swaps
    // of the columns left of the block, the row swaps and solve of the
    // columns right of the next one, and their update
    const int c_far = j0 + jb + nc, n_far = N - c_far;
    if (j0 + n_far > 0 || perm) {
      // (forked after the next column's update: started earlier, the rest
      // competed with that critical work for the SMs: n = 4096 LU 8.10 ->
      // 8.48 ms)
      if (cudaEventRecord(ev_fork, s) != cudaSuccess ||
          cudaStreamWaitEvent(aux, ev_fork, 0) != cudaSuccess)
        return BFX_ECUDA;
      if (j0 > 0 || perm)  // (perm: the block's swaps also go into the permutation)
        lu_laswp_kernel<<<static_cast<unsigned>(std::max<int64_t>(1, ceil_div(j0, LASWP_COLS))),
                          LASWP_THREADS, 0, aux>>>(A, lda, j0, jb, ipiv, 0, j0, 0, 0, perm, N);
      if (n_far > 0) {
        solve<<<static_cast<unsigned>(ceil_div(n_far, TRSM_COLS)), TRSM_COLS * 32, trsm_smem, aux>>>(
            A, lda, j0, jb, c_far, N, ipiv, np, Up, w.bp, w.kp);
        const bfx_status st = update(j0, jb, nc, n_far, Lp, aux, false);
        if (st != BFX_OK) return st;
      }
      if (cudaEventRecord(ev_rest, aux) != cudaSuccess) return BFX_ECUDA;
      rest_pending = true;
    }
  }
  if (rest_pending) {
    rest_pending = false;
    if (cudaStreamWaitEvent(s, ev_rest, 0) != cudaSuccess) return BFX_ECUDA;
  }
  return last_launch_status();
}

bfx_status lu_batched_block(bfx_mode mode, const BatchLu* d_sys, const int* h_n_desc, int S,
                            int nb, int J0, uint16_t* packA, uint16_t* packB, int64_t slot_rows,
                            int64_t kp, cudaStream_t s) {
  int S_act = 0;
  while (S_act < S && h_n_desc[S_act] > J0) ++S_act;
  if (S_act == 0) return BFX_OK;
  if (kp < nb || kp > SPLIT_KMAX || kp % 2 != 0) return BFX_EINVAL;
  const int nmax = h_n_desc[0];
  // once per process (thread-safe initialisation)
  static const bool attrs = [] {
    return cudaFuncSetAttribute(lu_trsm_batched_kernel<128>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(trsm_smem_bytes(128))) == cudaSuccess;
  }();
  if (!attrs) return BFX_ECUDA;
  bool paneled = false;
  if (nb <= 64) {
    // the whole block column of every system by the panel kernel: one CTA a
    // system (two, a cluster, above 512 rows)
    const int rows = nmax - J0;
    const int cs = static_cast<int>(ceil_div(rows, CLP_THREADS));
    if (cs <= 2) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = static_cast<unsigned>(cs);
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(static_cast<unsigned>(cs * S_act), 1, 1);
      cfg.blockDim = dim3(static_cast<unsigned>(cs == 1 ? round_up(rows, 32) : CLP_THREADS), 1, 1);
      cfg.stream = s;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      auto kern = nb <= 32 ? (cs == 1 ? lu_panel_batched_kernel<32, true> : lu_panel_batched_kernel<32, false>)
                           : (cs == 1 ? lu_panel_batched_kernel<64, true> : lu_panel_batched_kernel<64, false>);
      const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, d_sys, nb, J0, device_error_word());
      if (e == cudaSuccess)
        paneled = true;
      else
        cudaGetLastError();
    }
  }
  for (int j0 = J0; !paneled && j0 < J0 + nb; j0 += TILE_W) {
    int S_t = 0;
    while (S_t < S_act && h_n_desc[S_t] > j0) ++S_t;
    if (S_t == 0) break;
    // batch systems have n <= 1024: tiles of at most 2 rows a thread, in registers
    if (nmax - j0 <= PANEL_THREADS)
      lu_tile_regs_batched_kernel<1><<<S_t, PANEL_THREADS, 0, s>>>(d_sys, nb, J0, j0);
    else
      lu_tile_regs_batched_kernel<2><<<S_t, PANEL_THREADS, 0, s>>>(d_sys, nb, J0, j0);
    const int64_t work = static_cast<int64_t>(nmax - j0) * nb;
    const unsigned gx = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), 32)));
    lu_tile_update_batched_kernel<<<dim3(gx, S_t), 256, 0, s>>>(d_sys, nb, J0, j0);
  }
  // a CTA forms a system's swap set once and moves up to sixteen column
  // blocks (one CTA a system up to n = 512: the serial swap-set build,
  // repeated by every CTA of a system, cost more than the CTAs' parallelism
  // gained; four blocks a CTA: +0.3 ms a batch of 2000 systems)
  const unsigned cblk = static_cast<unsigned>(ceil_div(ceil_div(nmax, LASWP_COLS), 16));
  lu_laswp_batched_kernel<<<dim3(cblk, S_act), LASWP_THREADS, 0, s>>>(d_sys, nb, J0);
  const int tnb = nb <= 32 ? 32 : (nb <= 64 ? 64 : 128);
  const size_t tsmem = trsm_smem_bytes(tnb);
  const unsigned tblk = static_cast<unsigned>(ceil_div(nmax - J0, TRSM_COLS * TRSM_WCOLS));
  if (tnb == 32)
    lu_trsm_batched_kernel<32><<<dim3(tblk, S_act), TRSM_COLS * 32, tsmem, s>>>(d_sys, nb, J0);
  else if (tnb == 64)
    lu_trsm_batched_kernel<64><<<dim3(tblk, S_act), TRSM_COLS * 32, tsmem, s>>>(d_sys, nb, J0);
  else
    lu_trsm_batched_kernel<128><<<dim3(tblk, S_act), TRSM_COLS * 32, tsmem, s>>>(d_sys, nb, J0);
  const int np = mode_pieces(mode);
  const unsigned sblk = static_cast<unsigned>(ceil_div(nmax - J0, SPLIT_ROWS));
  lu_split_batched_kernel<<<dim3(sblk, S_act), SPLIT_THREADS, 0, s>>>(d_sys, nb, J0, np, packA,
                                                                      packB, slot_rows, kp);
  return last_launch_status();
}

size_t lu_workspace_bytes(bfx_mode mode, int64_t n, int nb) {
  const int np = mode_pieces(mode);
  if (n <= 0) return 0;
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
                   static_cast<cudaStream_t>(stream), nullptr);
}

}  // extern "C"
