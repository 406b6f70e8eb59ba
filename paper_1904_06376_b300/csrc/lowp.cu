// Single-type LU with residual-form refinement: the plain IR table of
// Sec. IV-B, which compares FP32 factors with factors computed entirely in
// one bfloat16 or one binary16 type.
//
// LU (per system): A is rounded to the type, then the unblocked right-looking
// LU with partial pivoting (pivot = first row of the largest |a| at or below
// the diagonal, whole rows swapped) runs with every division, product and
// difference done in FP32 (IEEE, round to nearest, no contraction) and its
// result rounded to the type; an exactly zero pivot column sets info (the
// first one) and is skipped.  Each element of the factors sees the same
// sequence of operations whatever the thread layout, so the factors are
// reproducible bit for bit.
//
// Refinement (Sec. III, residual form, FP64): x = (LU)^-1 P b, then up to
// max_iter times r = b - A x, d = (LU)^-1 P r, x += d; converged when
// |d|_inf <= tol |x|_inf, diverged at the first NaN or Inf entry.  Every sum
// runs in one fixed sequential order (residual rows left to right; forward
// substitution by columns, which adds each row's terms left to right;
// backward substitution row by row, left to right), with separate FP64
// multiply and subtract, so results do not depend on the launch.
//
// Layout: one warp per system (n <= 128); the factors live in shared memory
// as FP32 words holding values of the type.
#include "bfx_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace bfx {
namespace {

constexpr int LP_MAXN = 128;

template <int TYPE>
__device__ __forceinline__ float to_type(float v) {
  if constexpr (TYPE == BFX_LOWP_BF16) return __bfloat162float(__float2bfloat16_rn(v));
  else if constexpr (TYPE == BFX_LOWP_FP16) return __half2float(__float2half_rn(v));
  else return v;
}

// v <- (LU)^-1 P v for the factors in M (n x n, row stride n); lanes of one warp.
__device__ void lowp_solve(const float* M, const int32_t* piv, double* v, int n) {
  const int lane = threadIdx.x;
  if (lane == 0)
    for (int j = 0; j < n; ++j) {
      const int p = piv[j];
      if (p != j) {
        const double t = v[j];
        v[j] = v[p];
        v[p] = t;
      }
    }
  __syncwarp();
  // forward, unit lower: column l updates every row below it
  for (int l = 0; l < n - 1; ++l) {
    const double vl = v[l];
    for (int i = l + 1 + lane; i < n; i += 32)
      v[i] = __dsub_rn(v[i], __dmul_rn(static_cast<double>(M[i * n + l]), vl));
    __syncwarp();
  }
  // backward: row by row, each row's terms left to right
  if (lane == 0)
    for (int i = n - 1; i >= 0; --i) {
      double s = v[i];
      for (int l = i + 1; l < n; ++l) s = __dsub_rn(s, __dmul_rn(static_cast<double>(M[i * n + l]), v[l]));
      v[i] = __ddiv_rn(s, static_cast<double>(M[i * n + i]));
    }
  __syncwarp();
}

template <int TYPE>
__global__ void __launch_bounds__(32)
    lowp_lu_ir_kernel(int n, const float* __restrict__ A, const double* __restrict__ b,
                      const double* __restrict__ tol, int max_iter, double* __restrict__ x,
                      float* __restrict__ LU_out, int32_t* __restrict__ ipiv_out,
                      int32_t* __restrict__ iters, int32_t* __restrict__ conv,
                      int32_t* __restrict__ info_out) {
  extern __shared__ __align__(16) uint8_t lp_smem[];
  double* xv = reinterpret_cast<double*>(lp_smem);  // [n]
  double* r = xv + n;                                 // [n]
  float* M = reinterpret_cast<float*>(r + n);         // [n][n]
  int32_t* piv = reinterpret_cast<int32_t*>(M + n * n);  // [n]
  const int lane = threadIdx.x;
  const int64_t sys = blockIdx.x;
  const float* Ag = A + sys * n * n;
  const double* bg = b + sys * n;

  for (int e = lane; e < n * n; e += 32) M[e] = to_type<TYPE>(Ag[e]);
  __syncwarp();
  int info = 0;
  for (int k = 0; k < n; ++k) {
    // first row of the largest |a| (NaN is never larger; a NaN diagonal stays)
    float best = -1.0f;
    int bi = n;
    for (int i = k + lane; i < n; i += 32) {
      const float a = fabsf(M[i * n + k]);
      if (a > best) {
        best = a;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xFFFFFFFFu, best, o);
      const int oi = __shfl_xor_sync(0xFFFFFFFFu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    const float akk = M[k * n + k];
    const int p = (isnan(akk) || bi >= n) ? k : bi;
    const float amax = fabsf(M[p * n + k]);
    if (lane == 0) piv[k] = p;
    if (amax == 0.0f) {
      if (!info) info = k + 1;
      __syncwarp();
      continue;
    }
    if (p != k)
      for (int j = lane; j < n; j += 32) {
        const float t = M[k * n + j];
        M[k * n + j] = M[p * n + j];
        M[p * n + j] = t;
      }
    __syncwarp();
    const float pv = M[k * n + k];
    for (int i = k + 1 + lane; i < n; i += 32) M[i * n + k] = to_type<TYPE>(__fdiv_rn(M[i * n + k], pv));
    __syncwarp();
    const int w = n - k - 1;
    for (int e = lane; e < w * w; e += 32) {
      const int i = k + 1 + e / w, j = k + 1 + e % w;
      M[i * n + j] = to_type<TYPE>(__fsub_rn(M[i * n + j], to_type<TYPE>(__fmul_rn(M[i * n + k], M[k * n + j]))));
    }
    __syncwarp();
  }
  if (LU_out)
    for (int e = lane; e < n * n; e += 32) LU_out[sys * n * n + e] = M[e];
  if (ipiv_out)
    for (int j = lane; j < n; j += 32) ipiv_out[sys * n + j] = piv[j];

  // refinement
  for (int i = lane; i < n; i += 32) xv[i] = bg[i];
  __syncwarp();
  lowp_solve(M, piv, xv, n);
  const double tl = tol[sys];
  const float* Arow = Ag;
  int it = 0, ok = 0;
  while (it < max_iter) {
    for (int i = lane; i < n; i += 32) {
      double s = bg[i];
      for (int l = 0; l < n; ++l) s = __dsub_rn(s, __dmul_rn(static_cast<double>(Arow[i * n + l]), xv[l]));
      r[i] = s;
    }
    __syncwarp();
    lowp_solve(M, piv, r, n);
    double dn = 0.0, xn = 0.0;
    int bad = 0;
    for (int i = lane; i < n; i += 32) {
      const double xi = __dadd_rn(xv[i], r[i]);
      xv[i] = xi;
      if (!isfinite(r[i]) || !isfinite(xi)) bad = 1;
      dn = fmax(dn, fabs(r[i]));
      xn = fmax(xn, fabs(xi));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dn = fmax(dn, __shfl_xor_sync(0xFFFFFFFFu, dn, o));
      xn = fmax(xn, __shfl_xor_sync(0xFFFFFFFFu, xn, o));
      bad |= __shfl_xor_sync(0xFFFFFFFFu, bad, o);
    }
    __syncwarp();
    ++it;
    if (bad) break;
    if (dn <= tl * xn) {
      ok = 1;
      break;
    }
  }
  double* xg = x + sys * n;
  for (int i = lane; i < n; i += 32) xg[i] = xv[i];
  if (lane == 0) {
    iters[sys] = it;
    conv[sys] = ok;
    info_out[sys] = info;
  }
}

size_t lowp_smem(int n) {
  return sizeof(double) * 2 * n + sizeof(float) * n * n + sizeof(int32_t) * n;
}

}  // namespace

bfx_status launch_lowp_lu_ir(bfx_lowp type, int count, int n, const float* A, const double* b,
                             const double* tol, int max_iter, double* x, float* LU_out,
                             int32_t* ipiv_out, int32_t* iters, int32_t* conv, int32_t* info,
                             cudaStream_t s) {
  if (count == 0) return BFX_OK;
  const size_t smem = lowp_smem(n);
  auto run = [&](auto kern) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
      return BFX_ECUDA;
    kern<<<count, 32, smem, s>>>(n, A, b, tol, max_iter, x, LU_out, ipiv_out, iters, conv, info);
    return last_launch_status();
  };
  switch (type) {
    case BFX_LOWP_FP32: return run(lowp_lu_ir_kernel<BFX_LOWP_FP32>);
    case BFX_LOWP_BF16: return run(lowp_lu_ir_kernel<BFX_LOWP_BF16>);
    case BFX_LOWP_FP16: return run(lowp_lu_ir_kernel<BFX_LOWP_FP16>);
    default: return BFX_EINVAL;
  }
}

int lowp_max_n() { return LP_MAXN; }

}  // namespace bfx
