// Plain FP32 SIMT GEMM: the reference computation of Sec. II-C of the paper
// (Z <- FMA(x_l, y_l, Z) for l = 1..n) on the CUDA cores, used as the
// same-GPU baseline for the bfloat16-split tensor-core GEMM.
//
// 128 x 128 block tile, BK = 8, 256 threads, 8 x 8 outputs a thread (two 4x4
// quads per direction so shared-memory reads are conflict-free float4s),
// double-buffered shared memory with register prefetch.  Every output is
// accumulated with one fmaf per k in increasing k; zero-filled ragged edges
// only add exact zeros.  Epilogue: t = alpha*Z; C = beta == 0 ? t : fma(beta, C, t).
#include "bfx_internal.cuh"

namespace bfx {
namespace {

constexpr int SBM = 128, SBN = 128, SBK = 8;

template <bool VEC>
__global__ void __launch_bounds__(256)
    sgemm_kernel(int M, int N, int K, float alpha, const float* __restrict__ A, int64_t lda,
                 const float* __restrict__ B, int64_t ldb, float beta, float* __restrict__ C,
                 int64_t ldc) {
  __shared__ __align__(16) float As[2][SBK][SBM];
  __shared__ __align__(16) float Bs[2][SBK][SBN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * SBM, n0 = blockIdx.x * SBN;

  // global -> register staging for one BK slab
  const int a_row = tid >> 1, a_k = (tid & 1) * 4;  // A: 128 rows x 8 k
  const int b_k = tid >> 5, b_col = (tid & 31) * 4;  // B: 8 k x 128 cols
  float ra[4], rb[4];

  auto load_slab = [&](int k0) {
    const int gr = m0 + a_row;
    if (VEC && gr < M && k0 + a_k + 3 < K) {
      const float4 v = *reinterpret_cast<const float4*>(A + gr * lda + k0 + a_k);
      ra[0] = v.x; ra[1] = v.y; ra[2] = v.z; ra[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        ra[i] = (gr < M && k0 + a_k + i < K) ? A[gr * lda + k0 + a_k + i] : 0.0f;
    }
    const int gk = k0 + b_k, gc = n0 + b_col;
    if (VEC && gk < K && gc + 3 < N) {
      const float4 v = *reinterpret_cast<const float4*>(B + gk * ldb + gc);
      rb[0] = v.x; rb[1] = v.y; rb[2] = v.z; rb[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) rb[i] = (gk < K && gc + i < N) ? B[gk * ldb + gc + i] : 0.0f;
    }
  };
  auto store_slab = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 4; ++i) As[buf][a_k + i][a_row] = ra[i];
    *reinterpret_cast<float4*>(&Bs[buf][b_k][b_col]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  const int nslab = (K + SBK - 1) / SBK;
  load_slab(0);
  store_slab(0);
  __syncthreads();
  for (int s = 0; s < nslab; ++s) {
    const int buf = s & 1;
    if (s + 1 < nslab) load_slab((s + 1) * SBK);
#pragma unroll
    for (int kk = 0; kk < SBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4 + 64]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4 + 64]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (s + 1 < nslab) store_slab(buf ^ 1);
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = m0 + ty * 4 + (i & 3) + (i >> 2) * 64;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = n0 + tx * 4 + (j & 3) + (j >> 2) * 64;
      if (c >= N) continue;
      const float t = alpha * acc[i][j];
      float* dst = C + static_cast<int64_t>(r) * ldc + c;
      *dst = (beta == 0.0f) ? t : fmaf(beta, *dst, t);
    }
  }
}

}  // namespace

bfx_status launch_sgemm_simt(int64_t m, int64_t n, int64_t k, float alpha, const float* A,
                             int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                             int64_t ldc, cudaStream_t s) {
  if (m == 0 || n == 0) return BFX_OK;
  if (k == 0) return launch_scale(m, n, beta, C, ldc, s);
  if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) return BFX_EUNSUPPORTED;
  const int64_t gy = ceil_div(m, SBM), gx = ceil_div(n, SBN);
  if (gy > 65535 || gx > INT32_MAX) return BFX_EUNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  const bool vec = (lda % 4 == 0) && (ldb % 4 == 0) && aligned(A, 16) && aligned(B, 16);
  if (vec)
    sgemm_kernel<true><<<grid, 256, 0, s>>>(int(m), int(n), int(k), alpha, A, lda, B, ldb, beta,
                                            C, ldc);
  else
    sgemm_kernel<false><<<grid, 256, 0, s>>>(int(m), int(n), int(k), alpha, A, lda, B, ldb, beta,
                                             C, ldc);
  return last_launch_status();
}

}  // namespace bfx

// ---------------------------------------------------------------------------
// Arithmetic peaks of the CUDA cores, measured: the roofline denominators of
// the FP32 SIMT baseline (FFMA) and of the refinement's FP64 work (DFMA).
// Every thread runs 8 independent FMA chains (enough to cover the pipeline
// latency), one CTA of 256 threads per 1/8 of an SM's threads times 8 waves
// of the SMs; the chains' results are stored only under a condition the
// caller never meets, so the work cannot be dropped.
namespace bfx {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T seed, T* __restrict__ sink) {
  T a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = seed + static_cast<T>(threadIdx.x + q);
  const T m = static_cast<T>(0.999999), c = static_cast<T>(1e-7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = fma(a[q], m, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  if (s == static_cast<T>(-12345.0)) sink[threadIdx.x] = s;
}

template <typename T>
bfx_status fma_peak(double* tflops, cudaStream_t s) {
  const int sms = current_num_sms();
  if (sms <= 0) return BFX_ECUDA;
  const int grid = sms * 8, iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return BFX_ECUDA;
  }
  fma_peak_kernel<T><<<grid, 256, 0, s>>>(iters / 8, static_cast<T>(1.0), nullptr);  // warm-up
  cudaEventRecord(e0, s);
  fma_peak_kernel<T><<<grid, 256, 0, s>>>(iters, static_cast<T>(1.0), nullptr);
  cudaEventRecord(e1, s);
  float ms = 0.0f;
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return BFX_ECUDA;
  const double flops = 2.0 * 8.0 * 16.0 * iters * static_cast<double>(grid) * 256.0;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return last_launch_status();
}

}  // namespace
}  // namespace bfx

extern "C" BFX_API bfx_status bfx_measure_fma_peak(int fp64, double* h_tflops, bfx_stream stream) {
  if (!h_tflops) return BFX_EINVAL;
  return fp64 ? bfx::fma_peak<double>(h_tflops, static_cast<cudaStream_t>(stream))
              : bfx::fma_peak<float>(h_tflops, static_cast<cudaStream_t>(stream));
}
