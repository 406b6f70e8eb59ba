// Inner product x^T y from bfloat16 pieces (Sec. II-B .. II-G of the paper).
//
// Each element pair is split in registers (Sec. II-A) and every kept product
// x_l^(i) y_l^(j), exact in FP32 (Sec. I), is accumulated with one FMA into the
// FP32 accumulator of its level i+j (the paper's "equal levels" Z^(i+j)), the
// smallest level first.  A block reduces each level in a fixed tree; a second
// one-block kernel reduces the per-block partials level by level in a fixed
// order and combines the levels smallest first in FP32 (x3: Z0 + Z1;
// x6: Z0 + (Z1 + Z2); x9: Z0 + (Z1 + (Z2 + (Z3 + Z4)))).  Deterministic for a
// given grid.  Mode FP32 accumulates plain FMAs x_l y_l (Sec. II-C).
//
// HBM-bound: 8 bytes read per element pair; grid of 4 blocks a SM with
// 16-byte loads.
#include "bfx_internal.cuh"

namespace bfx {
namespace {

constexpr int DOT_THREADS = 256;
constexpr int DOT_LEVELS = 5;

__device__ __forceinline__ float bf16_val(float a) {
  return __bfloat162float(__float2bfloat16_rn(a));
}

// pieces of one element (same readings as the split kernel: Inf/NaN and the
// overflowing range are carried by hi alone / truncated hi).
__device__ __forceinline__ void pieces3(float a, float& h, float& m, float& l) {
  const uint32_t u = __float_as_uint(a);
  const uint32_t mag = u & 0x7FFFFFFFu;
  if (mag >= 0x7F800000u) {
    h = a;
    m = 0.0f;
    l = 0.0f;
    return;
  }
  h = (mag >= 0x7F7F8000u) ? __uint_as_float(u & 0xFFFF0000u) : bf16_val(a);
  const float r1 = __fsub_rn(a, h);
  m = bf16_val(r1);
  l = bf16_val(__fsub_rn(r1, m));
}

template <int MODE>
__device__ __forceinline__ void accumulate(float a, float b, float (&Z)[DOT_LEVELS]) {
  if (MODE == 0) {
    Z[0] = fmaf(a, b, Z[0]);
    return;
  }
  float x[3], y[3];
  pieces3(a, x[0], x[1], x[2]);
  pieces3(b, y[0], y[1], y[2]);
  if (MODE == 9) Z[4] = fmaf(x[2], y[2], Z[4]);
  if (MODE >= 8) {
    Z[3] = fmaf(x[1], y[2], Z[3]);
    Z[3] = fmaf(x[2], y[1], Z[3]);
  }
  if (MODE >= 6) {
    Z[2] = fmaf(x[0], y[2], Z[2]);
    Z[2] = fmaf(x[1], y[1], Z[2]);
    Z[2] = fmaf(x[2], y[0], Z[2]);
  }
  if (MODE >= 3) {
    Z[1] = fmaf(x[0], y[1], Z[1]);
    Z[1] = fmaf(x[1], y[0], Z[1]);
  }
  Z[0] = fmaf(x[0], y[0], Z[0]);
}

template <int MODE>
__global__ void __launch_bounds__(DOT_THREADS) dot_partial_kernel(int64_t n,
                                                                 const float* __restrict__ x,
                                                                 const float* __restrict__ y,
                                                                 bool vec, float* __restrict__ part) {
  float Z[DOT_LEVELS] = {0.f, 0.f, 0.f, 0.f, 0.f};
  const int64_t tid = blockIdx.x * static_cast<int64_t>(DOT_THREADS) + threadIdx.x;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * DOT_THREADS;
  if (vec) {
    const int64_t n4 = n / 4;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* y4 = reinterpret_cast<const float4*>(y);
    for (int64_t i = tid; i < n4; i += stride) {
      const float4 a = __ldcs(x4 + i), b = __ldcs(y4 + i);
      accumulate<MODE>(a.x, b.x, Z);
      accumulate<MODE>(a.y, b.y, Z);
      accumulate<MODE>(a.z, b.z, Z);
      accumulate<MODE>(a.w, b.w, Z);
    }
    for (int64_t i = n4 * 4 + tid; i < n; i += stride) accumulate<MODE>(x[i], y[i], Z);
  } else {
    for (int64_t i = tid; i < n; i += stride) accumulate<MODE>(x[i], y[i], Z);
  }
  __shared__ float red[DOT_LEVELS][DOT_THREADS];
#pragma unroll
  for (int lv = 0; lv < DOT_LEVELS; ++lv) red[lv][threadIdx.x] = Z[lv];
  __syncthreads();
  for (int s = DOT_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int lv = 0; lv < DOT_LEVELS; ++lv) red[lv][threadIdx.x] += red[lv][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x < DOT_LEVELS) part[blockIdx.x * DOT_LEVELS + threadIdx.x] = red[threadIdx.x][0];
}

template <int MODE>
__global__ void __launch_bounds__(DOT_THREADS) dot_final_kernel(int nblocks,
                                                               const float* __restrict__ part,
                                                               float* __restrict__ out) {
  __shared__ float red[DOT_LEVELS][DOT_THREADS];
#pragma unroll
  for (int lv = 0; lv < DOT_LEVELS; ++lv) {
    float s = 0.0f;
    for (int b = threadIdx.x; b < nblocks; b += DOT_THREADS) s += part[b * DOT_LEVELS + lv];
    red[lv][threadIdx.x] = s;
  }
  __syncthreads();
  for (int s = DOT_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int lv = 0; lv < DOT_LEVELS; ++lv) red[lv][threadIdx.x] += red[lv][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float Z0 = red[0][0], Z1 = red[1][0], Z2 = red[2][0], Z3 = red[3][0], Z4 = red[4][0];
    float z;
    switch (MODE) {
      case 0:
      case 1: z = Z0; break;
      case 3: z = Z0 + Z1; break;
      case 6: z = Z0 + (Z1 + Z2); break;
      case 8: z = Z0 + (Z1 + (Z2 + Z3)); break;
      default: z = Z0 + (Z1 + (Z2 + (Z3 + Z4))); break;
    }
    *out = z;
  }
}

int dot_blocks() {
  const int sms = current_num_sms() > 0 ? current_num_sms() : 148;
  return 4 * sms;
}

template <int MODE>
bfx_status run_dot(int64_t n, const float* x, const float* y, float* out, float* part, int g,
                   cudaStream_t s) {
  const bool vec = aligned(x, 16) && aligned(y, 16);
  dot_partial_kernel<MODE><<<g, DOT_THREADS, 0, s>>>(n, x, y, vec, part);
  dot_final_kernel<MODE><<<1, DOT_THREADS, 0, s>>>(g, part, out);
  return last_launch_status();
}

}  // namespace
}  // namespace bfx

using namespace bfx;

extern "C" {

BFX_API size_t bfx_dot_workspace_size(void) {
  return static_cast<size_t>(dot_blocks()) * DOT_LEVELS * sizeof(float);
}

BFX_API bfx_status bfx_dot_bf16xN(bfx_mode mode, int64_t n, const float* d_x, const float* d_y,
                                  float* d_result, void* d_ws, size_t ws_bytes,
                                  bfx_stream stream) {
  if (n < 0 || !d_result) return BFX_EINVAL;
  if (n > 0 && (!d_x || !d_y)) return BFX_EINVAL;
  if (mode != BFX_FP32 && mode_pieces(mode) == 0) return BFX_EINVAL;
  const int g = dot_blocks();
  const size_t need = static_cast<size_t>(g) * DOT_LEVELS * sizeof(float);
  if (!d_ws || ws_bytes < need) return BFX_ENOMEM;
  if (!aligned(d_ws, 16)) return BFX_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* part = static_cast<float*>(d_ws);
  switch (mode) {
    case BFX_FP32: return run_dot<0>(n, d_x, d_y, d_result, part, g, s);
    case BFX_X1: return run_dot<1>(n, d_x, d_y, d_result, part, g, s);
    case BFX_X3: return run_dot<3>(n, d_x, d_y, d_result, part, g, s);
    case BFX_X6: return run_dot<6>(n, d_x, d_y, d_result, part, g, s);
    case BFX_X8: return run_dot<8>(n, d_x, d_y, d_result, part, g, s);
    default: return run_dot<9>(n, d_x, d_y, d_result, part, g, s);
  }
}

}  // extern "C"
