// Split of FP32 values into bfloat16 pieces (Sec. II-A of the paper):
//   hi = (B16)a,  mid = (B16)(a - hi),  lo = (B16)(a - hi - mid)
// with (B16) the hardware round-to-nearest-even conversion (cvt.rn.bf16.f32).
// Both remainders are exact FP32 subtractions for |a| >= 2^-110 (Sec. II-F).
//
// bfx_split: bandwidth-bound streaming pass (reads 4 B, writes 2*npieces B per
// element).  Fast path: 8 consecutive elements per thread, two 16-byte loads,
// one 16-byte store per piece plane; grid of one full wave over the SMs.
// bfx_split_transpose: the same split written transposed through a shared-
// memory tile so both the FP32 reads and the bfloat16 writes are coalesced.
#include "bfx_internal.cuh"

namespace bfx {
namespace {

// split_elem (the per-element decomposition) lives in bfx_internal.cuh.

__device__ __forceinline__ uint4 pack8(const uint16_t* q) {
  uint4 o;
  o.x = q[0] | (static_cast<uint32_t>(q[1]) << 16);
  o.y = q[2] | (static_cast<uint32_t>(q[3]) << 16);
  o.z = q[4] | (static_cast<uint32_t>(q[5]) << 16);
  o.w = q[6] | (static_cast<uint32_t>(q[7]) << 16);
  return o;
}

template <int NP>
__global__ void __launch_bounds__(256) split_vec8_kernel(const float* __restrict__ x, int64_t ldx,
                                                         int64_t rows, int64_t cols8,
                                                         uint16_t* __restrict__ p0,
                                                         uint16_t* __restrict__ p1,
                                                         uint16_t* __restrict__ p2, int64_t ldp) {
  const int64_t total = rows * cols8;
  for (int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; v < total;
       v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = v / cols8;
    const int64_t c = (v - r * cols8) * 8;
    const float4* src = reinterpret_cast<const float4*>(x + r * ldx + c);
    const float4 a = __ldcs(src);
    const float4 b = __ldcs(src + 1);
    const float e[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint16_t h[8], m[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) split_elem(e[i], h[i], m[i], l[i]);
    const int64_t off = r * ldp + c;
    __stcs(reinterpret_cast<uint4*>(p0 + off), pack8(h));
    if (NP >= 2) __stcs(reinterpret_cast<uint4*>(p1 + off), pack8(m));
    if (NP >= 3) __stcs(reinterpret_cast<uint4*>(p2 + off), pack8(l));
  }
}

__global__ void __launch_bounds__(256) split_scalar_kernel(const float* __restrict__ x, int64_t ldx,
                                                           int64_t rows, int64_t cols, int np,
                                                           uint16_t* __restrict__ p0,
                                                           uint16_t* __restrict__ p1,
                                                           uint16_t* __restrict__ p2,
                                                           int64_t ldp) {
  const int64_t total = rows * cols;
  for (int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; v < total;
       v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = v / cols;
    const int64_t c = v - r * cols;
    uint16_t h, m, l;
    split_elem(x[r * ldx + c], h, m, l);
    const int64_t off = r * ldp + c;
    p0[off] = h;
    if (np >= 2) p1[off] = m;
    if (np >= 3) p2[off] = l;
  }
}

// 64 x 64 tile, 256 threads (32 x 8).  Reads rows of x coalesced, writes rows
// of the transposed pieces coalesced as pairs of bfloat16 (4 bytes a lane).
constexpr int TT = 64;
__global__ void __launch_bounds__(256) split_transpose_kernel(const float* __restrict__ x,
                                                              int64_t ldx, int64_t rows,
                                                              int64_t cols, int np,
                                                              uint16_t* __restrict__ p0,
                                                              uint16_t* __restrict__ p1,
                                                              uint16_t* __restrict__ p2,
                                                              int64_t ldp, bool pairs) {
  __shared__ float tile[TT][TT + 1];
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * TT;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * TT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < TT; i += 8) {
    const int64_t r = r0 + ty + i;
#pragma unroll
    for (int j = 0; j < TT; j += 32) {
      const int64_t c = c0 + tx + j;
      tile[ty + i][tx + j] = (r < rows && c < cols) ? x[r * ldx + c] : 0.0f;
    }
  }
  __syncthreads();
  // output row oc = c0 + (ty + i), output columns orr = r0 + 2*tx + {0,1}
#pragma unroll
  for (int i = 0; i < TT; i += 8) {
    const int64_t oc = c0 + ty + i;
    if (oc >= cols) continue;
    const int64_t orr = r0 + 2 * tx;
    uint16_t h0, m0, l0, h1, m1, l1;
    split_elem(tile[2 * tx][ty + i], h0, m0, l0);
    split_elem(tile[2 * tx + 1][ty + i], h1, m1, l1);
    const int64_t off = oc * ldp + orr;
    if (pairs && orr + 1 < rows && ((off & 1) == 0)) {
      *reinterpret_cast<uint32_t*>(p0 + off) = h0 | (static_cast<uint32_t>(h1) << 16);
      if (np >= 2) *reinterpret_cast<uint32_t*>(p1 + off) = m0 | (static_cast<uint32_t>(m1) << 16);
      if (np >= 3) *reinterpret_cast<uint32_t*>(p2 + off) = l0 | (static_cast<uint32_t>(l1) << 16);
    } else {
      if (orr < rows) {
        p0[off] = h0;
        if (np >= 2) p1[off] = m0;
        if (np >= 3) p2[off] = l0;
      }
      if (orr + 1 < rows) {
        p0[off + 1] = h1;
        if (np >= 2) p1[off + 1] = m1;
        if (np >= 3) p2[off + 1] = l1;
      }
    }
  }
}

__global__ void scale_kernel(int64_t m, int64_t n, float beta, float* __restrict__ C, int64_t ldc) {
  const int64_t total = m * n;
  for (int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; v < total;
       v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = v / n, c = v - r * n;
    C[r * ldc + c] = (beta == 0.0f) ? 0.0f : beta * C[r * ldc + c];
  }
}

int grid_for(int64_t work, int threads) {
  const int sms = current_num_sms() > 0 ? current_num_sms() : 148;
  const int64_t want = ceil_div(work, threads);
  const int64_t cap = static_cast<int64_t>(sms) * 8;  // one full wave of 256-thread blocks
  return static_cast<int>(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

bfx_status launch_split(int64_t rows, int64_t cols, const float* x, int64_t ldx, int npieces,
                        uint16_t* hi, uint16_t* mid, uint16_t* lo, int64_t ldp, cudaStream_t s) {
  if (rows == 0 || cols == 0) return BFX_OK;
  const bool vec = (cols % 8 == 0) && (ldx % 4 == 0) && (ldp % 8 == 0) && aligned(x, 16) &&
                   aligned(hi, 16) && (npieces < 2 || aligned(mid, 16)) &&
                   (npieces < 3 || aligned(lo, 16));
  if (vec) {
    const int64_t cols8 = cols / 8;
    const int grid = grid_for(rows * cols8, 256);
    switch (npieces) {
      case 1: split_vec8_kernel<1><<<grid, 256, 0, s>>>(x, ldx, rows, cols8, hi, mid, lo, ldp); break;
      case 2: split_vec8_kernel<2><<<grid, 256, 0, s>>>(x, ldx, rows, cols8, hi, mid, lo, ldp); break;
      default: split_vec8_kernel<3><<<grid, 256, 0, s>>>(x, ldx, rows, cols8, hi, mid, lo, ldp); break;
    }
  } else {
    const int grid = grid_for(rows * cols, 256);
    split_scalar_kernel<<<grid, 256, 0, s>>>(x, ldx, rows, cols, npieces, hi, mid, lo, ldp);
  }
  return last_launch_status();
}

bfx_status launch_split_transpose(int64_t rows, int64_t cols, const float* x, int64_t ldx,
                                  int npieces, uint16_t* hi, uint16_t* mid, uint16_t* lo,
                                  int64_t ldp, cudaStream_t s) {
  if (rows == 0 || cols == 0) return BFX_OK;
  const int64_t gx = ceil_div(cols, TT), gy = ceil_div(rows, TT);
  if (gy > 65535 || gx > INT32_MAX) return BFX_EUNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  const bool pairs = aligned(hi, 4) && (npieces < 2 || aligned(mid, 4)) &&
                     (npieces < 3 || aligned(lo, 4));
  split_transpose_kernel<<<grid, 256, 0, s>>>(x, ldx, rows, cols, npieces, hi, mid, lo, ldp,
                                              pairs);
  return last_launch_status();
}

bfx_status launch_scale(int64_t m, int64_t n, float beta, float* C, int64_t ldc, cudaStream_t s) {
  if (m == 0 || n == 0) return BFX_OK;
  scale_kernel<<<grid_for(m * n, 256), 256, 0, s>>>(m, n, beta, C, ldc);
  return last_launch_status();
}

}  // namespace bfx
