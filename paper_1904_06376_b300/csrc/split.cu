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
__device__ __forceinline__ void split8_store(const float4 a, const float4 b, uint16_t* p0,
                                             uint16_t* p1, uint16_t* p2, int64_t off) {
  const float e[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  uint16_t h[8], m[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) split_elem(e[i], h[i], m[i], l[i]);
  __stcs(reinterpret_cast<uint4*>(p0 + off), pack8(h));
  if (NP >= 2) __stcs(reinterpret_cast<uint4*>(p1 + off), pack8(m));
  if (NP >= 3) __stcs(reinterpret_cast<uint4*>(p2 + off), pack8(l));
}

// Contiguous rows (ldx == ldp == cols): one flat range, no index division;
// two groups of 8 elements a thread and iteration, all four 16-byte loads
// issued before the splits.  Block bid of nblocks.
template <int NP>
__device__ __forceinline__ void split_flat_body(const float* __restrict__ x, int64_t n8,
                                                uint16_t* __restrict__ p0, uint16_t* __restrict__ p1,
                                                uint16_t* __restrict__ p2, int bid, int nblocks) {
  const int64_t stride = static_cast<int64_t>(nblocks) * blockDim.x;
  const float4* src = reinterpret_cast<const float4*>(x);
  int64_t v = bid * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  for (; v + stride < n8; v += 2 * stride) {
    const float4 a0 = __ldcs(src + 2 * v), b0 = __ldcs(src + 2 * v + 1);
    const float4 a1 = __ldcs(src + 2 * (v + stride)), b1 = __ldcs(src + 2 * (v + stride) + 1);
    split8_store<NP>(a0, b0, p0, p1, p2, 8 * v);
    split8_store<NP>(a1, b1, p0, p1, p2, 8 * (v + stride));
  }
  if (v < n8) split8_store<NP>(__ldcs(src + 2 * v), __ldcs(src + 2 * v + 1), p0, p1, p2, 8 * v);
}
template <int NP>
__global__ void __launch_bounds__(256) split_flat_kernel(const float* __restrict__ x, int64_t n8,
                                                         uint16_t* __restrict__ p0,
                                                         uint16_t* __restrict__ p1,
                                                         uint16_t* __restrict__ p2) {
  split_flat_body<NP>(x, n8, p0, p1, p2, static_cast<int>(blockIdx.x), static_cast<int>(gridDim.x));
}

template <int NP>
__global__ void __launch_bounds__(256) split_vec8_kernel(const float* __restrict__ x, int64_t ldx,
                                                         int64_t rows, int64_t cols8,
                                                         uint16_t* __restrict__ p0,
                                                         uint16_t* __restrict__ p1,
                                                         uint16_t* __restrict__ p2, int64_t ldp) {
  // launched as a programmatic dependent (the LU's L21 pieces after the
  // panel): wait for the previous kernel; a no-op otherwise
  asm volatile("griddepcontrol.wait;" ::: "memory");
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
// Tile (bx, by) of the transposed split; tile: the caller's shared memory.
__device__ __forceinline__ void split_transpose_tile(float (*tile)[TT + 1], const float* __restrict__ x,
                                                     int64_t ldx, int64_t rows, int64_t cols, int np,
                                                     uint16_t* __restrict__ p0,
                                                     uint16_t* __restrict__ p1,
                                                     uint16_t* __restrict__ p2, int64_t ldp,
                                                     int pairs, int64_t bx, int64_t by) {
  const int64_t r0 = by * TT;
  const int64_t c0 = bx * TT;
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
  if (pairs == 2) {
    // 16-byte stores: thread t writes output row oc = c0 + t/8 (+32), output
    // columns r0 + 8*(t%8) .. +7, when that run is inside the matrix
    const int seg = (threadIdx.x & 7) * 8;
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
      const int ol = (threadIdx.x >> 3) + 32 * pass;
      const int64_t oc = c0 + ol;
      if (oc >= cols) continue;
      const int64_t orr = r0 + seg;
      uint16_t h[8], m[8], l[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) split_elem(tile[seg + q][ol], h[q], m[q], l[q]);
      const int64_t off = oc * ldp + orr;
      if (orr + 8 <= rows) {
        *reinterpret_cast<uint4*>(p0 + off) = pack8(h);
        if (np >= 2) *reinterpret_cast<uint4*>(p1 + off) = pack8(m);
        if (np >= 3) *reinterpret_cast<uint4*>(p2 + off) = pack8(l);
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (orr + q >= rows) break;
          p0[off + q] = h[q];
          if (np >= 2) p1[off + q] = m[q];
          if (np >= 3) p2[off + q] = l[q];
        }
      }
    }
    return;
  }
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
    if (pairs == 1 && orr + 1 < rows && ((off & 1) == 0)) {
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

__global__ void __launch_bounds__(256) split_transpose_kernel(const float* __restrict__ x,
                                                              int64_t ldx, int64_t rows,
                                                              int64_t cols, int np,
                                                              uint16_t* __restrict__ p0,
                                                              uint16_t* __restrict__ p1,
                                                              uint16_t* __restrict__ p2,
                                                              int64_t ldp, int pairs) {
  __shared__ float tile[TT][TT + 1];
  split_transpose_tile(tile, x, ldx, rows, cols, np, p0, p1, p2, ldp, pairs, blockIdx.x, blockIdx.y);
}

// Both operands of C = A B in one launch: CTAs [0, ga) split A as
// split_flat_kernel (contiguous rows), the others take B's transposed tiles
// (16-byte piece stores), so the two passes fill each other's tails instead
// of running one after the other.  Same bytes and results as the two
// kernels.
__global__ void __launch_bounds__(256)
    split_pair_kernel(const float* __restrict__ a, int64_t n8, int npa, uint16_t* __restrict__ a0,
                      uint16_t* __restrict__ a1, uint16_t* __restrict__ a2, int ga,
                      const float* __restrict__ b, int64_t ldb, int64_t rows, int64_t cols, int npb,
                      uint16_t* __restrict__ b0, uint16_t* __restrict__ b1,
                      uint16_t* __restrict__ b2, int64_t ldp, int64_t tiles_x) {
  __shared__ float tile[TT][TT + 1];
  const int bid = static_cast<int>(blockIdx.x);
  if (bid < ga) {
    if (npa == 1)
      split_flat_body<1>(a, n8, a0, a1, a2, bid, ga);
    else if (npa == 2)
      split_flat_body<2>(a, n8, a0, a1, a2, bid, ga);
    else
      split_flat_body<3>(a, n8, a0, a1, a2, bid, ga);
    return;
  }
  const int64_t t = bid - ga;
  split_transpose_tile(tile, b, ldb, rows, cols, npb, b0, b1, b2, ldp, 2, t % tiles_x, t / tiles_x);
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
  if (vec && ldx == cols && ldp == cols) {
    const int64_t n8 = rows * cols / 8;
    const int grid = grid_for(n8, 256);
    switch (npieces) {
      case 1: split_flat_kernel<1><<<grid, 256, 0, s>>>(x, n8, hi, mid, lo); break;
      case 2: split_flat_kernel<2><<<grid, 256, 0, s>>>(x, n8, hi, mid, lo); break;
      default: split_flat_kernel<3><<<grid, 256, 0, s>>>(x, n8, hi, mid, lo); break;
    }
  } else if (vec) {
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

// launch_split as a programmatic dependent of the previous kernel on s when
// the 8-wide form applies (the LU's L21 pieces), else launch_split
bfx_status launch_split_pdl(int64_t rows, int64_t cols, const float* x, int64_t ldx, int npieces,
                            uint16_t* hi, uint16_t* mid, uint16_t* lo, int64_t ldp, cudaStream_t s) {
  if (rows == 0 || cols == 0) return BFX_OK;
  const bool vec = (cols % 8 == 0) && (ldx % 4 == 0) && (ldp % 8 == 0) && aligned(x, 16) &&
                   aligned(hi, 16) && (npieces < 2 || aligned(mid, 16)) &&
                   (npieces < 3 || aligned(lo, 16)) && !(ldx == cols && ldp == cols);
  if (!vec) return launch_split(rows, cols, x, ldx, npieces, hi, mid, lo, ldp, s);
  const int64_t cols8 = cols / 8;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid_for(rows * cols8, 256)));
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  auto kern = npieces == 1 ? split_vec8_kernel<1> : (npieces == 2 ? split_vec8_kernel<2> : split_vec8_kernel<3>);
  return cudaLaunchKernelEx(&cfg, kern, x, ldx, rows, cols8, hi, mid, lo, ldp) == cudaSuccess ? BFX_OK
                                                                                              : BFX_ECUDA;
}


bfx_status launch_split_transpose(int64_t rows, int64_t cols, const float* x, int64_t ldx,
                                  int npieces, uint16_t* hi, uint16_t* mid, uint16_t* lo,
                                  int64_t ldp, cudaStream_t s) {
  if (rows == 0 || cols == 0) return BFX_OK;
  const int64_t gx = ceil_div(cols, TT), gy = ceil_div(rows, TT);
  if (gy > 65535 || gx > INT32_MAX) return BFX_EUNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  // 2: 16-byte stores (planes 16-byte aligned, ldp a multiple of 8);
  // 1: 4-byte pairs; 0: single elements
  const bool al16 = aligned(hi, 16) && (npieces < 2 || aligned(mid, 16)) &&
                    (npieces < 3 || aligned(lo, 16)) && ldp % 8 == 0;
  const bool al4 = aligned(hi, 4) && (npieces < 2 || aligned(mid, 4)) &&
                   (npieces < 3 || aligned(lo, 4));
  const int pairs = al16 ? 2 : (al4 ? 1 : 0);
  split_transpose_kernel<<<grid, 256, 0, s>>>(x, ldx, rows, cols, npieces, hi, mid, lo, ldp,
                                              pairs);
  return last_launch_status();
}

// A (rows_a x cols_a, split as is) and B (rows_b x cols_b, split transposed)
// in one launch when A's rows are contiguous (lda == ldpa == cols_a, 16-byte
// aligned) and B's piece planes take 16-byte stores; otherwise the two
// launches of launch_split and launch_split_transpose.
bfx_status launch_split_pair(int64_t rows_a, int64_t cols_a, const float* a, int64_t lda, int npa,
                             uint16_t* a0, uint16_t* a1, uint16_t* a2, int64_t ldpa,
                             int64_t rows_b, int64_t cols_b, const float* b, int64_t ldb, int npb,
                             uint16_t* b0, uint16_t* b1, uint16_t* b2, int64_t ldpb, cudaStream_t s) {
  const bool flat = rows_a > 0 && cols_a > 0 && cols_a % 8 == 0 && lda == cols_a && ldpa == cols_a &&
                    aligned(a, 16) && aligned(a0, 16) && (npa < 2 || aligned(a1, 16)) &&
                    (npa < 3 || aligned(a2, 16));
  const bool t16 = rows_b > 0 && cols_b > 0 && aligned(b0, 16) && (npb < 2 || aligned(b1, 16)) &&
                   (npb < 3 || aligned(b2, 16)) && ldpb % 8 == 0;
  const int64_t tx = ceil_div(cols_b, TT), ty = ceil_div(rows_b, TT);
  const int64_t n8 = rows_a * cols_a / 8;
  const int ga = grid_for(n8, 256);
  if (!flat || !t16 || static_cast<int64_t>(ga) + tx * ty > INT32_MAX) {
    const bfx_status st = launch_split(rows_a, cols_a, a, lda, npa, a0, a1, a2, ldpa, s);
    if (st != BFX_OK) return st;
    return launch_split_transpose(rows_b, cols_b, b, ldb, npb, b0, b1, b2, ldpb, s);
  }
  split_pair_kernel<<<static_cast<unsigned>(ga + tx * ty), 256, 0, s>>>(
      a, n8, npa, a0, a1, a2, ga, b, ldb, rows_b, cols_b, npb, b0, b1, b2, ldpb, tx);
  return last_launch_status();
}

bfx_status launch_scale(int64_t m, int64_t n, float beta, float* C, int64_t ldc, cudaStream_t s) {
  if (m == 0 || n == 0) return BFX_OK;
  scale_kernel<<<grid_for(m * n, 256), 256, 0, s>>>(m, n, beta, C, ldc);
  return last_launch_status();
}

}  // namespace bfx
