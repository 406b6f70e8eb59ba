// Internal helpers of the bfx library: argument checks, the device error
// word, and thin inline-PTX wrappers for the sm_100-family async machinery
// (mbarrier, TMA bulk tensor copies, tcgen05 tensor-core MMA / tensor memory).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bfx.h"

namespace bfx {

// ---------------------------------------------------------------- host side
// Device error word (one int per device).  Codes:
enum DeviceError : int {
  kErrNone = 0,
  kErrWaitFull = 1,      // MMA issuer waited too long for a TMA stage
  kErrWaitEmpty = 2,     // TMA producer waited too long for a free stage
  kErrWaitAccFull = 3,   // epilogue waited too long for an accumulator
  kErrWaitAccEmpty = 4,  // MMA issuer waited too long for the epilogue
  kErrWaitDrain = 5,     // final drain of in-flight MMAs expired
  kErrWaitBlock = 6,     // triangular solve waited too long for an earlier row block
  kErrWaitPanel = 7,     // cluster panel waited too long for a pivot exchange
};

int* device_error_word();  // nullptr on failure
int current_num_sms();
int current_cc();          // major*10 + minor, or -1
bool is_sm103();

inline bfx_status cuda_status(cudaError_t e) { return e == cudaSuccess ? BFX_OK : BFX_ECUDA; }
inline bfx_status last_launch_status() { return cuda_status(cudaGetLastError()); }

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }
inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int mode_pieces(bfx_mode mode);  // 0 for invalid / FP32
bool gemm_pieces(bfx_mode mode, int* npa, int* npb);  // GEMM pieces of A, B (x5: 2, 3)

// split launchers (split.cu)
bfx_status launch_split(int64_t rows, int64_t cols, const float* x, int64_t ldx, int npieces,
                        uint16_t* hi, uint16_t* mid, uint16_t* lo, int64_t ldp, cudaStream_t s);
bfx_status launch_split_transpose(int64_t rows, int64_t cols, const float* x, int64_t ldx,
                                  int npieces, uint16_t* hi, uint16_t* mid, uint16_t* lo,
                                  int64_t ldp, cudaStream_t s);
bfx_status launch_split_pair(int64_t rows_a, int64_t cols_a, const float* a, int64_t lda, int npa,
                             uint16_t* a0, uint16_t* a1, uint16_t* a2, int64_t ldpa,
                             int64_t rows_b, int64_t cols_b, const float* b, int64_t ldb, int npb,
                             uint16_t* b0, uint16_t* b1, uint16_t* b2, int64_t ldpb, cudaStream_t s);
// C = beta*C (k == 0 GEMM)
bfx_status launch_scale(int64_t m, int64_t n, float beta, float* C, int64_t ldc, cudaStream_t s);
// SIMT SGEMM (gemm_simt.cu)
bfx_status launch_sgemm_simt(int64_t m, int64_t n, int64_t k, float alpha, const float* A,
                             int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                             int64_t ldc, cudaStream_t s);
// Grouped tensor-core GEMM (many independent problems in one launch): the
// pieces of problem p are planes plane0 .. plane0+np-1 of two packed buffers
// (rows x kp bfloat16 each); tiles list the output tiles of all problems.
struct GroupTile {
  int prob, mb, nb, pad;
};
struct GroupProblem {
  float* C;
  int64_t ldc;
  int M, N, k_tiles, plane0, vec_c, pad;
};
int gemm_bk(bfx_mode mode);  // K-slice width of the mode's kernel
// Fused split + product: FP32 A (m x k, lda) and B (k x n, ldb) read by TMA
// and split in the kernel (lda, ldb multiples of 4, A, B 16-byte aligned).
bfx_status launch_gemm_fused(bfx_mode mode, int64_t m, int64_t n, int64_t k, float alpha,
                             const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                             float* C, int64_t ldc, cudaStream_t s);
bfx_status launch_gemm_grouped(bfx_mode mode, int bn, int num_tiles, const GroupTile* d_tiles,
                               const GroupProblem* d_probs, const uint16_t* Apack,
                               int64_t a_rows, const uint16_t* Bpack, int64_t b_rows,
                               int64_t planes, int64_t kp, float alpha, float beta,
                               cudaStream_t s);
// Batched LU (lu.cu): one descriptor per system, systems sorted by n descending.
struct BatchLu {
  float* A;  // n x n, leading dimension n, factored in place
  int n, pad;
  int32_t* ipiv;
  int32_t* info;
};
// One block column [J0, J0+nb) of the LU of every system with n > J0 (the
// first S_active descriptors): tiles, row swaps, block solve, and the pieces
// of L21 / U12^T written to the packs for a grouped trailing update (np
// planes of slot_rows x kp per system); the grouped GEMM itself is launched
// by the caller.  h_n_desc: the systems' n, descending, on the host.
bfx_status lu_batched_block(bfx_mode mode, const BatchLu* d_sys, const int* h_n_desc, int S,
                            int nb, int J0, uint16_t* packA, uint16_t* packB, int64_t slot_rows,
                            int64_t kp, cudaStream_t s);
// One batched solve launched directly (no graph) on s; the plan is left
// unbound, so bfx_batch_solve captures afresh afterwards (batched.cu).
bfx_status batch_solve_direct(bfx_batch_plan* P, const float* d_A, const double* d_b, double* d_x,
                              bfx_batch_status* d_status, void* d_ws, size_t ws_bytes,
                              cudaStream_t s);
// Batched refinement (ir.cu): one descriptor per system (same order as the
// BatchLu array).  All buffers are n x nrhs (FP64) or n x n (FP32), leading
// dimension n (resp. nrhs).
struct BatchIrState {
  int active, conv, stalled, iters;
  double dprev, anorm, bnorm, berr;
};
struct BatchIr {
  const float* A;   // the problem matrix (FP32)
  const float* LU;  // its factors
  const int32_t* ipiv;
  const int32_t* info;
  int32_t* perm;
  const double* b;
  double* x;
  double* r;
  double* d;
  double* Linv;  // inverses of the 64 x 64 diagonal blocks of L, then U
  double* Uinv;
  BatchIrState* st;
  bfx_batch_status* out;  // the caller's status slot of this system
  int n, nrhs;
};
struct BatchIrParams {
  double tol, tol_b, stall;
};
// The refinement of a batch, all on the device (launch sequence; no host
// decisions): prepare (norms, state), factors' permutation and inverse
// diagonal blocks, x0 = LU^-1 b, max_iter refinement steps (residual, solve,
// update with per-system stop decisions), final backward errors.
bfx_status ir_batched_prepare(const BatchIr* d_ir, int S, int nmax, cudaStream_t s);
bfx_status ir_batched_post_lu(const BatchIr* d_ir, int S, int nmax, cudaStream_t s);
bfx_status ir_batched_first_solve(const BatchIr* d_ir, int S, cudaStream_t s);
bfx_status ir_batched_step(const BatchIr* d_ir, int S, BatchIrParams p, cudaStream_t s);
bfx_status ir_batched_finish(const BatchIr* d_ir, int S, BatchIrParams p, cudaStream_t s);
// GMRES-IR for the systems still unconverged after ir_batched_finish
// (persistent grid of nslots CTAs, one Krylov slot of slot_doubles each).
bfx_status ir_batched_gmres(const BatchIr* d_ir, int S, int* d_queue, double* d_slots,
                            int64_t slot_doubles, int nslots, int m, BatchIrParams p,
                            int max_outer, double tau, cudaStream_t s);
int64_t batched_gmres_slot_doubles(int m, int nmax, int R);
// tcgen05 GEMM on pieces (gemm_tc.cu)
// pdl: launch as a programmatic dependent of the previous kernel on s
bfx_status launch_gemm_presplit(bfx_mode mode, int64_t m, int64_t n, int64_t k, float alpha,
                                const uint16_t* Ap, int64_t lda_p, int64_t a_plane,
                                const uint16_t* Btp, int64_t ldb_p, int64_t b_plane, float beta,
                                float* C, int64_t ldc, cudaStream_t s, bool pdl = false);
// FP64 collection of the mode's partial products (Sec. IV-A "d"); same piece
// layout as launch_gemm_presplit, C is FP64.
bfx_status launch_gemm_f64(bfx_mode mode, int64_t m, int64_t n, int64_t k, const uint16_t* Ap,
                           int64_t lda_p, int64_t a_plane, const uint16_t* Btp, int64_t ldb_p,
                           int64_t b_plane, double* C, int64_t ldc, cudaStream_t s);
// Single-type LU + FP64 refinement, one warp per system (lowp.cu).
bfx_status launch_lowp_lu_ir(bfx_lowp type, int count, int n, const float* A, const double* b,
                             const double* tol, int max_iter, double* x, float* LU_out,
                             int32_t* ipiv_out, int32_t* iters, int32_t* conv, int32_t* info,
                             cudaStream_t s);
int lowp_max_n();

// ---------------------------------------------------------------- device side
#if defined(__CUDACC__)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// FP32 -> FP64, exact, on the integer pipe for zeros and normal values (the
// exponent rebiased by 1023 - 127 = 896, the significand shifted into place);
// subnormals, Inf and NaN take the hardware conversion.  On B300 the
// hardware conversion shares the FP64 pipe, whose throughput bounds the
// FP64 refinement kernels that widen every FP32 matrix element they read.
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu, mant = u & 0x7FFFFFu;
  const uint64_t sign = static_cast<uint64_t>(u & 0x80000000u) << 32;
  if ((e == 0u && mant != 0u) || e == 0xFFu) return static_cast<double>(f);
  const uint64_t d = e == 0u ? sign
                             : (sign | (static_cast<uint64_t>(e + 896u) << 52) |
                                (static_cast<uint64_t>(mant) << 29));
  return __longlong_as_double(static_cast<long long>(d));
}
__device__ __forceinline__ double widen(double d) { return d; }

// ---- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity to complete; give up after
// `limit_ns` of wall time (set *err = code, return false) instead of hanging.
// backoff: sleep briefly between polls (for waiters that are not on the
// critical path, so their polling leaves the issue slots to the others).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err,
                                                  int code, uint64_t limit_ns = 4000000000ull,
                                                  bool backoff = false) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (backoff) __nanosleep(128);
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) {
      if (err) atomicCAS(err, 0, code);
      return false;
    }
  }
}

// ---- TMA (bulk tensor copies global -> shared, completion on an mbarrier)
__device__ __forceinline__ void tma_prefetch_desc(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, uint64_t* bar, int c0,
                                            int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_addr(dst)),
      "l"(tmap), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, uint64_t* bar, int c0,
                                            int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_addr(dst)),
      "l"(tmap), "r"(smem_addr(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// ---- tcgen05: tensor memory and MMA
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D(tmem) (+)= A(smem desc) * B(smem desc), bf16 inputs, f32 accumulate.
__device__ __forceinline__ void umma_bf16_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                             uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive once on an mbarrier when all previously issued tcgen05 ops of this
// thread have completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns; the wait is fused so the
// registers are only consumed after tcgen05.wait::ld.
__device__ __forceinline__ void tmem_ld16_wait(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])::"memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 16 consecutive 32-bit columns stored to tensor memory; waits
// until the stores have completed.
__device__ __forceinline__ void tmem_st16_wait(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Split of one FP32 value into its bfloat16 pieces (Sec. II-A):
// hi = (B16)a, mid = (B16)(a - hi), lo = (B16)(a - hi - mid), (B16) = RNE.
// Readings for values the paper does not cover: Inf/NaN go to hi (NaN made
// quiet, sign kept), mid = lo = +0; a finite value whose RNE would overflow
// to infinity takes hi = a truncated toward zero.
__device__ __forceinline__ uint16_t bf16_bits_rn(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_value(uint16_t h) {
  return __uint_as_float(static_cast<uint32_t>(h) << 16);
}
__device__ __forceinline__ void split_elem(float a, uint16_t& h, uint16_t& m, uint16_t& l) {
  const uint32_t u = __float_as_uint(a);
  const uint32_t mag = u & 0x7FFFFFFFu;
  if (mag >= 0x7F800000u) {
    h = static_cast<uint16_t>((u >> 16) | (mag > 0x7F800000u ? 0x0040u : 0u));
    m = 0;
    l = 0;
    return;
  }
  h = (mag >= 0x7F7F8000u) ? static_cast<uint16_t>(u >> 16) : bf16_bits_rn(a);
  const float r1 = __fsub_rn(a, bf16_value(h));
  m = bf16_bits_rn(r1);
  const float r2 = __fsub_rn(r1, bf16_value(m));
  l = bf16_bits_rn(r2);
}

// Shared-memory matrix descriptor for a K-major tile written by TMA with a
// 128-byte (layout 2) or 64-byte (layout 4) swizzle: rows of SW bytes, 8-row
// core groups SBO = 8*SW bytes apart; LBO unused for swizzled K-major tiles.
template <int SW>
__device__ __forceinline__ uint64_t smem_desc_kmajor(uint32_t saddr) {
  static_assert(SW == 128 || SW == 64, "swizzle");
  constexpr uint64_t layout = (SW == 128) ? 2ull : 4ull;
  constexpr uint64_t sbo = (8ull * SW) >> 4;
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= 1ull << 16;          // LBO (ignored for swizzled K-major)
  d |= sbo << 32;           // SBO
  d |= 1ull << 46;          // descriptor version for the sm_100 family
  d |= layout << 61;        // swizzle mode
  return d;
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major.
template <int M, int N>
__host__ __device__ constexpr uint32_t idesc_bf16_f32() {
  return (1u << 4)                           // D format: f32
         | (1u << 7)                         // A format: bf16
         | (1u << 10)                        // B format: bf16
         | (static_cast<uint32_t>(N >> 3) << 17)
         | (static_cast<uint32_t>(M >> 4) << 24);
}

#endif  // __CUDACC__

}  // namespace bfx
