// C-ABI entry points of the bfx library: argument validation, the device
// error word, workspace carving, and dispatch to the kernels of split.cu,
// gemm_simt.cu and gemm_tc.cu.
#include <cstring>

#include "bfx_internal.cuh"

namespace bfx {
namespace {

// One int per device; kernels with bounded waits record expiries here.
__device__ int g_device_error = 0;

constexpr int kMaxDevices = 64;
int* g_error_ptr[kMaxDevices] = {nullptr};
int g_num_sms[kMaxDevices] = {0};
int g_cc[kMaxDevices] = {0};

int current_device() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
  return d;
}

bool check_mode(bfx_mode mode) {
  return mode == BFX_FP32 || mode == BFX_X1 || mode == BFX_X3 || mode == BFX_X5 ||
         mode == BFX_X6 || mode == BFX_X8 || mode == BFX_X9;
}

}  // namespace

int* device_error_word() {
  const int d = current_device();
  if (d < 0) return nullptr;
  if (!g_error_ptr[d]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
    g_error_ptr[d] = static_cast<int*>(p);
  }
  return g_error_ptr[d];
}

int current_num_sms() {
  const int d = current_device();
  if (d < 0) return -1;
  if (g_num_sms[d] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess) return -1;
    g_num_sms[d] = v;
  }
  return g_num_sms[d];
}

int current_cc() {
  const int d = current_device();
  if (d < 0) return -1;
  if (g_cc[d] == 0) {
    int ma = 0, mi = 0;
    if (cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, d) != cudaSuccess ||
        cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, d) != cudaSuccess)
      return -1;
    g_cc[d] = ma * 10 + mi;
  }
  return g_cc[d];
}

bool is_sm103() { return current_cc() == 103; }

int mode_pieces(bfx_mode mode) {
  switch (mode) {
    case BFX_X1: return 1;
    case BFX_X3: return 2;
    case BFX_X6: return 3;
    case BFX_X8: return 3;
    case BFX_X9: return 3;
    default: return 0;
  }
}

// Pieces of A and of B a GEMM mode reads (x5: two and three); false if the
// mode has no tensor-core GEMM.
bool gemm_pieces(bfx_mode mode, int* npa, int* npb) {
  if (mode == BFX_X5) {
    *npa = 2;
    *npb = 3;
    return true;
  }
  *npa = *npb = mode_pieces(mode);
  return *npa > 0;
}

}  // namespace bfx

using namespace bfx;

extern "C" {

BFX_API int bfx_version(void) { return 100; }

BFX_API const char* bfx_status_string(bfx_status s) {
  switch (s) {
    case BFX_OK: return "ok";
    case BFX_EINVAL: return "invalid argument";
    case BFX_ENOMEM: return "workspace too small";
    case BFX_ECUDA: return "CUDA error";
    case BFX_EUNSUPPORTED: return "unsupported shape, alignment or device";
    case BFX_SINGULAR: return "exactly zero pivot";
    case BFX_NOT_CONVERGED: return "iterative refinement did not converge";
    case BFX_TIMEOUT: return "a bounded device-side wait expired";
    default: return "unknown status";
  }
}

BFX_API int bfx_num_sms(void) { return current_num_sms(); }

BFX_API bfx_status bfx_device_error(int* h_code, bfx_stream stream) {
  if (!h_code) return BFX_EINVAL;
  int* p = device_error_word();
  if (!p) return BFX_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(h_code, p, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return BFX_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return BFX_ECUDA;
  if (*h_code != 0) {
    if (cudaMemsetAsync(p, 0, sizeof(int), s) != cudaSuccess) return BFX_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BFX_ECUDA;
  }
  return BFX_OK;
}

static bfx_status check_split_args(int64_t rows, int64_t cols, const float* x, int64_t ldx,
                                   int npieces, const uint16_t* hi, const uint16_t* mid,
                                   const uint16_t* lo, int64_t ldp, int64_t min_ldp) {
  if (rows < 0 || cols < 0 || npieces < 1 || npieces > 3) return BFX_EINVAL;
  if (rows == 0 || cols == 0) return BFX_OK;
  if (ldx < cols || ldp < min_ldp) return BFX_EINVAL;
  if (!x || !hi || (npieces >= 2 && !mid) || (npieces >= 3 && !lo)) return BFX_EINVAL;
  return BFX_OK;
}

BFX_API bfx_status bfx_split(int64_t rows, int64_t cols, const float* d_x, int64_t ldx,
                             int npieces, uint16_t* d_hi, uint16_t* d_mid, uint16_t* d_lo,
                             int64_t ldp, bfx_stream stream) {
  bfx_status st = check_split_args(rows, cols, d_x, ldx, npieces, d_hi, d_mid, d_lo, ldp, cols);
  if (st != BFX_OK || rows == 0 || cols == 0) return st;
  return launch_split(rows, cols, d_x, ldx, npieces, d_hi, d_mid, d_lo, ldp,
                      static_cast<cudaStream_t>(stream));
}

BFX_API bfx_status bfx_split_transpose(int64_t rows, int64_t cols, const float* d_x, int64_t ldx,
                                       int npieces, uint16_t* d_hi, uint16_t* d_mid,
                                       uint16_t* d_lo, int64_t ldp, bfx_stream stream) {
  bfx_status st = check_split_args(rows, cols, d_x, ldx, npieces, d_hi, d_mid, d_lo, ldp, rows);
  if (st != BFX_OK || rows == 0 || cols == 0) return st;
  return launch_split_transpose(rows, cols, d_x, ldx, npieces, d_hi, d_mid, d_lo, ldp,
                                static_cast<cudaStream_t>(stream));
}

BFX_API bfx_status bfx_split_pair(int64_t rows_a, int64_t cols_a, const float* d_a, int64_t lda,
                                  int npa, uint16_t* d_a0, uint16_t* d_a1, uint16_t* d_a2,
                                  int64_t ldpa, int64_t rows_b, int64_t cols_b, const float* d_b,
                                  int64_t ldb, int npb, uint16_t* d_b0, uint16_t* d_b1,
                                  uint16_t* d_b2, int64_t ldpb, bfx_stream stream) {
  bfx_status st = check_split_args(rows_a, cols_a, d_a, lda, npa, d_a0, d_a1, d_a2, ldpa, cols_a);
  if (st != BFX_OK) return st;
  st = check_split_args(rows_b, cols_b, d_b, ldb, npb, d_b0, d_b1, d_b2, ldpb, rows_b);
  if (st != BFX_OK) return st;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (rows_a == 0 || cols_a == 0)
    return (rows_b == 0 || cols_b == 0)
               ? BFX_OK
               : launch_split_transpose(rows_b, cols_b, d_b, ldb, npb, d_b0, d_b1, d_b2, ldpb, s);
  if (rows_b == 0 || cols_b == 0)
    return launch_split(rows_a, cols_a, d_a, lda, npa, d_a0, d_a1, d_a2, ldpa, s);
  return launch_split_pair(rows_a, cols_a, d_a, lda, npa, d_a0, d_a1, d_a2, ldpa, rows_b, cols_b,
                           d_b, ldb, npb, d_b0, d_b1, d_b2, ldpb, s);
}

// Workspace of bfx_gemm_bf16xN: npa planes of A pieces (m x kp) followed by
// npb planes of transposed B pieces (n x kp), kp = k rounded up to 8, every
// plane starting on a 256-byte boundary.
static void gemm_ws_layout(int npa, int npb, int64_t m, int64_t n, int64_t k, int64_t* kp,
                           int64_t* a_plane, int64_t* b_plane, size_t* bytes) {
  *kp = round_up(k > 0 ? k : 1, 8);
  *a_plane = round_up(m * *kp, 128);
  *b_plane = round_up(n * *kp, 128);
  *bytes = (static_cast<size_t>(npa) * static_cast<size_t>(*a_plane) +
            static_cast<size_t>(npb) * static_cast<size_t>(*b_plane)) *
           2;
}

BFX_API size_t bfx_gemm_workspace_size(bfx_mode mode, int64_t m, int64_t n, int64_t k) {
  int npa, npb;
  if (!gemm_pieces(mode, &npa, &npb) || m <= 0 || n <= 0 || k <= 0) return 0;
  int64_t kp, ap, bp;
  size_t bytes;
  gemm_ws_layout(npa, npb, m, n, k, &kp, &ap, &bp, &bytes);
  return bytes;
}

static bfx_status check_gemm_args(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda,
                                  const void* B, int64_t ldb, const float* C, int64_t ldc) {
  if (m < 0 || n < 0 || k < 0) return BFX_EINVAL;
  if (m == 0 || n == 0) return BFX_OK;
  if (ldc < n || !C) return BFX_EINVAL;
  if (k > 0 && (!A || !B || lda < k)) return BFX_EINVAL;
  (void)ldb;
  return BFX_OK;
}

BFX_API bfx_status bfx_sgemm_simt(int64_t m, int64_t n, int64_t k, float alpha, const float* d_A,
                                  int64_t lda, const float* d_B, int64_t ldb, float beta,
                                  float* d_C, int64_t ldc, bfx_stream stream) {
  bfx_status st = check_gemm_args(m, n, k, d_A, lda, d_B, ldb, d_C, ldc);
  if (st != BFX_OK) return st;
  if (k > 0 && ldb < n) return BFX_EINVAL;
  return launch_sgemm_simt(m, n, k, alpha, d_A, lda, d_B, ldb, beta, d_C, ldc,
                           static_cast<cudaStream_t>(stream));
}

BFX_API bfx_status bfx_gemm_presplit(bfx_mode mode, int64_t m, int64_t n, int64_t k, float alpha,
                                     const uint16_t* d_Ap, int64_t lda_p, int64_t a_plane,
                                     const uint16_t* d_Btp, int64_t ldb_p, int64_t b_plane,
                                     float beta, float* d_C, int64_t ldc, bfx_stream stream) {
  int npa, npb;
  if (!gemm_pieces(mode, &npa, &npb)) return BFX_EINVAL;
  bfx_status st = check_gemm_args(m, n, k, d_Ap, lda_p, d_Btp, ldb_p, d_C, ldc);
  if (st != BFX_OK) return st;
  if (m == 0 || n == 0) return BFX_OK;
  if (k > 0) {
    if (ldb_p < k) return BFX_EINVAL;
    if ((npa > 1 && a_plane < (m - 1) * lda_p + k) || (npb > 1 && b_plane < (n - 1) * ldb_p + k))
      return BFX_EINVAL;
    if (lda_p % 8 || ldb_p % 8 || (npa > 1 && a_plane % 8) || (npb > 1 && b_plane % 8) ||
        !aligned(d_Ap, 16) || !aligned(d_Btp, 16))
      return BFX_EUNSUPPORTED;
  }
  if (m >= INT32_MAX || n >= INT32_MAX || k >= INT32_MAX) return BFX_EUNSUPPORTED;
  if (!is_sm103()) return BFX_EUNSUPPORTED;
  return launch_gemm_presplit(mode, m, n, k, alpha, d_Ap, lda_p, a_plane, d_Btp, ldb_p, b_plane,
                              beta, d_C, ldc, static_cast<cudaStream_t>(stream));
}

// Splits A (npa pieces) and the transpose of B (npb pieces) into the
// workspace laid out as gemm_ws_layout says.
static bfx_status split_operands(bfx_mode mode, int64_t m, int64_t n, int64_t k, const float* d_A,
                                 int64_t lda, const float* d_B, int64_t ldb, void* d_ws,
                                 size_t ws_bytes, uint16_t** Ap, uint16_t** Bp, int64_t* kp,
                                 int64_t* ap, int64_t* bp, cudaStream_t s) {
  int npa, npb;
  if (!gemm_pieces(mode, &npa, &npb)) return BFX_EINVAL;
  size_t need;
  gemm_ws_layout(npa, npb, m, n, k, kp, ap, bp, &need);
  if (!d_ws || ws_bytes < need) return BFX_ENOMEM;
  if (!aligned(d_ws, 256)) return BFX_EUNSUPPORTED;
  *Ap = static_cast<uint16_t*>(d_ws);
  *Bp = *Ap + npa * *ap;
  return launch_split_pair(m, k, d_A, lda, npa, *Ap, npa > 1 ? *Ap + *ap : nullptr,
                           npa > 2 ? *Ap + 2 * *ap : nullptr, *kp, k, n, d_B, ldb, npb, *Bp,
                           npb > 1 ? *Bp + *bp : nullptr, npb > 2 ? *Bp + 2 * *bp : nullptr, *kp, s);
}

BFX_API bfx_status bfx_gemm_bf16xN(bfx_mode mode, int64_t m, int64_t n, int64_t k, float alpha,
                                   const float* d_A, int64_t lda, const float* d_B, int64_t ldb,
                                   float beta, float* d_C, int64_t ldc, void* d_ws,
                                   size_t ws_bytes, bfx_stream stream) {
  if (!check_mode(mode)) return BFX_EINVAL;
  if (mode == BFX_FP32)
    return bfx_sgemm_simt(m, n, k, alpha, d_A, lda, d_B, ldb, beta, d_C, ldc, stream);
  bfx_status st = check_gemm_args(m, n, k, d_A, lda, d_B, ldb, d_C, ldc);
  if (st != BFX_OK) return st;
  if (m == 0 || n == 0) return BFX_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (k == 0) return launch_scale(m, n, beta, d_C, ldc, s);
  if (ldb < n) return BFX_EINVAL;
  if (m >= INT32_MAX || n >= INT32_MAX || k >= INT32_MAX) return BFX_EUNSUPPORTED;
  if (!is_sm103()) return BFX_EUNSUPPORTED;
  int64_t kp, ap, bp;
  uint16_t *Ap, *Bp;
  if ((st = split_operands(mode, m, n, k, d_A, lda, d_B, ldb, d_ws, ws_bytes, &Ap, &Bp, &kp, &ap,
                           &bp, s)) != BFX_OK)
    return st;
  return launch_gemm_presplit(mode, m, n, k, alpha, Ap, kp, ap, Bp, kp, bp, beta, d_C, ldc, s);
}

BFX_API bfx_status bfx_gemm_bf16xN_f64(bfx_mode mode, int64_t m, int64_t n, int64_t k,
                                       const float* d_A, int64_t lda, const float* d_B,
                                       int64_t ldb, double* d_C, int64_t ldc, void* d_ws,
                                       size_t ws_bytes, bfx_stream stream) {
  int npa, npb;
  if (!gemm_pieces(mode, &npa, &npb)) return BFX_EINVAL;
  if (m < 0 || n < 0 || k < 0) return BFX_EINVAL;
  if (m == 0 || n == 0) return BFX_OK;
  if (ldc < n || !d_C || k == 0 || !d_A || !d_B || lda < k || ldb < n) return BFX_EINVAL;
  if (m >= INT32_MAX || n >= INT32_MAX || k >= INT32_MAX) return BFX_EUNSUPPORTED;
  if (!is_sm103()) return BFX_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t kp, ap, bp;
  uint16_t *Ap, *Bp;
  bfx_status st;
  if ((st = split_operands(mode, m, n, k, d_A, lda, d_B, ldb, d_ws, ws_bytes, &Ap, &Bp, &kp, &ap,
                           &bp, s)) != BFX_OK)
    return st;
  return launch_gemm_f64(mode, m, n, k, Ap, kp, ap, Bp, kp, bp, d_C, ldc, s);
}

BFX_API bfx_status bfx_gemm_bf16xN_fused(bfx_mode mode, int64_t m, int64_t n, int64_t k,
                                         float alpha, const float* d_A, int64_t lda,
                                         const float* d_B, int64_t ldb, float beta, float* d_C,
                                         int64_t ldc, bfx_stream stream) {
  if (mode_pieces(mode) == 0) return BFX_EINVAL;
  bfx_status st = check_gemm_args(m, n, k, d_A, lda, d_B, ldb, d_C, ldc);
  if (st != BFX_OK) return st;
  if (m == 0 || n == 0) return BFX_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (k == 0) return launch_scale(m, n, beta, d_C, ldc, s);
  if (ldb < n) return BFX_EINVAL;
  if (m >= INT32_MAX || n >= INT32_MAX || k >= INT32_MAX) return BFX_EUNSUPPORTED;
  if (!is_sm103()) return BFX_EUNSUPPORTED;
  return launch_gemm_fused(mode, m, n, k, alpha, d_A, lda, d_B, ldb, beta, d_C, ldc, s);
}

BFX_API bfx_status bfx_lowp_lu_ir_batched(bfx_lowp type, int count, int n, const float* d_A,
                                          const double* d_b, const double* d_tol, int max_iter,
                                          double* d_x, float* d_LU, int32_t* d_ipiv,
                                          int32_t* d_iters, int32_t* d_conv, int32_t* d_info,
                                          bfx_stream stream) {
  if (type != BFX_LOWP_FP32 && type != BFX_LOWP_BF16 && type != BFX_LOWP_FP16) return BFX_EINVAL;
  if (count < 0 || n < 1 || max_iter < 0) return BFX_EINVAL;
  if (count == 0) return BFX_OK;
  if (!d_A || !d_b || !d_tol || !d_x || !d_iters || !d_conv || !d_info) return BFX_EINVAL;
  if (n > lowp_max_n()) return BFX_EUNSUPPORTED;
  if (!is_sm103()) return BFX_EUNSUPPORTED;
  return launch_lowp_lu_ir(type, count, n, d_A, d_b, d_tol, max_iter, d_x, d_LU, d_ipiv, d_iters,
                           d_conv, d_info, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
