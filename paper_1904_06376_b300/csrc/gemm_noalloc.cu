// Workspace-free bf16xN GEMM: bfx_gemm_bf16xN_noalloc.
//
// bfx_gemm_bf16xN needs a caller-provided workspace for the bfloat16 pieces.
// Some callers cannot provide one: code that runs inside a host application
// which owns every byte of device memory through its own pool and forbids
// libraries from calling cudaMalloc, or latency-critical loops where an
// allocation (and the device-wide synchronisation cudaMalloc/cudaFree may
// imply) is not acceptable.  For them this entry point keeps the pieces in a
// file-scope device array of fixed size.  The array is reserved on a device
// when the library's module is loaded there (with CUDA's lazy module loading,
// at the first launch of any of the library's kernels on that device, by any
// entry point), so every process using the library holds it on every device
// it uses until the process exits.
//
// The array's name, used in host code, is only a host-side stand-in for the
// symbol, not a device address.  Its device address is looked up once per
// device with cudaGetSymbolAddress (with that device current) on the first
// call on that device, and that address is what the kernels receive.
//
// Nothing in the array has to start at zero: every piece element the GEMM
// reads is written by the split kernels earlier in the same call, on the same
// stream.  All calls share the one array, so calls whose kernels overlap on
// the GPU (different streams, or different host threads on one device) race
// on it; serialise them.
#include "bfx_internal.cuh"

namespace bfx {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB a device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDev = 64;
void* g_noalloc_ptr[kMaxDev] = {nullptr};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
bfx_status noalloc_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return BFX_ECUDA;
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return BFX_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return BFX_OK;
}

}  // namespace
}  // namespace bfx

using namespace bfx;

extern "C" BFX_API bfx_status bfx_gemm_bf16xN_noalloc(bfx_mode mode, int64_t m, int64_t n,
                                                      int64_t k, float alpha, const float* d_A,
                                                      int64_t lda, const float* d_B, int64_t ldb,
                                                      float beta, float* d_C, int64_t ldc,
                                                      bfx_stream stream) {
  int npa = 0, npb = 0;
  if (!gemm_pieces(mode, &npa, &npb)) return BFX_EINVAL;  // X1, X3, X5, X6, X8, X9
  if (m < 0 || n < 0 || k < 0) return BFX_EINVAL;
  if (m == 0 || n == 0) return BFX_OK;
  if (!d_C || ldc < n) return BFX_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (k == 0) return launch_scale(m, n, beta, d_C, ldc, s);
  if (!d_A || !d_B || lda < k || ldb < n) return BFX_EINVAL;
  if (m >= INT32_MAX || n >= INT32_MAX || k >= INT32_MAX) return BFX_EUNSUPPORTED;
  // pieces: npa planes of A (m x kp) and npb planes of B^T (n x kp), kp = k
  // rounded up to 8, each plane on a 256-byte boundary
  const int64_t kp = round_up(k, 8);
  const int64_t ap = round_up(m * kp, 128);
  const int64_t bp = round_up(n * kp, 128);
  const double need = 2.0 * (npa * static_cast<double>(ap) + npb * static_cast<double>(bp));
  if (need > static_cast<double>(kNoAllocScratchBytes)) return BFX_ENOMEM;
  if (!is_sm103()) return BFX_EUNSUPPORTED;
  void* scratch = nullptr;
  bfx_status st = noalloc_scratch(&scratch);
  if (st != BFX_OK) return st;
  uint16_t* Ap = static_cast<uint16_t*>(scratch);
  uint16_t* Bp = Ap + npa * ap;
  st = launch_split(m, k, d_A, lda, npa, Ap, npa > 1 ? Ap + ap : nullptr,
                    npa > 2 ? Ap + 2 * ap : nullptr, kp, s);
  if (st != BFX_OK) return st;
  st = launch_split_transpose(k, n, d_B, ldb, npb, Bp, npb > 1 ? Bp + bp : nullptr,
                              npb > 2 ? Bp + 2 * bp : nullptr, kp, s);
  if (st != BFX_OK) return st;
  return launch_gemm_presplit(mode, m, n, k, alpha, Ap, kp, ap, Bp, kp, bp, beta, d_C, ldc, s);
}
