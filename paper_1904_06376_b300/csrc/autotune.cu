// Autotuner of the batched solve's tile shapes.
//
// A batch of small uneven systems has no single best blocking: the block
// width nb of the LU sets how many steps the factorisation takes and the
// depth (K) of every grouped trailing update, and the tile width of the
// grouped tensor-core GEMM sets how much of each 128 x BN tile is padding for
// the small trailing matrices (n - J0 - nb of them, down to a few rows).  The
// tuner runs the caller's own batch under every candidate (nb in {32, 64,
// 128} x tile width in {64, 128, 256}), each as the CUDA graph the batch
// would replay, times `reps` replays with CUDA events on the caller's stream,
// and returns the fastest.  Results are also kept in a process-wide table
// keyed by a coarse signature of the batch (mode, nrhs, max_iter, count and
// the size histogram), so later batches drawn from the same distribution can
// take the tuned shape without timing (bfx_batch_tuned_config).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "bfx_internal.cuh"

namespace {

std::mutex g_tune_mu;
std::map<std::string, bfx_batch_config> g_tuned;

std::string signature(bfx_mode mode, int count, const int32_t* h_n, int nrhs,
                      const bfx_ir_params* params) {
  // histogram of n over 8 bins of 128, each bin's share rounded to 1/20;
  // count rounded to two significant digits
  int hist[8] = {0};
  for (int s = 0; s < count; ++s) hist[std::min(7, (h_n[s] - 1) / 128)] += 1;
  int c2 = count;
  int scale = 1;
  while (c2 >= 100) {
    c2 /= 10;
    scale *= 10;
  }
  std::string key = std::to_string(static_cast<int>(mode)) + "/" + std::to_string(nrhs) + "/" +
                    std::to_string(params ? params->max_iter : 50) + "/" +
                    std::to_string(c2 * scale);
  for (int b = 0; b < 8; ++b) key += "/" + std::to_string((hist[b] * 20 + count / 2) / count);
  return key;
}

}  // namespace

extern "C" {

BFX_API bfx_status bfx_batch_autotune(bfx_mode mode, int count, const int32_t* h_n, int nrhs,
                                      const bfx_ir_params* params, const float* d_A,
                                      const double* d_b, double* d_x,
                                      bfx_batch_status* d_status, int reps, bfx_stream stream,
                                      bfx_batch_config* h_best, float* h_best_ms,
                                      bfx_tune_entry* h_table, int* h_table_len) {
  if (!h_best || !d_A || !d_b || !d_x || !d_status || reps < 1) return BFX_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nbs[3] = {32, 64, 128}, bns[3] = {64, 128, 256};
  std::vector<bfx_tune_entry> table;
  float best = 0.0f;
  bool have = false;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return BFX_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return BFX_ECUDA;
  }
  bfx_status fatal = BFX_OK;
  for (int i = 0; i < 3 && fatal == BFX_OK; ++i) {
    for (int j = 0; j < 3 && fatal == BFX_OK; ++j) {
      bfx_tune_entry en{};
      en.config.nb = nbs[i];
      en.config.gemm_bn = bns[j];
      en.ms = -1.0f;
      bfx_batch plan = nullptr;
      en.status = bfx_batch_create_config(&plan, mode, count, h_n, nrhs, params, &en.config);
      if (en.status != BFX_OK) {
        if (en.status != BFX_ENOMEM) fatal = static_cast<bfx_status>(en.status);  // invalid batch
        table.push_back(en);
        continue;
      }
      const size_t wsb = bfx_batch_workspace_size(plan);
      void* ws = nullptr;
      if (cudaMalloc(&ws, wsb) != cudaSuccess) {
        cudaGetLastError();  // clear the allocation failure; try the next shape
        en.status = BFX_ENOMEM;
        bfx_batch_destroy(plan);
        table.push_back(en);
        continue;
      }
      // first solve: builds and instantiates the graph (untimed)
      en.status = bfx_batch_solve(plan, d_A, d_b, d_x, d_status, ws, wsb, stream);
      std::vector<float> t;
      for (int r = 0; r < reps && en.status == BFX_OK; ++r) {
        if (cudaEventRecord(e0, s) != cudaSuccess) {
          en.status = BFX_ECUDA;
          break;
        }
        en.status = bfx_batch_solve(plan, d_A, d_b, d_x, d_status, ws, wsb, stream);
        float ms = 0.0f;
        if (en.status == BFX_OK &&
            (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
          en.status = BFX_ECUDA;
        t.push_back(ms);
      }
      cudaStreamSynchronize(s);
      bfx_batch_destroy(plan);
      cudaFree(ws);
      if (en.status == BFX_OK) {
        std::sort(t.begin(), t.end());
        en.ms = t[t.size() / 2];
        if (!have || en.ms < best) {
          best = en.ms;
          *h_best = en.config;
          have = true;
        }
      } else if (en.status == BFX_ECUDA) {
        fatal = BFX_ECUDA;
      }
      table.push_back(en);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (h_table_len) {
    const int n = std::min<int>(*h_table_len, static_cast<int>(table.size()));
    if (h_table)
      for (int k = 0; k < n; ++k) h_table[k] = table[k];
    *h_table_len = static_cast<int>(table.size());
  }
  if (fatal != BFX_OK) return fatal;
  if (!have) return BFX_ENOMEM;
  if (h_best_ms) *h_best_ms = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[signature(mode, count, h_n, nrhs, params)] = *h_best;
  return BFX_OK;
}

BFX_API bfx_status bfx_batch_tuned_config(bfx_mode mode, int count, const int32_t* h_n, int nrhs,
                                          const bfx_ir_params* params, bfx_batch_config* out) {
  if (!out || !h_n || count <= 0) return BFX_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(signature(mode, count, h_n, nrhs, params));
  if (it == g_tuned.end()) return BFX_EINVAL;
  *out = it->second;
  return BFX_OK;
}

}  // extern "C"
