// Batched LU + refinement of many uneven-size systems (host planning and the
// C ABI).  The kernels live in lu.cu (batched LU steps), gemm_tc.cu (grouped
// tensor-core GEMM) and ir.cu (batched refinement); this file sorts the
// systems by size, lays out the workspace, builds the per-step tile lists of
// the grouped trailing updates, and captures the whole launch sequence into
// one CUDA graph per set of buffers.
#include <algorithm>
#include <cstring>
#include <cmath>
#include <numeric>
#include <vector>

#include "bfx_internal.cuh"

namespace bfx {
// refinement step in the latency form (ir.cu)
bfx_status ir_batched_step_latency(const BatchIr* d_ir, int S, BatchIrParams p, cudaStream_t s);

namespace {

constexpr int kBatchNb = 64;      // default block-column width of the batched LU
constexpr int kBatchBn = 256;     // default tile width of the grouped trailing updates
constexpr int kBatchMaxN = 1024;  // largest system of a batch
constexpr int kSolveTB = 64;      // diagonal-block size of the refinement solves
constexpr int kGmresM = 256;      // Krylov length of the batched GMRES-IR (capped at n)
// refinement steps from this one on use the latency form (most systems have
// stopped by then: a step lasts as long as its slowest system's); on a batch
// of 2000 systems up to n = 512, switching at steps 4, 5 or 6 measured the
// same within 0.1 ms, at step 3 0.9 ms slower
constexpr int kLatencyStep = 5;
constexpr int kGmresOuter = 20;   // its refinement steps at most
constexpr double kGmresTau = 1e-10;
constexpr size_t kGmresSlotBudget = size_t(1) << 30;  // Krylov memory of all slots, at most

size_t take(size_t& off, size_t bytes) {
  const size_t o = off;
  off += (bytes + 255) / 256 * 256;
  return o;
}

}  // namespace
}  // namespace bfx

using namespace bfx;

struct bfx_batch_plan {
  bfx_mode mode;
  int S, nrhs, nb, bn, max_iter, np, nmax;
  int gmres, gm_slots;
  int64_t gm_slot_doubles;
  BatchIrParams p;
  std::vector<int> n;       // caller order
  std::vector<int> sorted;  // sorted[k] = caller index, n descending
  std::vector<int> n_desc;
  std::vector<int64_t> offA, offV, offN, offD;  // caller order (elements)
  int64_t totA = 0, totV = 0, totN = 0, totD = 0;
  int64_t kp = 0, slot_rows = 0;
  // workspace layout (byte offsets)
  size_t o_LU, o_ipiv, o_info, o_perm, o_r, o_d, o_Linv, o_Uinv, o_state, o_packA, o_packB;
  size_t o_lu_tab, o_ir_tab, o_tiles, o_probs, o_gm_queue, o_gm_slots, total;
  std::vector<int> step_J0, step_ntiles, step_nprobs;
  std::vector<size_t> step_tile_off, step_prob_off;  // element offsets into the tables
  int64_t ntiles_all = 0, nprobs_all = 0;
  // bound buffers and the captured graph
  const void* bA = nullptr;
  const void* bb = nullptr;
  void* bx = nullptr;
  void* bst = nullptr;
  void* bws = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

bfx_status enqueue(bfx_batch_plan* P, cudaStream_t s) {
  char* ws = static_cast<char*>(P->bws);
  float* LU = reinterpret_cast<float*>(ws + P->o_LU);
  const BatchLu* lu_tab = reinterpret_cast<const BatchLu*>(ws + P->o_lu_tab);
  const BatchIr* ir_tab = reinterpret_cast<const BatchIr*>(ws + P->o_ir_tab);
  const GroupTile* tiles = reinterpret_cast<const GroupTile*>(ws + P->o_tiles);
  const GroupProblem* probs = reinterpret_cast<const GroupProblem*>(ws + P->o_probs);
  uint16_t* packA = reinterpret_cast<uint16_t*>(ws + P->o_packA);
  uint16_t* packB = reinterpret_cast<uint16_t*>(ws + P->o_packB);
  if (cudaMemcpyAsync(LU, P->bA, sizeof(float) * P->totA, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(ws + P->o_info, 0, sizeof(int32_t) * P->S, s) != cudaSuccess)
    return BFX_ECUDA;
  bfx_status st = ir_batched_prepare(ir_tab, P->S, P->nmax, s);
  if (st != BFX_OK) return st;
  for (size_t k = 0; k < P->step_J0.size(); ++k) {
    st = lu_batched_block(P->mode, lu_tab, P->n_desc.data(), P->S, P->nb, P->step_J0[k], packA,
                          packB, P->slot_rows, P->kp, s);
    if (st != BFX_OK) return st;
    if (P->step_ntiles[k] > 0) {
      st = launch_gemm_grouped(P->mode, P->bn, P->step_ntiles[k], tiles + P->step_tile_off[k],
                               probs + P->step_prob_off[k], packA, P->slot_rows, packB,
                               P->slot_rows, static_cast<int64_t>(P->S) * P->np, P->kp, -1.0f,
                               1.0f, s);
      if (st != BFX_OK) return st;
    }
  }
  if ((st = ir_batched_post_lu(ir_tab, P->S, P->nmax, s)) != BFX_OK) return st;
  if ((st = ir_batched_first_solve(ir_tab, P->S, s)) != BFX_OK) return st;
  for (int it = 0; it < P->max_iter; ++it)
    if ((st = (it < kLatencyStep ? ir_batched_step : ir_batched_step_latency)(ir_tab, P->S, P->p, s)) !=
        BFX_OK)
      return st;
  if ((st = ir_batched_finish(ir_tab, P->S, P->p, s)) != BFX_OK) return st;
  if (!P->gmres) return BFX_OK;
  return ir_batched_gmres(ir_tab, P->S, reinterpret_cast<int*>(ws + P->o_gm_queue),
                          reinterpret_cast<double*>(ws + P->o_gm_slots), P->gm_slot_doubles,
                          P->gm_slots, kGmresM, P->p, kGmresOuter, kGmresTau, s);
}

// Fill the device tables for the bound buffers (host staging, one copy each).
bfx_status write_tables(bfx_batch_plan* P, cudaStream_t s) {
  char* ws = static_cast<char*>(P->bws);
  float* LU = reinterpret_cast<float*>(ws + P->o_LU);
  int32_t* ipiv = reinterpret_cast<int32_t*>(ws + P->o_ipiv);
  int32_t* info = reinterpret_cast<int32_t*>(ws + P->o_info);
  int32_t* perm = reinterpret_cast<int32_t*>(ws + P->o_perm);
  double* r = reinterpret_cast<double*>(ws + P->o_r);
  double* d = reinterpret_cast<double*>(ws + P->o_d);
  double* Linv = reinterpret_cast<double*>(ws + P->o_Linv);
  double* Uinv = reinterpret_cast<double*>(ws + P->o_Uinv);
  BatchIrState* state = reinterpret_cast<BatchIrState*>(ws + P->o_state);
  std::vector<BatchLu> lt(P->S);
  std::vector<BatchIr> it(P->S);
  for (int k = 0; k < P->S; ++k) {
    const int c = P->sorted[k];
    lt[k] = BatchLu{LU + P->offA[c], P->n[c], 0, ipiv + P->offN[c], info + c};
    BatchIr q{};
    q.A = static_cast<const float*>(P->bA) + P->offA[c];
    q.LU = LU + P->offA[c];
    q.ipiv = ipiv + P->offN[c];
    q.info = info + c;
    q.perm = perm + P->offN[c];
    q.b = static_cast<const double*>(P->bb) + P->offV[c];
    q.x = static_cast<double*>(P->bx) + P->offV[c];
    q.r = r + P->offV[c];
    q.d = d + P->offV[c];
    q.Linv = Linv + P->offD[c];
    q.Uinv = Uinv + P->offD[c];
    q.st = state + k;
    q.out = static_cast<bfx_batch_status*>(P->bst) + c;
    q.n = P->n[c];
    q.nrhs = P->nrhs;
    it[k] = q;
  }
  std::vector<GroupTile> tl;
  std::vector<GroupProblem> pr;
  const int bk = gemm_bk(P->mode);
  for (size_t st = 0; st < P->step_J0.size(); ++st) {
    const int J0 = P->step_J0[st];
    const int p0 = static_cast<int>(pr.size());
    for (int k = 0; k < P->S; ++k) {
      const int n = P->n_desc[k];
      if (n <= J0) break;
      const int JB = std::min(P->nb, n - J0);
      const int M = n - J0 - JB;
      if (M <= 0) continue;
      GroupProblem g{};
      g.C = lt[k].A + static_cast<int64_t>(J0 + JB) * n + J0 + JB;
      g.ldc = n;
      g.M = M;
      g.N = M;
      g.k_tiles = static_cast<int>(ceil_div(JB, bk));
      g.plane0 = k * P->np;
      g.vec_c = (n % 4 == 0) && aligned(g.C, 16);
      const int pi = static_cast<int>(pr.size()) - p0;
      pr.push_back(g);
      for (int mb = 0; mb < ceil_div(M, 128); ++mb)
        for (int nbk = 0; nbk < ceil_div(M, P->bn); ++nbk) tl.push_back(GroupTile{pi, mb, nbk, 0});
    }
  }
  if (static_cast<int64_t>(tl.size()) != P->ntiles_all || static_cast<int64_t>(pr.size()) != P->nprobs_all)
    return BFX_EINVAL;
  if (cudaMemcpyAsync(ws + P->o_lu_tab, lt.data(), sizeof(BatchLu) * lt.size(), cudaMemcpyHostToDevice,
                      s) != cudaSuccess ||
      cudaMemcpyAsync(ws + P->o_ir_tab, it.data(), sizeof(BatchIr) * it.size(), cudaMemcpyHostToDevice,
                      s) != cudaSuccess)
    return BFX_ECUDA;
  if (!tl.empty() && cudaMemcpyAsync(ws + P->o_tiles, tl.data(), sizeof(GroupTile) * tl.size(),
                                     cudaMemcpyHostToDevice, s) != cudaSuccess)
    return BFX_ECUDA;
  if (!pr.empty() && cudaMemcpyAsync(ws + P->o_probs, pr.data(), sizeof(GroupProblem) * pr.size(),
                                     cudaMemcpyHostToDevice, s) != cudaSuccess)
    return BFX_ECUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? BFX_OK : BFX_ECUDA;
}

}  // namespace

namespace bfx {
// One batched solve launched directly on stream s, without a graph: the
// serving loop's batches come with new buffers every time, so capturing
// would cost more than it saves.  Same launch sequence as the graph.
bfx_status batch_solve_direct(bfx_batch_plan* P, const float* d_A, const double* d_b, double* d_x,
                              bfx_batch_status* d_status, void* d_ws, size_t ws_bytes,
                              cudaStream_t s) {
  if (!P || !d_A || !d_b || !d_x || !d_status) return BFX_EINVAL;
  if (!d_ws || ws_bytes < P->total) return BFX_ENOMEM;
  if (!aligned(d_ws, 256)) return BFX_EUNSUPPORTED;
  if (!device_error_word()) return BFX_ECUDA;
  if (P->exec) {
    cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
  }
  P->bA = d_A;
  P->bb = d_b;
  P->bx = d_x;
  P->bst = d_status;
  P->bws = d_ws;
  bfx_status st = write_tables(P, s);
  if (st != BFX_OK) return st;
  st = enqueue(P, s);
  P->bA = nullptr;  // not bound to a graph: a later bfx_batch_solve captures afresh
  return st;
}
}  // namespace bfx

extern "C" {

BFX_API bfx_status bfx_batch_create_config(bfx_batch* out, bfx_mode mode, int count,
                                           const int32_t* h_n, int nrhs,
                                           const bfx_ir_params* params,
                                           const bfx_batch_config* config) {
  if (!out) return BFX_EINVAL;
  *out = nullptr;
  if (mode_pieces(mode) == 0 || count <= 0 || !h_n || nrhs < 1 || nrhs > 16) return BFX_EINVAL;
  for (int s = 0; s < count; ++s)
    if (h_n[s] < 1 || h_n[s] > kBatchMaxN) return BFX_EINVAL;
  bfx_ir_params ip{};
  ip.max_iter = 50;
  ip.tol = 1.1102230246251565e-16;
  ip.tol_b = -1.0;
  ip.stall = 0.5;
  ip.gmres = 1;
  if (params) ip = *params;
  if (ip.gmres < 0 || ip.gmres > 2) return BFX_EINVAL;
  if (ip.max_iter < 0 || ip.max_iter > 200) return BFX_EINVAL;
  bfx_batch_config cfg{kBatchNb, kBatchBn};
  if (config) {
    cfg.nb = config->nb ? config->nb : kBatchNb;
    cfg.gemm_bn = config->gemm_bn ? config->gemm_bn : kBatchBn;
  }
  if ((cfg.nb != 32 && cfg.nb != 64 && cfg.nb != 128) ||
      (cfg.gemm_bn != 64 && cfg.gemm_bn != 128 && cfg.gemm_bn != 256))
    return BFX_EINVAL;
  auto* P = new bfx_batch_plan();
  P->mode = mode;
  P->S = count;
  P->nrhs = nrhs;
  P->nb = cfg.nb;
  P->bn = cfg.gemm_bn;
  P->gmres = ip.gmres != 0;  // 1 and 2 both: GMRES-IR after plain refinement
  P->max_iter = ip.max_iter;
  P->np = mode_pieces(mode);
  P->n.assign(h_n, h_n + count);
  P->sorted.resize(count);
  std::iota(P->sorted.begin(), P->sorted.end(), 0);
  std::stable_sort(P->sorted.begin(), P->sorted.end(),
                   [&](int a, int b) { return P->n[a] > P->n[b]; });
  P->n_desc.resize(count);
  for (int k = 0; k < count; ++k) P->n_desc[k] = P->n[P->sorted[k]];
  P->nmax = P->n_desc[0];
  int64_t nmin = P->n_desc[count - 1];
  P->p.tol = ip.tol;
  P->p.stall = ip.stall;
  P->p.tol_b = ip.tol_b >= 0 ? ip.tol_b : 1.1102230246251565e-16 * std::sqrt(static_cast<double>(nmin));
  for (int s = 0; s < count; ++s) {
    const int64_t n = P->n[s];
    P->offA.push_back(P->totA);
    P->offV.push_back(P->totV);
    P->offN.push_back(P->totN);
    P->offD.push_back(P->totD);
    P->totA += n * n;
    P->totV += n * nrhs;
    P->totN += n;
    P->totD += ceil_div(n, kSolveTB) * kSolveTB * kSolveTB;
  }
  P->kp = P->nb;
  P->slot_rows = P->nmax;
  for (int J0 = 0; J0 < P->nmax; J0 += P->nb) {
    int nt = 0, npb = 0;
    for (int k = 0; k < count; ++k) {
      const int n = P->n_desc[k];
      if (n <= J0) break;
      const int M = n - J0 - std::min(P->nb, n - J0);
      if (M <= 0) continue;
      ++npb;
      nt += static_cast<int>(ceil_div(M, 128) * ceil_div(M, P->bn));
    }
    P->step_J0.push_back(J0);
    P->step_ntiles.push_back(nt);
    P->step_nprobs.push_back(npb);
    P->step_tile_off.push_back(P->ntiles_all);
    P->step_prob_off.push_back(P->nprobs_all);
    P->ntiles_all += nt;
    P->nprobs_all += npb;
  }
  size_t off = 0;
  P->o_LU = take(off, sizeof(float) * P->totA);
  P->o_ipiv = take(off, sizeof(int32_t) * P->totN);
  P->o_info = take(off, sizeof(int32_t) * count);
  P->o_perm = take(off, sizeof(int32_t) * P->totN);
  P->o_r = take(off, sizeof(double) * P->totV);
  P->o_d = take(off, sizeof(double) * P->totV);
  P->o_Linv = take(off, sizeof(double) * P->totD);
  P->o_Uinv = take(off, sizeof(double) * P->totD);
  P->o_state = take(off, sizeof(BatchIrState) * count);
  const size_t pack = sizeof(uint16_t) * static_cast<size_t>(count) * P->np * P->slot_rows * P->kp;
  P->o_packA = take(off, pack);
  P->o_packB = take(off, pack);
  P->o_lu_tab = take(off, sizeof(BatchLu) * count);
  P->o_ir_tab = take(off, sizeof(BatchIr) * count);
  P->o_tiles = take(off, sizeof(GroupTile) * std::max<int64_t>(1, P->ntiles_all));
  P->o_probs = take(off, sizeof(GroupProblem) * std::max<int64_t>(1, P->nprobs_all));
  if (P->gmres) {
    P->gm_slot_doubles = batched_gmres_slot_doubles(kGmresM, P->nmax, nrhs);
    const int64_t per = P->gm_slot_doubles * static_cast<int64_t>(sizeof(double));
    const int sms = current_num_sms() > 0 ? current_num_sms() : 148;
    int64_t slots = std::min<int64_t>(count, sms);
    slots = std::min<int64_t>(slots, std::max<int64_t>(1, static_cast<int64_t>(kGmresSlotBudget) / per));
    P->gm_slots = static_cast<int>(slots);
    P->o_gm_queue = take(off, sizeof(int));
    P->o_gm_slots = take(off, static_cast<size_t>(per) * slots);
  }
  P->total = off;
  *out = P;
  return BFX_OK;
}

BFX_API bfx_status bfx_batch_create(bfx_batch* out, bfx_mode mode, int count, const int32_t* h_n,
                                    int nrhs, const bfx_ir_params* params) {
  return bfx_batch_create_config(out, mode, count, h_n, nrhs, params, nullptr);
}

BFX_API bfx_status bfx_batch_get_config(bfx_batch plan, bfx_batch_config* out) {
  if (!plan || !out) return BFX_EINVAL;
  out->nb = plan->nb;
  out->gemm_bn = plan->bn;
  return BFX_OK;
}

BFX_API size_t bfx_batch_workspace_size(bfx_batch plan) { return plan ? plan->total : 0; }

BFX_API bfx_status bfx_batch_solve(bfx_batch P, const float* d_A, const double* d_b, double* d_x,
                                   bfx_batch_status* d_status, void* d_ws, size_t ws_bytes,
                                   bfx_stream stream) {
  if (!P || !d_A || !d_b || !d_x || !d_status) return BFX_EINVAL;
  if (!d_ws || ws_bytes < P->total) return BFX_ENOMEM;
  if (!aligned(d_ws, 256)) return BFX_EUNSUPPORTED;
  if (!is_sm103()) return BFX_EUNSUPPORTED;
  if (!device_error_word()) return BFX_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool same = P->exec && P->bA == d_A && P->bb == d_b && P->bx == d_x && P->bst == d_status &&
                    P->bws == d_ws;
  if (!same) {
    if (P->exec) {
      cudaGraphExecDestroy(P->exec);
      P->exec = nullptr;
    }
    P->bA = d_A;
    P->bb = d_b;
    P->bx = d_x;
    P->bst = d_status;
    P->bws = d_ws;
    bfx_status st = write_tables(P, s);
    if (st != BFX_OK) return st;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return BFX_ECUDA;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaStreamDestroy(cs);
      return BFX_ECUDA;
    }
    st = enqueue(P, cs);
    const cudaError_t ce = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st != BFX_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return st != BFX_OK ? st : BFX_ECUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&P->exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      P->exec = nullptr;
      return BFX_ECUDA;
    }
  }
  return cudaGraphLaunch(P->exec, s) == cudaSuccess ? BFX_OK : BFX_ECUDA;
}

BFX_API void bfx_batch_destroy(bfx_batch P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  delete P;
}

}  // extern "C"
