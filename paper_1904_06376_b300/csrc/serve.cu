// Serving runtime: continuous admission of solve requests of mixed sizes.
//
// A server owns one device-memory pool of a fixed budget (allocated once at
// creation) and a set of worker threads, each with its own CUDA stream.  A
// submitted request waits in a FIFO queue; it is admitted as soon as a worker
// is free AND the pool can hold its buffers (matrix, right-hand sides,
// solution and the solve workspace).  Admitted requests run concurrently, so
// kernels of different requests overlap on the device: the single-CTA panel
// tiles of one factorisation run beside the grouped or tensor-core updates of
// others.  Factors and refinement state stay in the request's device buffers
// for the whole solve; only A, b (in) and x (out) cross the bus.  Latency is
// measured from submission to completion.
// Continuous batching (batch_max_n > 0): a worker whose next request is small
// takes every waiting small request with the same nrhs (up to batch_max, as
// far as the pool has room) and solves them as one batch through the batched
// path (one grouped tensor-core update per LU step over all of them, per-
// system refinement decisions on the device), launched directly on its
// stream; requests arriving meanwhile form the next batch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "bfx_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// First-fit sub-allocator over one device allocation (256-byte granules).
class Pool {
 public:
  bool init(size_t bytes) {
    bytes_ = bytes / 256 * 256;
    if (cudaMalloc(&base_, bytes_) != cudaSuccess) {
      base_ = nullptr;
      return false;
    }
    free_[0] = bytes_;
    return true;
  }
  void release() {
    if (base_) cudaFree(base_);
    base_ = nullptr;
  }
  // offset or SIZE_MAX
  size_t alloc(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        used_ += bytes;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void free(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {  // merge right
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {  // merge left
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  char* base() const { return static_cast<char*>(base_); }
  size_t capacity() const { return bytes_; }
  size_t used() const { return used_; }

 private:
  void* base_ = nullptr;
  size_t bytes_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Request {
  int64_t ticket, n, nrhs;
  const float* hA;
  const double* hb;
  double* hx;
  Clock::time_point t_submit, t_start, t_done;
  bfx_request_result res{};
  bool done = false;
  size_t bytes = 0, off = 0;
};

// A batch of small requests solved together (continuous batching).
struct BatchJob {
  std::vector<Request*> reqs;
  bfx_batch plan = nullptr;
  size_t bytes = 0, off = 0;
  size_t oA = 0, ob = 0, ox = 0, ost = 0, ows = 0, wsb = 0;
};

}  // namespace

struct bfx_server_impl {
  bfx_server_config cfg{};
  int device = 0;
  Pool pool;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<int64_t, Request*> all;
  std::vector<std::thread> workers;
  int64_t next_ticket = 1;
  int running = 0;
  int batches = 0;
  bool stop = false;
  size_t peak_used = 0;
  int peak_running = 0;
};

namespace {

// Every request is solved with these parameters; the Krylov length is capped
// at 1024 so that a large request's reservation (the basis and Hessenberg
// matrices grow with gmres_m x n x nrhs) does not crowd the pool.
bfx_ir_params request_params(const bfx_server_config& cfg, int64_t n, int64_t nrhs) {
  bfx_ir_params p{};
  p.max_iter = 50;
  p.tol = 1.1102230246251565e-16;
  p.tol_b = -1.0;
  p.stall = 0.5;
  p.escalate = cfg.escalate;
  p.nb = cfg.nb;
  p.gmres = nrhs <= 16 ? cfg.gmres : 0;  // one Krylov basis per right-hand side, at most 16
  p.gmres_m = static_cast<int>(std::min<int64_t>(n, 1024));
  p.gmres_tol = 1e-10;
  // many concurrent solves: the preconditioner form with the least FP64 work
  // (explicit inverses cost n^3/3 FMAs per factorisation and save none)
  p.gmres_inverses = 0;
  return p;
}

constexpr int kBatchNb = 32, kBatchBn = 64;  // fixed tile shape of the serving batches
constexpr int kBatchMaxIter = 20;

bool is_small(const bfx_server_config& cfg, const Request* r) {
  return cfg.batch_max_n > 0 && r->n <= cfg.batch_max_n && r->nrhs <= 16;
}

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// Plan and pool layout of a batch of these requests (host only); false if
// the batch cannot be planned.
bool plan_batch(const bfx_server_config& cfg, BatchJob* J) {
  const int count = static_cast<int>(J->reqs.size());
  const int nrhs = static_cast<int>(J->reqs[0]->nrhs);
  std::vector<int32_t> ns(count);
  size_t sA = 0, sV = 0;
  for (int i = 0; i < count; ++i) {
    ns[i] = static_cast<int32_t>(J->reqs[i]->n);
    sA += sizeof(float) * J->reqs[i]->n * J->reqs[i]->n;
    sV += sizeof(double) * J->reqs[i]->n * nrhs;
  }
  bfx_ir_params p{};
  p.max_iter = kBatchMaxIter;
  p.tol = 1.1102230246251565e-16;
  p.tol_b = -1.0;
  p.stall = 0.5;
  p.escalate = 0;
  p.nb = kBatchNb;
  p.gmres = cfg.gmres ? 1 : 0;
  p.gmres_m = 0;
  p.gmres_tol = 0.0;
  bfx_batch_config bc{kBatchNb, kBatchBn};
  if (J->plan) bfx_batch_destroy(J->plan);
  J->plan = nullptr;
  if (bfx_batch_create_config(&J->plan, cfg.mode, count, ns.data(), nrhs, &p, &bc) != BFX_OK) {
    J->plan = nullptr;
    return false;
  }
  J->wsb = bfx_batch_workspace_size(J->plan);
  J->oA = 0;
  J->ob = J->oA + al256(sA);
  J->ox = J->ob + al256(sV);
  J->ost = J->ox + al256(sV);
  J->ows = J->ost + al256(sizeof(bfx_batch_status) * count);
  J->bytes = J->ows + al256(J->wsb);
  return true;
}

size_t request_bytes(const bfx_server_config& cfg, int64_t n, int64_t nrhs) {
  const size_t a = sizeof(float) * n * n;
  const size_t v = sizeof(double) * n * nrhs;
  const bfx_ir_params p = request_params(cfg, n, nrhs);
  const size_t ws = bfx_solve_ir_workspace_size(cfg.mode, n, nrhs, &p);
  return (a + 255) / 256 * 256 + 2 * ((v + 255) / 256 * 256) + ws + 256;
}

void finish_request(bfx_server_impl* S, Request* r, bfx_status status, const bfx_ir_result& ir) {
  r->t_done = Clock::now();
  r->res.status = status;
  r->res.converged = ir.converged;
  r->res.iters = ir.iters;
  r->res.info = ir.info;
  r->res.mode_used = ir.mode_used;
  r->res.refactorizations = ir.refactorizations;
  r->res.berr = ir.berr;
  r->res.gmres_steps = ir.gmres_steps;
  r->res.arnoldi = ir.arnoldi;
  r->res.latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  r->res.queue_s = std::chrono::duration<double>(r->t_start - r->t_submit).count();
  r->done = true;
}

// Solve a batch of small requests on stream st (continuous batching).
void run_batch(bfx_server_impl* S, BatchJob* J, cudaStream_t st) {
  const Clock::time_point t0 = Clock::now();
  for (Request* r : J->reqs) r->t_start = t0;
  char* base = S->pool.base() + J->off;
  float* dA = reinterpret_cast<float*>(base + J->oA);
  double* db = reinterpret_cast<double*>(base + J->ob);
  double* dx = reinterpret_cast<double*>(base + J->ox);
  auto* dst = reinterpret_cast<bfx_batch_status*>(base + J->ost);
  const int count = static_cast<int>(J->reqs.size());
  const int64_t R = J->reqs[0]->nrhs;
  bfx_status status = BFX_OK;
  int64_t oa = 0, ov = 0;
  for (Request* r : J->reqs) {
    if (cudaMemcpyAsync(dA + oa, r->hA, sizeof(float) * r->n * r->n, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(db + ov, r->hb, sizeof(double) * r->n * R, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
      status = BFX_ECUDA;
    oa += r->n * r->n;
    ov += r->n * R;
  }
  if (status == BFX_OK)
    status = bfx::batch_solve_direct(J->plan, dA, db, dx, dst, base + J->ows, J->wsb, st);
  std::vector<bfx_batch_status> hs(count);
  if (status == BFX_OK) {
    ov = 0;
    for (Request* r : J->reqs) {
      if (cudaMemcpyAsync(r->hx, dx + ov, sizeof(double) * r->n * R, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess)
        status = BFX_ECUDA;
      ov += r->n * R;
    }
    if (cudaMemcpyAsync(hs.data(), dst, sizeof(bfx_batch_status) * count, cudaMemcpyDeviceToHost,
                        st) != cudaSuccess)
      status = BFX_ECUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) status = BFX_ECUDA;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (int i = 0; i < count; ++i) {
      bfx_ir_result ir{};
      ir.mode_used = S->cfg.mode;
      bfx_status rs = status;
      if (status == BFX_OK) {
        ir.converged = hs[i].converged;
        ir.iters = hs[i].iters;
        ir.info = hs[i].info;
        ir.berr = hs[i].berr;
        ir.gmres_steps = hs[i].gmres_steps;
        rs = hs[i].info > 0 ? BFX_SINGULAR : (hs[i].converged ? BFX_OK : BFX_NOT_CONVERGED);
      }
      finish_request(S, J->reqs[i], rs, ir);
    }
    S->pool.free(J->off, J->bytes);
    S->running -= 1;
  }
  bfx_batch_destroy(J->plan);
  J->plan = nullptr;
}

void worker_main(bfx_server_impl* S) {
  cudaSetDevice(S->device);
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  const size_t bmax = S->cfg.batch_max > 0 ? static_cast<size_t>(S->cfg.batch_max) : 64;
  for (;;) {
    Request* r = nullptr;
    BatchJob job;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) break;
        if (!S->queue.empty()) {
          Request* h = S->queue.front();
          if (is_small(S->cfg, h)) {
            // every waiting small request with h's nrhs, in arrival order
            std::vector<Request*> cand;
            for (Request* q : S->queue)
              if (is_small(S->cfg, q) && q->nrhs == h->nrhs) {
                cand.push_back(q);
                if (cand.size() == bmax) break;
              }
            size_t off = SIZE_MAX;
            while (!cand.empty()) {  // as many as the pool holds (a prefix keeps h)
              job.reqs = cand;
              if (plan_batch(S->cfg, &job) && (off = S->pool.alloc(job.bytes)) != SIZE_MAX) break;
              cand.resize(cand.size() / 2);
            }
            if (off != SIZE_MAX) {
              job.off = off;
              S->batches += 1;
              for (Request* q : job.reqs) S->queue.erase(std::find(S->queue.begin(), S->queue.end(), q));
              S->running += 1;
              S->peak_running = std::max(S->peak_running, S->running);
              S->peak_used = std::max(S->peak_used, S->pool.used());
              break;
            }
            if (job.plan) bfx_batch_destroy(job.plan);
            job = BatchJob{};
          } else {
            const size_t off = S->pool.alloc(h->bytes);
            if (off != SIZE_MAX) {
              h->off = off;
              r = h;
              S->queue.pop_front();
              S->running += 1;
              S->peak_running = std::max(S->peak_running, S->running);
              S->peak_used = std::max(S->peak_used, S->pool.used());
              break;
            }
          }
        }
        S->cv_work.wait(lk);
      }
    }
    if (!job.reqs.empty() && job.plan) {
      run_batch(S, &job, st);
      S->cv_done.notify_all();
      S->cv_work.notify_all();
      continue;
    }
    if (!r) break;
    r->t_start = Clock::now();
    char* base = S->pool.base() + r->off;
    const int64_t n = r->n, R = r->nrhs;
    float* dA = reinterpret_cast<float*>(base);
    size_t o = (sizeof(float) * n * n + 255) / 256 * 256;
    double* db = reinterpret_cast<double*>(base + o);
    o += (sizeof(double) * n * R + 255) / 256 * 256;
    double* dx = reinterpret_cast<double*>(base + o);
    o += (sizeof(double) * n * R + 255) / 256 * 256;
    void* ws = base + o;
    const size_t wsb = r->bytes - o;
    bfx_status status = BFX_OK;
    if (cudaMemcpyAsync(dA, r->hA, sizeof(float) * n * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(db, r->hb, sizeof(double) * n * R, cudaMemcpyHostToDevice, st) != cudaSuccess)
      status = BFX_ECUDA;
    const bfx_ir_params p = request_params(S->cfg, n, R);
    bfx_ir_result ir{};
    if (status == BFX_OK)
      status = bfx_solve_ir(S->cfg.mode, n, R, dA, n, db, R, dx, R, &p, &ir, ws, wsb, st);
    if (status == BFX_OK || status == BFX_NOT_CONVERGED || status == BFX_SINGULAR) {
      if (cudaMemcpyAsync(r->hx, dx, sizeof(double) * n * R, cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        status = BFX_ECUDA;
    } else {
      cudaStreamSynchronize(st);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      finish_request(S, r, status, ir);
      S->pool.free(r->off, r->bytes);
      S->running -= 1;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

BFX_API bfx_status bfx_server_create(bfx_server* out, const bfx_server_config* cfg) {
  if (!out || !cfg) return BFX_EINVAL;
  *out = nullptr;
  if (cfg->budget_bytes < (1u << 20) || cfg->max_inflight < 1 || cfg->max_inflight > 256)
    return BFX_EINVAL;
  if (cfg->mode != BFX_FP32 && bfx::mode_pieces(cfg->mode) == 0) return BFX_EINVAL;
  if (cfg->gmres < 0 || cfg->gmres > 2) return BFX_EINVAL;
  if (cfg->batch_max_n < 0 || cfg->batch_max_n > 1024 || cfg->batch_max < 0) return BFX_EINVAL;
  if (cfg->batch_max_n > 0 && cfg->mode == BFX_FP32) return BFX_EINVAL;  // batches need pieces
  auto* S = new bfx_server_impl();
  S->cfg = *cfg;
  if (S->cfg.nb <= 0) S->cfg.nb = 64;
  if (cudaGetDevice(&S->device) != cudaSuccess || !S->pool.init(cfg->budget_bytes)) {
    delete S;
    return BFX_ENOMEM;
  }
  // one-time per-device lookups happen here, before any worker runs
  if (!bfx::device_error_word() || bfx::current_num_sms() <= 0 || bfx::current_cc() <= 0) {
    S->pool.release();
    delete S;
    return BFX_ECUDA;
  }
  for (int i = 0; i < cfg->max_inflight; ++i) S->workers.emplace_back(worker_main, S);
  *out = S;
  return BFX_OK;
}

BFX_API bfx_status bfx_server_submit(bfx_server S, int64_t n, int64_t nrhs, const float* h_A,
                                     const double* h_b, double* h_x, int64_t* ticket) {
  if (!S || !ticket || n < 1 || nrhs < 1 || nrhs > (1 << 20) || !h_A || !h_b || !h_x) return BFX_EINVAL;
  if (n >= (1 << 30)) return BFX_EUNSUPPORTED;
  auto* r = new Request();
  r->n = n;
  r->nrhs = nrhs;
  r->hA = h_A;
  r->hb = h_b;
  r->hx = h_x;
  r->bytes = request_bytes(S->cfg, n, nrhs);
  if (r->bytes > S->pool.capacity()) {
    delete r;
    return BFX_ENOMEM;  // can never fit the budget
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->ticket = S->next_ticket++;
    S->all[r->ticket] = r;
    S->queue.push_back(r);
  }
  *ticket = r->ticket;
  S->cv_work.notify_one();
  return BFX_OK;
}

// Waits until the request is done (timeout_s < 0: no limit).  BFX_OK and the
// result when done (the ticket is then released); BFX_TIMEOUT if still pending.
BFX_API bfx_status bfx_server_wait(bfx_server S, int64_t ticket, bfx_request_result* out,
                                   double timeout_s) {
  if (!S || !out) return BFX_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return BFX_EINVAL;
  Request* r = it->second;
  auto pred = [&] { return r->done; };
  if (timeout_s < 0)
    S->cv_done.wait(lk, pred);
  else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
    return BFX_TIMEOUT;
  *out = r->res;
  S->all.erase(it);
  delete r;
  return BFX_OK;
}

BFX_API bfx_status bfx_server_stats(bfx_server S, bfx_server_stats_t* out) {
  if (!S || !out) return BFX_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  out->queued = static_cast<int32_t>(S->queue.size());
  out->running = S->running;
  out->peak_running = S->peak_running;
  out->batches = S->batches;
  out->pool_bytes = S->pool.capacity();
  out->used_bytes = S->pool.used();
  out->peak_used_bytes = S->peak_used;
  return BFX_OK;
}

BFX_API void bfx_server_destroy(bfx_server S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->all) delete kv.second;
  S->pool.release();
  delete S;
}

}  // extern "C"
