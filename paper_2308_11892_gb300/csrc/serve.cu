// Serving: continuous batching of independent CPTR-GMRES solves.
//
// Requests are copied at submission and queued (a full queue answers
// CPTR_ERR_AGAIN).  A request is admitted as soon as a slot is free and its
// estimated device footprint fits in what is left of the HBM budget (first
// come, first served: the head of the queue is admitted first, so large
// requests are not starved).  A slot is a worker thread with its own CUDA
// stream that builds the request's context (create, setup); requests that
// arrive while others are on the GPU start as soon as memory and a slot free
// up, and their kernels overlap on the device.  A large request is then
// solved by its slot.  A small one (at most batch_max_cells cells) is handed
// to the batcher and its slot moves on: the batcher solves every small
// request that is set up and waiting in one launch (cptr_solve_batch, one
// thread block per system), while the next ones gather for the launch after
// it.  Each request owns its hierarchy and Krylov state until it finishes;
// its result does not depend on what else runs (every reduction has a fixed
// order, and a system's batched result is the same in any batch).
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ctx.h"

namespace {
struct Request {
  uint64_t id = 0;
  int N = 0;
  std::vector<int32_t> rp, ci;
  std::vector<double> v, rhs, x;
  double tol = 0.0;
  int maxit = 0;
  size_t footprint = 0;
  cptr_ctx* ctx = nullptr;  // set up, waiting for the batcher
  cptr_status st = CPTR_PENDING;
  cptr_info info{};
  bool done = false;
};

size_t estimate_footprint(long long N, long long nnzb, const cptr_params& p) {
  bool mixed = p.precision == CPTR_MIXED;
  long long m = p.restart;
  long long b = nnzb * (128 + 128 + (mixed ? 64 : 128) + (mixed ? 32 : 64) + 12);
  b += 4 * nnzb * 12 * 3 * 2;               // AMG levels (FP64 + apply copies), C_op ~ 3
  b += nnzb * 160;                          // setup scratch (strength, SpGEMM tables)
  b += (2 * m + 3) * 4 * N * 8;             // Krylov basis V, Z and vectors
  b += 64 * N + (64ll << 20);               // schedules, small buffers, slack
  if (p.mgr) b += nnzb * 128 + 32 * N;      // the unreduced matrix and right-hand side
  return (size_t)b;
}

// Whether cptr_solve_batch runs contexts made with these parameters.
bool batchable(const cptr_params& p) {
  return (p.precond == CPTR_PREC_CPTR || p.precond == CPTR_PREC_ILU) && !p.mgr &&
         p.smoother == CPTR_SMOOTH_L1_JACOBI && p.restart <= 32;
}

// Copies n bytes from a host or device pointer into host memory.  Host
// inputs are copied with memcpy so that submission never waits on the GPU.
bool copy_in(void* dst, const void* src, size_t n) {
  if (n == 0) return true;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, src) != cudaSuccess) {
    cudaGetLastError();
    a.type = cudaMemoryTypeUnregistered;
  }
  if (a.type == cudaMemoryTypeDevice) {
    if (cudaMemcpy(dst, src, n, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  }
  std::memcpy(dst, src, n);
  return true;
}

constexpr int kMaxBatch = 1024;  // systems per batched launch
}  // namespace

struct cptr_server {
  std::mutex mu;
  std::condition_variable cv;   // workers: the queue, memory, stop
  std::condition_variable bcv;  // batcher: small requests set up, stop
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> reqs;
  std::vector<std::shared_ptr<Request>> ready;  // set up, waiting for a batch
  std::vector<std::thread> workers;
  std::thread batcher;
  cptr_params p{};
  size_t budget = 0, in_use = 0;
  int max_slots = 1;
  int max_queued = 4096;
  int batch_cells = 0;
  int dev = 0;
  int workers_left = 0;
  uint64_t next_id = 1;
  bool stop = false;
  std::string err;  // the last failed request's message

  void note_failure(const Request& r, cptr_ctx* c, cptr_status st) {
    std::string m = "request " + std::to_string(r.id) + " (" + std::to_string(r.N) +
                     " cells): " + cptr_status_str(st);
    const char* e = c ? cptr_last_error(c) : "";
    if (e && *e) m += std::string(": ") + e;
    std::lock_guard<std::mutex> lk(mu);
    err = m;
  }

  void finish(Request& r) {
    // the request's input copies are no longer needed
    std::vector<int32_t>().swap(r.rp);
    std::vector<int32_t>().swap(r.ci);
    std::vector<double>().swap(r.v);
  }

  void worker() {
    cudaSetDevice(dev);
    for (;;) {
      std::shared_ptr<Request> r;
      int small_limit = 0;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] {
          return stop || (!queue.empty() &&
                          (in_use + queue.front()->footprint <= budget || in_use == 0));
        });
        if (queue.empty()) {
          if (stop) break;
          continue;
        }
        r = queue.front();
        queue.pop_front();
        in_use += r->footprint;
        small_limit = batch_cells;
      }
      if (r->N <= small_limit && batchable(p)) {
        if (prepare(*r)) {
          {
            std::lock_guard<std::mutex> lk(mu);
            ready.push_back(r);
          }
          bcv.notify_one();
          continue;  // the batcher finishes it
        }
      } else {
        run(*r);
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= r->footprint;
        r->done = true;
      }
      cv.notify_all();
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      --workers_left;
    }
    bcv.notify_one();
  }

  cptr_params request_params(const Request& r) const {
    cptr_params q = p;
    q.tol = r.tol;
    q.maxit = r.maxit;
    q.tri_tune = 0;  // shapes rarely repeat, and blocks of other requests share the SMs
    return q;
  }

  // Creates and sets up a small request's context; false when that failed
  // (the request is then finished with the failure).
  bool prepare(Request& r) {
    r.x.assign(r.rhs.size(), 0.0);
    cptr_params q = request_params(r);
    cptr_ctx* c = nullptr;
    cptr_status st = cptr_create(&c, r.N, 4, r.rp.data(), r.ci.data(), r.v.data(), &q);
    if (st == CPTR_OK) st = cptr_setup(c);
    finish(r);
    if (st == CPTR_OK) {
      r.ctx = c;
      return true;
    }
    if (c) cptr_get_info(c, &r.info);
    r.info.status = st;
    r.st = st;
    note_failure(r, c, st);
    cptr_destroy(c);
    return false;
  }

  void run(Request& r) {
    cptr_ctx* c = nullptr;
    r.x.assign(r.rhs.size(), 0.0);
    cptr_params q = request_params(r);
    cptr_status st = cptr_create(&c, r.N, 4, r.rp.data(), r.ci.data(), r.v.data(), &q);
    if (st == CPTR_OK) st = cptr_setup(c);
    if (st == CPTR_OK) st = cptr_solve(c, r.rhs.data(), r.x.data(), r.tol, r.maxit, &r.info);
    else if (c) cptr_get_info(c, &r.info);
    r.info.status = st;
    r.st = st;
    if (st != CPTR_OK && st != CPTR_ERR_MAXIT) note_failure(r, c, st);
    cptr_destroy(c);
    finish(r);
  }

  void batch_loop() {
    cudaSetDevice(dev);
    for (;;) {
      std::vector<std::shared_ptr<Request>> b;
      {
        std::unique_lock<std::mutex> lk(mu);
        bcv.wait(lk, [&] { return !ready.empty() || (stop && workers_left == 0); });
        if (ready.empty()) return;
        const size_t n = std::min<size_t>(ready.size(), kMaxBatch);
        b.assign(ready.begin(), ready.begin() + n);
        ready.erase(ready.begin(), ready.begin() + n);
      }
      const int n = (int)b.size();
      std::vector<cptr_ctx*> cs(n);
      std::vector<const double*> rhs(n);
      std::vector<double*> xs(n);
      std::vector<cptr_info> infos(n);
      for (int k = 0; k < n; ++k) {
        cs[k] = b[k]->ctx;
        rhs[k] = b[k]->rhs.data();
        xs[k] = b[k]->x.data();
      }
      // tol and maxit <= 0: each context's own (the request's)
      cptr_status st = cptr_solve_batch(cs.data(), n, rhs.data(), xs.data(), 0.0, 0, infos.data());
      const bool launched = st == CPTR_OK || st == CPTR_ERR_MAXIT || st == CPTR_ERR_BREAKDOWN;
      for (int k = 0; k < n; ++k) {
        Request& r = *b[k];
        if (launched) {
          r.info = infos[k];
          r.st = (cptr_status)infos[k].status;
        } else {
          cptr_get_info(r.ctx, &r.info);
          r.st = st;
          r.info.status = st;
          note_failure(r, cs[0], st);
        }
        cptr_destroy(r.ctx);
        r.ctx = nullptr;
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        for (auto& r : b) {
          in_use -= r->footprint;
          r->done = true;
        }
      }
      cv.notify_all();
    }
  }
};

extern "C" {

cptr_status cptr_server_create(cptr_server** out, size_t hbm_budget_bytes, int max_slots,
                               const cptr_params* params) {
  if (!out || max_slots < 1 || hbm_budget_bytes == 0) return CPTR_ERR_INVALID;
  cptr_server* s = new cptr_server();
  if (params) s->p = *params; else cptr_params_default(&s->p);
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  if (cudaGetDevice(&s->dev) != cudaSuccess) { cudaGetLastError(); delete s; return CPTR_ERR_CUDA; }
  s->workers_left = max_slots;
  for (int k = 0; k < max_slots; ++k) s->workers.emplace_back([s] { s->worker(); });
  s->batcher = std::thread([s] { s->batch_loop(); });
  *out = s;
  return CPTR_OK;
}

cptr_status cptr_server_set_limits(cptr_server* s, int max_queued, int batch_max_cells) {
  if (!s || max_queued < 1 || batch_max_cells < 0) return CPTR_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  s->max_queued = max_queued;
  s->batch_cells = batchable(s->p) ? batch_max_cells : 0;
  return batch_max_cells > 0 && !batchable(s->p) ? CPTR_ERR_INVALID : CPTR_OK;
}

cptr_status cptr_submit(cptr_server* s, int32_t n_cells, const int32_t* rowptr,
                        const int32_t* col, const double* vals, const double* rhs, double tol,
                        int maxit, uint64_t* req_id) {
  if (!s || n_cells <= 0 || !rowptr || !col || !vals || !rhs || !req_id) return CPTR_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return CPTR_ERR_INVALID;
    if ((int)s->queue.size() >= s->max_queued) return CPTR_ERR_AGAIN;
  }
  auto r = std::make_shared<Request>();
  r->N = n_cells;
  r->rp.resize(n_cells + 1);
  if (!copy_in(r->rp.data(), rowptr, sizeof(int32_t) * (n_cells + 1))) return CPTR_ERR_INVALID;
  long long nnzb = r->rp[n_cells];
  if (r->rp[0] != 0 || nnzb < n_cells) return CPTR_ERR_INVALID;
  r->ci.resize(nnzb);
  r->v.resize(16 * nnzb);
  r->rhs.resize(4 * (size_t)n_cells);
  if (!copy_in(r->ci.data(), col, sizeof(int32_t) * nnzb) ||
      !copy_in(r->v.data(), vals, sizeof(double) * 16 * nnzb) ||
      !copy_in(r->rhs.data(), rhs, sizeof(double) * 4 * (size_t)n_cells))
    return CPTR_ERR_INVALID;
  r->tol = tol > 0 ? tol : s->p.tol;
  r->maxit = maxit > 0 ? maxit : s->p.maxit;
  r->footprint = estimate_footprint(n_cells, nnzb, s->p);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return CPTR_ERR_INVALID;
    if ((int)s->queue.size() >= s->max_queued) return CPTR_ERR_AGAIN;
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    *req_id = r->id;
  }
  s->cv.notify_all();
  return CPTR_OK;
}

cptr_status cptr_poll(cptr_server* s, uint64_t req_id, double* x_out, cptr_info* info) {
  if (!s) return CPTR_ERR_INVALID;
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return CPTR_ERR_INVALID;
    r = it->second;
    if (!r->done) return CPTR_PENDING;
    s->reqs.erase(it);
  }
  if (x_out && !r->x.empty())
    std::memcpy(x_out, r->x.data(), sizeof(double) * r->x.size());
  if (info) *info = r->info;
  return r->st;
}

const char* cptr_server_last_error(cptr_server* s) {
  if (!s) return "";
  std::lock_guard<std::mutex> lk(s->mu);
  return s->err.c_str();
}

void cptr_server_destroy(cptr_server* s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // let queued work finish first
    s->cv.wait(lk, [&] { return s->queue.empty(); });
    s->stop = true;
  }
  s->cv.notify_all();
  for (auto& t : s->workers) t.join();
  s->bcv.notify_all();
  s->batcher.join();
  delete s;
}

}  // extern "C"
