// C ABI of libcptr (declared in include/cptr.h): context lifetime, setup,
// solve, single-step entry points and inspection.
#include <algorithm>
#include <chrono>
#include <thread>
#include <utility>
#include <cstring>
#include <cstdio>
#include <cstdlib>
#include <new>

#include "common.cuh"
#include "ctx.h"

// ------------------------------------------------------------------ helpers
thread_local cudaStream_t t_setup_stream = nullptr;

namespace {
// The host-mapped cycle-end flags come from a process-wide pool of pinned
// pages that is never returned: allocating and freeing pinned host memory
// synchronises with the device, which would serialise contexts that other
// threads create and destroy (a server's slots) behind every kernel running.
// One flag per 64-byte line, so that contexts do not share a line.
constexpr int kFlagStride = 16, kFlagsPerPage = 1024;
std::mutex g_flag_mu;
std::vector<std::pair<int*, int*>> g_flag_free;  // (host, device) addresses

cudaError_t flag_acquire(int** host, int** dev) {
  std::lock_guard<std::mutex> lk(g_flag_mu);
  if (g_flag_free.empty()) {
    int* hp = nullptr;
    int* dp = nullptr;
    cudaError_t e = cudaHostAlloc((void**)&hp, sizeof(int) * kFlagStride * kFlagsPerPage,
                                  cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) return e;
    e = cudaHostGetDevicePointer((void**)&dp, (void*)hp, 0);
    if (e != cudaSuccess) {
      cudaFreeHost(hp);
      return e;
    }
    for (int k = kFlagsPerPage - 1; k >= 0; --k)
      g_flag_free.emplace_back(hp + k * kFlagStride, dp + k * kFlagStride);
  }
  *host = g_flag_free.back().first;
  *dev = g_flag_free.back().second;
  g_flag_free.pop_back();
  return cudaSuccess;
}

void flag_release(int* host, int* dev) {
  std::lock_guard<std::mutex> lk(g_flag_mu);
  g_flag_free.emplace_back(host, dev);
}
}  // namespace

void* ctx_alloc(cptr_ctx* c, size_t bytes, bool setup_lifetime) {
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, cs(c));
  std::lock_guard<std::mutex> lk(c->mu);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    c->err = "device allocation of " + std::to_string(bytes) + " bytes failed";
    return nullptr;
  }
  (setup_lifetime ? c->allocs_setup : c->allocs_create).push_back(p);
  return p;
}

void ctx_set_err(cptr_ctx* c, const char* msg) {
  std::lock_guard<std::mutex> lk(c->mu);
  c->err = msg;
}

cptr_status ctx_cuda_fail(cptr_ctx* c, cudaError_t e, const char* what) {
  std::lock_guard<std::mutex> lk(c->mu);
  c->err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? CPTR_ERR_NOMEM : CPTR_ERR_CUDA;
}

cptr_status ctx_check_device_status(cptr_ctx* c) {
  int st = 0;
  CTX_CUDA(c, cudaMemcpyAsync(&st, &c->ctl->status, sizeof(int), cudaMemcpyDeviceToHost,
                              cs(c)));
  CTX_CUDA(c, cudaStreamSynchronize(cs(c)));
  CTX_CUDA(c, cudaGetLastError());
  if (st == DEV_TIMEOUT) {
    ctx_set_err(c, "a bounded device-side wait gave up");
    return CPTR_ERR_TIMEOUT;
  }
  if (st == DEV_BREAKDOWN) {
    ctx_set_err(c, "zero or non-finite pivot (decoupling, ILU(0) or coarse solve)");
    return CPTR_ERR_BREAKDOWN;
  }
  return CPTR_OK;
}

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Phase class of a ctx_phase name (its leading words).
static int phase_class(const char* name) {
  while (*name == ' ') ++name;
  auto is = [name](const char* p) { return strncmp(name, p, strlen(p)) == 0; };
  if (is("decouple") || is("mgr")) return CPTR_PHASE_DECOUPLE;
  if (is("strength")) return CPTR_PHASE_STRENGTH;
  if (is("pmis")) return CPTR_PHASE_PMIS;
  if (is("interp") || is("aggregate") || is("transpose")) return CPTR_PHASE_INTERP;
  if (is("spgemm")) return CPTR_PHASE_SPGEMM;
  if (is("coarse")) return CPTR_PHASE_COARSE;
  if (is("ilu")) return CPTR_PHASE_ILU;
  if (is("apply")) return CPTR_PHASE_BUFFERS;
  return -1;  // totals ("amg (total)") are not a phase of their own
}

void ctx_phase(cptr_ctx* c, const char* name) {
  if (!(c->timing || c->phase_on) || t_setup_stream) return;  // (main setup thread only)
  cudaStreamSynchronize(c->stream);
  double t = now_s();
  if (name) {
    if (c->timing) fprintf(stderr, "[cptr] %-28s %9.3f ms\n", name, 1e3 * (t - c->phase_t0));
    int k = phase_class(name);
    if (k >= 0) c->phase_ms[k] += 1e3 * (t - c->phase_t0);
  }
  c->phase_t0 = t;
}

void swap_stage(cptr_ctx* c) {
  StageStore& s = c->st2;
  std::swap(c->lev, s.lev);
  std::swap(c->W64, s.W64);
  std::swap(c->Wt, s.Wt);
  std::swap(c->AE, s.AE);
  std::swap(c->Cinv, s.Cinv);
  std::swap(c->ncoarse, s.ncoarse);
  std::swap(c->op_complexity, s.op_complexity);
  std::swap(c->rhat, s.rhat);
  std::swap(c->zc, s.zc);
  std::swap(c->se0, s.e0);
  std::swap(c->se1, s.e1);
}

static void free_list(cptr_ctx* c, std::vector<void*>& l) {
  for (void* p : l) cudaFreeAsync(p, c->stream);
  l.clear();
}

static void reset_setup_state(cptr_ctx* c) {
  krylov_release_graph(c);
  free_list(c, c->allocs_setup);
  c->lev.clear();
  c->W64 = nullptr; c->Wt = nullptr; c->AE = nullptr; c->Cinv = nullptr; c->ncoarse = 0;
  c->LU64 = nullptr; c->lvl_f = c->lvl_b = nullptr; c->ord_f = c->ord_b = nullptr;
  c->loff_f = c->loff_b = nullptr;
  c->Lrp = c->Lci = nullptr; c->Lv = nullptr; c->Urp = c->Uci = nullptr; c->Uv = nullptr;
  c->Dinv = nullptr; c->rhat = c->zc = c->r2 = c->u = c->y2 = c->zt = nullptr;
  c->nlev_f = c->nlev_b = c->npos_f = c->npos_b = 0;
  c->tf = TriSched(); c->tb = TriSched(); c->cf = CluSched(); c->cb = CluSched();
  c->sf = StripSched(); c->sb = StripSched(); c->strip = false;
  c->chf = ChainSched(); c->chb = ChainSched(); c->chain = false;
  c->st2 = StageStore();
  c->strip_rf = c->strip_uf = c->strip_rb = c->strip_yb = nullptr;
  c->chunked = c->cluster = false;
  c->rhsf = c->rhsb = nullptr;
  c->op_complexity = 0.0;
  c->setup_done = false;
}

static cptr_status check_params(const cptr_params& p, std::string& why) {
  if (p.restart < 1 || p.restart > 63) { why = "restart must be in [1, 63]"; return CPTR_ERR_INVALID; }
  if (p.maxit < 0) { why = "maxit must be >= 0"; return CPTR_ERR_INVALID; }
  if (!(p.tol >= 0.0)) { why = "tol must be >= 0"; return CPTR_ERR_INVALID; }
  if (p.precision != CPTR_FP64 && p.precision != CPTR_MIXED) { why = "bad precision"; return CPTR_ERR_INVALID; }
  if (p.precond < CPTR_PREC_NONE || p.precond > CPTR_PREC_CPTR3) { why = "bad precond"; return CPTR_ERR_INVALID; }
  if (p.precond == CPTR_PREC_CPTR3 && p.e1 < 0) { why = "CPTR3 needs two elliptic unknowns"; return CPTR_ERR_INVALID; }
  if (p.e0 < 0 || p.e0 > 3 || p.e1 < -1 || p.e1 > 3 || p.e0 == p.e1) { why = "bad elliptic unknowns"; return CPTR_ERR_INVALID; }
  if (p.pmax < 1 || p.pmax > 64) { why = "pmax must be in [1, 64]"; return CPTR_ERR_INVALID; }
  if (p.max_coarse < 1 || p.max_levels < 1) { why = "bad coarsening limits"; return CPTR_ERR_INVALID; }
  if (!(p.theta >= 0.0 && p.theta <= 1.0)) { why = "theta must be in [0, 1]"; return CPTR_ERR_INVALID; }
  if (p.mgr != 0 && p.mgr != 1) { why = "mgr must be 0 or 1"; return CPTR_ERR_INVALID; }
  if (p.agg < 0 || p.agg > 2) { why = "agg must be 0, 1 or 2"; return CPTR_ERR_INVALID; }
  if (p.nu_pre < 0 || p.nu_pre > 8 || p.nu_post < 0 || p.nu_post > 8) { why = "nu_pre and nu_post must be in [0, 8]"; return CPTR_ERR_INVALID; }
  if (p.smoother != CPTR_SMOOTH_L1_JACOBI && p.smoother != CPTR_SMOOTH_HYBRID_GS) { why = "bad smoother"; return CPTR_ERR_INVALID; }
  if (p.tri_tune != 0 && p.tri_tune != 1) { why = "tri_tune must be 0 or 1"; return CPTR_ERR_INVALID; }
  if (p.coarsen != CPTR_COARSEN_PMIS && p.coarsen != CPTR_COARSEN_HMIS) { why = "bad coarsen"; return CPTR_ERR_INVALID; }
  if (p.mgr && (p.e0 == 2 || p.e1 == 2)) { why = "mgr eliminates unknown 2: it cannot be elliptic"; return CPTR_ERR_INVALID; }
  return CPTR_OK;
}

// ------------------------------------------------------------------ ABI
extern "C" {

void cptr_params_default(cptr_params* p) {
  if (!p) return;
  p->restart = 30;
  p->maxit = 200;
  p->tol = 1e-6;
  p->precision = CPTR_FP64;
  p->theta = 0.25;
  p->pmax = 4;
  p->max_coarse = 256;
  p->max_levels = 25;
  p->precond = CPTR_PREC_CPTR;
  p->use_graphs = 1;
  p->seed = 0x5eed;
  p->e0 = 0;
  p->e1 = 3;
  p->mgr = 0;
  p->agg = 0;
  p->nu_pre = 1;
  p->nu_post = 1;
  p->smoother = CPTR_SMOOTH_L1_JACOBI;
  p->tri_tune = 1;
  p->coarsen = CPTR_COARSEN_PMIS;
}

const char* cptr_status_str(cptr_status s) {
  switch (s) {
    case CPTR_OK: return "ok";
    case CPTR_ERR_INVALID: return "invalid argument";
    case CPTR_ERR_NOMEM: return "out of device memory";
    case CPTR_ERR_CUDA: return "CUDA error";
    case CPTR_ERR_MAXIT: return "maximum iterations reached";
    case CPTR_ERR_BREAKDOWN: return "numerical breakdown";
    case CPTR_ERR_TIMEOUT: return "device wait timed out";
    case CPTR_ERR_AGAIN: return "try again";
    case CPTR_PENDING: return "pending";
  }
  return "unknown status";
}

const char* cptr_last_error(const cptr_ctx* c) { return c ? c->err.c_str() : "null context"; }

void cptr_destroy(cptr_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  krylov_release_graph(c);
  free_list(c, c->allocs_setup);
  free_list(c, c->allocs_create);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->hflag) flag_release((int*)c->hflag, c->hflag_dev);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->stream2) cudaStreamDestroy(c->stream2);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

cptr_status cptr_create(cptr_ctx** out, int32_t n_cells, int32_t bs, const int32_t* rowptr,
                        const int32_t* col, const double* vals, const cptr_params* params) {
  if (!out) return CPTR_ERR_INVALID;
  *out = nullptr;
  if (n_cells <= 0 || bs != 4 || !rowptr || !col || !vals) return CPTR_ERR_INVALID;
  // 32-bit counts throughout: the first AMG level holds 4 entries per block
  constexpr int32_t kMaxCount = INT32_MAX / 4;
  if (n_cells > kMaxCount) return CPTR_ERR_INVALID;
  cptr_ctx* c = new (std::nothrow) cptr_ctx();
  if (!c) return CPTR_ERR_NOMEM;
  if (params) c->p = *params; else cptr_params_default(&c->p);
  std::string why;
  if (check_params(c->p, why) != CPTR_OK) { delete c; return CPTR_ERR_INVALID; }
  c->mixed = c->p.precision == CPTR_MIXED;
  {
    const char* tm = getenv("CPTR_TIMING");
    c->timing = tm && tm[0] == '1';
    const char* fb = getenv("CPTR_SETUP_FALLBACK");
    c->force_fallback = fb && fb[0] == '1';
    const char* sp = getenv("CPTR_SPGEMM_PATH");
    c->spgemm_path = sp ? atoi(sp) : 0;
    const char* ip = getenv("CPTR_INTERP_PATH");
    c->interp_path = ip ? atoi(ip) : 0;
    const char* sp_ = getenv("CPTR_STRIP_P");
    c->strip_p = sp_ ? std::max(0, atoi(sp_)) : 0;
    const char* rc_ = getenv("CPTR_STRIP_RC");
    c->strip_rc = rc_ ? std::max(0, atoi(rc_)) : 0;
    const char* rg_ = getenv("CPTR_STRIP_RING");
    c->strip_ring = rg_ ? std::max(0, atoi(rg_)) : 0;
    const char* lg_ = getenv("CPTR_LVL_GRID");
    c->lvl_grid_forced = lg_ ? std::max(0, atoi(lg_)) : 0;
  }
  c->N = n_cells;
  cudaError_t e = cudaGetDevice(&c->dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) { cudaGetLastError(); delete c; return CPTR_ERR_CUDA; }
  c->stream = c->own_stream;
  {
    // keep freed stream-ordered memory in the pool for the next setup
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, c->dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  }
  int32_t ends[2] = {0, 0};
  e = cudaMemcpy(&ends[0], rowptr, sizeof(int32_t), cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(&ends[1], rowptr + n_cells, sizeof(int32_t), cudaMemcpyDefault);
  if (e != cudaSuccess) { cudaGetLastError(); cptr_destroy(c); return CPTR_ERR_INVALID; }
  if (ends[0] != 0 || ends[1] < n_cells || ends[1] > kMaxCount) {
    cptr_destroy(c);
    return CPTR_ERR_INVALID;
  }
  c->nnzb = ends[1];
  cptr_status st = CPTR_OK;
  c->rp = (int32_t*)ctx_alloc(c, sizeof(int32_t) * (n_cells + 1), false);
  c->ci = (int32_t*)ctx_alloc(c, sizeof(int32_t) * (size_t)c->nnzb, false);
  c->diag = (int32_t*)ctx_alloc(c, sizeof(int32_t) * (size_t)n_cells, false);
  c->v = (double*)ctx_alloc(c, sizeof(double) * 16 * (size_t)c->nnzb, false);
  c->ctl = (Ctl*)ctx_alloc(c, sizeof(Ctl), false);
  if (!c->rp || !c->ci || !c->diag || !c->v || !c->ctl) { cptr_destroy(c); return CPTR_ERR_NOMEM; }
  if (c->p.mgr) {
    c->vfull = (double*)ctx_alloc(c, sizeof(double) * 16 * (size_t)c->nnzb, false);
    c->bfull = (double*)ctx_alloc(c, sizeof(double) * 4 * (size_t)n_cells, false);
    c->mgr_flag = (int*)ctx_alloc(c, sizeof(int), false);
    if (!c->vfull || !c->bfull || !c->mgr_flag) { cptr_destroy(c); return CPTR_ERR_NOMEM; }
  }
  double* vdst = c->p.mgr ? c->vfull : c->v;  // with mgr, v receives the reduced operator
  e = cudaMemcpyAsync(c->rp, rowptr, sizeof(int32_t) * (n_cells + 1), cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->ci, col, sizeof(int32_t) * (size_t)c->nnzb, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(vdst, vals, sizeof(double) * 16 * (size_t)c->nnzb, cudaMemcpyDefault, c->stream);
  Ctl h{};
  h.one = 1;
  h.m = c->p.restart;
  h.maxit = c->p.maxit;
  h.spin = c->spin_limit;
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    int* hf = nullptr;
    e = flag_acquire(&hf, &c->hflag_dev);
    c->hflag = hf;
  }
  if (e != cudaSuccess) { cudaGetLastError(); cptr_destroy(c); return CPTR_ERR_CUDA; }
  *c->hflag = 0;
  st = setup_validate(c);
  if (st == CPTR_OK) st = krylov_alloc(c);
  if (st == CPTR_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = CPTR_ERR_CUDA;
  if (st != CPTR_OK) { cptr_destroy(c); return st; }
  *out = c;
  return CPTR_OK;
}

cptr_status cptr_update_values(cptr_ctx* c, const double* vals) {
  if (!c || !vals) return CPTR_ERR_INVALID;
  CTX_CUDA(c, cudaMemcpyAsync(c->p.mgr ? c->vfull : c->v, vals,
                              sizeof(double) * 16 * (size_t)c->nnzb, cudaMemcpyDefault, c->stream));
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  reset_setup_state(c);
  return CPTR_OK;
}

cptr_status cptr_set_stream(cptr_ctx* c, void* stream) {
  if (!c) return CPTR_ERR_INVALID;
  cudaStream_t ns = stream ? (cudaStream_t)stream : c->own_stream;
  if (ns == c->stream) return CPTR_OK;
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  c->stream = ns;
  krylov_release_graph(c);  // graphs are replayed on any stream, but capture needs a fresh one
  return CPTR_OK;
}

cptr_status cptr_setup(cptr_ctx* c) {
  if (!c) return CPTR_ERR_INVALID;
  auto t0 = std::chrono::steady_clock::now();
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  reset_setup_state(c);
  CTX_CUDA(c, cudaMemsetAsync(&c->ctl->status, 0, sizeof(int), c->stream));
  for (double& v : c->phase_ms) v = 0.0;
  cptr_status st = CPTR_OK;
  if (c->p.mgr) {
    // the reduced operator replaces v before anything (both setup streams) reads it
    st = mgr_reduce(c);
    ctx_phase(c, "mgr reduction");
    if (st) return st;
  }
  const bool cptr3 = c->p.precond == CPTR_PREC_CPTR3;
  bool first = c->p.precond == CPTR_PREC_CPTR || c->p.precond == CPTR_PREC_FIRST || cptr3;
  bool second = c->p.precond == CPTR_PREC_CPTR || c->p.precond == CPTR_PREC_ILU || cptr3;
  // the first stage's elliptic unknowns: CPTR3 builds the pressure stage here
  // and its temperature stage after the ILU(0) setup has joined
  c->se0 = c->p.e0;
  c->se1 = cptr3 ? -1 : c->p.e1;
  ctx_phase(c, nullptr);
  if (first && second) {
    // ILU(0) of A does not depend on the AMG hierarchy: its level sets,
    // schedules and factorisation run on the second stream from their own
    // host thread (both setups synchronise with the host between phases)
    cptr_status ilu_st = CPTR_OK;
    bool sched_done = false;  // the solve schedule was built on the ILU thread too
    CTX_CUDA(c, cudaEventRecord(c->ev_fork, c->stream));
    auto ilu_work = [c, &ilu_st, &sched_done] {
      double tw = now_s();
      t_setup_stream = c->stream2;
      if (cudaSetDevice(c->dev) != cudaSuccess ||
          cudaStreamWaitEvent(c->stream2, c->ev_fork, 0) != cudaSuccess) {
        cudaGetLastError();
        ilu_st = CPTR_ERR_CUDA;
      } else {
        ilu_st = setup_ilu_factor(c);
        // a decided schedule is only built (nothing is timed): it can run here
        if (!ilu_st && tune_decided(c)) {
          ilu_st = setup_ilu_schedule(c);
          sched_done = true;
        }
      }
      if (cudaEventRecord(c->ev_join, c->stream2) != cudaSuccess && !ilu_st) ilu_st = CPTR_ERR_CUDA;
      if (c->phase_on) {
        cudaStreamSynchronize(c->stream2);
        c->phase_ms[CPTR_PHASE_ILU_CONCURRENT] = 1e3 * (now_s() - tw);
      }
      t_setup_stream = nullptr;
    };
    std::thread ilu;
    bool threaded = true;
    try {
      ilu = std::thread(ilu_work);
    } catch (...) {  // no thread available: the same work, after the AMG setup
      threaded = false;
    }
    st = setup_decouple(c);
    ctx_phase(c, "decouple");
    if (!st) st = setup_amg(c);
    ctx_phase(c, "amg (total)");
    if (threaded) ilu.join();
    else ilu_work();
    CTX_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    if (!st) st = ilu_st;
    if (!st && !sched_done) st = setup_ilu_schedule(c);
  } else {
    if (first) {
      st = setup_decouple(c);
      ctx_phase(c, "decouple");
      if (!st) st = setup_amg(c);
      ctx_phase(c, "amg (total)");
    }
    if (!st && second) st = setup_ilu(c);
  }
  ctx_phase(c, "ilu (total)");
  if (!st && cptr3) {
    // CPTR3's temperature stage (Section 3.3): its own decoupling onto T and a
    // scalar AMG, built in the first-stage fields and then stored aside
    c->st2 = StageStore();
    c->st2.e0 = c->p.e1;
    c->st2.e1 = -1;
    swap_stage(c);
    st = setup_decouple(c);
    ctx_phase(c, "decouple");
    if (!st) st = setup_amg(c);
    ctx_phase(c, "amg (total)");
    if (!st) st = setup_apply_buffers(c);
    swap_stage(c);
  }
  if (!st) st = setup_apply_buffers(c);
  ctx_phase(c, "apply buffers");
  if (!st) st = ctx_check_device_status(c);
  if (st) return st;
  c->setup_done = true;
  c->info.setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  c->info.amg_levels = (int)c->lev.size();
  c->info.ilu_levels = c->nlev_f;
  c->info.tri_schedule = c->cluster ? 1 : c->strip ? 2 : c->chain ? 3 : c->chunked ? c->tf.R : 0;
  c->info.op_complexity = c->op_complexity;
  return CPTR_OK;
}

cptr_status cptr_solve(cptr_ctx* c, const double* rhs, double* x, double tol, int maxit,
                       cptr_info* info) {
  if (!c || !rhs || !x) return CPTR_ERR_INVALID;
  if (!c->setup_done) { ctx_set_err(c, "cptr_setup has not been called"); return CPTR_ERR_INVALID; }
  if (tol <= 0.0) tol = c->p.tol;
  if (maxit <= 0) maxit = c->p.maxit;
  auto t0 = std::chrono::steady_clock::now();
  size_t nb = sizeof(double) * 4 * (size_t)c->N;
  CTX_CUDA(c, cudaMemcpyAsync(c->p.mgr ? c->bfull : c->bd, rhs, nb, cudaMemcpyDefault, c->stream));
  CTX_CUDA(c, cudaMemcpyAsync(c->xd, x, nb, cudaMemcpyDefault, c->stream));
  if (c->p.mgr) mgr_rhs(c);  // reduced rhs into bd; eliminated entries of x set to 0
  cptr_status st = krylov_solve(c, tol, maxit);
  if (c->p.mgr) mgr_recover(c);
  cudaError_t e = cudaMemcpyAsync(x, c->xd, nb, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess && st == CPTR_OK) st = ctx_cuda_fail(c, e, "copy of the solution");
  if (st == CPTR_OK || st == CPTR_ERR_MAXIT) {
    cptr_status d = ctx_check_device_status(c);
    if (d != CPTR_OK) st = d;
  }
  c->info.solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  c->info.status = st;
  c->info.launches = c->nlaunch;
  if (info) *info = c->info;
  return st;
}

cptr_status cptr_spmv(cptr_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return CPTR_ERR_INVALID;
  if (c->p.mgr && !c->setup_done) {
    ctx_set_err(c, "with mgr the operator is the reduced one, formed by cptr_setup");
    return CPTR_ERR_INVALID;
  }
  launch_spmv(c, x, false, y, nullptr);
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

cptr_status cptr_apply(cptr_ctx* c, int which, const double* in, double* out) {
  if (!c || !in || !out) return CPTR_ERR_INVALID;
  if (!c->setup_done) { ctx_set_err(c, "cptr_setup has not been called"); return CPTR_ERR_INVALID; }
  const bool cptr3 = c->p.precond == CPTR_PREC_CPTR3;
  bool first = c->p.precond == CPTR_PREC_CPTR || c->p.precond == CPTR_PREC_FIRST || cptr3;
  bool second = c->p.precond == CPTR_PREC_CPTR || c->p.precond == CPTR_PREC_ILU || cptr3;
  if ((which == CPTR_APPLY_ILU && !second) ||
      (which >= CPTR_APPLY_RESTRICT && which <= CPTR_APPLY_CORRECTION && !first)) {
    ctx_set_err(c, "this piece is not part of the configured preconditioner");
    return CPTR_ERR_INVALID;
  }
  return launch_apply_piece(c, which, in, out);
}

int cptr_amg_levels(const cptr_ctx* c) { return c ? (int)c->lev.size() : 0; }

cptr_status cptr_level_info(const cptr_ctx* c, int level, int32_t* info) {
  if (!c || !info || level < 0 || level >= (int)c->lev.size()) return CPTR_ERR_INVALID;
  const Level& L = c->lev[level];
  bool last = level == (int)c->lev.size() - 1;
  info[0] = L.A.n;
  info[1] = L.A.nnz;
  info[2] = last ? 0 : L.nc;
  info[3] = last ? 0 : L.P.nnz;
  return CPTR_OK;
}

cptr_status cptr_copy(const cptr_ctx* cc, int level, int what, void* dst) {
  cptr_ctx* c = const_cast<cptr_ctx*>(cc);
  if (!c || !dst || !c->setup_done) return CPTR_ERR_INVALID;
  const void* src = nullptr;
  size_t bytes = 0;
  if (what == CPTR_COPY_W || what == CPTR_COPY_ILU || what == CPTR_COPY_ILU_LEVEL) {
    if (what == CPTR_COPY_W) { src = c->W64; bytes = sizeof(double) * 4 * (size_t)c->N; }
    if (what == CPTR_COPY_ILU) { src = c->LU64; bytes = sizeof(double) * 16 * (size_t)c->nnzb; }
    if (what == CPTR_COPY_ILU_LEVEL) { src = c->lvl_f; bytes = sizeof(int32_t) * (size_t)c->N; }
  } else {
    if (level < 0 || level >= (int)c->lev.size()) return CPTR_ERR_INVALID;
    const Level& L = c->lev[level];
    bool last = level == (int)c->lev.size() - 1;
    switch (what) {
      case CPTR_COPY_A_ROWPTR: src = L.A.rp; bytes = sizeof(int32_t) * (L.A.n + 1); break;
      case CPTR_COPY_A_COL: src = L.A.ci; bytes = sizeof(int32_t) * (size_t)L.A.nnz; break;
      case CPTR_COPY_A_VAL: src = L.A.v; bytes = sizeof(double) * (size_t)L.A.nnz; break;
      case CPTR_COPY_P_ROWPTR: if (!last) { src = L.P.rp; bytes = sizeof(int32_t) * (L.P.n + 1); } break;
      case CPTR_COPY_P_COL: if (!last) { src = L.P.ci; bytes = sizeof(int32_t) * (size_t)L.P.nnz; } break;
      case CPTR_COPY_P_VAL: if (!last) { src = L.P.v; bytes = sizeof(double) * (size_t)L.P.nnz; } break;
      case CPTR_COPY_CF: if (!last) { src = L.cf; bytes = sizeof(int32_t) * (size_t)L.A.n; } break;
      case CPTR_COPY_DL1: if (!last) { src = L.dl1; bytes = sizeof(double) * (size_t)L.A.n; } break;
      default: return CPTR_ERR_INVALID;
    }
  }
  if (!src) return CPTR_ERR_INVALID;
  if (bytes == 0) return CPTR_OK;
  CTX_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  return CPTR_OK;
}

cptr_status cptr_set_spin_limit(cptr_ctx* c, unsigned polls) {
  if (!c) return CPTR_ERR_INVALID;
  c->spin_limit = polls ? polls : kSpinDefault;
  CTX_CUDA(c, cudaMemcpyAsync(&c->ctl->spin, &c->spin_limit, sizeof(unsigned),
                              cudaMemcpyHostToDevice, c->stream));
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  return CPTR_OK;
}

cptr_status cptr_setup_timing(cptr_ctx* c, int enable) {
  if (!c) return CPTR_ERR_INVALID;
  c->phase_on = enable != 0;
  return CPTR_OK;
}

cptr_status cptr_setup_phases(const cptr_ctx* c, double* ms) {
  if (!c || !ms) return CPTR_ERR_INVALID;
  for (int k = 0; k < CPTR_PHASE_COUNT; ++k) ms[k] = c->phase_ms[k];
  return CPTR_OK;
}

cptr_status cptr_get_info(const cptr_ctx* c, cptr_info* info) {
  if (!c || !info) return CPTR_ERR_INVALID;
  *info = c->info;
  info->launches = c->nlaunch;
  return CPTR_OK;
}

}  // extern "C"
