// Internal (non-ABI) definitions shared by the host code of libcptr.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "cptr.h"

// Device CSR (scalar), FP64 values.
struct DCSR {
  int n = 0, m = 0, nnz = 0;
  int32_t* rp = nullptr;
  int32_t* ci = nullptr;
  double* v = nullptr;
};

// One level of the system-AMG hierarchy.
struct Level {
  DCSR A;                   // FP64 level operator (setup result)
  int32_t* func = nullptr;  // unknown (function) tag per row
  int32_t* cf = nullptr;    // +1 coarse, -1 fine (non-coarsest levels)
  int32_t* cidx = nullptr;  // coarse index of each C point (non-coarsest levels)
  DCSR P, R;                // interpolation and its transpose (FP64)
  double* dl1 = nullptr;    // l1 diagonal (FP64)
  int nc = 0;
  // apply-precision copies (float in CPTR_MIXED, double in CPTR_FP64)
  void* Av = nullptr;
  void* Pv = nullptr;
  void* Rv = nullptr;
  void* dinv = nullptr;
  // work vectors in apply precision
  void* b = nullptr;
  void* x = nullptr;
  void* r = nullptr;
  void* x2 = nullptr;
  void* t = nullptr;  // second smoothing iterate (V(nu_pre, nu_post) sweeps)
  int lanes = 4;  // lanes per row for the level's row-parallel kernels
};

// Schedule and factor arrays of one chunked triangular solve: rows are cut
// into chunks of R consecutive rows (from the top for the lower triangle,
// from the bottom for the upper one); inside a chunk rows are listed by their
// level in the chunk-local dependency graph.
struct TriSched {
  int R = 0;                 // rows per chunk
  int nch = 0;               // chunks
  int cap_blocks = 0;        // factor blocks a chunk may stage in shared memory
  int lev_cap = 0;           // most local levels in one chunk
  size_t smem = 0;           // dynamic shared memory of the solve kernel
  int32_t* clp = nullptr;    // chunk -> first level index
  int32_t* lvp = nullptr;    // level -> first schedule position
  int32_t* ord = nullptr;    // schedule position -> row
  int32_t* rp = nullptr;     // factor blocks per position (CSR over positions)
  int32_t* ci = nullptr;
  void* v = nullptr;         // blocks, apply precision
  void* dinv = nullptr;      // inv(U_ii) per position (upper only)
  long long nnz = 0;
};

// Level-synchronous schedule of one triangular solve on a thread-block
// cluster: rows listed level by level, each level cut into nq contiguous
// slices (one per CTA of the cluster), factor blocks in position order.
struct CluSched {
  int nq = 0;                // CTAs in the cluster
  int nlev = 0;
  int rows_cap = 0;          // most rows of one slice
  int blk_cap = 0;           // most factor blocks of one slice
  size_t smem = 0;           // dynamic shared memory of the solve kernel
  int4* desc = nullptr;      // [nq][nlev] {first pos, end pos, first block, end block}
  int32_t* ord = nullptr;    // position -> row
  int32_t* pos = nullptr;    // row -> position
  int32_t* rp = nullptr;     // factor blocks per position (CSR over positions)
  int32_t* ci = nullptr;
  void* v = nullptr;         // blocks, apply precision
  void* dinv = nullptr;      // inv(U_ii) per position (upper only)
  int32_t* pos2 = nullptr;   // forward only: backward position of each position's row
  int32_t* loc = nullptr;    // per block: (owner CTA << 24) | slot of its dependency
  int ycap = 0;              // most rows one CTA owns (solution slots in shared memory)
  int32_t* dest = nullptr;   // [nq][ycap] output index of every slot (-1 unused)
  long long nnz = 0;         // factor blocks
};

// Strip-owned schedule of one triangular solve (large systems): rows cut into
// P contiguous index strips, one CTA each, walked level by level in steps that
// a producer warp stages into shared memory.
struct StripSched {
  int P = 0;                 // strips (CTAs)
  int S = 0;                 // rows per strip
  int RC = 0;                // rows of the shared-memory solution ring
  int nsteps = 0;
  unsigned ring_bytes = 0;   // staging ring of the solve kernel
  size_t smem = 0;           // dynamic shared memory of the solve kernel
  int32_t* sptr = nullptr;   // [P+1] steps of each strip
  int4* step = nullptr;      // [nsteps] {first pos, end pos, first block, end block}
  int4* meta = nullptr;      // [N] per position {row, block range in step, other position}
  int32_t* loc = nullptr;    // per block: ring slot (high bit set) or global position
  void* v = nullptr;         // blocks, apply precision
  void* dinv = nullptr;      // inv(U_ii) per position (upper only)
  int32_t* ord = nullptr;    // position -> row
  int32_t* pos = nullptr;    // row -> position
  long long nnz = 0;         // factor blocks
  long long nblk_padded = 0; // blocks including per-step padding
};

// Chain schedule of one triangular solve: rows linked into chains (each row
// follows its dependency of highest level), one quad walking each chain.
struct ChainSched {
  int nchains = 0;
  int32_t* cptr = nullptr;   // [nchains+1] first position of each chain
  int4* meta = nullptr;      // [N] per position {row, first block, blocks, predecessor slot}
  int32_t* ci = nullptr;     // per block: dependency row
  void* v = nullptr;         // blocks, apply precision
  void* dinv = nullptr;      // inv(U_ii) per position (upper only)
  long long nnz = 0;
};

// Device-resident control block of one context.
struct Ctl {
  int j;          // Arnoldi column of the step being executed
  int active;     // 1 while the current restart cycle continues
  int k;          // columns completed in the current cycle
  int iters;      // total GMRES iterations
  int maxit;
  int m;          // restart length
  int status;     // DEV_* error word
  int conv;       // 1 once the residual estimate met the tolerance
  int zero;       // constant 0 (column index for single applications)
  int one;        // constant 1 ("active" flag for single applications)
  int pad[2];
  double bnorm, tol_abs, beta, hn;
  unsigned red_ctr[8];  // tickets of the last-block reductions
  unsigned fwd_ctr;     // work counters of the sync-free triangular solves
  unsigned bwd_ctr;
  unsigned fac_ctr;     // work counter of the ILU(0) factorisation
  unsigned spin;        // polls a triangular-solve dependency wait makes before giving up
};

// Arnoldi column at which the CGS2 multi-dot is profiled: the average column
// of the last solve (half the columns its longest cycle used), restart/2 before
// any solve.
inline int mdot_profile_column(const cptr_info& info, int restart) {
  int cols = info.iters > 0 ? (info.iters < restart ? info.iters : restart) : restart;
  return cols / 2;
}

// Default number of polls before a triangular-solve dependency wait gives up.
constexpr unsigned kSpinDefault = 1u << 21;


// The temperature stage of CPTR3 (a second decoupled first stage), kept aside
// while the pressure stage occupies the context's first-stage fields.
struct StageStore {
  std::vector<Level> lev;
  double* W64 = nullptr;
  void* Wt = nullptr;
  void* AE = nullptr;
  double* Cinv = nullptr;
  int ncoarse = 0;
  double op_complexity = 0.0;
  void* rhat = nullptr;
  void* zc = nullptr;
  int e0 = 3, e1 = -1;  // its elliptic unknowns
};

struct cptr_ctx {
  int N = 0, nnzb = 0;
  cptr_params p{};
  // elliptic unknowns of the first stage being built or applied: p.e0/p.e1,
  // or one unknown at a time for CPTR3 (see swap_stage)
  int se0 = 0, se1 = 3;
  StageStore st2;  // CPTR3's temperature stage
  bool mixed = false;
  int dev = 0, nsm = 0;
  // A kernel's dynamic shared-memory limit is one setting per process, not per
  // context: a kernel whose launches differ in size raises it to the device's
  // per-block maximum, never to the size of one launch, so that a context
  // launching with more shared memory cannot find the limit lowered by another
  // context's setup running in another thread.
  int smem_optin = 48 * 1024;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  // second stream: the ILU(0) setup runs on it, from its own host thread,
  // beside the AMG setup on `stream`
  cudaStream_t stream2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // matrix (device, FP64)
  int32_t* rp = nullptr;
  int32_t* ci = nullptr;
  int32_t* diag = nullptr;  // position of the diagonal block per row
  double* v = nullptr;      // the operator GMRES works on (reduced when p.mgr)
  // first MGR reduction (p.mgr): the given matrix, the given right-hand side
  // and the reduction's status word
  double* vfull = nullptr;
  double* bfull = nullptr;
  int* mgr_flag = nullptr;

  // decoupling
  double* W64 = nullptr;  // N x 4 (2x2 row-major per cell)
  void* Wt = nullptr;     // apply-precision copy
  void* AE = nullptr;     // nnzb x 8: E columns of A (4x2 per block), apply precision

  // system AMG
  std::vector<Level> lev;
  int ncoarse = 0;
  double* Cinv = nullptr;  // dense inverse of the coarsest operator (FP64)
  double op_complexity = 0.0;

  // ILU(0)
  double* LU64 = nullptr;  // nnzb x 16 factors in the input block order
  int32_t* lvl_f = nullptr;
  int32_t* lvl_b = nullptr;
  int nlev_f = 0, nlev_b = 0;
  int npos_f = 0, npos_b = 0;          // padded schedule lengths
  int32_t* ord_f = nullptr;            // schedule position -> row (-1 = padding)
  int32_t* ord_b = nullptr;
  int32_t* loff_f = nullptr;           // first schedule position of each level (nlev + 1)
  int32_t* loff_b = nullptr;
  int32_t* Lrp = nullptr;              // strictly lower blocks in forward order
  int32_t* Lci = nullptr;
  void* Lv = nullptr;
  int32_t* Urp = nullptr;              // strictly upper blocks in backward order
  int32_t* Uci = nullptr;
  void* Uv = nullptr;
  void* Dinv = nullptr;                // inv(U_ii) in backward order
  long long nnzL = 0, nnzU = 0;        // strictly lower / upper blocks
  TriSched tf, tb;                     // chunked forward / backward solves
  bool chunked = false;                // use tf/tb (else the level-padded kernels)
  CluSched cf, cb;                     // cluster forward / backward solves
  bool cluster = false;                // use cf/cb
  ChainSched chf, chb;                 // chain forward / backward solves
  bool chain = false;                  // use chf/chb
  StripSched sf, sb;                   // strip forward / backward solves
  bool strip = false;                  // use sf/sb
  void* strip_rf = nullptr;            // 4N: forward rhs in forward position order
  void* strip_uf = nullptr;            // 4N: forward output (polled), forward position order
  void* strip_rb = nullptr;            // 4N: backward rhs in backward position order
  void* strip_yb = nullptr;            // 4N: backward output (polled), backward position order
  void* rhsf = nullptr;                // 4N: forward rhs in forward level order (cluster path)
  void* rhsb = nullptr;                // 4N: backward rhs in backward level order (cluster path)
  unsigned spin_limit = kSpinDefault;  // Ctl::spin of every later solve (cptr_set_spin_limit)
  int tuned_R = -1;                    // autotuned schedule: -1 not tuned, 0 level kernels,
                                       // 1 cluster, 2 strips, 3 chains, > 3 chunk rows
  int fac_epoch = 0;
  int32_t* fac_done = nullptr;
  void* flush_buf = nullptr;           // 256 MiB buffer written to flush L2 (profiling)

  // preconditioner work vectors (apply precision)
  void* rhat = nullptr;  // 2N
  void* zc = nullptr;    // 2N: V-cycle output
  void* r2 = nullptr;    // 4N
  void* u = nullptr;     // 4N forward solve output
  void* y2 = nullptr;    // 4N backward solve output
  void* zt = nullptr;    // 4N preconditioner output for single applications

  // Krylov (FP64 except Z in CPTR_MIXED)
  double* V = nullptr;     // (m+1) x 4N
  void* Z = nullptr;       // m x 4N
  double* w = nullptr;     // 4N
  double* xd = nullptr;    // 4N solution
  double* bd = nullptr;    // 4N rhs
  double* H = nullptr;     // (m+1) x m, column-major (rotated)
  double* cs = nullptr;
  double* sn = nullptr;
  double* g = nullptr;
  double* yv = nullptr;
  double* h1 = nullptr;
  double* h2 = nullptr;
  double* part = nullptr;  // NB x (m+1) reduction partials
  int NB = 0;              // blocks of the Krylov kernels
  int NBd = 0;             // blocks of the CGS2 dot and norm kernels (one wave of their own)
  Ctl* ctl = nullptr;
  volatile int* hflag = nullptr;  // mapped host mirror of ctl->active
  int* hflag_dev = nullptr;

  // CUDA graph of one Arnoldi step
  cudaGraphExec_t step_exec = nullptr;

  // bookkeeping
  std::atomic<long long> nlaunch{0};  // kernels launched by this context
  long long step_kernels = 0;  // kernel nodes of the captured Arnoldi step
  std::vector<void*> allocs_create;  // freed by cptr_destroy
  std::vector<void*> allocs_setup;   // freed by the next cptr_setup / destroy
  cptr_info info{};
  std::string err;
  std::mutex mu;  // guards err and the allocation lists (two setup threads)
  bool setup_done = false;
  bool timing = false;  // CPTR_TIMING=1: print setup phase times to stderr
  bool phase_on = false;  // cptr_setup_timing: record setup phase wall times
  double phase_ms[CPTR_PHASE_COUNT] = {};  // per phase, last cptr_setup
  bool force_fallback = false;  // CPTR_SETUP_FALLBACK=1: thread-per-row setup kernels only
  // test hooks: one SpGEMM path for every row (CPTR_SPGEMM_PATH: 1 ordered-table
  // block kernel, 2 bucketed block kernel, 3 global-scratch kernel) and one
  // ext+i path (CPTR_INTERP_PATH: 1 wide blocks, 2 global-scratch kernel)
  int spgemm_path = 0, interp_path = 0;
  // test hooks of the strip triangular solves: strips, solution-ring rows and
  // staging-ring bytes (CPTR_STRIP_P, CPTR_STRIP_RC, CPTR_STRIP_RING; 0 = automatic)
  int strip_p = 0, strip_rc = 0, strip_ring = 0;
  // thread blocks of the level-scheduled triangular solves (0: chosen by the
  // tuner; CPTR_LVL_GRID forces a value)
  int lvl_grid = 0, lvl_grid_forced = 0;
  double phase_t0 = 0.0;
};

// Exchanges the first-stage fields (hierarchy, decoupling, work vectors and
// elliptic unknowns) with the stored second stage.
void swap_stage(cptr_ctx* c);

// Stream for the work this host thread issues for the context: the ILU(0)
// setup thread sets an override to the context's second stream.
extern thread_local cudaStream_t t_setup_stream;
inline cudaStream_t cs(const cptr_ctx* c) { return t_setup_stream ? t_setup_stream : c->stream; }

// Phase marker for CPTR_TIMING (synchronises the stream only when enabled).
void ctx_phase(cptr_ctx* c, const char* name);

// Wraps one kernel-launch statement and counts it for the context.
#define KL(c, ...)       \
  do {                   \
    __VA_ARGS__;         \
    ++(c)->nlaunch;      \
  } while (0)

// ---- internal helpers (api.cu) ----
void* ctx_alloc(cptr_ctx* c, size_t bytes, bool setup_lifetime);
// Records the reason of a failure (under the context's lock: both setup
// threads may fail at the same time).
void ctx_set_err(cptr_ctx* c, const char* msg);
cptr_status ctx_cuda_fail(cptr_ctx* c, cudaError_t e, const char* what);
// the same check in a function returning nothing: the failure is recorded in
// the context's error and status (CPTR_ERR_CUDA at the next status check)
#define CTX_CUDA_V(c, call)                                            \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) { ctx_cuda_fail((c), e_, #call); return; }  \
  } while (0)
#define CTX_CUDA(c, call)                                              \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) return ctx_cuda_fail((c), e_, #call);       \
  } while (0)
#define CTX_ALLOC(c, ptr, type, count, setup)                                       \
  do {                                                                              \
    (ptr) = (type*)ctx_alloc((c), sizeof(type) * (size_t)(count) + 16, (setup));    \
    if (!(ptr)) return CPTR_ERR_NOMEM;                                              \
  } while (0)
cptr_status ctx_check_device_status(cptr_ctx* c);

// ---- scan.cu ----
// Exclusive scan of n int32 values into out[0..n] (out[n] = total); returns
// the total through *total_host when non-null (synchronises the stream).
cptr_status scan_i32(cptr_ctx* c, const int32_t* in, int32_t* out, int n, int* total_host);
cptr_status scan_i64(cptr_ctx* c, const int32_t* in, long long* out, int n, long long* total_host);

// ---- setup_amg.cu ----
cptr_status setup_validate(cptr_ctx* c);
cptr_status setup_decouple(cptr_ctx* c);
cptr_status setup_amg(cptr_ctx* c);

// ---- mgr.cu (first MGR reduction, Section 3.4) ----
cptr_status mgr_reduce(cptr_ctx* c);  // vfull -> v; synchronous, checks the input
void mgr_rhs(cptr_ctx* c);            // bfull -> bd, and xd[.,2] = 0
void mgr_recover(cptr_ctx* c);        // xd[.,2] from the constraint rows

// ---- setup_ilu.cu ----
cptr_status setup_ilu(cptr_ctx* c);
cptr_status setup_ilu_factor(cptr_ctx* c);
cptr_status setup_ilu_schedule(cptr_ctx* c);
cptr_status build_level_solve_arrays(cptr_ctx* c);  // level-padded schedule arrays

// ---- sptrsv.cu ----
// Builds the chunked schedules for R rows per chunk (apply precision).
cptr_status build_chunked(cptr_ctx* c, int R);
// Times candidate chunk sizes (and the level-padded kernels) and keeps the best.
cptr_status tune_triangular(cptr_ctx* c);
bool tune_decided(cptr_ctx* c);
// Forward then backward chunked solve: y2 = (LU)^-1 r2, z = P zc + y2 at
// zbase + (*jptr)*stride (zc may be null).
void launch_tri_chunked(cptr_ctx* c, const void* zc, void* zbase, const int* jptr, size_t stride,
                        const int* active, int which /*0 both, 1 fwd, 2 bwd*/);

// ---- sptrsv_cluster.cu ----
// Builds the level-synchronous cluster schedules (CPTR_ERR_INVALID when a
// level slice does not fit in shared memory or no cluster can be launched).
cptr_status build_cluster(cptr_ctx* c);
// Forward then backward cluster solve, same contract as launch_tri_chunked.
void launch_tri_cluster(cptr_ctx* c, const void* zc, void* zbase, const int* jptr, size_t stride,
                        const int* active, int which);

// ---- sptrsv_strip.cu ----
// Builds the strip schedules (CPTR_ERR_INVALID when a step cannot be staged).
cptr_status build_strip(cptr_ctx* c);
// Forward then backward strip solve, same contract as launch_tri_chunked.
void launch_tri_strip(cptr_ctx* c, const void* zc, void* zbase, const int* jptr, size_t stride,
                      const int* active, int which);

// ---- sptrsv_chain.cu ----
// Builds the chain schedules (CPTR_ERR_INVALID when a dependency points to a
// later chain, which could make a solve wait on an unclaimed chain).
cptr_status build_chain(cptr_ctx* c);
void launch_tri_chain(cptr_ctx* c, const void* zc, void* zbase, const int* jptr, size_t stride,
                      const int* active, int which);

// ---- apply.cu ----
// Convert the FP64 hierarchy to the apply precision and size work buffers.
cptr_status setup_apply_buffers(cptr_ctx* c);
// z = M^-1 v with v = vbase + (*jptr)*stride and output zbase + (*jptr)*stride
// (apply precision); kernels do nothing while *active == 0.
void launch_precond(cptr_ctx* c, const double* vbase, void* zbase, const int* jptr,
                    const int* active);
cptr_status launch_apply_piece(cptr_ctx* c, int which, const double* in, double* out);
// Level-padded forward + backward solves of c->r2 (no first-stage combine).
void launch_level_solves(cptr_ctx* c, void* zbase);
// Profiling of single apply kernels: prepare=true runs the untimed preparation,
// prepare=false the launch being timed (CPTR_KERNEL_ILU_*, VC_PRE0, CORRECTION).
cptr_status profile_apply_kernel(cptr_ctx* c, int kernel, bool prepare);
// Same for CPTR_KERNEL_SPMV and CPTR_KERNEL_MDOT (krylov.cu).
cptr_status profile_krylov_kernel(cptr_ctx* c, int kernel, bool prepare);

// ---- krylov.cu ----
void launch_spmv(cptr_ctx* c, const void* x, bool x_f32, double* y, const double* b);
// Raises the kernel's dynamic shared-memory limit to what the device allows
// beside the kernel's static shared memory (see cptr_ctx::smem_optin).
inline cudaError_t raise_smem_limit(const cptr_ctx* c, const void* kernel) {
  cudaFuncAttributes a{};
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              c->smem_optin - (int)a.sharedSizeBytes);
}
cptr_status krylov_alloc(cptr_ctx* c);
cptr_status krylov_solve(cptr_ctx* c, double tol, int maxit);
void krylov_release_graph(cptr_ctx* c);
