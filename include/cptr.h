/*
 * cptr.h -- C ABI of libcptr.so: CPTR-preconditioned flexible GMRES on one
 * GB300 GPU (sm_103a).
 *
 * Problem (paper Section 3): solve A x = b, where A is a Jacobian with four
 * interleaved unknowns per cell (p, rho_CO2, rho_H2O, T), using
 * right-preconditioned GMRES (maximum 200 iterations, relative tolerance 1e-6)
 * and the two-stage preconditioner of Eq. 3,
 *     M^-1 = M1^-1 + M2^-1 (I - A M1^-1),
 * with M1^-1 = [[0,0],[0,Mee^-1]] on the elliptic unknowns {p, T}
 * (Section 3.2, CPTR split), Mee^-1 one V-cycle of a system AMG (Section
 * 3.1/3.2), M2^-1 an ILU(0) of the global matrix (Section 3.1), and the
 * first-stage operator obtained by Quasi-IMPES decoupling (Section 5.2).
 *
 * Conventions shared by every entry point:
 *  - Block CSR with 4x4 blocks: rowptr[n_cells+1] and col[nnzb] are int32,
 *    columns strictly increasing inside each row, the diagonal block present;
 *    vals holds nnzb*16 doubles, each block row-major.  Vectors are 4*n_cells
 *    doubles, cell-major (unknown u of cell i at index 4*i+u).
 *  - Pointers may be host memory (pageable or pinned) or device memory of the
 *    current CUDA device; the library detects which.  The library never keeps a
 *    caller pointer: inputs are copied, outputs written before return.
 *  - Errors are returned, never aborted on.  cptr_last_error() gives a
 *    human-readable reason for the last failure on a context.
 *  - A context is not thread-safe; use one per thread or serialise calls.  A
 *    server (cptr_server_*) is thread-safe.
 *  - All device work of a context runs on its stream (cptr_set_stream).
 */
#ifndef CPTR_H
#define CPTR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CPTR_OK = 0,
  CPTR_ERR_INVALID = 1,    /* bad argument, malformed BSR, call out of order */
  CPTR_ERR_NOMEM = 2,      /* device allocation failed */
  CPTR_ERR_CUDA = 3,       /* CUDA runtime error (see cptr_last_error) */
  CPTR_ERR_MAXIT = 4,      /* GMRES reached maxit; x holds the last iterate */
  CPTR_ERR_BREAKDOWN = 5,  /* zero/non-finite pivot, singular coarse system, NaN */
  CPTR_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up (never a hang) */
  CPTR_ERR_AGAIN = 7,      /* server: queue full, try later */
  CPTR_PENDING = 8         /* server: request not finished yet */
} cptr_status;

typedef struct cptr_ctx cptr_ctx;        /* opaque, library-owned */
typedef struct cptr_server cptr_server;  /* opaque, library-owned */

enum {
  CPTR_PREC_NONE = 0,
  CPTR_PREC_CPTR = 1,   /* Eq. 3 with the (p, T) system-AMG first stage (default) */
  CPTR_PREC_ILU = 2,    /* ILU(0) alone */
  CPTR_PREC_FIRST = 3,  /* the first stage alone */
  CPTR_PREC_CPTR3 = 4   /* CPTR3 (Section 3.3): a pressure stage (decoupling onto e0 and a
                           scalar AMG), then a temperature stage on the residual it leaves
                           (decoupling onto e1 and a scalar AMG), then ILU(0) on the residual
                           of both, z = y_p + y_T + y_ILU, i.e. Eq. 3 applied twice.  The
                           single-piece calls of cptr_apply act on the pressure stage */
};
enum { CPTR_FP64 = 0, CPTR_MIXED = 1 };

typedef struct {
  int restart;        /* FGMRES(m) restart length, 1..63 (default 30) */
  int maxit;          /* maximum GMRES iterations (default 200, Section 3) */
  double tol;         /* relative tolerance on ||b - A x|| / ||b|| (default 1e-6) */
  int precision;      /* CPTR_FP64: everything FP64; CPTR_MIXED: V-cycle and ILU(0)
                         apply in FP32 inside FP64 flexible GMRES (default FP64) */
  double theta;       /* AMG strength threshold (default 0.25) */
  int pmax;           /* ext+i truncation, entries per row (default 4, Section 3.1) */
  int max_coarse;     /* coarsest level size (default 256) */
  int max_levels;     /* maximum AMG levels (default 25) */
  int precond;        /* CPTR_PREC_* (default CPTR_PREC_CPTR) */
  int use_graphs;     /* capture the Arnoldi step in a CUDA graph (default 1) */
  uint64_t seed;      /* PMIS random weights (default 0x5eed) */
  int e0, e1;         /* elliptic unknowns inside a block (default 0 = p, 3 = T: CPTR,
                         Section 3.2); e1 = -1 keeps e0 alone in the first stage (CPR,
                         Section 3.1: W_i is 1x3, the first-stage system is scalar) */
  int mgr;            /* 1: first MGR reduction (Section 3.4) before CPTR.  Equation row 2
                         of every cell must be a volume constraint on the cell's own
                         unknowns (row 2 of every off-diagonal block zero, A_ii[2,2] != 0);
                         unknown 2 (the last density) is eliminated with it exactly,
                         At_ij[r,s] = A_ij[r,s] - A_ij[r,2] (A_jj[2,s] / A_jj[2,2]), and
                         FGMRES runs on the reduced system (row and column 2 of its blocks
                         are the identity), with the tolerance relative to the reduced
                         right-hand side; cptr_solve takes and returns the full system's
                         rhs and x, recovering unknown 2 from the constraint rows.
                         cptr_setup returns CPTR_ERR_INVALID for a non-local row 2 and
                         CPTR_ERR_BREAKDOWN for a zero pivot.  e0 and e1 must not be 2.
                         Default 0 */
  int agg;            /* 1: one aggregate level (Section 3.1 lists it among the AMG
                         defaults): the first AMG level is coarsened twice (PMIS on A, then
                         PMIS on the Galerkin operator A1 = P1^T A P1 of the first split),
                         interpolates in two stages, P = P1 P2 truncated to pmax entries
                         per row by the ext+i rule, and its coarse operator is P^T A P;
                         A1 is not kept as a level.
                         2: BoomerAMG's form of it: the first split's C points are split
                         again on distance-two strength (j depends strongly on i, or on
                         one of i's strong dependencies), and the level interpolates by
                         multipass interpolation (direct from strong C neighbours, then
                         through strong neighbours interpolated in earlier passes, with
                         same-sign couplings lumped into the diagonal), truncated to pmax
                         entries per row.  Default 0 */
  int nu_pre;         /* V-cycle smoothing sweeps before the coarse correction (0..8,
                         default 1; Section 3.1: "one V-cycle") */
  int nu_post;        /* sweeps after it (0..8, default 1) */
  int smoother;       /* CPTR_SMOOTH_L1_JACOBI (default; Section 3.1 "first order
                         relaxation") or CPTR_SMOOTH_HYBRID_GS: rows in blocks of 32,
                         Gauss-Seidel in row order inside a block (reverse order after the
                         coarse correction) with the l1 diagonal as pivot, the sweep's
                         starting values for rows of other blocks */
  int tri_tune;       /* 1 (default): cptr_setup picks the ILU(0) triangular-solve
                         schedule by timing the candidates once per matrix shape (cached
                         per process); 0: by a rule without timing (one thread-block
                         cluster walking the levels when its rows fit, else level
                         kernels).  Schedules are bit-identical, so this changes speed
                         only.  Servers use the rule for every request. */
  int coarsen;        /* C/F splitting of every AMG level: CPTR_COARSEN_PMIS (default, on
                         the GPU) or CPTR_COARSEN_HMIS (Section 3.1).  HMIS on one domain
                         is the first pass of classical Ruge-Stueben coarsening: the
                         undecided point with the most points depending strongly on it
                         (ties: the smaller index) becomes C, its strong dependents F,
                         the counts are updated, until no undecided point has dependents;
                         the rest become F.  The pass is sequential: it runs on the host
                         (strength graph copied down, splitting copied up), the rest of
                         the setup on the GPU. */
} cptr_params;
enum { CPTR_COARSEN_PMIS = 0, CPTR_COARSEN_HMIS = 1 };
enum { CPTR_SMOOTH_L1_JACOBI = 0, CPTR_SMOOTH_HYBRID_GS = 1 };

typedef struct {
  int iters;            /* GMRES iterations (= preconditioner applications) */
  double rel_resid;     /* true ||b - A x|| / ||b|| at return */
  double setup_s;       /* last cptr_setup wall time (seconds) */
  double solve_s;       /* last cptr_solve wall time (seconds) */
  int amg_levels;       /* levels of the system-AMG hierarchy */
  int ilu_levels;       /* level sets of the ILU(0) lower triangle */
  double op_complexity; /* sum_l nnz(A_l) / nnz(A_0) */
  int status;           /* cptr_status of the last solve */
  long long launches;   /* kernels this context has launched since cptr_create
                           (graph launches count their kernel nodes) */
  int tri_schedule;     /* ILU(0) triangular-solve schedule chosen at setup: 0 level
                           kernels, 1 one cluster walking the levels, 2 index strips
                           owned by thread blocks, 3 dependency chains, > 3 chunks of
                           that many rows */
} cptr_info;

/* Fills *p with the defaults listed above. */
void cptr_params_default(cptr_params* p);

/* Creates a context from a 4x4 BSR matrix and copies it to the device.
 * bs must be 4.  Validation: indices in range, columns strictly increasing,
 * diagonal block present, n_cells and nnzb = rowptr[n_cells] at most
 * 2^29 - 1 (the scalar AMG operator of the first level holds four 32-bit
 * indexed entries per block) (CPTR_ERR_INVALID otherwise).  params may be NULL
 * (defaults).  On success *out owns device memory until cptr_destroy. */
cptr_status cptr_create(cptr_ctx** out, int32_t n_cells, int32_t bs, const int32_t* rowptr,
                        const int32_t* col, const double* vals, const cptr_params* params);

/* Replaces the matrix values (same pattern; with mgr the full, unreduced matrix);
 * cptr_setup must be called again. */
cptr_status cptr_update_values(cptr_ctx* c, const double* vals);

/* Sets the CUDA stream (a cudaStream_t) used by all later work; NULL selects the
 * context's own stream.  The caller keeps ownership of the stream. */
cptr_status cptr_set_stream(cptr_ctx* c, void* stream);

/* Builds the preconditioner on the device: Quasi-IMPES decoupling of the
 * (p, T) system, the system-AMG hierarchy (strength, PMIS, ext+i truncated to
 * pmax, Galerkin products, l1 diagonals, dense coarsest inverse) and the block
 * ILU(0) factors with their level schedule.  Synchronous. */
cptr_status cptr_setup(cptr_ctx* c);

/* Solves A x = rhs by flexible GMRES(restart) preconditioned with Eq. 3.
 * rhs: 4N doubles; x: 4N doubles, in: initial guess, out: solution (also on
 * CPTR_ERR_MAXIT, which returns the last iterate).  tol <= 0 and maxit <= 0
 * select the context's parameters.  info may be NULL.  Synchronous. */
cptr_status cptr_solve(cptr_ctx* c, const double* rhs, double* x, double tol, int maxit,
                       cptr_info* info);

/* Solves n small systems in one launch: one thread block per system runs the
 * whole flexible GMRES(restart) loop with the Eq. 3 preconditioner on the
 * device (block SpMV, restriction, V-cycle, correction, ILU(0) level by level,
 * CGS2, Givens rotations, restarts, true residual), with no host
 * synchronisation per iteration; the systems advance concurrently.  The same
 * algorithm and stopping rules as cptr_solve, with sums in a fixed order that
 * does not depend on the batch: a system's result is identical alone and in
 * any batch (it agrees with cptr_solve's to rounding, not bit for bit).
 * ctxs: n distinct contexts on one device and of one precision, each set up
 * by cptr_setup, with precond CPTR_PREC_CPTR (CPTR or CPR) or CPTR_PREC_ILU,
 * mgr = 0, the l1-Jacobi smoother and restart <= 32 (CPTR_ERR_INVALID
 * otherwise, reason in cptr_last_error(ctxs[0])).  rhs[k], x[k] (in: initial
 * guess, out: solution) are 4 N_k doubles, host or device.  tol <= 0 and
 * maxit <= 0 select each context's parameters.  infos (n entries) may be NULL.
 * Runs on the stream of ctxs[0] after every context's earlier work; returns
 * CPTR_OK when all converged, else the first failure (a breakdown before
 * CPTR_ERR_MAXIT); every x[k] is written.  Meant for systems of up to tens of
 * thousands of cells: one block per system. */
cptr_status cptr_solve_batch(cptr_ctx* const* ctxs, int n, const double* const* rhs,
                             double* const* x, double tol, int maxit, cptr_info* infos);

/* Frees every device and host resource of the context.  NULL is ignored. */
void cptr_destroy(cptr_ctx* c);

/* ---- single steps of the hot path (device pointers, asynchronous on the
 *      context stream; valid after cptr_setup) ---- */

/* y = A x, FP64 block SpMV (the outer Krylov operator: with mgr the reduced
 * one, which exists after cptr_setup; before it the call is refused). */
cptr_status cptr_spmv(cptr_ctx* c, const double* x, double* y);

enum {
  CPTR_APPLY_PRECOND = 0,     /* out(4N) = M^-1 in(4N), Eq. 3 */
  CPTR_APPLY_RESTRICT = 1,    /* out(ne N) = R in(4N): r_e - W r_h per cell (ne = 2, or
                                 1 for CPR) */
  CPTR_APPLY_VCYCLE = 2,      /* out(ne N) = one V-cycle on Ahat applied to in(ne N) */
  CPTR_APPLY_FIRST = 3,       /* out(4N) = P Vcycle(R in) = M1^-1 in */
  CPTR_APPLY_CORRECTION = 4,  /* out(4N) = in - A M1^-1 in */
  CPTR_APPLY_ILU = 5          /* out(4N) = (L U)^-1 in */
};
/* One preconditioner piece; in/out are FP64 device arrays (converted to and
 * from FP32 inside in CPTR_MIXED mode). */
cptr_status cptr_apply(cptr_ctx* c, int which, const double* in, double* out);

/* ---- inspection (host outputs, synchronous; for tests and tooling) ---- */
enum {
  CPTR_LVL_N = 0, CPTR_LVL_NNZ = 1, CPTR_LVL_NC = 2, CPTR_LVL_NNZP = 3
};
/* Number of AMG levels (0 before setup). */
int cptr_amg_levels(const cptr_ctx* c);
/* info[4] = {n, nnz(A_l), n_coarse, nnz(P_l)} of level l. */
cptr_status cptr_level_info(const cptr_ctx* c, int level, int32_t* info);
enum {
  CPTR_COPY_A_ROWPTR = 0, CPTR_COPY_A_COL = 1, CPTR_COPY_A_VAL = 2,
  CPTR_COPY_P_ROWPTR = 3, CPTR_COPY_P_COL = 4, CPTR_COPY_P_VAL = 5,
  CPTR_COPY_CF = 6, CPTR_COPY_DL1 = 7, CPTR_COPY_W = 8, CPTR_COPY_ILU = 9,
  CPTR_COPY_ILU_LEVEL = 10
};
/* Copies one FP64/int32 array of the hierarchy to host memory dst (sized by
 * cptr_level_info; W is N*4 doubles, ILU is nnzb*16 doubles in the input block
 * order, ILU_LEVEL is N int32; level is ignored for those three). */
cptr_status cptr_copy(const cptr_ctx* c, int level, int what, void* dst);
/* Last solve/setup statistics. */
cptr_status cptr_get_info(const cptr_ctx* c, cptr_info* info);

/* Bounded device waits: a triangular-solve dependency wait (a row waiting for a
 * value another thread block computes) gives up after `polls` reads that all
 * found the value unwritten, records the failure and lets the kernel finish;
 * the solve then returns CPTR_ERR_TIMEOUT (never a hang).  polls = 0 restores
 * the default of 2^21 reads (well over a second).  A context that timed out
 * solves normally again once the limit is large enough (the next cptr_solve
 * clears the failure).  Small limits exist to exercise that error path. */
cptr_status cptr_set_spin_limit(cptr_ctx* c, unsigned polls);

/* ---- setup phase timing (where cptr_setup spends its time) ----
 * With timing enabled, cptr_setup synchronises its stream at every phase
 * boundary (which slows it slightly) and records each phase's wall time in
 * milliseconds; cptr_setup_phases copies the CPTR_PHASE_COUNT values of the
 * last cptr_setup into ms (zeros while timing is off).  The ILU(0) setup runs
 * on a second stream and host thread while the AMG hierarchy is built:
 * CPTR_PHASE_ILU_CONCURRENT is its own wall time (overlapping the AMG phases),
 * CPTR_PHASE_ILU the time the setup still waits for it afterwards. */
enum {
  CPTR_PHASE_DECOUPLE = 0,     /* Quasi-IMPES decoupling (and the MGR reduction) */
  CPTR_PHASE_STRENGTH = 1,     /* strength of connection and its transpose, all levels */
  CPTR_PHASE_PMIS = 2,         /* C/F splitting, all levels */
  CPTR_PHASE_INTERP = 3,       /* ext+i interpolation, truncation, transpose, all levels */
  CPTR_PHASE_SPGEMM = 4,       /* Galerkin products A P and P^T (A P), all levels */
  CPTR_PHASE_COARSE = 5,       /* dense inverse of the coarsest operator */
  CPTR_PHASE_ILU = 6,          /* ILU(0) work left after the AMG setup */
  CPTR_PHASE_BUFFERS = 7,      /* apply-precision copies and work buffers */
  CPTR_PHASE_ILU_CONCURRENT = 8,
  CPTR_PHASE_COUNT = 9
};
cptr_status cptr_setup_timing(cptr_ctx* c, int enable);
cptr_status cptr_setup_phases(const cptr_ctx* c, double* ms);

/* ---- kernel timing (roofline evidence) ----
 * Runs one kernel of the hot path `reps` times on the context's current data
 * (valid after cptr_setup and one cptr_solve), each launch preceded by an
 * untimed L2 flush (a 256 MiB device write) and by the untimed preparation the
 * kernel needs (sentinel reset for the triangular solves, the forward solve
 * before a backward one).  Returns the mean launch duration in milliseconds
 * measured with CUDA events on the context stream, and the algorithmic bytes
 * one launch must move (matrix and index data read once, vectors read and
 * written once).  Synchronous. */
enum {
  CPTR_KERNEL_SPMV = 0,        /* FP64 block SpMV w = A z */
  CPTR_KERNEL_ILU_FWD = 1,     /* forward block triangular solve */
  CPTR_KERNEL_ILU_BWD = 2,     /* backward block triangular solve + combine */
  CPTR_KERNEL_VC_PRE0 = 3,     /* fused l1-Jacobi + residual on the finest AMG level */
  CPTR_KERNEL_CORRECTION = 4,  /* r - A P zc (elliptic columns of A) */
  CPTR_KERNEL_MDOT = 5         /* CGS2 first-pass multi-dot at the average Arnoldi column of
                                  the last solve (min(iterations, restart) / 2 + 1 basis
                                  vectors; restart/2 + 1 before any solve) */
};
cptr_status cptr_profile_kernel(cptr_ctx* c, int kernel, int reps, double* avg_ms,
                                double* bytes);

/* Floating-point operations one launch of `kernel` (a CPTR_KERNEL_* value) must
 * do, an FMA counting two: SpMV 32 per block; forward solve 32 per block of L;
 * backward solve 32 per block of U and per row (D^-1) plus 4 per row (the
 * first-stage part, Eq. 3); finest-level smoothing 2 per nonzero and 3 per
 * row; correction 8 per elliptic column per block plus 4 per row; multi-dot 8
 * per cell per basis vector.  *fp64 = 1 when the kernel computes in FP64 (SpMV
 * and the multi-dot always; the preconditioner kernels unless precision is
 * mixed).  Valid after cptr_setup; CPTR_ERR_INVALID otherwise.  Host only. */
cptr_status cptr_kernel_flops(const cptr_ctx* c, int kernel, double* flops, int* fp64);

/* The device's measured FMA throughput, the compute roof of the kernels above:
 * `reps` timed launches (after one untimed) on `stream` (NULL: the legacy
 * default stream) of a kernel whose threads (8 blocks of 256 per SM) each run
 * eight independent chains x <- x a + b of `iters` steps, in FP64 (fp64 != 0)
 * or FP32.  *tflops = 2 x FMAs / mean CUDA-event launch time, in TFLOP/s.
 * With a = 1 and b = 1/2 every step is exact, and every thread's result is
 * checked on the host against its closed form (CPTR_ERR_BREAKDOWN if one
 * differs: the launches did not do their work).  iters must be at most 2^30
 * (FP64) or 2^21 (FP32) for that to hold (CPTR_ERR_INVALID otherwise).
 * Allocates and frees its own 10 KiB-per-SM output; synchronous; not for use
 * inside a stream capture. */
cptr_status cptr_fma_rate(int fp64, int iters, int reps, void* stream, double* tflops);

/* ---- serving: continuous batching of independent solves ---- */
/* Creates a server on the current device that admits requests while their
 * estimated device footprint fits in hbm_budget_bytes, with max_slots worker
 * threads (one CUDA stream each) building and solving them concurrently.
 * Every request uses params (NULL: defaults) with its own tol and maxit, and
 * the triangular-solve schedule rule of tri_tune = 0 (shapes rarely repeat,
 * and the blocks of concurrent requests share the SMs). */
cptr_status cptr_server_create(cptr_server** out, size_t hbm_budget_bytes, int max_slots,
                               const cptr_params* params);
/* max_queued: submitted requests not yet admitted (default 4096); a submit
 * beyond it returns CPTR_ERR_AGAIN.  batch_max_cells: requests of at most that
 * many cells are, once set up, solved together by cptr_solve_batch (every
 * small request set up and waiting goes into the next batched launch);
 * 0 (default) solves every request on its own.  CPTR_ERR_INVALID for
 * batch_max_cells > 0 when the server's params are not ones cptr_solve_batch
 * runs (the limit is then 0). */
cptr_status cptr_server_set_limits(cptr_server* s, int max_queued, int batch_max_cells);
/* Queues one solve (BSR system + rhs, host or device pointers, copied before
 * return; never blocks on the GPU).  *req_id identifies it for cptr_poll.
 * CPTR_ERR_AGAIN when max_queued requests are already waiting. */
cptr_status cptr_submit(cptr_server* s, int32_t n_cells, const int32_t* rowptr,
                        const int32_t* col, const double* vals, const double* rhs, double tol,
                        int maxit, uint64_t* req_id);
/* CPTR_PENDING while running; otherwise the request's final status, with the
 * solution copied to x_out (host, 4N doubles) and info filled.  A finished
 * request is released after a successful poll. */
cptr_status cptr_poll(cptr_server* s, uint64_t req_id, double* x_out, cptr_info* info);
/* The message of the last request that failed ("" if none): the request,
 * its size, the status and the context's cptr_last_error.  Valid until the
 * next failure or cptr_server_destroy. */
const char* cptr_server_last_error(cptr_server* s);
/* Waits for all requests and frees the server. */
void cptr_server_destroy(cptr_server* s);

/* ---- residual without allocation ----
 * The paper has no counterpart to this call; it is a library service.
 * For callers that must not allocate device memory when they need a residual:
 * code that runs while its stream is being captured into a CUDA graph, and
 * applications whose device memory belongs to their own pool or framework
 * allocator.  It computes r = b - A x (A: BSR with 4x4 row-major blocks, FP64)
 * and rnorm = ||r||_2, the same products as cptr_spmv, with no context.
 * n_cells, rowptr (n_cells+1), col, vals (16 doubles per block), x, b, r
 * (4*n_cells doubles each) and rnorm (one double) are DEVICE pointers owned by
 * the caller; r must not overlap x or b, and x must be 16-byte aligned (it is
 * read two doubles at a time; a misaligned x returns CPTR_ERR_INVALID).  Work is queued on `stream` (a
 * cudaStream_t; NULL = the legacy default stream) and the call returns without
 * waiting.  The reduction's scratch (one partial sum per 64 cells and a
 * completion counter) is a fixed array in the library's device memory, so the
 * call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine); it is limited to CPTR_NOALLOC_MAX_CELLS cells, and larger sizes,
 * n_cells <= 0 and null pointers return CPTR_ERR_INVALID before anything runs.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  The address is kept per device index for the life of
 * the process: after a cudaDeviceReset the next call would use a stale
 * address, so do not reset a device between calls.  Every call on a device shares the one array, so calls
 * that may run at the same time on the GPU (different streams, no ordering
 * between them) race and may return a wrong rnorm; calls ordered on one stream
 * are safe.  The counter is cleared on the stream before each launch. */
#define CPTR_NOALLOC_MAX_CELLS 262144
cptr_status cptr_residual_noalloc(int32_t n_cells, const int32_t* rowptr, const int32_t* col,
                                  const double* vals, const double* x, const double* b,
                                  double* r, double* rnorm, void* stream);

/* ---- diagnostics ---- */
const char* cptr_status_str(cptr_status s);
const char* cptr_last_error(const cptr_ctx* c);

#ifdef __cplusplus
}
#endif
#endif /* CPTR_H */
