// cptr_profile_kernel: CUDA-event timing of single hot-path kernels with the
// algorithmic byte count of one launch (the numerator of a roofline fraction).
#include "common.cuh"
#include "ctx.h"

namespace {
// Bytes a launch must move: matrix values and indices read once, vectors read
// and written once (reuse of gathered vector entries through the caches is not
// counted).
double algorithmic_bytes(const cptr_ctx* c, int kernel) {
  double N = c->N, nnzb = c->nnzb;
  double T = c->mixed ? 4.0 : 8.0;
  switch (kernel) {
    case CPTR_KERNEL_SPMV:
      return 132.0 * nnzb + 4.0 * (N + 1) + 64.0 * N;
    case CPTR_KERNEL_ILU_FWD: {
      double np = (c->chunked || c->cluster || c->strip || c->chain) ? N : (double)c->npos_f;
      return (double)c->nnzL * (16 * T + 4) + 8.0 * np + 4 + 12.0 * N * T;
    }
    case CPTR_KERNEL_ILU_BWD: {
      double np = (c->chunked || c->cluster || c->strip || c->chain) ? N : (double)c->npos_b;
      return (double)c->nnzU * (16 * T + 4) + 8.0 * np + 4 + 16.0 * T * np + 12.0 * N * T +
             (c->lev.empty() ? 0.0 : (c->se1 < 0 ? 1.0 : 2.0) * N * T);
    }
    case CPTR_KERNEL_VC_PRE0: {
      double n = c->lev[0].A.n, nnz = c->lev[0].A.nnz;
      return nnz * (T + 4) + 4.0 * (n + 1) + 4.0 * n * T;
    }
    case CPTR_KERNEL_CORRECTION: {
      // e columns of every block (4 x ne), the ne-vector z_c, r in, r2 and the
      // sentinel reset out
      double ne = c->se1 < 0 ? 1.0 : 2.0;
      return nnzb * (4 * ne * T + 4) + 4.0 * (N + 1) + 32.0 * N + ne * N * T + 8.0 * N * T;
    }
    case CPTR_KERNEL_MDOT:
      return (double)(mdot_profile_column(c->info, c->p.restart) + 2) * 32.0 * N;
  }
  return 0.0;
}
}  // namespace

extern "C" cptr_status cptr_profile_kernel(cptr_ctx* c, int kernel, int reps, double* avg_ms,
                                           double* bytes) {
  if (!c || !avg_ms || reps < 1) return CPTR_ERR_INVALID;
  if (!c->setup_done) { ctx_set_err(c, "cptr_setup has not been called"); return CPTR_ERR_INVALID; }
  if (kernel < CPTR_KERNEL_SPMV || kernel > CPTR_KERNEL_MDOT) return CPTR_ERR_INVALID;
  const size_t kFlush = 256ull << 20;
  if (!c->flush_buf) {
    c->flush_buf = ctx_alloc(c, kFlush, false);
    if (!c->flush_buf) return CPTR_ERR_NOMEM;
  }
  bool kry = kernel == CPTR_KERNEL_SPMV || kernel == CPTR_KERNEL_MDOT;
  cudaEvent_t e0, e1;
  CTX_CUDA(c, cudaEventCreate(&e0));
  CTX_CUDA(c, cudaEventCreate(&e1));
  double total = 0.0;
  cptr_status st = CPTR_OK;
  for (int r = 0; r < reps && st == CPTR_OK; ++r) {
    CTX_CUDA(c, cudaMemsetAsync(c->flush_buf, r & 0xff, kFlush, c->stream));
    st = kry ? profile_krylov_kernel(c, kernel, true) : profile_apply_kernel(c, kernel, true);
    if (st) break;
    CTX_CUDA(c, cudaEventRecord(e0, c->stream));
    st = kry ? profile_krylov_kernel(c, kernel, false) : profile_apply_kernel(c, kernel, false);
    CTX_CUDA(c, cudaEventRecord(e1, c->stream));
    CTX_CUDA(c, cudaEventSynchronize(e1));
    float ms = 0.f;
    CTX_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
    total += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  st = ctx_check_device_status(c);
  if (st) return st;
  *avg_ms = total / reps;
  if (bytes) *bytes = algorithmic_bytes(c, kernel);
  return CPTR_OK;
}
