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

// ---------------------------------------------------------------- flop model
namespace {
// Floating-point operations one launch must do (an FMA counts two), in the
// precision the kernel computes in: the compute roof beside the byte count.
double algorithmic_flops(const cptr_ctx* c, int kernel, int* fp64) {
  double N = c->N, nnzb = c->nnzb;
  *fp64 = !c->mixed;
  switch (kernel) {
    case CPTR_KERNEL_SPMV:  // a 4x4 block times a 4-vector per block
      *fp64 = 1;
      return 32.0 * nnzb;
    case CPTR_KERNEL_ILU_FWD:  // r_i - sum L_ij y_j (unit lower factor)
      return 32.0 * (double)c->nnzL;
    case CPTR_KERNEL_ILU_BWD:  // D_i^-1 (y_i - sum U_ij x_j), then the first-stage part added
      return 32.0 * (double)c->nnzU + 32.0 * N + 4.0 * N;
    case CPTR_KERNEL_VC_PRE0: {  // r = b - A x, x += D_l1^-1 r on the finest level
      double n = c->lev[0].A.n, nnz = c->lev[0].A.nnz;
      return 2.0 * nnz + 3.0 * n;
    }
    case CPTR_KERNEL_CORRECTION: {  // r - A P zc: ne elliptic columns of every block
      double ne = c->se1 < 0 ? 1.0 : 2.0;
      return 8.0 * ne * nnzb + 4.0 * N;
    }
    case CPTR_KERNEL_MDOT:  // h_i = V_i . w for the columns 0..j
      *fp64 = 1;
      return 8.0 * N * (double)(mdot_profile_column(c->info, c->p.restart) + 1);
  }
  return 0.0;
}

// Eight independent chains x <- x a + b per thread.  With a = 1 and b = 1/2
// every step is exact, so each thread's sum has a closed form the host checks:
// the timed launches did all their FMAs.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T a, T b, int iters, T* out) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)((threadIdx.x & 7) + k);
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cptr_status fma_rate(int iters, int reps, cudaStream_t st, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CPTR_ERR_CUDA;
  const int kThreads = 256, blocks = 8 * sms;
  const size_t nt = (size_t)blocks * kThreads;
  T* out = nullptr;
  if (cudaMalloc(&out, nt * sizeof(T)) != cudaSuccess) return CPTR_ERR_NOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cptr_status rc = CPTR_OK;
  double total = 0.0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = CPTR_ERR_CUDA;
  // one untimed launch first (module load, clocks up), then the timed ones
  for (int r = -1; r < reps && rc == CPTR_OK; ++r) {
    if (cudaEventRecord(e0, st) != cudaSuccess) { rc = CPTR_ERR_CUDA; break; }
    k_fma_chains<T><<<blocks, kThreads, 0, st>>>((T)1, (T)0.5, iters, out);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess) { rc = CPTR_ERR_CUDA; break; }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = CPTR_ERR_CUDA; break; }
    if (r >= 0) total += ms;
  }
  if (rc == CPTR_OK) {
    std::vector<T> h(nt);
    if (cudaMemcpy(h.data(), out, nt * sizeof(T), cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = CPTR_ERR_CUDA;
    } else {
      for (size_t t = 0; t < nt && rc == CPTR_OK; ++t) {
        const double x0 = 8.0 * (double)((t % kThreads) & 7) + 28.0;  // sum of the 8 starts
        if ((double)h[t] != x0 + 4.0 * (double)iters) rc = CPTR_ERR_BREAKDOWN;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc == CPTR_OK)
    *tflops = 2.0 * 8.0 * (double)nt * (double)iters / (total / reps * 1e-3) * 1e-12;
  return rc;
}
}  // namespace

extern "C" cptr_status cptr_kernel_flops(const cptr_ctx* c, int kernel, double* flops, int* fp64) {
  if (!c || !flops || !fp64) return CPTR_ERR_INVALID;
  if (!c->setup_done) return CPTR_ERR_INVALID;
  if (kernel < CPTR_KERNEL_SPMV || kernel > CPTR_KERNEL_MDOT) return CPTR_ERR_INVALID;
  *flops = algorithmic_flops(c, kernel, fp64);
  return CPTR_OK;
}

extern "C" cptr_status cptr_fma_rate(int fp64, int iters, int reps, void* stream, double* tflops) {
  if (!tflops || reps < 1 || iters < 1) return CPTR_ERR_INVALID;
  // the chains and each thread's sum of eight stay exact while they fit the
  // significand in steps of 1/2
  if (fp64 ? iters > (1 << 30) : iters > (1 << 21)) return CPTR_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return fp64 ? fma_rate<double>(iters, reps, st, tflops) : fma_rate<float>(iters, reps, st, tflops);
}
