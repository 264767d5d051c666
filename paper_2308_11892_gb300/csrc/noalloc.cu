// Residual and residual norm for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they need a residual: code running while a stream is being captured
// into a CUDA graph, solver loops embedded in an application whose memory is
// owned by a custom pool or a framework allocator, or latency-critical paths
// that must not touch the allocator at all.  cptr_residual_noalloc serves them:
// it is the block SpMV residual r = b - A x fused with the two-level norm
// reduction used by the Krylov kernels, but its reduction scratch (one partial
// sum per thread block and a completion ticket) lives in a fixed array in the
// library's own device memory instead of in a context.
#include <mutex>

#include "common.cuh"
#include "cptr.h"

namespace {

constexpr int kRowsPerBlock = 64;  // 256 threads, four lanes per block row
constexpr int kMaxBlocks = CPTR_NOALLOC_MAX_CELLS / kRowsPerBlock;  // 4096
static_assert(kMaxBlocks * kRowsPerBlock == CPTR_NOALLOC_MAX_CELLS, "scratch sizing");

// Scratch: kMaxBlocks partial sums followed by the ticket counter.  Every GPU
// that loads the library holds this array (about 32 KiB) until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kMaxBlocks + 2];

__global__ void __launch_bounds__(256) k_residual_norm(int N, const int32_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci,
                                                       const double* __restrict__ v,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ b,
                                                       double* __restrict__ r, double* rnorm,
                                                       double* scratch) {
  double* part = scratch;
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch + kMaxBlocks);
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i = (int)(g >> 2), q = (int)(g & 3);
  double s2 = 0.0;
  if (i < N) {
    double acc = 0.0;
    const double* a = v + 16 * (size_t)rp[i] + 4 * q;
    for (int t = rp[i]; t < rp[i + 1]; ++t, a += 16) {
      double xj[4];
      ld4(x + 4 * (size_t)ci[t], xj);
      acc += a[0] * xj[0] + a[1] * xj[1] + a[2] * xj[2] + a[3] * xj[3];
    }
    size_t o = 4 * (size_t)i + q;
    double ri = b[o] - acc;
    r[o] = ri;
    s2 = ri * ri;
  }
  __shared__ double red[8];
  s2 = warp_sum(s2);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
  if (last_block_ticket(ticket) && threadIdx.x == 0) {
    double t = 0.0;
    for (unsigned bk = 0; bk < gridDim.x; ++bk) t += part[bk];
    *rnorm = sqrt(t);
    *ticket = 0u;
  }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_mu;
double* g_ptr[64] = {nullptr};

}  // namespace

extern "C" cptr_status cptr_residual_noalloc(int32_t n_cells, const int32_t* rowptr,
                                             const int32_t* col, const double* vals,
                                             const double* x, const double* b, double* r,
                                             double* rnorm, void* stream) {
  if (n_cells <= 0 || !rowptr || !col || !vals || !x || !b || !r || !rnorm)
    return CPTR_ERR_INVALID;
  if (n_cells > CPTR_NOALLOC_MAX_CELLS) return CPTR_ERR_INVALID;  // beyond the fixed scratch
  if (reinterpret_cast<uintptr_t>(x) % 16 != 0) return CPTR_ERR_INVALID;  // read as double2
  int blocks = (n_cells + kRowsPerBlock - 1) / kRowsPerBlock;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return CPTR_ERR_CUDA;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
      // first call on this device: translate the symbol to a device address
      double* p = nullptr;
      if (cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch) != cudaSuccess ||
          !p) {
        cudaGetLastError();
        return CPTR_ERR_CUDA;
      }
      g_ptr[dev] = p;
    }
    scratch = g_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the ticket must start at zero (a previous call leaves it at zero, but a
  // call that failed mid-way might not)
  if (cudaMemsetAsync(scratch + kMaxBlocks, 0, sizeof(unsigned), s) != cudaSuccess) {
    cudaGetLastError();
    return CPTR_ERR_CUDA;
  }
  k_residual_norm<<<blocks, 4 * kRowsPerBlock, 0, s>>>(n_cells, rowptr, col, vals, x, b, r, rnorm,
                                                        scratch);
  if (cudaGetLastError() != cudaSuccess) return CPTR_ERR_CUDA;
  return CPTR_OK;
}
