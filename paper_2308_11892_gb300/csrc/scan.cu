// Device exclusive prefix sums used by the setup phase (row pointers,
// schedule offsets, scratch offsets).  Three passes: tile sums, a one-block
// scan of the tile sums, tile scans with carried offsets.
#include "common.cuh"
#include "ctx.h"

namespace {
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kTile = kScanThreads * kScanItems;

template <class TO>
__global__ void k_tile_sums(const int32_t* __restrict__ in, int n, TO* __restrict__ sums) {
  __shared__ TO sm[kScanThreads / 32];
  long long base = (long long)blockIdx.x * kTile;
  TO s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    long long i = base + (long long)k * kScanThreads + threadIdx.x;
    if (i < n) s += (TO)in[i];
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    TO t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += sm[w];
    sums[blockIdx.x] = t;
  }
}

// single block exclusive scan of nb values (in place), total written to sums[nb]
template <class TO>
__global__ void k_scan_sums(TO* sums, int nb) {
  __shared__ TO carry;
  __shared__ TO warp_tot[kScanThreads / 32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += kScanThreads) {
    int i = base + threadIdx.x;
    TO v = (i < nb) ? sums[i] : 0;
    // inclusive warp scan
    TO x = v;
    for (int o = 1; o < 32; o <<= 1) {
      TO y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      TO t = (threadIdx.x < kScanThreads / 32) ? warp_tot[threadIdx.x] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        TO y = __shfl_up_sync(0xffffffffu, t, o);
        if (threadIdx.x >= o) t += y;
      }
      if (threadIdx.x < kScanThreads / 32) warp_tot[threadIdx.x] = t;
    }
    __syncthreads();
    TO wpre = (threadIdx.x >= 32) ? warp_tot[(threadIdx.x >> 5) - 1] : 0;
    if (i < nb) sums[i] = carry + wpre + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

template <class TO>
__global__ void k_tile_scan(const int32_t* __restrict__ in, int n, const TO* __restrict__ sums,
                            TO* __restrict__ out) {
  __shared__ TO warp_tot[kScanThreads / 32];
  __shared__ TO carry;
  long long base = (long long)blockIdx.x * kTile;
  if (threadIdx.x == 0) carry = sums[blockIdx.x];
  __syncthreads();
  for (int k = 0; k < kScanItems; ++k) {
    long long i = base + (long long)k * kScanThreads + threadIdx.x;
    TO v = (i < n) ? (TO)in[i] : 0;
    TO x = v;
    for (int o = 1; o < 32; o <<= 1) {
      TO y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      TO t = (threadIdx.x < kScanThreads / 32) ? warp_tot[threadIdx.x] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        TO y = __shfl_up_sync(0xffffffffu, t, o);
        if (threadIdx.x >= o) t += y;
      }
      if (threadIdx.x < kScanThreads / 32) warp_tot[threadIdx.x] = t;
    }
    __syncthreads();
    TO wpre = (threadIdx.x >= 32) ? warp_tot[(threadIdx.x >> 5) - 1] : 0;
    if (i < n) out[i] = carry + wpre + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

template <class TO>
cptr_status scan_impl(cptr_ctx* c, const int32_t* in, TO* out, int n, TO* total_host) {
  int nb = n > 0 ? ceil_div(n, kTile) : 1;
  TO* sums = (TO*)ctx_alloc(c, sizeof(TO) * (nb + 1), true);
  if (!sums) return CPTR_ERR_NOMEM;
  if (n > 0) {
    KL(c, k_tile_sums<TO><<<nb, kScanThreads, 0, cs(c)>>>(in, n, sums));
    KL(c, k_scan_sums<TO><<<1, kScanThreads, 0, cs(c)>>>(sums, nb));
    KL(c, k_tile_scan<TO><<<nb, kScanThreads, 0, cs(c)>>>(in, n, sums, out));
  } else {
    CTX_CUDA(c, cudaMemsetAsync(out, 0, sizeof(TO), cs(c)));
  }
  CTX_CUDA(c, cudaGetLastError());
  if (total_host) {
    CTX_CUDA(c, cudaMemcpyAsync(total_host, out + n, sizeof(TO), cudaMemcpyDeviceToHost,
                                cs(c)));
    CTX_CUDA(c, cudaStreamSynchronize(cs(c)));
  }
  return CPTR_OK;
}
}  // namespace

cptr_status scan_i32(cptr_ctx* c, const int32_t* in, int32_t* out, int n, int* total_host) {
  return scan_impl<int32_t>(c, in, out, n, total_host);
}
cptr_status scan_i64(cptr_ctx* c, const int32_t* in, long long* out, int n,
                     long long* total_host) {
  return scan_impl<long long>(c, in, out, n, total_host);
}
