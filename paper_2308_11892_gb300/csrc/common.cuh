// Device-side helpers shared by the CUDA translation units of libcptr.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Error codes written into the device status word (first writer wins).
enum { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BREAKDOWN = 2 };

// Bounded spin: a device wait gives up after this many polls, records
// DEV_TIMEOUT and returns (it never traps and never loops forever).
#ifndef CPTR_SPIN_LIMIT
#define CPTR_SPIN_LIMIT (1u << 21)
#endif

__device__ __forceinline__ void dev_fail(int* status, int code) { atomicCAS(status, DEV_OK, code); }

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  int v;
  asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int ld_acquire_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_i32(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- "not yet written" sentinels for the sync-free triangular solves.
// Signalling-NaN payloads that arithmetic never produces (the GPU returns the
// canonical quiet NaN), so a value doubles as its own ready flag.
#define SENT_F32 0x7fbadbadu
#define SENT_F64 0x7ff4badbadbadbadull

__device__ __forceinline__ float sentinel_of(float) { return __uint_as_float(SENT_F32); }
__device__ __forceinline__ double sentinel_of(double) {
  return __longlong_as_double((long long)SENT_F64);
}
__device__ __forceinline__ bool is_sentinel(float v) { return __float_as_uint(v) == SENT_F32; }
__device__ __forceinline__ bool is_sentinel(double v) {
  return (unsigned long long)__double_as_longlong(v) == SENT_F64;
}
// ---- IEEE comparisons of doubles with zero, evaluated on the bit pattern.
// Each returns exactly what the comparison it names returns (NaN included),
// but runs on the integer pipes: GB300 issues FP64 compares on its narrow
// FP64 pipe, which the setup kernels otherwise saturate.
__device__ __forceinline__ unsigned long long dmag(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ bool d_isnan(double x) { return dmag(x) > 0x7ff0000000000000ull; }
__device__ __forceinline__ bool d_eq0(double x) { return dmag(x) == 0; }   // x == 0.0
__device__ __forceinline__ bool d_neg(double x) {                         // sign bit
  return __double_as_longlong(x) < 0;
}
__device__ __forceinline__ bool d_lt0(double x) {                         // x < 0.0
  return d_neg(x) && !d_eq0(x) && !d_isnan(x);
}
__device__ __forceinline__ bool d_gt0(double x) {                         // x > 0.0
  return !d_neg(x) && !d_eq0(x) && !d_isnan(x);
}
__device__ __forceinline__ bool d_ge0(double x) { return !d_lt0(x) && !d_isnan(x); }  // x >= 0.0

// a > b and a >= b for doubles as in IEEE (false when either is NaN; -0 ==
// +0), through a monotone integer key of the bit pattern
__device__ __forceinline__ long long d_key(double x) {
  const long long b = __double_as_longlong(x);
  return b < 0 ? -(b & 0x7fffffffffffffffll) : b;
}
__device__ __forceinline__ bool d_gt(double a, double b) {
  return !d_isnan(a) && !d_isnan(b) && d_key(a) > d_key(b);
}
__device__ __forceinline__ bool d_ge(double a, double b) {
  return !d_isnan(a) && !d_isnan(b) && d_key(a) >= d_key(b);
}
// -x (a sign flip)
__device__ __forceinline__ double d_neg_of(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

// A computed value equal to the sentinel bit pattern (only possible by copying
// an input that already held it) is replaced by the canonical NaN.
template <class T>
__device__ __forceinline__ T desentinel(T v) {
  return is_sentinel(v) ? (T)__int_as_float(0x7fffffff) : v;
}

// 4-vector volatile load / store (L1 bypassed, element-wise single-copy atomic).
__device__ __forceinline__ void ld_volatile4(const float* p, float* o) {
  asm volatile("ld.volatile.global.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3])
               : "l"(p));
}
__device__ __forceinline__ void ld_volatile4(const double* p, double* o) {
  asm volatile("ld.volatile.global.v2.f64 {%0,%1}, [%2];" : "=d"(o[0]), "=d"(o[1]) : "l"(p));
  asm volatile("ld.volatile.global.v2.f64 {%0,%1}, [%2];" : "=d"(o[2]), "=d"(o[3]) : "l"(p + 2));
}
__device__ __forceinline__ void st_volatile(float* p, float v) {
  asm volatile("st.volatile.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void st_volatile(double* p, double v) {
  asm volatile("st.volatile.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// 4-vector plain loads of float/double data as double.
__device__ __forceinline__ void ld4(const double* p, double* o) {
  double2 a = __ldg(reinterpret_cast<const double2*>(p));
  double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld4(const float* p, double* o) {
  float4 a = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void ld4(const float* p, float* o) {
  float4 a = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid-wide "last block" detection for deterministic two-level reductions:
// every block writes its partial, fences, and takes a ticket; the block with
// the last ticket sees all partials and combines them in block order.
__device__ __forceinline__ bool last_block_ticket(unsigned* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// a0 x0 + a1 x1 + a2 x2 + a3 x3 with a fixed rounding sequence (one product,
// then three fused multiply-adds).  Every triangular-solve kernel uses it, so
// all schedules (level kernels, any chunk size) give bit-identical results
// whatever contraction the compiler would choose at each call site.
__device__ __forceinline__ float dot4(const float* a, const float* x) {
  float t = __fmul_rn(a[0], x[0]);
  t = __fmaf_rn(a[1], x[1], t);
  t = __fmaf_rn(a[2], x[2], t);
  return __fmaf_rn(a[3], x[3], t);
}
__device__ __forceinline__ double dot4(const double* a, const double* x) {
  double t = __dmul_rn(a[0], x[0]);
  t = __fma_rn(a[1], x[1], t);
  t = __fma_rn(a[2], x[2], t);
  return __fma_rn(a[3], x[3], t);
}
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

__host__ __device__ __forceinline__ int ceil_div(long long a, long long b) {
  return (int)((a + b - 1) / b);
}
