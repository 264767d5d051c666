// Level-ordered block triangular solves on one thread-block cluster, with
// the solution held in distributed shared memory.
//
// The ILU(0) solves of a 7-point system in natural order have one level per
// anti-diagonal plane, and every row depends on rows of the level just before
// it.  A sync-free schedule spread over all SMs pays a cross-SM hand-off
// through L2 on every level.  Here one cluster of up to 16 CTAs (one per SM of
// a GPC) walks the levels in order: each CTA takes a contiguous slice of every
// level's rows and keeps the solution of all its rows in its own shared
// memory.  Solution slots start as a sentinel NaN; a row reads each dependency
// from the owning CTA's shared memory (DSMEM, ld.shared::cluster, or its own)
// until no entry is the sentinel, so levels need no cluster barrier; a CTA
// barrier per level only recycles the staged buffers.  The outputs are written
// to global memory once, after the last level and a final cluster barrier.
// The block pointers, dependency locations (owner CTA, slot), factor blocks,
// inverse diagonals and right-hand side of each level slice are contiguous and
// staged by TMA bulk copies (cp.async.bulk + mbarrier), double-buffered one
// level ahead.  The schedule is built only when the solution fits in the
// cluster's shared memory.  Each row's sum uses the same rounding sequence as
// every other schedule (dot4, sub_rn), so results are bit-identical to them.
#include <algorithm>
#include <cstdio>
#include <vector>

#include <cub/device/device_radix_sort.cuh>

#include "common.cuh"
#include "ctx.h"

namespace {

constexpr int kT = 256;
constexpr int kCluThreads = 512;
constexpr size_t kCluSmemBudget = 220 * 1024;
inline int nblk(long long n, int per = kT) { return n > 0 ? ceil_div(n, per) : 1; }

// ------------------------------------------------------------------ TMA / cluster helpers
__device__ __forceinline__ unsigned saddr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes,
                                          uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(b))
      : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on an mbarrier phase; false after CPTR_SPIN_LIMIT polls
__device__ __forceinline__ bool bar_wait(uint64_t* b, unsigned parity) {
  for (unsigned s = 0; s < (unsigned)CPTR_SPIN_LIMIT; ++s)
    if (bar_try(b, parity)) return true;
  return false;
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
template <class T>
__device__ __forceinline__ void lds4(const T* p, T* o) {
  if (sizeof(T) == 4) {
    float4 a = *reinterpret_cast<const float4*>(p);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  } else {
    double2 a = *reinterpret_cast<const double2*>(p);
    double2 b = *(reinterpret_cast<const double2*>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
}

// ------------------------------------------------------------------ shared-memory layout
// [3 mbarriers | desc table (nlev int4) | solution (ycap x 4 T) | buffer 0 | buffer 1]
// one buffer: srp [rows+9] | loc [blks+8] (ints) | rhs [rows*4 T] |
//             dinv [rows*16 T] (backward) | v [blks*16 T]
struct CluBuf {
  size_t srp, loc, rhs, dinv, v, size;
};
__host__ __device__ inline size_t r128(size_t b) { return (b + 127) & ~(size_t)127; }
__host__ __device__ inline CluBuf clu_buf(int rows, int blks, int ts, bool upper) {
  CluBuf B;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o += r128(bytes); return at; };
  B.srp = take(4 * ((size_t)rows + 9));
  B.loc = take(4 * ((size_t)blks + 8));
  B.rhs = take((size_t)rows * 4 * ts);
  B.dinv = take(upper ? (size_t)rows * 16 * ts : 0);
  B.v = take((size_t)blks * 16 * ts);
  B.size = o;
  return B;
}
__host__ __device__ inline size_t clu_desc_off() { return 128; }
__host__ __device__ inline size_t clu_y_off(int nlev) { return clu_desc_off() + r128((size_t)nlev * 16); }
__host__ __device__ inline size_t clu_buf_off(int nlev, int ycap, int ts) {
  return clu_y_off(nlev) + r128((size_t)ycap * 4 * ts);
}
__host__ __device__ inline size_t clu_smem(int nlev, int ycap, int rows, int blks, int ts,
                                           bool upper) {
  return clu_buf_off(nlev, ycap, ts) + 2 * clu_buf(rows, blks, ts, upper).size;
}
// 4-vector from the shared memory of CTA `rank` of the cluster
__device__ __forceinline__ void ld_dsmem4(unsigned laddr, unsigned rank, float* o) {
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(laddr), "r"(rank));
  asm volatile("ld.shared::cluster.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3])
               : "r"(ra)
               : "memory");
}
__device__ __forceinline__ void ld_dsmem4(unsigned laddr, unsigned rank, double* o) {
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(laddr), "r"(rank));
  asm volatile("ld.shared::cluster.v2.f64 {%0,%1}, [%2];" : "=d"(o[0]), "=d"(o[1]) : "r"(ra) : "memory");
  asm volatile("ld.shared::cluster.v2.f64 {%0,%1}, [%2];" : "=d"(o[2]), "=d"(o[3]) : "r"(ra + 16) : "memory");
}

// A dependency's solution vector, from this CTA's shared memory or the
// owner's (DSMEM), read again until none of its four entries is the "not yet
// written" sentinel; false after `limit` reads, or as soon as the
// context's status records a failure (so that one lost row ends every wait).
template <class T>
__device__ __forceinline__ bool ld_dep4(const T* ys, unsigned ys_addr, unsigned slot,
                                        unsigned owner, unsigned q, T* o, const int* status,
                                        unsigned limit) {
  for (unsigned s = 0; s < limit; ++s) {
    if ((s & 1023u) == 1023u && ld_volatile_i32(status) != DEV_OK) return false;
    if (owner == q) {
      const volatile T* p = ys + 4 * (size_t)slot;
      o[0] = p[0]; o[1] = p[1]; o[2] = p[2]; o[3] = p[3];
    } else {
      ld_dsmem4(ys_addr + slot * 4u * (unsigned)sizeof(T), owner, o);
    }
    if (!is_sentinel(o[0]) && !is_sentinel(o[1]) && !is_sentinel(o[2]) && !is_sentinel(o[3]))
      return true;
  }
  return false;
}

}  // namespace

namespace {

// Copies int32 elements [e0, e1) of src into dst (16-byte aligned); returns the
// offset of element e0 inside dst.  The source allocation must extend at least
// 12 bytes past element e1 - 1 (rounding up to a 16-byte multiple).
__device__ __forceinline__ int copy_ints(int* dst, const int32_t* src, int e0, int e1,
                                         uint64_t* b, unsigned* bytes) {
  int a0 = e0 & ~3;
  int a1 = (e1 + 3) & ~3;
  if (e1 > e0) {
    unsigned n = 4u * (unsigned)(a1 - a0);
    bulk_copy(dst, src + a0, n, b);
    *bytes += n;
  }
  return e0 - a0;
}

// Bytes that one level slice will bring in (must match the copies issued).
__device__ __forceinline__ unsigned int_bytes(int e0, int e1) {
  return e1 > e0 ? 4u * (unsigned)(((e1 + 3) & ~3) - (e0 & ~3)) : 0u;
}

// UPPER = false: y_i = rhs_i - sum_{k<i} L_ik y_k; at the end y_i is written to
//   outp at the row's backward-schedule position (the backward solve's rhs).
// UPPER = true:  y_i = inv(U_ii)(rhs_i - sum_{j>i} U_ij y_j); at the end
//   z_i = P zc_i + y_i.
// rhsp is in this schedule's position order.  desc[q * nlev + l] = {first
// position, end position, first block, end block} of CTA q's slice of level l;
// loc[k] = (owner CTA << 24) | slot of the dependency of block k; the rows of a
// CTA occupy consecutive slots, level after level.
template <class T, bool UPPER>
__global__ void __launch_bounds__(kCluThreads) k_tri_cluster(
    int nlev, int rows_cap, int blk_cap, int ycap, const int4* __restrict__ desc,
    const int32_t* __restrict__ srp, const int32_t* __restrict__ loc, const T* __restrict__ sv,
    const T* __restrict__ sdinv, const T* __restrict__ rhsp, const int32_t* __restrict__ dest,
    T* __restrict__ outp, const T* __restrict__ zc, int e0,
    int e1, T* __restrict__ zbase, const int* jptr, size_t stride, Ctl* ctl, const int* active) {
  if (!*active) return;  // the same flag for every CTA: the whole cluster leaves
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm);  // [0], [1]: buffers; [2]: descriptors
  int4* sdesc = reinterpret_cast<int4*>(sm + clu_desc_off());
  T* ys = reinterpret_cast<T*>(sm + clu_y_off(nlev));
  const unsigned ys_addr = saddr(ys);
  const CluBuf B = clu_buf(rows_cap, blk_cap, (int)sizeof(T), UPPER);
  unsigned char* buf0 = sm + clu_buf_off(nlev, ycap, (int)sizeof(T));
  const unsigned q = cluster_rank();
  // the last warp only stages data (lane 0 issues the bulk copies); the other
  // warps compute rows, four lanes per row
  const int tid = threadIdx.x, r = tid & 3, quad = tid >> 2;
  const int nquad = (blockDim.x - 32) >> 2;
  const int producer = blockDim.x - 32;  // thread that issues the copies
  const bool computes = tid < producer;
  const unsigned qmask = 0xFu << ((tid & 31) & ~3);
  const int q0 = (tid & 31) & ~3;
  int* status = &ctl->status;
  const unsigned lim = ctl->spin;
  __shared__ int s_bad;
  if (tid == 0) {
    s_bad = 0;
    bar_init(&bars[0]);
    bar_init(&bars[1]);
    bar_init(&bars[2]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int l) {  // producer thread: stage level l's slice
    unsigned char* bb = buf0 + (size_t)(l & 1) * B.size;
    uint64_t* bar = &bars[l & 1];
    const int4 d = sdesc[l];
    const unsigned nr = (unsigned)(d.y - d.x), nb = (unsigned)(d.w - d.z);
    unsigned bytes = int_bytes(d.x, d.y + 1) + int_bytes(d.z, d.w) + nr * 4u * (unsigned)sizeof(T) +
                     nb * 16u * (unsigned)sizeof(T);
    if (UPPER) bytes += nr * 16u * (unsigned)sizeof(T);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    bar_expect(bar, bytes);
    unsigned got = 0;
    copy_ints(reinterpret_cast<int*>(bb + B.srp), srp, d.x, d.y + 1, bar, &got);
    copy_ints(reinterpret_cast<int*>(bb + B.loc), loc, d.z, d.w, bar, &got);
    if (nr) {
      bulk_copy(bb + B.rhs, rhsp + 4 * (size_t)d.x, nr * 4u * (unsigned)sizeof(T), bar);
      if (UPPER) bulk_copy(bb + B.dinv, sdinv + 16 * (size_t)d.x, nr * 16u * (unsigned)sizeof(T), bar);
    }
    if (nb) bulk_copy(bb + B.v, sv + 16 * (size_t)d.z, nb * 16u * (unsigned)sizeof(T), bar);
  };
  if (tid == producer) {
    unsigned nb = (unsigned)nlev * 16u;
    bar_expect(&bars[2], nb);
    bulk_copy(sdesc, desc + (size_t)q * nlev, nb, &bars[2]);
  }
  if (!__syncthreads_and(bar_wait(&bars[2], 0)) && tid == 0) {
    dev_fail(status, DEV_TIMEOUT);
    s_bad = 1;
  }
  __syncthreads();
  int last_issued = -1;  // producer: the latest level whose copies were issued
  if (tid == producer && !s_bad) {
    issue(0);
    last_issued = 0;
  }
  // every slot starts as "not yet written"; every DSMEM reader must be able
  // to rely on its peers having started (and filled their slots)
  for (int x = tid; x < 4 * ycap; x += blockDim.x) ys[x] = sentinel_of(T());
  cluster_sync();
  int base = 0;  // slot of this CTA's first row of the current level
  for (int l = 0; l < nlev; ++l) {
    const int b = l & 1;
    if (!computes) {
      // producer warp: stage level l+1 into the buffer level l-1 used (its
      // readers passed the previous CTA barrier), then wait at this level's
      __syncwarp();
      if (tid == producer && l + 1 < nlev && !s_bad) {
        issue(l + 1);
        last_issued = l + 1;
      }
      __syncwarp();
      __syncthreads();
      continue;
    }
    // each warp decides for itself (a warp that gives up leaves its rows
    // unwritten; their readers then end their waits on the failed status)
    const bool waited = !s_bad && bar_wait(&bars[b], (unsigned)(l >> 1) & 1u);
    const bool ok = __all_sync(0xffffffffu, waited);
    if (!waited) {
      dev_fail(status, DEV_TIMEOUT);
      s_bad = 1;  // read again only after the next CTA barrier
    }
    const int4 d = sdesc[l];
    const int nrows = d.y - d.x;
    if (ok) {
      const unsigned char* bb = buf0 + (size_t)b * B.size;
      const int* s_srp = reinterpret_cast<const int*>(bb + B.srp) + (d.x & 3);
      const int* s_loc = reinterpret_cast<const int*>(bb + B.loc) + (d.z & 3);
      const T* s_rhs = reinterpret_cast<const T*>(bb + B.rhs);
      const T* s_dinv = reinterpret_cast<const T*>(bb + B.dinv);
      const T* s_v = reinterpret_cast<const T*>(bb + B.v);
      const int nround = (nrows + nquad - 1) / nquad;  // uniform: quads shuffle together
      for (int t0 = 0; t0 < nround; ++t0) {
        const int t = t0 * nquad + quad;
        const bool live = t < nrows;
        T y = 0;
        if (live) {
          T acc = s_rhs[4 * t + r];
          const int kb = s_srp[t] - d.z, ke = s_srp[t + 1] - d.z;
          // four dependencies at a time: lane r fetches the solution vector of
          // dependency k + r (own shared memory, or the owner's through DSMEM)
          // and the quad shares the four vectors by shuffles
          // (the factor rows are loaded before the dependencies arrive, and the
          // four dot products are independent; only the subtractions form a
          // chain, in the same order as before)
          for (int k = kb; k < ke; k += 4) {
            const int nk = min(4, ke - k);
            T a[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (u < nk) lds4(s_v + 16 * (size_t)(k + u) + 4 * r, a[u]);
            T mine[4] = {0, 0, 0, 0};
            if (k + r < ke) {
              const unsigned w = (unsigned)s_loc[k + r];
              if (!ld_dep4(ys, ys_addr, w & 0xFFFFFFu, w >> 24, q, mine, status, lim))
                dev_fail(status, DEV_TIMEOUT);
            }
            T d[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              T x[4];
#pragma unroll
              for (int cc = 0; cc < 4; ++cc) x[cc] = __shfl_sync(qmask, mine[cc], q0 + u);
              d[u] = u < nk ? dot4(a[u], x) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (u < nk) acc = sub_rn(acc, d[u]);
          }
          y = acc;
        }
        if (UPPER) {
          T s0 = __shfl_sync(qmask, y, q0 + 0);
          T s1 = __shfl_sync(qmask, y, q0 + 1);
          T s2 = __shfl_sync(qmask, y, q0 + 2);
          T s3 = __shfl_sync(qmask, y, q0 + 3);
          if (live) {
            T dd[4];
            lds4(s_dinv + 16 * (size_t)t + 4 * r, dd);
            T sv4[4] = {s0, s1, s2, s3};
            y = dot4(dd, sv4);
          }
        }
        if (live) ys[4 * (size_t)(base + t) + r] = desentinel(y);
      }
    }
    base += nrows;
    __syncthreads();  // this CTA's buffers of level l are free again
  }
  cluster_sync();  // no peer reads this CTA's slots any more
  // outputs, from this CTA's own slots: dest[q * ycap + slot] is the backward
  // position (forward solve) or the row (backward solve) of the slot, -1 if unused
  if (computes && !s_bad) {
    T* z = UPPER ? zbase + (size_t)(*jptr) * stride : nullptr;
    const int32_t* dq = dest + (size_t)q * ycap;
    constexpr int kU = 8;
    for (int sb = quad; sb < ycap; sb += nquad * kU) {
      int dd[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int sl = sb + u * nquad;
        dd[u] = sl < ycap ? dq[sl] : -1;
      }
      T y1[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        y1[u] = 0;
        if (UPPER && zc && dd[u] >= 0) {
          if (r == e0) y1[u] = zc[(e1 < 0 ? 1 : 2) * (size_t)dd[u]];
          else if (r == e1) y1[u] = zc[2 * (size_t)dd[u] + 1];
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        if (dd[u] < 0) continue;
        const T y = ys[4 * (size_t)(sb + u * nquad) + r];
        if (!UPPER) outp[4 * (size_t)dd[u] + r] = y;
        else z[4 * (size_t)dd[u] + r] = y1[u] + y;
      }
    }
  }
  // after a timeout, copies still in flight must land before the CTA exits
  if (tid == producer && s_bad) {
    bar_wait(&bars[2], 0);
    for (int l = last_issued; l >= 0 && l >= last_issued - 1; --l)
      bar_wait(&bars[l & 1], (unsigned)(l >> 1) & 1u);
  }
}

}  // namespace

namespace {

// ------------------------------------------------------------------ schedule kernels
__global__ void k_clu_count(int N, const int32_t* __restrict__ lvl, int32_t* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) atomicAdd(&cnt[lvl[i]], 1);
}
__global__ void k_clu_iota(int N, int32_t* __restrict__ v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) v[i] = i;
}
__global__ void k_clu_pos(int N, const int32_t* __restrict__ ord, int32_t* __restrict__ pos) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) pos[ord[p]] = p;
}
__global__ void k_clu_nblk(int N, const int32_t* __restrict__ ord, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ diag, bool upper,
                          int32_t* __restrict__ cnt) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int i = ord[p];
  cnt[p] = upper ? rp[i + 1] - diag[i] - 1 : diag[i] - rp[i];
}
template <class T>
__global__ void k_clu_blocks(int N, const int32_t* __restrict__ ord, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ ci, const int32_t* __restrict__ diag,
                             const double* __restrict__ LU, bool upper,
                             const int32_t* __restrict__ srp, int32_t* __restrict__ sci,
                             T* __restrict__ sv, T* __restrict__ dinv) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int i = ord[p];
  int t0 = upper ? diag[i] + 1 : rp[i];
  int o = srp[p], n = srp[p + 1] - o;
  for (int a = 0; a < n; ++a) {
    sci[o + a] = ci[t0 + a];
    for (int q = 0; q < 16; ++q) sv[16 * (size_t)(o + a) + q] = (T)LU[16 * (size_t)(t0 + a) + q];
  }
  if (dinv)
    for (int q = 0; q < 16; ++q) dinv[16 * (size_t)p + q] = (T)LU[16 * (size_t)diag[i] + q];
}
// slice q of level l: rows [lp[l] + n q / nq, lp[l] + n (q+1) / nq)
__global__ void k_clu_desc(int nlev, int nq, const int32_t* __restrict__ lp,
                           const int32_t* __restrict__ srp, int4* __restrict__ desc,
                           int* __restrict__ caps) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nlev * nq) return;
  int q = g / nlev, l = g % nlev;
  long long a = lp[l], n = lp[l + 1] - a;
  int s0 = (int)(a + n * q / nq), s1 = (int)(a + n * (q + 1) / nq);
  int k0 = srp[s0], k1 = srp[s1];
  desc[(size_t)q * nlev + l] = make_int4(s0, s1, k0, k1);
  atomicMax(&caps[0], s1 - s0);
  atomicMax(&caps[1], k1 - k0);
}
// owner CTA and slot of every position (slots of a CTA: its rows, level after level)
__global__ void k_clu_slots(int nlev, int nq, const int4* __restrict__ desc,
                            const int32_t* __restrict__ base, int32_t* __restrict__ owner) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nlev * nq) return;
  int4 d = desc[g];
  int q = g / nlev;
  for (int p = d.x; p < d.y; ++p) owner[p] = (q << 24) | (base[g] + p - d.x);
}
// dependency location of every block: owner word of the column's position
__global__ void k_clu_loc(long long nb, const int32_t* __restrict__ sci,
                          const int32_t* __restrict__ pos, const int32_t* __restrict__ owner,
                          int32_t* __restrict__ loc) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nb) loc[k] = owner[pos[sci[k]]];
}
// slot -> output index (backward position for the forward solve, row for the backward)
__global__ void k_clu_dest(int N, int ycap, const int32_t* __restrict__ owner,
                           const int32_t* __restrict__ val, int32_t* __restrict__ dest) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  unsigned w = (unsigned)owner[p];
  dest[(size_t)(w >> 24) * ycap + (w & 0xFFFFFFu)] = val[p];
}
__global__ void k_clu_pos2(int N, const int32_t* __restrict__ ord_f,
                           const int32_t* __restrict__ pos_b, int32_t* __restrict__ pos2) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) pos2[p] = pos_b[ord_f[p]];
}
template <class T>
__global__ void k_clu_gather(int N, const int32_t* __restrict__ ord, const T* __restrict__ in,
                             T* __restrict__ out, const int* active) {
  if (!*active) return;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 4ll * N) return;
  int p = (int)(g >> 2), r = (int)(g & 3);
  out[g] = in[4 * (size_t)ord[p] + r];
}

}  // namespace

namespace {

// ------------------------------------------------------------------ host side
// Positions (rows by level) and factor blocks of one direction; *lp_out gets
// the level pointers (nlev + 1 positions).
template <class T>
cptr_status build_rows(cptr_ctx* c, bool upper, CluSched& S, int32_t** lp_out) {
  const int N = c->N;
  const int nlev = upper ? c->nlev_b : c->nlev_f;
  const int32_t* lvl = upper ? c->lvl_b : c->lvl_f;
  cudaStream_t s = cs(c);
  S.nlev = nlev;
  int32_t *cnt, *lp, *bcnt;
  CTX_ALLOC(c, cnt, int32_t, nlev + 1, true);
  CTX_ALLOC(c, lp, int32_t, nlev + 1, true);
  CTX_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nlev + 1), s));
  KL(c, k_clu_count<<<nblk(N), kT, 0, s>>>(N, lvl, cnt));
  int tot = 0;
  cptr_status st = scan_i32(c, cnt, lp, nlev, &tot);
  if (st) return st;
  // int arrays carry 16 elements of slack for the rounded-up bulk copies
  CTX_ALLOC(c, S.ord, int32_t, N + 16, true);
  CTX_ALLOC(c, S.pos, int32_t, N + 16, true);
  // rows sorted by level, by index inside a level (a stable radix sort), so a
  // level slice is a contiguous index range and most dependencies stay in the
  // owning CTA
  int32_t *iota, *keys;
  CTX_ALLOC(c, iota, int32_t, N + 1, true);
  CTX_ALLOC(c, keys, int32_t, N + 1, true);
  KL(c, k_clu_iota<<<nblk(N), kT, 0, s>>>(N, iota));
  int bits = 1;
  while ((1 << bits) < nlev) ++bits;
  size_t tmp_bytes = 0;
  CTX_CUDA(c, cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, lvl, keys, iota, S.ord, N, 0,
                                              bits, s));
  void* tmp = ctx_alloc(c, tmp_bytes + 16, true);
  if (!tmp) return CPTR_ERR_NOMEM;
  CTX_CUDA(c, cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, lvl, keys, iota, S.ord, N, 0, bits,
                                              s));
  ++c->nlaunch;
  KL(c, k_clu_pos<<<nblk(N), kT, 0, s>>>(N, S.ord, S.pos));
  CTX_ALLOC(c, bcnt, int32_t, N + 1, true);
  CTX_ALLOC(c, S.rp, int32_t, N + 16, true);
  KL(c, k_clu_nblk<<<nblk(N), kT, 0, s>>>(N, S.ord, c->rp, c->diag, upper, bcnt));
  int nb = 0;
  st = scan_i32(c, bcnt, S.rp, N, &nb);
  if (st) return st;
  S.nnz = nb;
  CTX_ALLOC(c, S.ci, int32_t, (size_t)nb + 16, true);
  CTX_ALLOC(c, S.loc, int32_t, (size_t)nb + 16, true);
  S.v = ctx_alloc(c, sizeof(T) * 16 * ((size_t)nb + 1), true);
  if (!S.v) return CPTR_ERR_NOMEM;
  T* dinv = nullptr;
  if (upper) {
    dinv = (T*)ctx_alloc(c, sizeof(T) * 16 * ((size_t)N + 1), true);
    if (!dinv) return CPTR_ERR_NOMEM;
  }
  S.dinv = dinv;
  KL(c, k_clu_blocks<T><<<nblk(N), kT, 0, s>>>(N, S.ord, c->rp, c->ci, c->diag, c->LU64, upper,
                                                S.rp, S.ci, (T*)S.v, dinv));
  *lp_out = lp;
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

// Slices for nq CTAs, slots and dependency locations; CPTR_ERR_INVALID when
// the kernel's shared memory would exceed the budget.
cptr_status build_slices(cptr_ctx* c, CluSched& S, const int32_t* lp, int nq, int ts, bool upper) {
  cudaStream_t s = cs(c);
  const int nlev = S.nlev, N = c->N;
  int4* desc;
  CTX_ALLOC(c, desc, int4, (size_t)nq * nlev + 1, true);
  int* caps;
  CTX_ALLOC(c, caps, int, 2, true);
  CTX_CUDA(c, cudaMemsetAsync(caps, 0, 2 * sizeof(int), s));
  KL(c, k_clu_desc<<<nblk((long long)nq * nlev), kT, 0, s>>>(nlev, nq, lp, S.rp, desc, caps));
  std::vector<int4> hd((size_t)nq * nlev);
  int hc[2] = {0, 0};
  CTX_CUDA(c, cudaMemcpyAsync(hd.data(), desc, sizeof(int4) * hd.size(), cudaMemcpyDeviceToHost, s));
  CTX_CUDA(c, cudaMemcpyAsync(hc, caps, sizeof(hc), cudaMemcpyDeviceToHost, s));
  CTX_CUDA(c, cudaStreamSynchronize(s));
  std::vector<int32_t> hb((size_t)nq * nlev);
  int ycap = 1;
  for (int q = 0; q < nq; ++q) {
    int acc = 0;
    for (int l = 0; l < nlev; ++l) {
      const int4& d = hd[(size_t)q * nlev + l];
      hb[(size_t)q * nlev + l] = acc;
      acc += d.y - d.x;
    }
    ycap = std::max(ycap, acc);
  }
  S.nq = nq;
  S.desc = desc;
  S.rows_cap = std::max(hc[0], 1);
  S.blk_cap = std::max(hc[1], 1);
  S.ycap = ycap;
  S.smem = clu_smem(nlev, ycap, S.rows_cap, S.blk_cap, ts, upper);
  if (S.smem > kCluSmemBudget || ycap >= (1 << 24)) return CPTR_ERR_INVALID;
  int32_t *base, *owner;
  CTX_ALLOC(c, base, int32_t, hb.size() + 1, true);
  CTX_ALLOC(c, owner, int32_t, N + 1, true);
  CTX_CUDA(c, cudaMemcpyAsync(base, hb.data(), sizeof(int32_t) * hb.size(), cudaMemcpyHostToDevice, s));
  KL(c, k_clu_slots<<<nblk((long long)nq * nlev), kT, 0, s>>>(nlev, nq, desc, base, owner));
  KL(c, k_clu_loc<<<nblk(S.nnz), kT, 0, s>>>(S.nnz, S.ci, S.pos, owner, S.loc));
  CTX_ALLOC(c, S.dest, int32_t, (size_t)nq * ycap + 16, true);
  CTX_CUDA(c, cudaMemsetAsync(S.dest, 0xFF, sizeof(int32_t) * ((size_t)nq * ycap + 16), s));
  KL(c, k_clu_dest<<<nblk(N), kT, 0, s>>>(N, ycap, owner, upper ? S.ord : S.pos2, S.dest));
  // the host vectors above go out of scope: finish the upload first
  CTX_CUDA(c, cudaStreamSynchronize(s));
  return CPTR_OK;
}

template <class T, bool UPPER>
cptr_status launchable(cptr_ctx* c, int nq, size_t smem, bool* ok) {
  auto kern = k_tri_cluster<T, UPPER>;
  CTX_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  CTX_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kCluSmemBudget));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nq);
  cfg.blockDim = dim3(kCluThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = nq;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int ncl = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ncl = 0;
  }
  *ok = ncl >= 1;
  return CPTR_OK;
}

template <class T>
cptr_status build_cluster_t(cptr_ctx* c) {
  const int ts = (int)sizeof(T);
  int32_t *lp_f = nullptr, *lp_b = nullptr;
  cptr_status st = build_rows<T>(c, true, c->cb, &lp_b);
  if (!st) st = build_rows<T>(c, false, c->cf, &lp_f);
  if (st) return st;
  CTX_ALLOC(c, c->cf.pos2, int32_t, c->N + 16, true);
  KL(c, k_clu_pos2<<<nblk(c->N), kT, 0, cs(c)>>>(c->N, c->cf.ord, c->cb.pos, c->cf.pos2));
  bool found = false;
  for (int nq : {16, 8}) {
    st = build_slices(c, c->cf, lp_f, nq, ts, false);
    if (st == CPTR_ERR_INVALID) continue;
    if (st) return st;
    st = build_slices(c, c->cb, lp_b, nq, ts, true);
    if (st == CPTR_ERR_INVALID) continue;
    if (st) return st;
    bool okf = false, okb = false;
    st = launchable<T, false>(c, nq, c->cf.smem, &okf);
    if (!st) st = launchable<T, true>(c, nq, c->cb.smem, &okb);
    if (st) return st;
    if (okf && okb) { found = true; break; }
  }
  if (!found) return CPTR_ERR_INVALID;
  c->nnzL = c->cf.nnz;  // strictly lower / upper blocks (the byte and flop models)
  c->nnzU = c->cb.nnz;
  size_t n4 = 4 * (size_t)c->N;
  c->rhsf = ctx_alloc(c, sizeof(T) * n4 + 16, true);
  c->rhsb = ctx_alloc(c, sizeof(T) * n4 + 16, true);
  if (!c->rhsf || !c->rhsb) return CPTR_ERR_NOMEM;
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

template <class T, bool UPPER>
void launch_dir(cptr_ctx* c, const CluSched& S, const T* rhsp, T* outp, const T* zc, T* zbase,
                const int* jptr, size_t stride, const int* active) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(S.nq);
  cfg.blockDim = dim3(kCluThreads);
  cfg.dynamicSmemBytes = S.smem;
  cfg.stream = cs(c);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = S.nq;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  KL(c, cudaLaunchKernelEx(&cfg, k_tri_cluster<T, UPPER>, S.nlev, S.rows_cap, S.blk_cap, S.ycap,
                           (const int4*)S.desc, (const int32_t*)S.rp, (const int32_t*)S.loc,
                           (const T*)S.v, (const T*)S.dinv, rhsp, (const int32_t*)S.dest,
                           outp, zc, c->se0, c->se1, zbase, jptr,
                           stride, c->ctl, active));
}

template <class T>
void launch_t(cptr_ctx* c, const T* zc, T* zbase, const int* jptr, size_t stride,
              const int* active, int which) {
  if (which != 2) {
    KL(c, k_clu_gather<T><<<nblk(4ll * c->N), kT, 0, cs(c)>>>(
              c->N, c->cf.ord, (const T*)c->r2, (T*)c->rhsf, active));
    launch_dir<T, false>(c, c->cf, (const T*)c->rhsf, (T*)c->rhsb, nullptr, nullptr, jptr,
                         stride, active);
  }
  if (which != 1)
    launch_dir<T, true>(c, c->cb, (const T*)c->rhsb, nullptr, zc, zbase, jptr, stride, active);
}

}  // namespace

cptr_status build_cluster(cptr_ctx* c) {
  return c->mixed ? build_cluster_t<float>(c) : build_cluster_t<double>(c);
}

void launch_tri_cluster(cptr_ctx* c, const void* zc, void* zbase, const int* jptr, size_t stride,
                        const int* active, int which) {
  if (c->mixed)
    launch_t<float>(c, (const float*)zc, (float*)zbase, jptr, stride, active, which);
  else
    launch_t<double>(c, (const double*)zc, (double*)zbase, jptr, stride, active, which);
}
