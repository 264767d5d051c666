// Chunked sync-free block triangular solves for the ILU(0) second stage.
//
// Rows are cut into chunks of R consecutive rows; chunks are claimed by
// thread blocks in dependency order (top-down for L, bottom-up for U), so a
// chunk only ever waits on chunks claimed earlier by running blocks.  Inside a
// chunk the rows follow their levels in the chunk-local dependency graph, one
// __syncthreads per level, with the chunk's solution kept in shared memory.
// The chunk's factor blocks (and inverse diagonal blocks) are staged into
// shared memory by one TMA bulk copy (cp.async.bulk + mbarrier) issued right
// after the claim, so the copy overlaps the wait for upstream chunks.
// Dependencies on other chunks are read through their values, which start as
// a sentinel NaN; every wait is bounded and reports DEV_TIMEOUT.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <tuple>
#include <mutex>
#include <map>

#include "common.cuh"
#include "ctx.h"

namespace {

constexpr int kT = 256;
inline int nblk(long long n, int per = kT) { return n > 0 ? ceil_div(n, per) : 1; }

// ------------------------------------------------------------------ schedule
__device__ __forceinline__ int chunk_of(int i, int N, int R, bool upper) {
  return upper ? (N - 1 - i) / R : i / R;
}

__global__ void k_local_level_sweep(int N, int R, bool upper, const int32_t* __restrict__ rp,
                                    const int32_t* __restrict__ ci,
                                    const int32_t* __restrict__ diag, int32_t* lvl, int* changed) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int ch = chunk_of(i, N, R, upper);
  int t0 = upper ? diag[i] + 1 : rp[i];
  int t1 = upper ? rp[i + 1] : diag[i];
  int m = 0;
  for (int t = t0; t < t1; ++t) {
    int j = ci[t];
    if (chunk_of(j, N, R, upper) != ch) continue;
    int q = ld_volatile_i32(lvl + j) + 1;
    m = q > m ? q : m;
  }
  if (m != lvl[i]) {
    lvl[i] = m;
    *changed = 1;
  }
}

__global__ void k_chunk_maxlvl(int N, int R, bool upper, const int32_t* __restrict__ lvl,
                               int32_t* __restrict__ cmax) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) atomicMax(&cmax[chunk_of(i, N, R, upper)], lvl[i] + 1);
}

__global__ void k_chunk_count(int N, int R, bool upper, const int32_t* __restrict__ lvl,
                              const int32_t* __restrict__ clp, int32_t* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) atomicAdd(&cnt[clp[chunk_of(i, N, R, upper)] + lvl[i]], 1);
}

__global__ void k_chunk_fill(int N, int R, bool upper, const int32_t* __restrict__ lvl,
                             const int32_t* __restrict__ clp, const int32_t* __restrict__ lvp,
                             int32_t* __restrict__ cur, int32_t* __restrict__ ord) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int L = clp[chunk_of(i, N, R, upper)] + lvl[i];
  ord[lvp[L] + atomicAdd(&cur[L], 1)] = i;
}

__global__ void k_pos_counts(int npos, const int32_t* __restrict__ ord,
                             const int32_t* __restrict__ rp, const int32_t* __restrict__ diag,
                             bool upper, int32_t* __restrict__ cnt) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npos) return;
  int i = ord[p];
  cnt[p] = upper ? rp[i + 1] - diag[i] - 1 : diag[i] - rp[i];
}

template <class T>
__global__ void k_pos_fill(int npos, const int32_t* __restrict__ ord,
                           const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const int32_t* __restrict__ diag, const double* __restrict__ LU,
                           bool upper, const int32_t* __restrict__ srp, int32_t* __restrict__ sci,
                           T* __restrict__ sv, T* __restrict__ dinv) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npos) return;
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

__global__ void k_max_levels(int nch, const int32_t* __restrict__ cmax, int* out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nch) atomicMax(out, cmax[c]);
}

// blocks of each chunk (for the shared-memory capacity)
__global__ void k_chunk_blocks(int nch, int N, int R, const int32_t* __restrict__ srp,
                               int* maxblk) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nch) return;
  int p0 = c * R, p1 = min(N, (c + 1) * R);
  atomicMax(maxblk, srp[p1] - srp[p0]);
}

// ------------------------------------------------------------------ TMA helpers
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

template <class T>
__device__ __forceinline__ bool wait_vec4(const T* p, T* o, int* status, unsigned limit) {
  for (unsigned s = 0;; ++s) {
    ld_volatile4(p, o);
    if (!is_sentinel(o[0]) && !is_sentinel(o[1]) && !is_sentinel(o[2]) && !is_sentinel(o[3]))
      return true;
    if (s + 1 >= limit) {  // `limit` polls saw the sentinel
      dev_fail(status, DEV_TIMEOUT);
      return false;
    }
    if ((s & 255u) == 255u && ld_volatile_i32(status) != DEV_OK) return false;
  }
}

template <class T>
__device__ __forceinline__ void ld4s(const T* p, T* o) {
  if (sizeof(T) == 4) {
    float4 a = *reinterpret_cast<const float4*>(p);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  } else {
    double2 a = *reinterpret_cast<const double2*>(p);
    double2 b = *(reinterpret_cast<const double2*>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
}

// ------------------------------------------------------------------ solve kernel
// UPPER = false: out_i = rhs_i - sum_{k<i} L_ik out_k (writes the sentinel into
//   `pre`, the backward solve's output, for every row it finishes).
// UPPER = true:  out_i = inv(U_ii) (rhs_i - sum_{j>i} U_ij out_j), and
//   z_i = P zc_i + out_i.
// Shared memory per chunk (all staged by TMA bulk copies on one mbarrier):
//   blocks [cap_blocks*16 T] | dinv [R*16 T, upper] | u [R*4 T] | rhs [R*4 T] |
//   ord [R+4] | srp [R+8] | lvp [lev_cap+8] | sci [cap_blocks+8]   (ints)
struct TriSmem {
  size_t blk, dinv, u, rhs, ord, srp, lvp, sci, total;
};
__host__ __device__ inline TriSmem tri_layout(int R, int cap_blocks, int lev_cap, int tsize,
                                              bool upper) {
  TriSmem L;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o += (bytes + 15) & ~(size_t)15; return at; };
  L.blk = take((size_t)cap_blocks * 16 * tsize);
  L.dinv = take(upper ? (size_t)R * 16 * tsize : 0);
  L.u = take((size_t)R * 4 * tsize);
  L.rhs = take((size_t)R * 4 * tsize);
  L.ord = take(4 * ((size_t)R + 4));
  L.srp = take(4 * ((size_t)R + 8));
  L.lvp = take(4 * ((size_t)lev_cap + 8));
  L.sci = take(4 * ((size_t)cap_blocks + 8));
  L.total = o;
  return L;
}

template <class T, bool UPPER>
__global__ void __launch_bounds__(256) k_tri_chunk(
    int N, int R, int nch, int lev_cap, const int32_t* __restrict__ clp,
    const int32_t* __restrict__ lvp, const int32_t* __restrict__ ord,
    const int32_t* __restrict__ srp, const int32_t* __restrict__ sci, const T* __restrict__ sv,
    const T* __restrict__ dinv, int cap_blocks, const T* __restrict__ rhs, T* out,
    T* __restrict__ pre, const T* __restrict__ zc, int e0, int e1, T* __restrict__ zbase,
    const int* jptr, size_t stride, Ctl* ctl, const int* active) {
  if (!*active) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  const TriSmem Ly = tri_layout(R, cap_blocks, lev_cap, (int)sizeof(T), UPPER);
  T* sblk = reinterpret_cast<T*>(smraw + Ly.blk);
  T* sdinv = reinterpret_cast<T*>(smraw + Ly.dinv);
  T* su = reinterpret_cast<T*>(smraw + Ly.u);
  T* srhs = reinterpret_cast<T*>(smraw + Ly.rhs);
  int* sord = reinterpret_cast<int*>(smraw + Ly.ord);
  int* ssrp = reinterpret_cast<int*>(smraw + Ly.srp);
  int* slvp = reinterpret_cast<int*>(smraw + Ly.lvp);
  int* ssci = reinterpret_cast<int*>(smraw + Ly.sci);
  __shared__ uint64_t bar;
  __shared__ int s_chunk, s_c0, s_c1;
  unsigned* ctr = UPPER ? &ctl->bwd_ctr : &ctl->fwd_ctr;
  int* status = &ctl->status;
  const unsigned lim = ctl->spin;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  unsigned phase = 0;
  const int r = threadIdx.x & 3, quad = threadIdx.x >> 2, nquads = blockDim.x >> 2;
  const unsigned qmask = 0xFu << ((threadIdx.x & 31) & ~3);
  const int q0 = (threadIdx.x & 31) & ~3;
  T* z = UPPER ? zbase + (size_t)(*jptr) * stride : nullptr;
  for (;;) {
    if (threadIdx.x == 0) {
      int cc = (int)atomicAdd(ctr, 1u);
      s_chunk = cc;
      if (cc < nch) { s_c0 = clp[cc]; s_c1 = clp[cc + 1]; }
    }
    __syncthreads();
    const int c = s_chunk;
    if (c >= nch) break;
    const int lev0 = s_c0, lev1 = s_c1;
    const int lo = UPPER ? max(0, N - (c + 1) * R) : c * R;
    const int hi = UPPER ? N - c * R : min(N, (c + 1) * R);
    const int p0 = c * R, np = hi - lo;
    const int k0 = srp[p0], k1 = srp[p0 + np];
    const int nb = k1 - k0;
    const int ka = k0 & ~3;           // sci copied from a 16-byte aligned start
    const int la = lev0 & ~3;         // lvp likewise
    const bool staged = nb <= cap_blocks && (lev1 - la + 1) <= lev_cap + 4;
    if (threadIdx.x == 0) {
      auto r16 = [](unsigned b) { return (b + 15u) & ~15u; };
      unsigned b_rhs = (unsigned)(np * 4 * sizeof(T));
      unsigned b_ord = r16(4u * np), b_srp = r16(4u * (np + 1));
      unsigned b_lvp = r16(4u * (lev1 + 1 - la)), b_sci = r16(4u * (k1 - ka));
      unsigned b_blk = (unsigned)(nb * 16 * sizeof(T));
      unsigned b_dinv = UPPER ? (unsigned)(np * 16 * sizeof(T)) : 0u;
      unsigned bytes = b_rhs + (staged ? b_ord + b_srp + b_lvp + b_sci + b_blk : 0u) + b_dinv;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bar, bytes);
      bulk_g2s(srhs, rhs + 4 * (size_t)lo, b_rhs, &bar);
      if (staged) {
        bulk_g2s(sord, ord + p0, b_ord, &bar);
        bulk_g2s(ssrp, srp + p0, b_srp, &bar);
        bulk_g2s(slvp, lvp + la, b_lvp, &bar);
        if (b_sci) bulk_g2s(ssci, sci + ka, b_sci, &bar);
        if (b_blk) bulk_g2s(sblk, sv + 16 * (size_t)k0, b_blk, &bar);
      }
      if (UPPER) bulk_g2s(sdinv, dinv + 16 * (size_t)p0, b_dinv, &bar);
    }
    bool done = false;
    for (unsigned s = 0; s <= CPTR_SPIN_LIMIT; ++s)
      if (mbar_try_wait(&bar, phase)) { done = true; break; }
    phase ^= 1u;
    // block-uniform decision: if any thread gave up, the whole block stops,
    // but only after the copies it issued have landed in its shared memory
    if (__syncthreads_or(!done)) {
      if (threadIdx.x == 0) {
        dev_fail(status, DEV_TIMEOUT);
        for (unsigned s = 0; s <= CPTR_SPIN_LIMIT; ++s)
          if (mbar_try_wait(&bar, phase ^ 1u)) break;
      }
      __syncthreads();
      return;
    }
    // schedule accessors: shared memory when staged, global otherwise
    auto LVP = [&](int lev) { return staged ? slvp[lev - la] : lvp[lev]; };
    auto ORD = [&](int p) { return staged ? sord[p - p0] : ord[p]; };
    auto SRP = [&](int p) { return staged ? ssrp[p - p0] : srp[p]; };
    auto SCI = [&](int k) { return staged ? ssci[k - ka] : sci[k]; };
    // Values of the first four dependencies of the quad's first row in a level,
    // loaded from other chunks one level ahead (before the barrier) so that the
    // L2 round trip overlaps it; a value still holding the sentinel is waited for.
    T pf[4][4];
    auto prefetch = [&](int lev) {
      if (lev >= lev1) return;
      int pp = LVP(lev) + quad;
      if (pp >= LVP(lev + 1)) return;
      int kb = SRP(pp), ke = SRP(pp + 1);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int k = kb + u;
        if (k < ke) {
          int j = SCI(k);
          if (j < lo || j >= hi) ld_volatile4(out + 4 * (size_t)j, pf[u]);
        }
      }
    };
    prefetch(lev0);
    for (int lev = lev0; lev < lev1; ++lev) {
      const int pe = LVP(lev + 1);
      bool first = true;
      for (int p = LVP(lev) + quad; p < pe; p += nquads, first = false) {
        const int i = ORD(p);
        T acc = srhs[4 * (i - lo) + r];
        const int kb = SRP(p), ke = SRP(p + 1);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          int k = kb + u;
          if (k < ke) {
            int j = SCI(k);
            T a[4], x[4];
            if (staged) ld4s(sblk + 16 * (size_t)(k - k0) + 4 * r, a);
            else ld4(sv + 16 * (size_t)k + 4 * r, a);
            if (j >= lo && j < hi) {
              ld4s(su + 4 * (j - lo), x);
            } else if (first && !is_sentinel(pf[u][0]) && !is_sentinel(pf[u][1]) &&
                       !is_sentinel(pf[u][2]) && !is_sentinel(pf[u][3])) {
              x[0] = pf[u][0]; x[1] = pf[u][1]; x[2] = pf[u][2]; x[3] = pf[u][3];
            } else {
              wait_vec4(out + 4 * (size_t)j, x, status, lim);
            }
            acc = sub_rn(acc, dot4(a, x));
          }
        }
        for (int k = kb + 4; k < ke; ++k) {
          int j = SCI(k);
          T a[4], x[4];
          if (staged) ld4s(sblk + 16 * (size_t)(k - k0) + 4 * r, a);
          else ld4(sv + 16 * (size_t)k + 4 * r, a);
          if (j >= lo && j < hi) ld4s(su + 4 * (j - lo), x);
          else wait_vec4(out + 4 * (size_t)j, x, status, lim);
          acc = sub_rn(acc, dot4(a, x));
        }
        T y = acc;
        if (UPPER) {
          T s0 = __shfl_sync(qmask, acc, q0 + 0);
          T s1 = __shfl_sync(qmask, acc, q0 + 1);
          T s2 = __shfl_sync(qmask, acc, q0 + 2);
          T s3 = __shfl_sync(qmask, acc, q0 + 3);
          T d[4];
          ld4s(sdinv + 16 * (size_t)(p - p0) + 4 * r, d);
          T sv4[4] = {s0, s1, s2, s3};
          y = dot4(d, sv4);
        }
        y = desentinel(y);
        su[4 * (i - lo) + r] = y;
        st_volatile(out + 4 * (size_t)i + r, y);
        if (!UPPER) {
          pre[4 * (size_t)i + r] = sentinel_of(T(0));
        } else {
          T y1 = 0;
          if (zc) {
            const int ne = e1 < 0 ? 1 : 2;
            if (r == e0) y1 = zc[ne * (size_t)i];
            else if (r == e1) y1 = zc[ne * (size_t)i + 1];
          }
          z[4 * (size_t)i + r] = y1 + y;
        }
      }
      prefetch(lev + 1);
      __syncthreads();
    }
  }
}

template <class T>
__global__ void k_sentinel_fill(long long n, T* __restrict__ u, Ctl* ctl) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) { ctl->fwd_ctr = 0u; ctl->bwd_ctr = 0u; }
  if (i < n) u[i] = sentinel_of(T(0));
}

// ------------------------------------------------------------------ host
const size_t kSmemBudget = 200 * 1024;

cptr_status compute_local_levels(cptr_ctx* c, int R, bool upper, int32_t* lvl) {
  int N = c->N;
  const int kBatch = 16;
  int* changed;
  CTX_ALLOC(c, changed, int, kBatch, true);
  CTX_CUDA(c, cudaMemsetAsync(lvl, 0, sizeof(int32_t) * N, cs(c)));
  for (int it = 0;; it += kBatch) {
    if (it > R + 2 * kBatch) {
      ctx_set_err(c, "chunk-local level computation did not converge");
      return CPTR_ERR_BREAKDOWN;
    }
    CTX_CUDA(c, cudaMemsetAsync(changed, 0, sizeof(int) * kBatch, cs(c)));
    for (int b = 0; b < kBatch; ++b)
      KL(c, k_local_level_sweep<<<nblk(N), kT, 0, cs(c)>>>(N, R, upper, c->rp, c->ci, c->diag,
                                                               lvl, changed + b));
    int h[kBatch];
    CTX_CUDA(c, cudaMemcpyAsync(h, changed, sizeof(h), cudaMemcpyDeviceToHost, cs(c)));
    CTX_CUDA(c, cudaStreamSynchronize(cs(c)));
    if (!h[kBatch - 1]) break;
  }
  return CPTR_OK;
}

template <class T>
cptr_status build_dir(cptr_ctx* c, int R, bool upper, TriSched& S) {
  int N = c->N;
  S = TriSched();
  S.R = R;
  S.nch = ceil_div(N, R);
  int32_t *lvl, *cmax, *cnt, *cur;
  CTX_ALLOC(c, lvl, int32_t, N + 1, true);
  cptr_status st = compute_local_levels(c, R, upper, lvl);
  if (st) return st;
  CTX_ALLOC(c, cmax, int32_t, S.nch + 1, true);
  CTX_ALLOC(c, S.clp, int32_t, S.nch + 1, true);
  CTX_CUDA(c, cudaMemsetAsync(cmax, 0, sizeof(int32_t) * (S.nch + 1), cs(c)));
  KL(c, k_chunk_maxlvl<<<nblk(N), kT, 0, cs(c)>>>(N, R, upper, lvl, cmax));
  {
    int* mx;
    CTX_ALLOC(c, mx, int, 1, true);
    CTX_CUDA(c, cudaMemsetAsync(mx, 0, sizeof(int), cs(c)));
    KL(c, k_max_levels<<<nblk(S.nch), kT, 0, cs(c)>>>(S.nch, cmax, mx));
    CTX_CUDA(c, cudaMemcpyAsync(&S.lev_cap, mx, sizeof(int), cudaMemcpyDeviceToHost, cs(c)));
    CTX_CUDA(c, cudaStreamSynchronize(cs(c)));
  }
  int TL = 0;
  st = scan_i32(c, cmax, S.clp, S.nch, &TL);
  if (st) return st;
  CTX_ALLOC(c, cnt, int32_t, TL + 1, true);
  CTX_ALLOC(c, cur, int32_t, TL + 1, true);
  CTX_ALLOC(c, S.lvp, int32_t, TL + 1, true);
  CTX_ALLOC(c, S.ord, int32_t, N + 1, true);
  CTX_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (TL + 1), cs(c)));
  CTX_CUDA(c, cudaMemsetAsync(cur, 0, sizeof(int32_t) * (TL + 1), cs(c)));
  KL(c, k_chunk_count<<<nblk(N), kT, 0, cs(c)>>>(N, R, upper, lvl, S.clp, cnt));
  st = scan_i32(c, cnt, S.lvp, TL, nullptr);
  if (st) return st;
  KL(c, k_chunk_fill<<<nblk(N), kT, 0, cs(c)>>>(N, R, upper, lvl, S.clp, S.lvp, cur, S.ord));
  int32_t* pc;
  CTX_ALLOC(c, pc, int32_t, N + 1, true);
  CTX_ALLOC(c, S.rp, int32_t, N + 1, true);
  KL(c, k_pos_counts<<<nblk(N), kT, 0, cs(c)>>>(N, S.ord, c->rp, c->diag, upper, pc));
  int tot = 0;
  st = scan_i32(c, pc, S.rp, N, &tot);
  if (st) return st;
  S.nnz = tot;
  CTX_ALLOC(c, S.ci, int32_t, tot + 1, true);
  S.v = ctx_alloc(c, sizeof(T) * (16 * (size_t)tot + 16), true);
  if (!S.v) return CPTR_ERR_NOMEM;
  if (upper) {
    S.dinv = ctx_alloc(c, sizeof(T) * (16 * (size_t)N + 16), true);
    if (!S.dinv) return CPTR_ERR_NOMEM;
  }
  KL(c, k_pos_fill<T><<<nblk(N), kT, 0, cs(c)>>>(N, S.ord, c->rp, c->ci, c->diag, c->LU64,
                                                     upper, S.rp, S.ci, (T*)S.v, (T*)S.dinv));
  int* mb;
  CTX_ALLOC(c, mb, int, 1, true);
  CTX_CUDA(c, cudaMemsetAsync(mb, 0, sizeof(int), cs(c)));
  KL(c, k_chunk_blocks<<<nblk(S.nch), kT, 0, cs(c)>>>(S.nch, N, R, S.rp, mb));
  int maxblk = 0;
  CTX_CUDA(c, cudaMemcpyAsync(&maxblk, mb, sizeof(int), cudaMemcpyDeviceToHost, cs(c)));
  CTX_CUDA(c, cudaStreamSynchronize(cs(c)));
  size_t fixed = tri_layout(R, 0, S.lev_cap, (int)sizeof(T), upper).total;
  if (fixed + 256 > kSmemBudget) return CPTR_ERR_INVALID;
  long long cap = (long long)((kSmemBudget - fixed - 256) / (16 * sizeof(T) + 4));
  S.cap_blocks = (int)std::min<long long>(cap, maxblk);
  S.smem = tri_layout(R, S.cap_blocks, S.lev_cap, (int)sizeof(T), upper).total;
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

template <class T>
void launch_t(cptr_ctx* c, const T* zc, T* zbase, const int* jptr, size_t stride,
              const int* active, int which) {
  cudaStream_t s = cs(c);
  const TriSched& F = c->tf;
  const TriSched& B = c->tb;
  // as many blocks as fit at once (shared memory per SM ~228 KB), at most one per chunk
  auto per_sm = [](size_t smem) { return std::max<int>(1, std::min<int>(8, (int)(227000 / (smem + 1024)))); };
  int gf = std::min(F.nch, c->nsm * per_sm(F.smem));
  int gb = std::min(B.nch, c->nsm * per_sm(B.smem));
  if (which != 2)
    KL(c, k_tri_chunk<T, false><<<gf, 256, F.smem, s>>>(
              c->N, F.R, F.nch, F.lev_cap, F.clp, F.lvp, F.ord, F.rp, F.ci, (const T*)F.v, nullptr,
              F.cap_blocks, (const T*)c->r2, (T*)c->u, (T*)c->y2, nullptr, 0, 0, nullptr, jptr,
              stride, c->ctl, active));
  if (which != 1)
    KL(c, k_tri_chunk<T, true><<<gb, 256, B.smem, s>>>(
              c->N, B.R, B.nch, B.lev_cap, B.clp, B.lvp, B.ord, B.rp, B.ci, (const T*)B.v,
              (const T*)B.dinv,
              B.cap_blocks, (const T*)c->u, (T*)c->y2, nullptr, zc, c->se0, c->se1, zbase, jptr,
              stride, c->ctl, active));
}

template <class T>
cptr_status set_smem_attrs(cptr_ctx* c) {
  CTX_CUDA(c, cudaFuncSetAttribute(k_tri_chunk<T, false>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget));
  CTX_CUDA(c, cudaFuncSetAttribute(k_tri_chunk<T, true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget));
  return CPTR_OK;
}

template <class T>
cptr_status build_t(cptr_ctx* c, int R) {
  cptr_status st = set_smem_attrs<T>(c);
  if (st) return st;
  st = build_dir<T>(c, R, false, c->tf);
  if (!st) st = build_dir<T>(c, R, true, c->tb);
  if (st) return st;
  c->nnzL = c->tf.nnz;
  c->nnzU = c->tb.nnz;
  c->chunked = true;
  return CPTR_OK;
}

// time forward + backward solves with zero right-hand sides (values do not
// matter, only the dependency propagation)
// R: 0 level kernels, 1 cluster, > 1 chunked
template <class T>
cptr_status time_solves(cptr_ctx* c, int R, float* ms_out) {
  cudaStream_t s = cs(c);
  long long n4 = 4ll * c->N;
  CTX_CUDA(c, cudaMemsetAsync(c->r2, 0, sizeof(T) * n4, s));
  cudaEvent_t e0, e1;
  CTX_CUDA(c, cudaEventCreate(&e0));
  CTX_CUDA(c, cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    KL(c, k_sentinel_fill<T><<<nblk(n4), kT, 0, s>>>(n4, (T*)c->u, c->ctl));
    CTX_CUDA(c, cudaEventRecord(e0, s));
    if (R > 3)
      launch_t<T>(c, nullptr, (T*)c->zt, &c->ctl->zero, (size_t)n4, &c->ctl->one, 0);
    else if (R == 3)
      launch_tri_chain(c, nullptr, c->zt, &c->ctl->zero, (size_t)n4, &c->ctl->one, 0);
    else if (R == 2)
      launch_tri_strip(c, nullptr, c->zt, &c->ctl->zero, (size_t)n4, &c->ctl->one, 0);
    else if (R == 1)
      launch_tri_cluster(c, nullptr, c->zt, &c->ctl->zero, (size_t)n4, &c->ctl->one, 0);
    else
      launch_level_solves(c, c->zt);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
      // a candidate that cannot launch is skipped, never chosen
      if (c->timing) fprintf(stderr, "[cptr]   tri solve launch failed: %s\n", cudaGetErrorString(le));
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return CPTR_ERR_INVALID;
    }
    CTX_CUDA(c, cudaEventRecord(e1, s));
    CTX_CUDA(c, cudaEventSynchronize(e1));
    float ms = 0.f;
    CTX_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = best;
  return ctx_check_device_status(c);
}

// Tuner decisions shared by every context of the process, keyed by what
// determines them: device, cells, blocks, forward and backward level counts
// and the apply precision.  Every schedule computes bit-identical results, so a
// decision taken on another matrix of the same shape can only cost speed; it
// spares each new context (a served request, a new Newton system) the trial
// solves of every candidate.
struct TuneKey {
  int dev, n, nnzb, nlev_f, nlev_b, mixed;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, n, nnzb, nlev_f, nlev_b, mixed) <
           std::tie(o.dev, o.n, o.nnzb, o.nlev_f, o.nlev_b, o.mixed);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune_cache;

template <class T>
cptr_status tune_t(cptr_ctx* c) {
  const char* env = getenv("CPTR_TRI_R");
  int forced = env ? atoi(env) : -1;
  if (forced >= 0) c->tuned_R = forced;
  // without timing: a cluster when its rows fit, else level kernels
  if (c->tuned_R < 0 && !c->p.tri_tune) c->tuned_R = 1;
  const TuneKey key{c->dev, c->N, c->nnzb, c->nlev_f, c->nlev_b, c->mixed ? 1 : 0};
  if (c->tuned_R < 0) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) c->tuned_R = it->second;
  }
  c->chunked = c->cluster = c->strip = c->chain = false;
  if (c->tuned_R == 0) return build_level_solve_arrays(c);
  if (c->tuned_R == 1) {
    cptr_status st = build_cluster(c);
    if (st != CPTR_ERR_INVALID) {
      c->cluster = st == CPTR_OK;
      return st;
    }
    return build_level_solve_arrays(c);  // no cluster fits: level kernels
  }
  if (c->tuned_R == 2) {
    cptr_status st = build_strip(c);
    if (st != CPTR_ERR_INVALID) {
      c->strip = st == CPTR_OK;
      return st;
    }
    return build_level_solve_arrays(c);  // a step does not fit: level kernels
  }
  if (c->tuned_R == 3) {
    cptr_status st = build_chain(c);
    if (st != CPTR_ERR_INVALID) {
      c->chain = st == CPTR_OK;
      return st;
    }
    return build_level_solve_arrays(c);  // chains that could wait on later ones: level kernels
  }
  if (c->tuned_R > 3) {
    cptr_status st = build_t<T>(c, c->tuned_R);
    if (st != CPTR_ERR_INVALID) return st;
    c->chunked = false;  // the chunk does not fit in shared memory: level kernels
    return build_level_solve_arrays(c);
  }
  // work buffers for timing
  size_t n4 = 4 * (size_t)c->N;
  if (!c->r2) {
    c->r2 = ctx_alloc(c, sizeof(T) * n4 + 16, true);
    c->u = ctx_alloc(c, sizeof(T) * n4 + 16, true);
    c->y2 = ctx_alloc(c, sizeof(T) * n4 + 16, true);
    c->zt = ctx_alloc(c, sizeof(T) * n4 + 16, true);
    if (!c->r2 || !c->u || !c->y2 || !c->zt) return CPTR_ERR_NOMEM;
  }
  std::vector<int> cand = {0, 1, 2, 3};
  for (int R : {128, 256, 512, 1024, 2048})
    if (R <= 2 * c->N) cand.push_back(R);
  int best_R = 0;
  float best_ms = 1e30f;
  // A chunked schedule needs every chunk resident at once: with more chunks
  // than thread blocks that fit on the GPU, the persistent blocks walk the
  // dependency chains one chunk after another (on a 200x200x100 grid that is
  // seconds per solve), so such chunk sizes are not candidates.
  auto per_sm = [](size_t smem) {
    return std::max<int>(1, std::min<int>(8, (int)(227000 / (smem + 1024))));
  };
  for (int R : cand) {
    if (R > 3 && (long long)ceil_div(c->N, R) > 8ll * c->nsm) continue;
    cptr_status st = (R == 0) ? build_level_solve_arrays(c)
                     : (R == 1) ? build_cluster(c) : (R == 2) ? build_strip(c)
                     : (R == 3) ? build_chain(c) : build_t<T>(c, R);
    if (st == CPTR_ERR_INVALID) continue;  // does not fit in shared memory
    if (st) return st;
    if (R > 3 && (c->tf.nch > c->nsm * per_sm(c->tf.smem) ||
                  c->tb.nch > c->nsm * per_sm(c->tb.smem)))
      continue;
    c->chunked = R > 3;
    c->cluster = R == 1;
    c->strip = R == 2;
    c->chain = R == 3;
    float ms = 0.f;
    st = time_solves<T>(c, R, &ms);
    if (st == CPTR_ERR_INVALID) continue;
    if (st) return st;
    if (c->timing) fprintf(stderr, "[cptr]   tri solve R=%-5d %8.3f ms\n", R, ms);
    if (ms < best_ms) { best_ms = ms; best_R = R; }
  }
  c->tuned_R = best_R;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best_R;
  }
  c->chunked = c->cluster = c->strip = c->chain = false;
  if (best_R == 0) return build_level_solve_arrays(c);
  if (best_R == 1) {
    cptr_status st = build_cluster(c);
    c->cluster = st == CPTR_OK;
    return st;
  }
  if (best_R == 2) {
    cptr_status st = build_strip(c);
    c->strip = st == CPTR_OK;
    return st;
  }
  if (best_R == 3) {
    cptr_status st = build_chain(c);
    c->chain = st == CPTR_OK;
    return st;
  }
  return build_t<T>(c, best_R);
}

}  // namespace

cptr_status build_chunked(cptr_ctx* c, int R) {
  return c->mixed ? build_t<float>(c, R) : build_t<double>(c, R);
}

// Whether the schedule is already decided (forced, tuned by an earlier setup
// of this context, or cached for this shape): then building it times nothing.
bool tune_decided(cptr_ctx* c) {
  const char* env = getenv("CPTR_TRI_R");
  if ((env && atoi(env) >= 0) || c->tuned_R >= 0 || !c->p.tri_tune) return true;
  const TuneKey key{c->dev, c->N, c->nnzb, c->nlev_f, c->nlev_b, c->mixed ? 1 : 0};
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune_cache.count(key) > 0;
}

cptr_status tune_triangular(cptr_ctx* c) {
  return c->mixed ? tune_t<float>(c) : tune_t<double>(c);
}

void launch_tri_chunked(cptr_ctx* c, const void* zc, void* zbase, const int* jptr, size_t stride,
                        const int* active, int which) {
  if (c->mixed)
    launch_t<float>(c, (const float*)zc, (float*)zbase, jptr, stride, active, which);
  else
    launch_t<double>(c, (const double*)zc, (double*)zbase, jptr, stride, active, which);
}
