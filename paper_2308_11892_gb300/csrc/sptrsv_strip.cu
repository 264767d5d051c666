// Strip-owned block triangular solves for the ILU(0) second stage of large
// systems (hundreds of thousands of rows and more).
//
// The rows are cut into P contiguous index strips (counted from the first row
// for the lower triangle, from the last for the upper one), one per CTA, and
// each CTA walks its own strip level by level in the global level order of the
// ILU(0) level sets (rows of a level, by index), one CTA barrier per step.
// Most dependencies of a row lie in its own strip at an earlier level: the CTA
// keeps the solutions of its most recent rows in a shared-memory ring and reads
// them from there.  Dependencies on other strips (and on own rows that have
// left the ring) are read from a global array in schedule-position order whose
// entries start as a sentinel NaN, polled until final (bounded).  A CTA only
// waits on strips that started before it (strips are assigned by a ticket in
// start order), so the solve progresses even when not every CTA is resident.
// A producer warp stages each step (row records, right-hand sides, dependency
// codes, factor blocks and, for the upper solve, inverse diagonal blocks) into a
// shared-memory byte ring with TMA bulk copies, up to kNB steps ahead of the
// rows being computed.  Each row's sum uses the same rounding sequence as every
// other schedule (dot4, sub_rn, in block order), so results are bit-identical.
#include <algorithm>
#include <cstdio>
#include <vector>

#include <cub/device/device_radix_sort.cuh>

#include "common.cuh"
#include "ctx.h"

namespace {

constexpr int kT = 256;
constexpr int kStripWarps = 16;                        // warps computing rows
constexpr int kStripThreads = 32 * (kStripWarps + 1);  // + one producer warp
constexpr int kNB = 8;                                 // steps staged ahead
// row rounds whose cross-strip dependencies are read one step ahead
template <class T> struct Prefetch { static constexpr int n = sizeof(T) == 4 ? 3 : 1; };
constexpr unsigned kLocal = 0x80000000u;               // dependency code: ring slot
inline int nblk(long long n, int per = kT) { return n > 0 ? ceil_div(n, per) : 1; }

// ------------------------------------------------------------------ device helpers
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
__device__ __forceinline__ bool bar_wait(uint64_t* b, unsigned parity) {
  for (unsigned s = 0; s < (unsigned)CPTR_SPIN_LIMIT; ++s)
    if (bar_try(b, parity)) return true;
  return false;
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
// A final value from the global position-ordered array: read until none of its
// four entries is the sentinel; false after `limit` reads or as soon as
// the context records a failure.
template <class T>
__device__ __forceinline__ bool poll4(const T* p, T* o, const int* status, unsigned limit) {
  for (unsigned s = 0;; ++s) {
    ld_volatile4(p, o);
    if (!is_sentinel(o[0]) && !is_sentinel(o[1]) && !is_sentinel(o[2]) && !is_sentinel(o[3]))
      return true;
    if (s + 1 >= limit) return false;  // `limit` polls saw the sentinel
    if ((s & 255u) == 255u && ld_volatile_i32(status) != DEV_OK) return false;
  }
}

// Bytes one step occupies in the ring (must match the copies issued):
// meta [nr int4] | rhs [nr*4 T] | loc [nb int] | v [nb*16 T] | dinv [nr*16 T]
__host__ __device__ inline unsigned step_bytes(int nr, int nb, int ts, bool upper) {
  return (unsigned)nr * (16u + 4u * ts + (upper ? 16u * ts : 0u)) + (unsigned)nb * (4u + 16u * ts);
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
// barrier among the warps that compute rows (the producer warp is not part of it)
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(32 * kStripWarps) : "memory");
}

// UPPER = false: y_i = rhs_i - sum_{k<i} L_ik y_k; also writes y_i as the
//   backward solve's right-hand side (at the row's backward position) and
//   resets the backward poll array there to the sentinel.
// UPPER = true:  y_i = inv(U_ii)(rhs_i - sum_{j>i} U_ij y_j), z_i = P zc_i + y_i.
// step[s] = {first position, end position, first block, end block} (blocks
// numbered with each step padded to a multiple of four), sptr[q]..sptr[q+1]
// the steps of strip q; meta[p] = {row, first block, end block (both relative
// to the step's first block), backward position (forward only)}; loc[k] =
// kLocal | ring slot, or the global position of the dependency.
// The producer warp stages step u into ring space and ring slot u % kNB once
// that slot's previous step is consumed (empty barrier) and arms full[u % kNB];
// the computing warps wait on full, compute the step's rows, synchronise among
// themselves (the ring entries written become readable) and release the slot.
template <class T, bool UPPER>
__global__ void __launch_bounds__(kStripThreads, 1) k_tri_strip(
    int RC, unsigned ring_bytes, const int32_t* __restrict__ sptr, const int4* __restrict__ step,
    const int4* __restrict__ meta, const int32_t* __restrict__ loc, const T* __restrict__ sv,
    const T* __restrict__ sdinv, const T* __restrict__ rhsp, T* outp, T* __restrict__ nextp,
    T* __restrict__ nextout, const T* __restrict__ zc, int e0, int e1, T* __restrict__ zbase,
    const int* jptr, size_t stride, unsigned* ticket, Ctl* ctl, const int* active) {
  if (!*active) return;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sm);                  // [kNB]
  uint64_t* empty = full + kNB;                                      // [kNB]
  int4* sinfo = reinterpret_cast<int4*>(sm + 16 * kNB);              // [kNB] {pos, nr, nb, off}
  T* ys = reinterpret_cast<T*>(sm + 32 * kNB);                       // [RC][4]
  unsigned char* ring = sm + 32 * kNB + (size_t)RC * 4 * sizeof(T);
  const int tid = threadIdx.x, r = tid & 3, quad = tid >> 2;
  const int nquad = kStripWarps * 8;
  const unsigned qmask = 0xFu << ((tid & 31) & ~3);
  const int q0 = (tid & 31) & ~3;
  int* status = &ctl->status;
  __shared__ int s_q;
  __shared__ volatile int s_bad;
  if (tid == 0) {
    s_q = (int)atomicAdd(ticket, 1u);  // strips in start order: waits only on earlier ones
    s_bad = 0;
    for (int b = 0; b < kNB; ++b) {
      bar_init(&full[b]);
      bar_init(&empty[b]);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int q = s_q;
  const int s0 = sptr[q], s1 = sptr[q + 1];
  const int nsteps = s1 - s0;
  if (nsteps <= 0) return;

  if (tid >= 32 * kStripWarps) {
    // ---------------- producer warp (lane 0 issues; the warp loads descriptors)
    const int lane = tid & 31;
    int live = 0, t_done = 0, t_issue = 0;
    unsigned head = 0, tail = 0;
    int4 dcur = lane < nsteps ? step[s0 + lane] : make_int4(0, 0, 0, 0);
    int4 dnext = 32 + lane < nsteps ? step[s0 + 32 + lane] : make_int4(0, 0, 0, 0);
    int dbase = 0;  // step index held by lane 0 of dcur
    unsigned tail_of[kNB];
#pragma unroll
    for (int b = 0; b < kNB; ++b) tail_of[b] = 0;
    // the oldest live step is consumed: its ring space comes back
    auto retire = [&]() -> bool {
      const int b = t_done % kNB;
      if (!bar_wait(&empty[b], (unsigned)(t_done / kNB) & 1u)) return false;
      ++t_done;
      --live;
      if (live > 0) {
#pragma unroll
        for (int bb = 0; bb < kNB; ++bb)
          if (bb == t_done % kNB) tail = tail_of[bb];
      }
      return true;
    };
    bool ok = true;
    for (int u = 0; u < nsteps && ok; ++u) {
      if (u - dbase == 32) {  // next 32 descriptors
        dcur = dnext;
        dbase += 32;
        dnext = dbase + 32 + lane < nsteps ? step[s0 + dbase + 32 + lane] : make_int4(0, 0, 0, 0);
      }
      const int src = u - dbase;
      int4 d;
      d.x = __shfl_sync(0xffffffffu, dcur.x, src);
      d.y = __shfl_sync(0xffffffffu, dcur.y, src);
      d.z = __shfl_sync(0xffffffffu, dcur.z, src);
      d.w = __shfl_sync(0xffffffffu, dcur.w, src);
      const int nr = d.y - d.x, nbp = (d.w - d.z + 3) & ~3;
      const unsigned sz = step_bytes(nr, nbp, (int)sizeof(T), UPPER);
      if (lane == 0) {
        if (u - t_done >= kNB) ok = retire();  // the slot's previous step
        unsigned off = 0;
        while (ok) {
          if (live == 0) {
            head = tail = 0;
            off = 0;
            break;
          }
          if (head > tail) {
            if (head + sz <= ring_bytes) { off = head; break; }
            if (sz <= tail) { off = 0; break; }
          } else if (head < tail) {
            if (head + sz <= tail) { off = head; break; }
          }
          ok = retire();  // no room yet: wait for the oldest step
        }
        if (ok && s_bad) ok = false;
        if (ok) {
          const int b = u % kNB;
          sinfo[b] = make_int4(d.x, nr, nbp, (int)off);
#pragma unroll
          for (int bb = 0; bb < kNB; ++bb)
            if (bb == b) tail_of[bb] = off;
          unsigned char* base = ring + off;
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bar_expect(&full[b], sz);
          const unsigned bm = (unsigned)nr * 16u, br = (unsigned)nr * 4u * sizeof(T);
          const unsigned bl = (unsigned)nbp * 4u, bv = (unsigned)nbp * 16u * sizeof(T);
          if (nr) {
            bulk_copy(base, meta + d.x, bm, &full[b]);
            bulk_copy(base + bm, rhsp + 4 * (size_t)d.x, br, &full[b]);
          }
          if (nbp) {
            bulk_copy(base + bm + br, loc + d.z, bl, &full[b]);
            bulk_copy(base + bm + br + bl, sv + 16 * (size_t)d.z, bv, &full[b]);
          }
          if (UPPER && nr)
            bulk_copy(base + bm + br + bl + bv, sdinv + 16 * (size_t)d.x,
                      (unsigned)nr * 16u * sizeof(T), &full[b]);
          head = off + sz;
          ++live;
          t_issue = u + 1;
        } else {
          dev_fail(status, DEV_TIMEOUT);
          s_bad = 1;
        }
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    }
    // copies still in flight must land before the CTA exits
    if (lane == 0)
      for (int u = max(0, t_issue - kNB); u < t_issue; ++u)
        bar_wait(&full[u % kNB], (unsigned)(u / kNB) & 1u);
    return;
  }

  // ---------------- computing warps
  const int pbase = step[s0].x;  // first position of the strip
  const unsigned lim = ctl->spin;
  T* z = UPPER ? zbase + (size_t)(*jptr) * stride : nullptr;
  constexpr int kPF = Prefetch<T>::n;
  // Values of the dependencies in other strips (first group of four of the
  // rows of the first kPF rounds) are read one step ahead, while the current
  // step computes, so that the L2 round trip overlaps it; a value that still
  // holds the sentinel is polled again when the row needs it.
  T pf[kPF][4];
#pragma unroll
  for (int u = 0; u < kPF; ++u) pf[u][0] = pf[u][1] = pf[u][2] = pf[u][3] = sentinel_of(T(0));
  for (int t = 0; t < nsteps; ++t) {
    const int b = t % kNB;
    const bool waited = !s_bad && bar_wait(&full[b], (unsigned)(t / kNB) & 1u);
    if (!waited && !s_bad) {
      dev_fail(status, DEV_TIMEOUT);
      s_bad = 1;
    }
    T pn[kPF][4];
#pragma unroll
    for (int u = 0; u < kPF; ++u) pn[u][0] = pn[u][1] = pn[u][2] = pn[u][3] = sentinel_of(T(0));
    if (t + 1 < nsteps && !s_bad &&
        bar_try(&full[(t + 1) % kNB], (unsigned)((t + 1) / kNB) & 1u)) {
      const int4 in1 = sinfo[(t + 1) % kNB];
      const unsigned char* b1 = ring + in1.w;
      const int4* m1 = reinterpret_cast<const int4*>(b1);
      const int* l1 = reinterpret_cast<const int*>(b1 + (size_t)in1.y * (16 + 4 * sizeof(T)));
#pragma unroll
      for (int u = 0; u < kPF; ++u) {
        const int k1 = u * nquad + quad;
        if (k1 < in1.y) {
          const int4 mt1 = m1[k1];
          if (mt1.y + r < mt1.z) {
            const unsigned w = (unsigned)l1[mt1.y + r];
            if (!(w & kLocal)) ld_volatile4(outp + 4 * (size_t)w, pn[u]);
          }
        }
      }
    }
    if (__all_sync(0xffffffffu, waited)) {
      const int4 info = sinfo[b];
      const int nr = info.y, nbp = info.z;
      const unsigned char* base = ring + info.w;
      const int4* s_meta = reinterpret_cast<const int4*>(base);
      const T* s_rhs = reinterpret_cast<const T*>(base + (size_t)nr * 16);
      const int* s_loc = reinterpret_cast<const int*>(base + (size_t)nr * (16 + 4 * sizeof(T)));
      const T* s_v = reinterpret_cast<const T*>(base + (size_t)nr * (16 + 4 * sizeof(T)) +
                                                (size_t)nbp * 4);
      const T* s_dinv = s_v + 16 * (size_t)nbp;
      const int nround = (nr + nquad - 1) / nquad;
      // one row per quad and round; pre = the prefetched first-group value (or sentinel)
      auto row = [&](int k, const T* pre) {
        const bool live_row = k < nr;
        int4 mt = make_int4(0, 0, 0, 0);
        T y = 0;
        if (live_row) {
          mt = s_meta[k];
          T acc = s_rhs[4 * k + r];
          const int kb = mt.y, ke = mt.z;
          for (int kk = kb; kk < ke; kk += 4) {
            const int nk = min(4, ke - kk);
            T a[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (u < nk) lds4(s_v + 16 * (size_t)(kk + u) + 4 * r, a[u]);
            // lane r fetches the solution vector of dependency kk + r
            T mine[4] = {0, 0, 0, 0};
            if (kk + r < ke) {
              const unsigned w = (unsigned)s_loc[kk + r];
              if (w & kLocal) {
                lds4(ys + 4 * (size_t)(w & ~kLocal), mine);
              } else if (kk == kb && pre && !is_sentinel(pre[0]) && !is_sentinel(pre[1]) &&
                         !is_sentinel(pre[2]) && !is_sentinel(pre[3])) {
                mine[0] = pre[0]; mine[1] = pre[1]; mine[2] = pre[2]; mine[3] = pre[3];
              } else if (!poll4(outp + 4 * (size_t)w, mine, status, lim)) {
                dev_fail(status, DEV_TIMEOUT);
              }
            }
            T dd[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              T x[4];
#pragma unroll
              for (int cc = 0; cc < 4; ++cc) x[cc] = __shfl_sync(qmask, mine[cc], q0 + u);
              dd[u] = u < nk ? dot4(a[u], x) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (u < nk) acc = sub_rn(acc, dd[u]);
          }
          y = acc;
        }
        if (UPPER) {
          T s0v = __shfl_sync(qmask, y, q0 + 0);
          T s1v = __shfl_sync(qmask, y, q0 + 1);
          T s2v = __shfl_sync(qmask, y, q0 + 2);
          T s3v = __shfl_sync(qmask, y, q0 + 3);
          if (live_row) {
            T dv[4];
            lds4(s_dinv + 16 * (size_t)k + 4 * r, dv);
            T sv4[4] = {s0v, s1v, s2v, s3v};
            y = dot4(dv, sv4);
          }
        }
        if (live_row) {
          y = desentinel(y);
          const int p = info.x + k;
          ys[4 * (size_t)((p - pbase) % RC) + r] = y;
          st_volatile(outp + 4 * (size_t)p + r, y);
          if (!UPPER) {
            nextp[4 * (size_t)mt.w + r] = y;
            nextout[4 * (size_t)mt.w + r] = sentinel_of(T(0));
          } else {
            const int i = mt.x;
            T y1 = 0;
            if (zc) {
              const int ne = e1 < 0 ? 1 : 2;
              if (r == e0) y1 = zc[ne * (size_t)i];
              else if (r == e1) y1 = zc[ne * (size_t)i + 1];
            }
            z[4 * (size_t)i + r] = y1 + y;
          }
        }
      };
#pragma unroll
      for (int u = 0; u < kPF; ++u)
        if (u < nround) row(u * nquad + quad, pf[u]);
      for (int t0 = kPF; t0 < nround; ++t0) row(t0 * nquad + quad, nullptr);
    }
#pragma unroll
    for (int u = 0; u < kPF; ++u) {
      pf[u][0] = pn[u][0]; pf[u][1] = pn[u][1]; pf[u][2] = pn[u][2]; pf[u][3] = pn[u][3];
    }
    consumers_sync();  // the step's ring entries are written; its staged data is no longer read
    if (tid == 0) bar_arrive(&empty[b]);
  }
}

// r2 (natural order) -> forward rhs in forward position order, and the forward
// poll array to the sentinel; the strip tickets restart at zero.
template <class T>
__global__ void k_strip_gather(int N, const int32_t* __restrict__ ord, const T* __restrict__ in,
                               T* __restrict__ out, T* __restrict__ poll, Ctl* ctl,
                               const int* active) {
  if (!*active) return;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0) { ctl->fwd_ctr = 0u; ctl->bwd_ctr = 0u; }
  if (g >= 4ll * N) return;
  int p = (int)(g >> 2), r = (int)(g & 3);
  out[g] = in[4 * (size_t)ord[p] + r];
  poll[g] = sentinel_of(T(0));
}

// ------------------------------------------------------------------ schedule kernels
__device__ __forceinline__ int strip_of(int i, int N, int S, bool upper) {
  return upper ? (N - 1 - i) / S : i / S;
}
__global__ void k_st_keys(int N, int S, int nlev, bool upper, const int32_t* __restrict__ lvl,
                          int32_t* __restrict__ key, int32_t* __restrict__ iota,
                          int32_t* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  // upper rows are listed from the last one: sort key by (strip, level, N-1-i)
  int row = upper ? N - 1 - i : i;
  int k = strip_of(row, N, S, upper) * nlev + lvl[row];
  key[i] = k;
  iota[i] = row;
  atomicAdd(&cnt[k], 1);
}
__global__ void k_st_pos(int N, const int32_t* __restrict__ ord, int32_t* __restrict__ pos) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) pos[ord[p]] = p;
}
__global__ void k_st_nblk(int N, const int32_t* __restrict__ ord, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ diag, bool upper, int32_t* __restrict__ cnt) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int i = ord[p];
  cnt[p] = upper ? rp[i + 1] - diag[i] - 1 : diag[i] - rp[i];
}
// Sub-steps of each (strip, level) bucket: consecutive rows, cut when the
// step's ring bytes would exceed cap.  pass 0 counts them into nsub[bucket];
// pass 1 writes {first position, end position, raw block count, 0} at sbase.
__global__ void k_st_split(int nbk, const int32_t* __restrict__ cscan,
                           const int32_t* __restrict__ bscan, unsigned cap, int ts, bool upper,
                           int pass, int32_t* __restrict__ nsub, const int32_t* __restrict__ sbase,
                           int4* __restrict__ desc) {
  int bk = blockIdx.x * blockDim.x + threadIdx.x;
  if (bk >= nbk) return;
  int p0 = cscan[bk], p1 = cscan[bk + 1];
  int n = 0, a = p0;
  while (a < p1) {
    int e = a + 1;
    while (e < p1) {
      int nb = bscan[e + 1] - bscan[a];
      if (step_bytes(e + 1 - a, (nb + 3) & ~3, ts, upper) > cap) break;
      ++e;
    }
    if (pass == 1) desc[sbase[bk] + n] = make_int4(a, e, bscan[e] - bscan[a], 0);
    ++n;
    a = e;
  }
  if (pass == 0) nsub[bk] = n;
}
__global__ void k_st_padcnt(int ns, const int4* __restrict__ desc, int32_t* __restrict__ cnt) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < ns) cnt[s] = (desc[s].z + 3) & ~3;
}
// final descriptors (padded block ranges) and per-position records; pblk[p] is
// the global index of position p's first block, pend[p] its step's end position
__global__ void k_st_meta(int ns, int4* __restrict__ desc, const int32_t* __restrict__ pbscan,
                          const int32_t* __restrict__ bscan, const int32_t* __restrict__ ord,
                          const int32_t* __restrict__ other, int ts, bool upper,
                          int4* __restrict__ meta, int32_t* __restrict__ pend,
                          int32_t* __restrict__ pblk, unsigned* __restrict__ max_bytes) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  int4 d = desc[s];
  int k0 = pbscan[s];
  desc[s] = make_int4(d.x, d.y, k0, k0 + d.z);
  atomicMax(max_bytes, step_bytes(d.y - d.x, (d.z + 3) & ~3, ts, upper));
  for (int p = d.x; p < d.y; ++p) {
    int kb = bscan[p] - bscan[d.x];
    int ke = kb + bscan[p + 1] - bscan[p];
    meta[p] = make_int4(ord[p], kb, ke, other ? other[ord[p]] : 0);
    pend[p] = d.y;
    pblk[p] = k0 + kb;
  }
}
// factor blocks, dependency codes and inverse diagonals of every position
template <class T>
__global__ void k_st_fill(int N, int S, int RC, bool upper, const int4* __restrict__ meta,
                          const int32_t* __restrict__ pend, const int32_t* __restrict__ pblk,
                          const int32_t* __restrict__ pos,
                          const int32_t* __restrict__ sfirst, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ ci, const int32_t* __restrict__ diag,
                          const double* __restrict__ LU, int32_t* __restrict__ loc,
                          T* __restrict__ sv, T* __restrict__ dinv) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int4 mt = meta[p];
  int i = mt.x;
  int t0 = upper ? diag[i] + 1 : rp[i];
  int q = strip_of(i, N, S, upper);
  size_t k0 = (size_t)pblk[p];
  for (int a = 0; a < mt.z - mt.y; ++a) {
    int j = ci[t0 + a];
    int pj = pos[j];
    unsigned w;
    if (strip_of(j, N, S, upper) == q && pj >= pend[p] - RC)
      w = kLocal | (unsigned)((pj - sfirst[q]) % RC);
    else
      w = (unsigned)pj;
    loc[k0 + a] = (int32_t)w;
    for (int e = 0; e < 16; ++e) sv[16 * (k0 + a) + e] = (T)LU[16 * (size_t)(t0 + a) + e];
  }
  if (upper)
    for (int e = 0; e < 16; ++e) dinv[16 * (size_t)p + e] = (T)LU[16 * (size_t)diag[i] + e];
}
__global__ void k_st_first(int P, int nlev, const int32_t* __restrict__ cscan,
                           const int32_t* __restrict__ sscan, int32_t* __restrict__ sfirst,
                           int32_t* __restrict__ sptr) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > P) return;
  sptr[q] = sscan[(size_t)q * nlev];
  if (q < P) sfirst[q] = cscan[(size_t)q * nlev];
}

// ------------------------------------------------------------------ host side
constexpr size_t kStripSmem = 220 * 1024;

template <class T>
cptr_status build_dir(cptr_ctx* c, bool upper, int P, StripSched& S, const int32_t* other) {
  const int N = c->N, ts = (int)sizeof(T);
  const int nlev = upper ? c->nlev_b : c->nlev_f;
  const int32_t* lvl = upper ? c->lvl_b : c->lvl_f;
  cudaStream_t s = cs(c);
  S = StripSched();
  S.P = P;
  S.S = ceil_div(N, P);
  // solution ring: the largest power of two of rows within a quarter of the budget
  S.RC = 1;
  while ((size_t)S.RC * 2 * 4 * ts <= kStripSmem / 4 && S.RC * 2 <= (1 << 20)) S.RC *= 2;
  if (c->strip_rc > 0) S.RC = c->strip_rc;  // test hook: a small ring evicts own rows
  const size_t fixed = 32 * kNB + (size_t)S.RC * 4 * ts;
  if (fixed + 4096 > kStripSmem) return CPTR_ERR_INVALID;
  S.ring_bytes = (unsigned)((kStripSmem - fixed) & ~(size_t)127);
  if (c->strip_ring > 0) S.ring_bytes = std::min<unsigned>(S.ring_bytes, (unsigned)c->strip_ring & ~127u);
  S.smem = fixed + S.ring_bytes;
  const long long nbk = (long long)P * nlev;
  if (nbk >= (1ll << 31)) return CPTR_ERR_INVALID;
  int32_t *key, *keys_out, *iota, *cnt, *cscan;
  CTX_ALLOC(c, key, int32_t, N + 1, true);
  CTX_ALLOC(c, keys_out, int32_t, N + 1, true);
  CTX_ALLOC(c, iota, int32_t, N + 1, true);
  CTX_ALLOC(c, cnt, int32_t, nbk + 1, true);
  CTX_ALLOC(c, cscan, int32_t, nbk + 1, true);
  CTX_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nbk + 1), s));
  KL(c, k_st_keys<<<nblk(N), kT, 0, s>>>(N, S.S, nlev, upper, lvl, key, iota, cnt));
  cptr_status st = scan_i32(c, cnt, cscan, (int)nbk, nullptr);
  if (st) return st;
  // rows by (strip, level, index in the solve's direction): a stable radix sort
  CTX_ALLOC(c, S.ord, int32_t, N + 16, true);
  CTX_ALLOC(c, S.pos, int32_t, N + 16, true);
  int bits = 1;
  while ((1ll << bits) < nbk) ++bits;
  size_t tmp_bytes = 0;
  CTX_CUDA(c, cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, key, keys_out, iota, S.ord, N,
                                              0, bits, s));
  void* tmp = ctx_alloc(c, tmp_bytes + 16, true);
  if (!tmp) return CPTR_ERR_NOMEM;
  CTX_CUDA(c, cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, key, keys_out, iota, S.ord, N, 0,
                                              bits, s));
  ++c->nlaunch;
  KL(c, k_st_pos<<<nblk(N), kT, 0, s>>>(N, S.ord, S.pos));
  // factor blocks per position and their prefix sums
  int32_t *bcnt, *bscan;
  CTX_ALLOC(c, bcnt, int32_t, N + 1, true);
  CTX_ALLOC(c, bscan, int32_t, N + 1, true);
  KL(c, k_st_nblk<<<nblk(N), kT, 0, s>>>(N, S.ord, c->rp, c->diag, upper, bcnt));
  int nbraw = 0;
  st = scan_i32(c, bcnt, bscan, N, &nbraw);
  if (st) return st;
  // steps: each (strip, level) bucket split into pieces that fit half the ring
  const unsigned cap = S.ring_bytes / 2;
  int32_t *nsub, *sscan;
  CTX_ALLOC(c, nsub, int32_t, nbk + 1, true);
  CTX_ALLOC(c, sscan, int32_t, nbk + 1, true);
  KL(c, k_st_split<<<nblk(nbk), kT, 0, s>>>((int)nbk, cscan, bscan, cap, ts, upper, 0, nsub,
                                             nullptr, nullptr));
  int ns = 0;
  st = scan_i32(c, nsub, sscan, (int)nbk, &ns);
  if (st) return st;
  S.nsteps = ns;
  CTX_ALLOC(c, S.step, int4, (size_t)ns + 1, true);
  KL(c, k_st_split<<<nblk(nbk), kT, 0, s>>>((int)nbk, cscan, bscan, cap, ts, upper, 1, nullptr,
                                             sscan, S.step));
  int32_t *pcnt, *pbscan;
  CTX_ALLOC(c, pcnt, int32_t, (size_t)ns + 1, true);
  CTX_ALLOC(c, pbscan, int32_t, (size_t)ns + 1, true);
  KL(c, k_st_padcnt<<<nblk(ns), kT, 0, s>>>(ns, S.step, pcnt));
  int nbp = 0;
  st = scan_i32(c, pcnt, pbscan, ns, &nbp);
  if (st) return st;
  S.nnz = nbraw;
  S.nblk_padded = nbp;
  CTX_ALLOC(c, S.meta, int4, (size_t)N + 1, true);
  int32_t *pend, *pblk;
  CTX_ALLOC(c, pend, int32_t, N + 1, true);
  CTX_ALLOC(c, pblk, int32_t, N + 1, true);
  unsigned* maxb;
  CTX_ALLOC(c, maxb, unsigned, 1, true);
  CTX_CUDA(c, cudaMemsetAsync(maxb, 0, sizeof(unsigned), s));
  KL(c, k_st_meta<<<nblk(ns), kT, 0, s>>>(ns, S.step, pbscan, bscan, S.ord, other, ts, upper,
                                           S.meta, pend, pblk, maxb));
  unsigned maxb_h = 0;
  CTX_CUDA(c, cudaMemcpyAsync(&maxb_h, maxb, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CTX_CUDA(c, cudaStreamSynchronize(s));
  if (maxb_h > S.ring_bytes) return CPTR_ERR_INVALID;  // a single row exceeds the staging ring
  CTX_ALLOC(c, S.sptr, int32_t, P + 1, true);
  int32_t* sfirst;
  CTX_ALLOC(c, sfirst, int32_t, P + 1, true);
  KL(c, k_st_first<<<nblk(P + 1), kT, 0, s>>>(P, nlev, cscan, sscan, sfirst, S.sptr));
  CTX_ALLOC(c, S.loc, int32_t, (size_t)nbp + 16, true);
  CTX_CUDA(c, cudaMemsetAsync(S.loc, 0, sizeof(int32_t) * ((size_t)nbp + 16), s));
  S.v = ctx_alloc(c, sizeof(T) * 16 * ((size_t)nbp + 1), true);
  if (!S.v) return CPTR_ERR_NOMEM;
  CTX_CUDA(c, cudaMemsetAsync(S.v, 0, sizeof(T) * 16 * ((size_t)nbp + 1), s));
  if (upper) {
    S.dinv = ctx_alloc(c, sizeof(T) * 16 * ((size_t)N + 1), true);
    if (!S.dinv) return CPTR_ERR_NOMEM;
  }
  KL(c, k_st_fill<T><<<nblk(N), kT, 0, s>>>(N, S.S, S.RC, upper, S.meta, pend, pblk, S.pos, sfirst,
                                             c->rp, c->ci, c->diag, c->LU64, S.loc, (T*)S.v,
                                             (T*)S.dinv));
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

template <class T>
cptr_status build_strip_t(cptr_ctx* c) {
  const int P = c->strip_p > 0 ? c->strip_p : c->nsm;
  CTX_CUDA(c, cudaFuncSetAttribute(k_tri_strip<T, false>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStripSmem));
  CTX_CUDA(c, cudaFuncSetAttribute(k_tri_strip<T, true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStripSmem));
  // the backward schedule first: the forward one records backward positions
  cptr_status st = build_dir<T>(c, true, P, c->sb, nullptr);
  if (!st) st = build_dir<T>(c, false, P, c->sf, c->sb.pos);
  if (st) return st;
  size_t n4 = 4 * (size_t)c->N;
  c->strip_rf = ctx_alloc(c, sizeof(T) * n4 + 16, true);
  c->strip_uf = ctx_alloc(c, sizeof(T) * n4 + 16, true);
  c->strip_rb = ctx_alloc(c, sizeof(T) * n4 + 16, true);
  c->strip_yb = ctx_alloc(c, sizeof(T) * n4 + 16, true);
  if (!c->strip_rf || !c->strip_uf || !c->strip_rb || !c->strip_yb) return CPTR_ERR_NOMEM;
  c->nnzL = c->sf.nnz;
  c->nnzU = c->sb.nnz;
  CTX_CUDA(c, cudaStreamSynchronize(cs(c)));
  return CPTR_OK;
}

template <class T, bool UPPER>
void launch_dir(cptr_ctx* c, const StripSched& S, const T* rhsp, T* outp, T* nextp, T* nextout,
                const T* zc, T* zbase, const int* jptr, size_t stride, const int* active) {
  KL(c, k_tri_strip<T, UPPER><<<S.P, kStripThreads, S.smem, cs(c)>>>(
            S.RC, S.ring_bytes, S.sptr, (const int4*)S.step, (const int4*)S.meta, S.loc,
            (const T*)S.v, (const T*)S.dinv, rhsp, outp, nextp, nextout, zc, c->se0, c->se1,
            zbase, jptr, stride, UPPER ? &c->ctl->bwd_ctr : &c->ctl->fwd_ctr, c->ctl, active));
}

template <class T>
void launch_t(cptr_ctx* c, const T* zc, T* zbase, const int* jptr, size_t stride,
              const int* active, int which) {
  if (which != 2) {
    KL(c, k_strip_gather<T><<<nblk(4ll * c->N), kT, 0, cs(c)>>>(
              c->N, c->sf.ord, (const T*)c->r2, (T*)c->strip_rf, (T*)c->strip_uf, c->ctl, active));
    launch_dir<T, false>(c, c->sf, (const T*)c->strip_rf, (T*)c->strip_uf, (T*)c->strip_rb,
                         (T*)c->strip_yb, nullptr, nullptr, jptr, stride, active);
  }
  if (which != 1)
    launch_dir<T, true>(c, c->sb, (const T*)c->strip_rb, (T*)c->strip_yb, nullptr, nullptr, zc,
                        zbase, jptr, stride, active);
}

}  // namespace

cptr_status build_strip(cptr_ctx* c) {
  return c->mixed ? build_strip_t<float>(c) : build_strip_t<double>(c);
}

void launch_tri_strip(cptr_ctx* c, const void* zc, void* zbase, const int* jptr, size_t stride,
                      const int* active, int which) {
  if (c->mixed)
    launch_t<float>(c, (const float*)zc, (float*)zbase, jptr, stride, active, which);
  else
    launch_t<double>(c, (const double*)zc, (double*)zbase, jptr, stride, active, which);
}
