// Chain schedule for the ILU(0) block triangular solves.
//
// Level-synchronous schedules pay a synchronisation (a CTA barrier, or a
// hand-off through L2) on every level of the dependency graph: 498 levels per
// triangle on a 200x200x100 grid in natural order.  Here the rows are linked
// into chains instead: the predecessor of a row is its dependency of highest
// level (ties: the closest row), and each row continues the chain of its
// predecessor if it is that row's first successor (a natural-order 7-point
// grid gives its x-lines).  One quad (four lanes, lane r computing component r)
// walks a chain row after row, so the dependency on the previous row never
// leaves registers; the other dependencies are read from the global solution
// array, whose entries start as a sentinel NaN, polled until final (bounded).
// Chains are claimed in the order of their heads' (level, index), and the
// schedule is only built when every cross-chain dependency points to a chain
// that comes earlier in that order: a quad then only waits on chains already
// claimed by running quads, so the solve progresses whatever is resident.
// Rows use the library's common rounding sequence (dot4, sub_rn, in block
// order), so results are bit-identical to every other schedule.
#include <algorithm>
#include <climits>
#include <cstdio>

#include <cub/device/device_radix_sort.cuh>

#include "common.cuh"
#include "ctx.h"

namespace {

constexpr int kT = 256;
constexpr int kPre = 4;  // factor blocks of a row held in registers (more: loaded in the loop)
inline int nblk(long long n, int per = kT) { return n > 0 ? ceil_div(n, per) : 1; }

template <class T>
__device__ __forceinline__ bool ready4(const T* o) {
  return !is_sentinel(o[0]) && !is_sentinel(o[1]) && !is_sentinel(o[2]) && !is_sentinel(o[3]);
}
// bounded poll with a short back-off between misses
template <class T>
__device__ __forceinline__ void poll_vec(const T* p, T* o, int* status, unsigned limit) {
  for (unsigned s = 0;; ++s) {
    ld_volatile4(p, o);
    if (ready4(o)) return;
    if (s + 1 >= limit) {  // `limit` polls saw the sentinel
      dev_fail(status, DEV_TIMEOUT);
      return;
    }
    __nanosleep(32);
    if ((s & 255u) == 255u && ld_volatile_i32(status) != DEV_OK) return;
  }
}

// meta[p] = {row, first block, block count, slot of the in-chain predecessor
// among the row's blocks (-1 for a chain head)}; blocks of a position are
// consecutive in cv/cci (factor values, dependency rows), in CSR order.
// UPPER = false: out_i = rhs_i - sum_{k<i} L_ik out_k; y2_i reset to the sentinel.
// UPPER = true:  out_i = inv(U_ii)(rhs_i - sum_{j>i} U_ij out_j), z_i = P zc_i + out_i.
template <class T, bool UPPER>
__global__ void __launch_bounds__(256) k_tri_chain(
    int nchains, const int32_t* __restrict__ cptr, const int4* __restrict__ meta,
    const int32_t* __restrict__ cci, const T* __restrict__ cv, const T* __restrict__ cdinv,
    const T* __restrict__ rhs, T* out, T* __restrict__ reset, const T* __restrict__ zc, int e0,
    int e1, T* __restrict__ zbase, const int* jptr, size_t stride, unsigned* ctr, Ctl* ctl,
    const int* active) {
  if (!*active) return;
  const int lane = threadIdx.x & 31, r = lane & 3, q0 = lane & ~3;
  const unsigned qm = 0xFu << q0;
  int* status = &ctl->status;
  const unsigned lim = ctl->spin;
  T* z = UPPER ? zbase + (size_t)(*jptr) * stride : nullptr;
  for (;;) {
    int c = 0;
    if (r == 0) c = (int)atomicAdd(ctr, 1u);
    c = __shfl_sync(qm, c, q0);
    if (c >= nchains) return;
    const int p0 = cptr[c], p1 = cptr[c + 1];
    T yprev[4] = {0, 0, 0, 0};  // the quad's previous row, all four components
    // row p's record and first blocks, loaded one row ahead
    int4 mt = meta[p0];
    T a[kPre][4];
    int col[kPre];
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
      col[u] = u < mt.z ? cci[mt.y + u] : 0;
      if (u < mt.z) ld4(cv + 16 * (size_t)(mt.y + u) + 4 * r, a[u]);
    }
    T b = rhs[4 * (size_t)mt.x + r];
    T dcur[4] = {0, 0, 0, 0};  // inv(U_ii) of the row (backward), also one row ahead
    if (UPPER) ld4(cdinv + 16 * (size_t)p0 + 4 * r, dcur);
    for (int p = p0; p < p1; ++p) {
      // next row's data in flight while this row waits and computes
      int4 mn = make_int4(0, 0, 0, 0);
      T an[kPre][4];
      int coln[kPre];
      T bn = 0;
      T dn[4] = {0, 0, 0, 0};
      if (p + 1 < p1) {
        if (UPPER) ld4(cdinv + 16 * (size_t)(p + 1) + 4 * r, dn);
        mn = meta[p + 1];
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
          coln[u] = u < mn.z ? cci[mn.y + u] : 0;
          if (u < mn.z) ld4(cv + 16 * (size_t)(mn.y + u) + 4 * r, an[u]);
        }
        bn = rhs[4 * (size_t)mn.x + r];
      }
      // this row's dependencies on other chains: every value read at once,
      // those still holding the sentinel polled again in block order
      T x[kPre][4];
#pragma unroll
      for (int u = 0; u < kPre; ++u)
        if (u < mt.z && u != mt.w) ld_volatile4(out + 4 * (size_t)col[u], x[u]);
      T acc = b;
#pragma unroll
      for (int u = 0; u < kPre; ++u) {
        if (u < mt.z) {
          if (u == mt.w) {
            x[u][0] = yprev[0]; x[u][1] = yprev[1]; x[u][2] = yprev[2]; x[u][3] = yprev[3];
          } else if (!ready4(x[u])) {
            poll_vec(out + 4 * (size_t)col[u], x[u], status, lim);
          }
          acc = sub_rn(acc, dot4(a[u], x[u]));
        }
      }
      for (int u = kPre; u < mt.z; ++u) {  // rows with many dependencies
        const int k = mt.y + u;
        T a1[4], x1[4];
        ld4(cv + 16 * (size_t)k + 4 * r, a1);
        if (u == mt.w) {
          x1[0] = yprev[0]; x1[1] = yprev[1]; x1[2] = yprev[2]; x1[3] = yprev[3];
        } else {
          poll_vec(out + 4 * (size_t)cci[k], x1, status, lim);
        }
        acc = sub_rn(acc, dot4(a1, x1));
      }
      T y = acc;
      T s0 = __shfl_sync(qm, acc, q0 + 0), s1 = __shfl_sync(qm, acc, q0 + 1);
      T s2 = __shfl_sync(qm, acc, q0 + 2), s3 = __shfl_sync(qm, acc, q0 + 3);
      if (UPPER) {
        T sv4[4] = {s0, s1, s2, s3};
        y = dot4(dcur, sv4);
        s0 = __shfl_sync(qm, y, q0 + 0); s1 = __shfl_sync(qm, y, q0 + 1);
        s2 = __shfl_sync(qm, y, q0 + 2); s3 = __shfl_sync(qm, y, q0 + 3);
      }
      y = desentinel(y);
      yprev[0] = desentinel(s0); yprev[1] = desentinel(s1);
      yprev[2] = desentinel(s2); yprev[3] = desentinel(s3);
      const int i = mt.x;
      st_volatile(out + 4 * (size_t)i + r, y);
      if (!UPPER) {
        reset[4 * (size_t)i + r] = sentinel_of(T(0));
      } else {
        T y1 = 0;
        if (zc) {
          const int ne = e1 < 0 ? 1 : 2;
          if (r == e0) y1 = zc[ne * (size_t)i];
          else if (r == e1) y1 = zc[ne * (size_t)i + 1];
        }
        z[4 * (size_t)i + r] = y1 + y;
      }
      mt = mn;
      b = bn;
      dcur[0] = dn[0]; dcur[1] = dn[1]; dcur[2] = dn[2]; dcur[3] = dn[3];
#pragma unroll
      for (int u = 0; u < kPre; ++u) {
        col[u] = coln[u];
        a[u][0] = an[u][0]; a[u][1] = an[u][1]; a[u][2] = an[u][2]; a[u][3] = an[u][3];
      }
    }
  }
}

// ------------------------------------------------------------------ schedule kernels
// predecessor: the dependency of highest level, ties broken by the closest row
__global__ void k_ch_pred(int N, bool upper, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ ci, const int32_t* __restrict__ diag,
                          const int32_t* __restrict__ lvl, int32_t* __restrict__ pred,
                          int32_t* __restrict__ next) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int t0 = upper ? diag[i] + 1 : rp[i], t1 = upper ? rp[i + 1] : diag[i];
  int best = -1, bl = -1;
  for (int t = t0; t < t1; ++t) {
    int j = ci[t], l = lvl[j];
    bool closer = best < 0 || (upper ? j < best : j > best);
    if (l > bl || (l == bl && closer)) { bl = l; best = j; }
  }
  pred[i] = best;
  next[i] = upper ? -1 : INT_MAX;
}
// first successor of each row: the closest row naming it as predecessor
__global__ void k_ch_next(int N, bool upper, const int32_t* __restrict__ pred,
                          int32_t* __restrict__ next) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int j = pred[i];
  if (j < 0) return;
  if (upper) atomicMax(&next[j], i);
  else atomicMin(&next[j], i);
}
// heads: key (level, index in the solve's direction) for the sort, -1 for others
__global__ void k_ch_heads(int N, bool upper, const int32_t* __restrict__ pred,
                           const int32_t* __restrict__ next, const int32_t* __restrict__ lvl,
                           int nlev_bits, long long* __restrict__ key, int32_t* __restrict__ row,
                           int32_t* __restrict__ nheads) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int j = pred[i];
  bool head = j < 0 || next[j] != i;
  long long dir = upper ? (long long)(N - 1 - i) : (long long)i;
  key[i] = head ? (((long long)lvl[i] << 32) | dir) : LLONG_MAX;
  row[i] = i;
  if (head) atomicAdd(nheads, 1);
}
// length of every chain (walking the successor links)
__global__ void k_ch_len(int nch, int N, bool upper, const int32_t* __restrict__ heads,
                         const int32_t* __restrict__ pred, const int32_t* __restrict__ next,
                         int32_t* __restrict__ len, int32_t* __restrict__ chain_of) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nch) return;
  int i = heads[c], n = 0;
  for (;;) {
    chain_of[i] = c;
    ++n;
    int s = next[i];
    if (s < 0 || s >= N || pred[s] != i) break;
    i = s;
  }
  len[c] = n;
}
__global__ void k_ch_fillord(int nch, int N, const int32_t* __restrict__ heads,
                             const int32_t* __restrict__ pred, const int32_t* __restrict__ next,
                             const int32_t* __restrict__ cptr, int32_t* __restrict__ ord) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nch) return;
  int i = heads[c], p = cptr[c];
  for (;;) {
    ord[p++] = i;
    int s = next[i];
    if (s < 0 || s >= N || pred[s] != i) break;
    i = s;
  }
}
__global__ void k_ch_nblk(int N, bool upper, const int32_t* __restrict__ ord,
                          const int32_t* __restrict__ rp, const int32_t* __restrict__ diag,
                          int32_t* __restrict__ cnt) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int i = ord[p];
  cnt[p] = upper ? rp[i + 1] - diag[i] - 1 : diag[i] - rp[i];
}
// records, factor blocks and dependency rows of every position; a dependency
// on another chain must point to an earlier chain (else *bad is set)
template <class T>
__global__ void k_ch_fill(int N, bool upper, const int32_t* __restrict__ ord,
                          const int32_t* __restrict__ bscan, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ ci, const int32_t* __restrict__ diag,
                          const double* __restrict__ LU, const int32_t* __restrict__ pred,
                          const int32_t* __restrict__ chain_of, int4* __restrict__ meta,
                          int32_t* __restrict__ cci, T* __restrict__ cv, T* __restrict__ dinv,
                          int* __restrict__ bad) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int i = ord[p];
  int t0 = upper ? diag[i] + 1 : rp[i];
  int k0 = bscan[p], n = bscan[p + 1] - k0;
  int slot = -1;
  const bool has_pred = pred[i] >= 0 && p > 0 && ord[p - 1] == pred[i] &&
                        chain_of[pred[i]] == chain_of[i];
  for (int a = 0; a < n; ++a) {
    int j = ci[t0 + a];
    cci[k0 + a] = j;
    if (has_pred && j == pred[i]) slot = a;
    else if (chain_of[j] > chain_of[i]) atomicOr(bad, 1);  // same chain: an earlier row of it
    for (int e = 0; e < 16; ++e) cv[16 * (size_t)(k0 + a) + e] = (T)LU[16 * (size_t)(t0 + a) + e];
  }
  meta[p] = make_int4(i, k0, n, slot);
  if (dinv)
    for (int e = 0; e < 16; ++e) dinv[16 * (size_t)p + e] = (T)LU[16 * (size_t)diag[i] + e];
}

// ------------------------------------------------------------------ host side
template <class T>
cptr_status build_dir(cptr_ctx* c, bool upper, ChainSched& S) {
  const int N = c->N;
  const int32_t* lvl = upper ? c->lvl_b : c->lvl_f;
  cudaStream_t s = cs(c);
  S = ChainSched();
  int32_t *pred, *next, *rows, *heads_sorted, *nheads, *chain_of, *len;
  long long *key, *key_sorted;
  CTX_ALLOC(c, pred, int32_t, N + 1, true);
  CTX_ALLOC(c, next, int32_t, N + 1, true);
  CTX_ALLOC(c, rows, int32_t, N + 1, true);
  CTX_ALLOC(c, heads_sorted, int32_t, N + 1, true);
  CTX_ALLOC(c, nheads, int32_t, 1, true);
  CTX_ALLOC(c, chain_of, int32_t, N + 1, true);
  CTX_ALLOC(c, key, long long, N + 1, true);
  CTX_ALLOC(c, key_sorted, long long, N + 1, true);
  KL(c, k_ch_pred<<<nblk(N), kT, 0, s>>>(N, upper, c->rp, c->ci, c->diag, lvl, pred, next));
  KL(c, k_ch_next<<<nblk(N), kT, 0, s>>>(N, upper, pred, next));
  CTX_CUDA(c, cudaMemsetAsync(nheads, 0, sizeof(int32_t), s));
  KL(c, k_ch_heads<<<nblk(N), kT, 0, s>>>(N, upper, pred, next, lvl, 0, key, rows, nheads));
  size_t tmp_bytes = 0;
  CTX_CUDA(c, cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, key, key_sorted, rows,
                                              heads_sorted, N, 0, 64, s));
  void* tmp = ctx_alloc(c, tmp_bytes + 16, true);
  if (!tmp) return CPTR_ERR_NOMEM;
  CTX_CUDA(c, cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, key, key_sorted, rows,
                                              heads_sorted, N, 0, 64, s));
  ++c->nlaunch;
  int nch = 0;
  CTX_CUDA(c, cudaMemcpyAsync(&nch, nheads, sizeof(int), cudaMemcpyDeviceToHost, s));
  CTX_CUDA(c, cudaStreamSynchronize(s));
  if (nch <= 0) return CPTR_ERR_INVALID;
  S.nchains = nch;
  CTX_ALLOC(c, len, int32_t, nch + 1, true);
  CTX_ALLOC(c, S.cptr, int32_t, nch + 1, true);
  KL(c, k_ch_len<<<nblk(nch), kT, 0, s>>>(nch, N, upper, heads_sorted, pred, next, len, chain_of));
  int tot = 0;
  cptr_status st = scan_i32(c, len, S.cptr, nch, &tot);
  if (st) return st;
  if (tot != N) {  // every row lies on exactly one chain
    ctx_set_err(c, "chain schedule: rows not covered by the chains");
    return CPTR_ERR_INVALID;
  }
  int32_t* ord;
  CTX_ALLOC(c, ord, int32_t, N + 1, true);
  KL(c, k_ch_fillord<<<nblk(nch), kT, 0, s>>>(nch, N, heads_sorted, pred, next, S.cptr, ord));
  int32_t *bcnt, *bscan;
  CTX_ALLOC(c, bcnt, int32_t, N + 1, true);
  CTX_ALLOC(c, bscan, int32_t, N + 1, true);
  KL(c, k_ch_nblk<<<nblk(N), kT, 0, s>>>(N, upper, ord, c->rp, c->diag, bcnt));
  int nb = 0;
  st = scan_i32(c, bcnt, bscan, N, &nb);
  if (st) return st;
  S.nnz = nb;
  CTX_ALLOC(c, S.meta, int4, N + 1, true);
  CTX_ALLOC(c, S.ci, int32_t, (size_t)nb + 16, true);
  S.v = ctx_alloc(c, sizeof(T) * 16 * ((size_t)nb + 1), true);
  if (!S.v) return CPTR_ERR_NOMEM;
  if (upper) {
    S.dinv = ctx_alloc(c, sizeof(T) * 16 * ((size_t)N + 1), true);
    if (!S.dinv) return CPTR_ERR_NOMEM;
  }
  int* bad;
  CTX_ALLOC(c, bad, int, 1, true);
  CTX_CUDA(c, cudaMemsetAsync(bad, 0, sizeof(int), s));
  KL(c, k_ch_fill<T><<<nblk(N), kT, 0, s>>>(N, upper, ord, bscan, c->rp, c->ci, c->diag, c->LU64,
                                             pred, chain_of, S.meta, S.ci, (T*)S.v, (T*)S.dinv,
                                             bad));
  int hbad = 0;
  CTX_CUDA(c, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CTX_CUDA(c, cudaStreamSynchronize(s));
  CTX_CUDA(c, cudaGetLastError());
  // a dependency on a later chain could make a quad wait on an unclaimed chain
  return hbad ? CPTR_ERR_INVALID : CPTR_OK;
}

template <class T>
cptr_status build_chain_t(cptr_ctx* c) {
  cptr_status st = build_dir<T>(c, false, c->chf);
  if (!st) st = build_dir<T>(c, true, c->chb);
  if (st) return st;
  c->nnzL = c->chf.nnz;
  c->nnzU = c->chb.nnz;
  return CPTR_OK;
}

template <class T>
void launch_t(cptr_ctx* c, const T* zc, T* zbase, const int* jptr, size_t stride,
              const int* active, int which) {
  cudaStream_t s = cs(c);
  const int grid = c->nsm * 8;
  if (which != 2)
    KL(c, k_tri_chain<T, false><<<grid, 256, 0, s>>>(
              c->chf.nchains, c->chf.cptr, (const int4*)c->chf.meta, c->chf.ci, (const T*)c->chf.v,
              nullptr, (const T*)c->r2, (T*)c->u, (T*)c->y2, nullptr, 0, 0, nullptr, jptr, stride,
              &c->ctl->fwd_ctr, c->ctl, active));
  if (which != 1)
    KL(c, k_tri_chain<T, true><<<grid, 256, 0, s>>>(
              c->chb.nchains, c->chb.cptr, (const int4*)c->chb.meta, c->chb.ci, (const T*)c->chb.v,
              (const T*)c->chb.dinv, (const T*)c->u, (T*)c->y2, nullptr, zc, c->se0, c->se1,
              zbase, jptr, stride, &c->ctl->bwd_ctr, c->ctl, active));
}

}  // namespace

cptr_status build_chain(cptr_ctx* c) {
  return c->mixed ? build_chain_t<float>(c) : build_chain_t<double>(c);
}

void launch_tri_chain(cptr_ctx* c, const void* zc, void* zbase, const int* jptr, size_t stride,
                      const int* active, int which) {
  if (c->mixed)
    launch_t<float>(c, (const float*)zc, (float*)zbase, jptr, stride, active, which);
  else
    launch_t<double>(c, (const double*)zc, (double*)zbase, jptr, stride, active, which);
}
