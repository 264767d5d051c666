// Block ILU(0) of the 4x4 BSR matrix on the device (paper Section 3.1: the
// second stage is ILU with zero fill-in on the global matrix), natural order,
// no pivoting: for each row i and each k < i in row i (ascending),
//   L_ik = A_ik inv(U_kk);  A_ij -= L_ik U_kj  for j > k present in rows i and k;
// then inv(U_ii) is stored in place of the diagonal block.
//
// Rows are factorised by a sync-free kernel that follows the level schedule of
// the lower triangle (level(i) = 1 + max level(k), k < i in row i): a warp
// claims the next row of the schedule, waits (bounded) for the rows it needs,
// and publishes completion with a release flag.  The same schedule, and the
// one of the upper triangle, order the triangular solves.
#include <vector>

#include "common.cuh"
#include "ctx.h"

namespace {

constexpr int kT = 256;
inline int nblk(long long n, int per = kT) { return n > 0 ? ceil_div(n, per) : 1; }

// level(i) = 1 + max over dependencies (0 if none) in one pass.  Warps claim
// groups of 32 rows in dependency order (increasing index for the lower
// triangle, decreasing for the upper), so every dependency of a row belongs to
// a group claimed earlier by a running warp; a row waits until its
// dependencies' levels are written (-1 before), polling a bounded number of times.
__global__ void __launch_bounds__(256) k_level_syncfree(int N, const int32_t* __restrict__ rp,
                                                        const int32_t* __restrict__ ci,
                                                        const int32_t* __restrict__ diag,
                                                        int32_t* lvl, bool upper, unsigned* ctr,
                                                        int* status) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned g0 = 0;
    if (lane == 0) g0 = atomicAdd(ctr, 32u);
    g0 = __shfl_sync(0xffffffffu, g0, 0);
    if (g0 >= (unsigned)N) return;
    const int k = (int)g0 + lane;
    // A lane that gives up leaves its row unwritten and the whole warp stops
    // at the vote below: every lane must reach the next __shfl_sync, so no
    // lane may leave the kernel on its own.
    bool quit = false;
    if (k < N) {
      const int i = upper ? N - 1 - k : k;
      const int t0 = upper ? diag[i] + 1 : rp[i];
      const int t1 = upper ? rp[i + 1] : diag[i];
      int m = 0;
      for (int t = t0; t < t1 && !quit; ++t) {
        const int32_t* pj = lvl + ci[t];
        int q = ld_volatile_i32(pj);
        for (unsigned sp = 0; q < 0; ++sp) {
          if ((sp & 255u) == 255u) {
            if (ld_volatile_i32(status) != DEV_OK) { quit = true; break; }
            if (sp > CPTR_SPIN_LIMIT) {
              dev_fail(status, DEV_TIMEOUT);
              quit = true;
              break;
            }
          }
          q = ld_volatile_i32(pj);
        }
        m = q + 1 > m ? q + 1 : m;
      }
      if (!quit) st_release_i32(lvl + i, m);
    }
    if (__any_sync(0xffffffffu, quit)) return;
  }
}

__global__ void k_level_count(int N, const int32_t* __restrict__ lvl, int32_t* __restrict__ cnt,
                              int* maxlvl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  atomicAdd(&cnt[lvl[i]], 1);
  atomicMax(maxlvl, lvl[i]);
}

__global__ void k_pad8(int n, const int32_t* __restrict__ cnt, int32_t* __restrict__ pc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pc[i] = (cnt[i] + 7) & ~7;
}

__global__ void k_level_fill(int N, const int32_t* __restrict__ lvl, const int32_t* __restrict__ off,
                             int32_t* __restrict__ cur, int32_t* __restrict__ ord) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int L = lvl[i];
  ord[off[L] + atomicAdd(&cur[L], 1)] = i;
}

// 4x4 inverse by Gauss-Jordan elimination with partial pivoting.
__device__ bool inv4(const double* M, double* out) {
  double a[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 8; ++c) a[r][c] = (c < 4) ? M[r * 4 + c] : (c - 4 == r ? 1.0 : 0.0);
  for (int c = 0; c < 4; ++c) {
    int p = c;
    double best = fabs(a[c][c]);
    for (int r = c + 1; r < 4; ++r)
      if (fabs(a[r][c]) > best) { best = fabs(a[r][c]); p = r; }
    if (!(best > 0.0) || !isfinite(best)) return false;
    if (p != c)
      for (int k = 0; k < 8; ++k) { double t = a[c][k]; a[c][k] = a[p][k]; a[p][k] = t; }
    double d = a[c][c];
    for (int k = 0; k < 8; ++k) a[c][k] /= d;
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      double f = a[r][c];
      for (int k = 0; k < 8; ++k) a[r][k] -= f * a[c][k];
    }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) out[r * 4 + c] = a[r][c + 4];
  return true;
}

// The same Gauss-Jordan inversion executed by a full warp: lane 8*r + k holds
// entry k of row r of the augmented 4x8 matrix [M | I].  Pivot choice, row
// swap, scaling and elimination perform exactly the operations of inv4 on the
// same values, so the result is identical.  M and out may alias (shared memory).
__device__ bool inv4_warp(const double* M, double* out) {
  const int lane = threadIdx.x & 31, r = lane >> 3, k = lane & 7;
  double a = (k < 4) ? M[r * 4 + k] : (k - 4 == r ? 1.0 : 0.0);
  bool ok = true;
  for (int c = 0; c < 4; ++c) {
    // candidate pivots a[rr][c], rr = c..3 (first maximum wins, as in inv4);
    // |x| and the comparisons run on bit patterns with IEEE results (a NaN
    // never wins; a NaN first candidate is kept)
    int p = c;
    unsigned long long best = dmag(__shfl_sync(0xffffffffu, a, 8 * c + c));
    for (int rr = c + 1; rr < 4; ++rr) {
      const unsigned long long v = dmag(__shfl_sync(0xffffffffu, a, 8 * rr + c));
      if (v > best && v <= 0x7ff0000000000000ull && best <= 0x7ff0000000000000ull) {
        best = v;
        p = rr;
      }
    }
    if (best == 0 || best >= 0x7ff0000000000000ull) ok = false;  // !(best > 0) || !isfinite
    // swap rows c and p
    double from_p = __shfl_sync(0xffffffffu, a, 8 * p + k);
    double from_c = __shfl_sync(0xffffffffu, a, 8 * c + k);
    if (r == c) a = from_p;
    else if (r == p) a = from_c;
    // scale row c by its pivot
    double d = __shfl_sync(0xffffffffu, a, 8 * c + c);
    if (r == c) a = a / d;
    // eliminate column c from the other rows
    double pivrow = __shfl_sync(0xffffffffu, a, 8 * c + k);
    double f = __shfl_sync(0xffffffffu, a, 8 * r + c);
    if (r != c) a = a - f * pivrow;
  }
  __syncwarp();
  if (k >= 4) out[r * 4 + (k - 4)] = a;
  __syncwarp();
  return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ bool wait_flag(const int* flag, int epoch, int* status) {
  for (unsigned s = 0;; ++s) {
    if (ld_acquire_i32(flag) == epoch) return true;
    if (s >= 32) __nanosleep(128);  // back off: fewer polls competing with working warps
    if ((s & 255u) == 255u) {
      if (ld_volatile_i32(status) != DEV_OK) return false;
      if (s > CPTR_SPIN_LIMIT) {
        dev_fail(status, DEV_TIMEOUT);
        return false;
      }
    }
  }
}

// One warp per row; lanes 0..15 hold one entry (r, c) of a 4x4 block product.
__global__ void __launch_bounds__(256) k_ilu_factor(int npos, const int32_t* __restrict__ ord,
                                                    const int32_t* __restrict__ rp,
                                                    const int32_t* __restrict__ ci,
                                                    const int32_t* __restrict__ diag, double* LU,
                                                    int* done, int epoch, Ctl* ctl) {
  int lane = threadIdx.x & 31;
  int r = lane >> 2, c = lane & 3;
  bool act = lane < 16;
  for (;;) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(&ctl->fac_ctr, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= (unsigned)npos) return;
    int i = ord[item];
    if (i < 0) continue;
    int t0 = rp[i], td = diag[i], t1 = rp[i + 1];
    for (int t = t0; t < td; ++t) {
      int k = ci[t];
      if (lane == 0) wait_flag(done + k, epoch, &ctl->status);
      __syncwarp();
      const double* Ukk = LU + 16 * (size_t)diag[k];  // holds inv(U_kk)
      double* Aik = LU + 16 * (size_t)t;
      double s = 0.0;
      if (act)
        for (int q = 0; q < 4; ++q) s += __ldcg(Aik + r * 4 + q) * __ldcg(Ukk + q * 4 + c);
      __syncwarp();
      if (act) Aik[r * 4 + c] = s;
      __syncwarp();
      // A_ij -= L_ik U_kj for j > k present in both rows
      int k1 = rp[k + 1];
      int t2 = diag[k] + 1;
      for (int t3 = t + 1; t3 < t1; ++t3) {
        int j = ci[t3];
        while (t2 < k1 && ci[t2] < j) ++t2;
        if (t2 < k1 && ci[t2] == j) {
          const double* Ukj = LU + 16 * (size_t)t2;
          double p = 0.0;
          if (act)
            for (int q = 0; q < 4; ++q) p += __ldcg(Aik + r * 4 + q) * __ldcg(Ukj + q * 4 + c);
          __syncwarp();
          if (act) LU[16 * (size_t)t3 + r * 4 + c] = __ldcg(LU + 16 * (size_t)t3 + r * 4 + c) - p;
          __syncwarp();
        }
      }
    }
    if (lane == 0) {
      double blk[16], inv[16];
      double* Dii = LU + 16 * (size_t)td;
      for (int q = 0; q < 16; ++q) blk[q] = __ldcg(Dii + q);
      if (!inv4(blk, inv)) {
        dev_fail(&ctl->status, DEV_BREAKDOWN);
        for (int q = 0; q < 16; ++q) inv[q] = 0.0;
      }
      for (int q = 0; q < 16; ++q) Dii[q] = inv[q];
      __threadfence();
      st_release_i32(done + i, epoch);
    }
    __syncwarp();
  }
}

// Same factorisation with the row staged in shared memory: one warp per row,
// row i's blocks and columns loaded once (while its dependencies finish), and
// for every dependency k one parallel load of inv(U_kk) and of row k's upper
// part.  Column matches are found lane-parallel by binary search; the block
// products keep the sequential order of the definition (same results).  Rows
// longer than kRowMax blocks set *overflow and are left to k_ilu_factor.
constexpr int kRowMax = 32;
constexpr int kFacWarps = 4;
struct FacWarpSmem {
  double bi[kRowMax][16];
  double bk[kRowMax][16];
  double uinv[16];
  int ci[kRowMax];
  int ck[kRowMax];
  int match[kRowMax];
  int mt[kRowMax];
};

__global__ void __launch_bounds__(32 * kFacWarps) k_ilu_factor_staged(
    int npos, const int32_t* __restrict__ ord, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const int32_t* __restrict__ diag, double* LU, int* done,
    int epoch, Ctl* ctl, int* overflow) {
  extern __shared__ __align__(16) unsigned char fsm[];
  FacWarpSmem& W = reinterpret_cast<FacWarpSmem*>(fsm)[threadIdx.x >> 5];
  int lane = threadIdx.x & 31;
  int r = (lane >> 2) & 3, c = lane & 3;
  bool act = lane < 16;
  for (;;) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(&ctl->fac_ctr, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= (unsigned)npos) return;
    int i = ord[item];
    if (i < 0) continue;
    int t0 = rp[i], t1 = rp[i + 1], ni = t1 - t0, di = diag[i] - t0;
    if (ni > kRowMax) {
      if (lane == 0) atomicExch(overflow, 1);
      continue;  // left for the fallback kernel
    }
    if (lane < ni) W.ci[lane] = ci[t0 + lane];
    for (int q = lane; q < 16 * ni; q += 32) W.bi[q >> 4][q & 15] = LU[16 * (size_t)t0 + q];
    __syncwarp();
    for (int e = 0; e < di; ++e) {
      int k = W.ci[e];
      if (lane == 0) wait_flag(done + k, epoch, &ctl->status);
      __syncwarp();
      int kd = diag[k], nu = rp[k + 1] - kd - 1;
      if (nu > kRowMax) nu = kRowMax;  // rows that long are flagged by their own warp
      if (lane < 16) W.uinv[lane] = __ldcg(LU + 16 * (size_t)kd + lane);
      if (lane < nu) W.ck[lane] = __ldcg(ci + kd + 1 + lane);
      for (int q = lane; q < 16 * nu; q += 32)
        W.bk[q >> 4][q & 15] = __ldcg(LU + 16 * (size_t)(kd + 1) + q);
      __syncwarp();
      // L_ik = A_ik inv(U_kk)
      double s = 0.0;  // (the sum starts at its first product: 0.0 + x only loses -0.0)
      if (act) {
        s = W.bi[e][r * 4] * W.uinv[c];
        for (int q = 1; q < 4; ++q) s += W.bi[e][r * 4 + q] * W.uinv[q * 4 + c];
      }
      __syncwarp();
      if (act) W.bi[e][r * 4 + c] = s;
      // matches of row i's later columns in row k's upper part (rows hold at
      // most 32 blocks: one later column per lane), as a compact list
      {
        const int t3 = e + 1 + lane;
        int pos = -1;
        if (t3 < ni) {
          int j = W.ci[t3], lo = 0, hi = nu - 1;
          while (lo <= hi) {
            int mid = (lo + hi) >> 1;
            int x = W.ck[mid];
            if (x == j) { pos = mid; break; }
            if (x < j) lo = mid + 1; else hi = mid - 1;
          }
        }
        const unsigned mm = __ballot_sync(0xffffffffu, pos >= 0);
        if (pos >= 0) {
          const int slot = __popc(mm & ((1u << lane) - 1u));
          W.mt[slot] = t3;
          W.match[slot] = pos;
        }
        __syncwarp();
        // A_ij -= L_ik U_kj for the matched j, two blocks at a time (lanes
        // 16..31 take the odd matches): every block still gets its one update
        // for this k, with the same products in the same order
        const int nm = __popc(mm), hw = lane >> 4;
        for (int a = 0; a < nm; a += 2) {
          const int q3 = a + hw;
          if (q3 < nm) {
            const int tt = W.mt[q3], m = W.match[q3];
            double p = W.bi[e][r * 4] * W.bk[m][c];
            for (int q = 1; q < 4; ++q) p += W.bi[e][r * 4 + q] * W.bk[m][q * 4 + c];
            W.bi[tt][r * 4 + c] = W.bi[tt][r * 4 + c] - p;
          }
        }
        __syncwarp();
      }
    }
    if (!inv4_warp(W.bi[di], W.bi[di])) {
      if (lane == 0) dev_fail(&ctl->status, DEV_BREAKDOWN);
      if (lane < 16) W.bi[di][lane] = 0.0;
    }
    __syncwarp();
    for (int q = lane; q < 16 * ni; q += 32) LU[16 * (size_t)t0 + q] = W.bi[q >> 4][q & 15];
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release_i32(done + i, epoch);
    __syncwarp();
  }
}

__global__ void k_max_row(int N, const int32_t* __restrict__ rp, int* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) atomicMax(out, rp[i + 1] - rp[i]);
}

__global__ void k_sched_counts(int npos, const int32_t* __restrict__ ord,
                               const int32_t* __restrict__ rp, const int32_t* __restrict__ diag,
                               bool upper, int32_t* __restrict__ cnt) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npos) return;
  int i = ord[p];
  int n = 0;
  if (i >= 0) n = upper ? rp[i + 1] - diag[i] - 1 : diag[i] - rp[i];
  cnt[p] = n;
}

template <class T>
__global__ void k_sched_fill(int npos, const int32_t* __restrict__ ord,
                             const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const int32_t* __restrict__ diag, const double* __restrict__ LU,
                             bool upper, const int32_t* __restrict__ srp, int32_t* __restrict__ sci,
                             T* __restrict__ sv, T* __restrict__ dinv) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npos) return;
  int i = ord[p];
  if (i < 0) {
    if (dinv)
      for (int q = 0; q < 16; ++q) dinv[16 * (size_t)p + q] = 0;
    return;
  }
  int t0 = upper ? diag[i] + 1 : rp[i];
  int o = srp[p], n = srp[p + 1] - o;
  for (int a = 0; a < n; ++a) {
    sci[o + a] = ci[t0 + a];
    for (int q = 0; q < 16; ++q) sv[16 * (size_t)(o + a) + q] = (T)LU[16 * (size_t)(t0 + a) + q];
  }
  if (dinv)
    for (int q = 0; q < 16; ++q) dinv[16 * (size_t)p + q] = (T)LU[16 * (size_t)diag[i] + q];
}

// level sets by repeated sweeps until a sweep changes nothing
cptr_status compute_levels(cptr_ctx* c, bool upper, int32_t* lvl, int* nlev) {
  int N = c->N;
  unsigned* ctr;
  CTX_ALLOC(c, ctr, unsigned, 1, true);
  CTX_CUDA(c, cudaMemsetAsync(ctr, 0, sizeof(unsigned), cs(c)));
  CTX_CUDA(c, cudaMemsetAsync(lvl, 0xFF, sizeof(int32_t) * N, cs(c)));
  KL(c, k_level_syncfree<<<c->nsm * 8, 256, 0, cs(c)>>>(N, c->rp, c->ci, c->diag, lvl, upper,
                                                             ctr, &c->ctl->status));
  CTX_CUDA(c, cudaGetLastError());
  cptr_status st = ctx_check_device_status(c);
  if (st) {
    ctx_set_err(c, "level-set computation timed out");
    return st;
  }
  int32_t* cnt;
  int* mx;
  CTX_ALLOC(c, cnt, int32_t, N + 1, true);
  CTX_ALLOC(c, mx, int, 1, true);
  CTX_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (N + 1), cs(c)));
  CTX_CUDA(c, cudaMemsetAsync(mx, 0, sizeof(int), cs(c)));
  KL(c, k_level_count<<<nblk(N), kT, 0, cs(c)>>>(N, lvl, cnt, mx));
  int hm = 0;
  CTX_CUDA(c, cudaMemcpyAsync(&hm, mx, sizeof(int), cudaMemcpyDeviceToHost, cs(c)));
  CTX_CUDA(c, cudaStreamSynchronize(cs(c)));
  *nlev = hm + 1;
  return CPTR_OK;
}

cptr_status build_schedule(cptr_ctx* c, const int32_t* lvl, int nlev, int32_t** ord, int* npos,
                           int32_t** offs) {
  int N = c->N;
  int32_t *cnt, *pc, *off, *cur;
  CTX_ALLOC(c, cnt, int32_t, nlev + 1, true);
  CTX_ALLOC(c, pc, int32_t, nlev + 1, true);
  CTX_ALLOC(c, off, int32_t, nlev + 1, true);
  CTX_ALLOC(c, cur, int32_t, nlev + 1, true);
  int* mx;
  CTX_ALLOC(c, mx, int, 1, true);
  CTX_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nlev + 1), cs(c)));
  CTX_CUDA(c, cudaMemsetAsync(cur, 0, sizeof(int32_t) * (nlev + 1), cs(c)));
  KL(c, k_level_count<<<nblk(N), kT, 0, cs(c)>>>(N, lvl, cnt, mx));
  KL(c, k_pad8<<<nblk(nlev), kT, 0, cs(c)>>>(nlev, cnt, pc));
  int tot = 0;
  cptr_status st = scan_i32(c, pc, off, nlev, &tot);
  if (st) return st;
  CTX_ALLOC(c, *ord, int32_t, tot + 8, true);
  CTX_CUDA(c, cudaMemsetAsync(*ord, 0xFF, sizeof(int32_t) * (tot + 8), cs(c)));
  KL(c, k_level_fill<<<nblk(N), kT, 0, cs(c)>>>(N, lvl, off, cur, *ord));
  *npos = tot;
  *offs = off;  // first (padded) position of each level, nlev + 1 entries
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

template <class T>
cptr_status build_solve_arrays(cptr_ctx* c, bool upper) {
  int npos = upper ? c->npos_b : c->npos_f;
  const int32_t* ord = upper ? c->ord_b : c->ord_f;
  int32_t *cnt, *srp, *sci;
  CTX_ALLOC(c, cnt, int32_t, npos + 1, true);
  CTX_ALLOC(c, srp, int32_t, npos + 1, true);
  KL(c, k_sched_counts<<<nblk(npos), kT, 0, cs(c)>>>(npos, ord, c->rp, c->diag, upper, cnt));
  int tot = 0;
  cptr_status st = scan_i32(c, cnt, srp, npos, &tot);
  if (st) return st;
  CTX_ALLOC(c, sci, int32_t, tot + 1, true);
  T* sv;
  CTX_ALLOC(c, sv, T, 16 * (size_t)tot + 16, true);
  T* dinv = nullptr;
  if (upper) CTX_ALLOC(c, dinv, T, 16 * (size_t)npos + 16, true);
  KL(c, k_sched_fill<T><<<nblk(npos), kT, 0, cs(c)>>>(npos, ord, c->rp, c->ci, c->diag, c->LU64,
                                                    upper, srp, sci, sv, dinv));
  if (upper) {
    c->Urp = srp; c->Uci = sci; c->Uv = sv; c->Dinv = dinv;
    c->nnzU = tot;
  } else {
    c->Lrp = srp; c->Lci = sci; c->Lv = sv;
    c->nnzL = tot;
  }
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

}  // namespace

// Level sets, schedules and the factorisation (issued on cs(c); may run on
// the second stream beside the AMG setup).
cptr_status setup_ilu_factor(cptr_ctx* c) {
  int N = c->N;
  cptr_status st;
  CTX_ALLOC(c, c->lvl_f, int32_t, N + 1, true);
  CTX_ALLOC(c, c->lvl_b, int32_t, N + 1, true);
  st = compute_levels(c, false, c->lvl_f, &c->nlev_f);
  if (st) return st;
  st = compute_levels(c, true, c->lvl_b, &c->nlev_b);
  if (st) return st;
  ctx_phase(c, "  ilu level sets");
  st = build_schedule(c, c->lvl_f, c->nlev_f, &c->ord_f, &c->npos_f, &c->loff_f);
  if (st) return st;
  st = build_schedule(c, c->lvl_b, c->nlev_b, &c->ord_b, &c->npos_b, &c->loff_b);
  if (st) return st;
  ctx_phase(c, "  ilu schedules");
  // factorisation in place on a copy of A
  CTX_ALLOC(c, c->LU64, double, 16 * (size_t)c->nnzb, true);
  CTX_CUDA(c, cudaMemcpyAsync(c->LU64, c->v, sizeof(double) * 16 * (size_t)c->nnzb,
                              cudaMemcpyDeviceToDevice, cs(c)));
  if (!c->fac_done) {
    CTX_ALLOC(c, c->fac_done, int32_t, N + 1, false);
    CTX_CUDA(c, cudaMemsetAsync(c->fac_done, 0, sizeof(int32_t) * (N + 1), cs(c)));
  }
  c->fac_epoch += 1;
  CTX_CUDA(c, cudaMemsetAsync(&c->ctl->fac_ctr, 0, sizeof(unsigned), cs(c)));
  int* mrow;
  CTX_ALLOC(c, mrow, int, 2, true);
  CTX_CUDA(c, cudaMemsetAsync(mrow, 0, 2 * sizeof(int), cs(c)));
  KL(c, k_max_row<<<nblk(N), kT, 0, cs(c)>>>(N, c->rp, mrow));
  int hm = 0;
  CTX_CUDA(c, cudaMemcpyAsync(&hm, mrow, sizeof(int), cudaMemcpyDeviceToHost, cs(c)));
  CTX_CUDA(c, cudaStreamSynchronize(cs(c)));
  if (hm <= kRowMax && !c->force_fallback) {
    size_t smem = kFacWarps * sizeof(FacWarpSmem);
    KL(c, k_ilu_factor_staged<<<c->nsm * 8, 32 * kFacWarps, smem, cs(c)>>>(
              c->npos_f, c->ord_f, c->rp, c->ci, c->diag, c->LU64, c->fac_done, c->fac_epoch,
              c->ctl, mrow + 1));
  } else {
    KL(c, k_ilu_factor<<<c->nsm * 4, 256, 0, cs(c)>>>(c->npos_f, c->ord_f, c->rp, c->ci,
                                                          c->diag, c->LU64, c->fac_done,
                                                          c->fac_epoch, c->ctl));
  }
  CTX_CUDA(c, cudaGetLastError());
  st = ctx_check_device_status(c);
  if (st) return st;
  ctx_phase(c, "  ilu factorisation");
  return CPTR_OK;
}

// The triangular-solve schedule (its tuner times trial solves, so it runs
// alone on the context's stream).
cptr_status setup_ilu_schedule(cptr_ctx* c) {
  cptr_status st = tune_triangular(c);
  ctx_phase(c, "  ilu solve schedule");
  return st;
}

cptr_status setup_ilu(cptr_ctx* c) {
  cptr_status st = setup_ilu_factor(c);
  return st ? st : setup_ilu_schedule(c);
}

cptr_status build_level_solve_arrays(cptr_ctx* c) {
  cptr_status st;
  if (c->mixed) {
    st = build_solve_arrays<float>(c, false);
    if (!st) st = build_solve_arrays<float>(c, true);
  } else {
    st = build_solve_arrays<double>(c, false);
    if (!st) st = build_solve_arrays<double>(c, true);
  }
  return st;
}
