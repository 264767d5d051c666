// Preconditioner application (Eq. 3) on the device, in the apply precision T
// (float in CPTR_MIXED, double in CPTR_FP64):
//   rhat = R v                                  (Quasi-IMPES restriction)
//   zc   = one V(1,1)-cycle of the system AMG on Ahat applied to rhat
//   r2   = v - A P zc                           (injection + residual correction)
//   y2   = (L U)^-1 r2                          (ILU(0), sync-free level-ordered solves)
//   z    = P zc + y2
// Every kernel first reads an "active" flag so that the same launch sequence
// can sit in a CUDA graph and become a no-op once GMRES has stopped.
#include "common.cuh"
#include "ctx.h"

namespace {

constexpr int kT = 256;
inline int nblk(long long n, int per = kT) { return n > 0 ? ceil_div(n, per) : 1; }

// ------------------------------------------------------------------ conversions
template <class T>
__global__ void k_convert(long long n, const double* __restrict__ in, T* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (T)in[i];
}

template <class T>
__global__ void k_inverse(int n, const double* __restrict__ d, T* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (T)(1.0 / d[i]);
}

// AE[t][r][s] = A_t[r][e_s]: the elliptic columns of every block (4x2; the
// second column is zero when e has one unknown, e1 < 0).
template <class T>
__global__ void k_extract_ae(int nnzb, const double* __restrict__ v, int e0, int e1,
                             T* __restrict__ ae) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  const double* B = v + 16 * (size_t)t;
  for (int r = 0; r < 4; ++r) {
    ae[8 * (size_t)t + 2 * r + 0] = (T)B[r * 4 + e0];
    ae[8 * (size_t)t + 2 * r + 1] = e1 < 0 ? T(0) : (T)B[r * 4 + e1];
  }
}

// ------------------------------------------------------------------ restriction
// rhat_i = r_i[e] - W_i r_i[h]: ne = 2 values per cell (CPTR) or 1 (CPR, e1 < 0).
// TIN: double for a Krylov vector, T for a residual the preconditioner formed
// (CPTR3's temperature stage restricts the pressure stage's corrected residual).
template <class T, class TIN = double>
__global__ void k_restrict(int N, const TIN* __restrict__ vbase, const int* jptr, size_t stride,
                           const T* __restrict__ W, int e0, int e1, int h0, int h1, int h2,
                           T* __restrict__ rhat, const int* active, Ctl* ctl) {
  if (!*active) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) { ctl->fwd_ctr = 0u; ctl->bwd_ctr = 0u; }
  if (i >= N) return;
  const TIN* r = vbase + (size_t)(*jptr) * stride + 4 * (size_t)i;
  double rv[4];
  ld4(r, rv);
  const T* w = W + 4 * (size_t)i;
  if (e1 >= 0) {
    T re0 = (T)rv[e0], re1 = (T)rv[e1], rh0 = (T)rv[h0], rh1 = (T)rv[h1];
    T a = re0 - w[0] * rh0 - w[1] * rh1;
    T b = re1 - w[2] * rh0 - w[3] * rh1;
    rhat[2 * (size_t)i] = a;
    rhat[2 * (size_t)i + 1] = b;
  } else {
    T a = (T)rv[e0] - w[0] * (T)rv[h0] - w[1] * (T)rv[h1] - w[2] * (T)rv[h2];
    rhat[i] = a;
  }
}

// ------------------------------------------------------------------ V-cycle
// LANES consecutive lanes cooperate on one row of a scalar CSR operator.
template <int LANES, class T>
__device__ __forceinline__ T row_dot(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const T* __restrict__ val, const T* __restrict__ x, int i,
                                     int sl) {
  T s = 0;
  for (int t = rp[i] + sl; t < rp[i + 1]; t += LANES) s += val[t] * x[ci[t]];
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LANES);
  return s;
}

// x = Dinv b (pre-smoothing from x0 = 0) and r = b - A x in one pass.
template <int LANES, class T>
__global__ void k_vc_pre(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const T* __restrict__ val, const T* __restrict__ dinv,
                         const T* __restrict__ b, T* __restrict__ x, T* __restrict__ r,
                         const int* active) {
  if (!*active || n <= 0) return;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i = (int)(g / LANES), sl = (int)(g % LANES);
  bool ok = i < n;
  int ii = ok ? i : n - 1;
  T s = 0;
  for (int t = rp[ii] + sl; ok && t < rp[ii + 1]; t += LANES) {
    int j = ci[t];
    s += val[t] * (dinv[j] * b[j]);
  }
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LANES);
  if (ok && sl == 0) {
    T bi = b[i];
    x[i] = dinv[i] * bi;
    r[i] = bi - s;
  }
}

// y = M x for a scalar CSR M (restriction by R).
template <int LANES, class T>
__global__ void k_csr_mv(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const T* __restrict__ val, const T* __restrict__ x, T* __restrict__ y,
                         const int* active) {
  if (!*active || n <= 0) return;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i = (int)(g / LANES), sl = (int)(g % LANES);
  bool ok = i < n;
  int ii = ok ? i : n - 1;
  T s = 0;
  for (int t = rp[ii] + sl; ok && t < rp[ii + 1]; t += LANES) s += val[t] * x[ci[t]];
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LANES);
  if (ok && sl == 0) y[i] = s;
}

// x += P xc (prolongation, at most pmax entries per row).
template <class T>
__global__ void k_prolong(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const T* __restrict__ val, const T* __restrict__ xc, T* __restrict__ x,
                          const int* active) {
  if (!*active) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T s = 0;
  for (int t = rp[i]; t < rp[i + 1]; ++t) s += val[t] * xc[ci[t]];
  x[i] += s;
}

// xout = xin + Dinv (b - A xin) (post-smoothing).
template <int LANES, class T>
__global__ void k_vc_post(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const T* __restrict__ val, const T* __restrict__ dinv,
                          const T* __restrict__ b, const T* __restrict__ xin, T* __restrict__ xout,
                          const int* active) {
  if (!*active || n <= 0) return;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i = (int)(g / LANES), sl = (int)(g % LANES);
  bool ok = i < n;
  int ii = ok ? i : n - 1;
  T s = 0;
  for (int t = rp[ii] + sl; ok && t < rp[ii + 1]; t += LANES) s += val[t] * xin[ci[t]];
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LANES);
  if (ok && sl == 0) xout[i] = xin[i] + dinv[i] * (b[i] - s);
}

// r = b - A x.
template <int LANES, class T>
__global__ void k_vc_resid(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const T* __restrict__ val, const T* __restrict__ b,
                           const T* __restrict__ x, T* __restrict__ r, const int* active) {
  if (!*active || n <= 0) return;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i = (int)(g / LANES), sl = (int)(g % LANES);
  bool ok = i < n;
  int ii = ok ? i : n - 1;
  T s = 0;
  for (int t = rp[ii] + sl; ok && t < rp[ii + 1]; t += LANES) s += val[t] * x[ci[t]];
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LANES);
  if (ok && sl == 0) r[i] = b[i] - s;
}

// One hybrid l1-Gauss-Seidel sweep: one warp per block of kHgsBlock rows
// relaxes them in order (backward: in reverse), x_i += d_i^-1 (b_i - sum_j
// a_ij x_j), with the newest values of the block's rows and xin (the sweep's
// start) for every other row.  The block's row entries are first staged into
// shared memory, with the values of columns outside the block gathered then,
// so that the sequential part reads shared memory only; a block with more than
// kHgsStage entries reads its rows from global memory instead.
constexpr int kHgsBlock = 32;
constexpr int kHgsWarps = 4;
constexpr int kHgsStage = 512;
template <class T>
__global__ void __launch_bounds__(32 * kHgsWarps) k_hgs(
    int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const T* __restrict__ val, const T* __restrict__ dinv, const T* __restrict__ b,
    const T* __restrict__ xin, T* __restrict__ xout, int backward, const int* active) {
  if (!*active) return;
  __shared__ T xw_all[kHgsWarps][kHgsBlock];
  __shared__ T cv_all[kHgsWarps][kHgsStage];   // coefficient
  __shared__ T xe_all[kHgsWarps][kHgsStage];   // value of a column outside the block
  __shared__ int lc_all[kHgsWarps][kHgsStage]; // column inside the block (0..31), or -1
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k0 = (blockIdx.x * kHgsWarps + warp) * kHgsBlock;
  if (k0 >= n) return;
  const int k1 = min(k0 + kHgsBlock, n);
  T* xw = xw_all[warp];
  T* cv = cv_all[warp];
  T* xe = xe_all[warp];
  int* lc = lc_all[warp];
  if (k0 + lane < k1) xw[lane] = xin[k0 + lane];
  const int e0 = rp[k0], e1 = rp[k1];
  const bool staged = e1 - e0 <= kHgsStage;
  if (staged)
    for (int t = e0 + lane; t < e1; t += 32) {
      const int j = ci[t];
      const bool in = j >= k0 && j < k1;
      cv[t - e0] = val[t];
      lc[t - e0] = in ? j - k0 : -1;
      xe[t - e0] = in ? T(0) : xin[j];
    }
  __syncwarp();
  for (int q = 0; q < k1 - k0; ++q) {
    const int i = backward ? k1 - 1 - q : k0 + q;
    T s = 0;
    if (staged) {
      for (int t = rp[i] - e0 + lane; t < rp[i + 1] - e0; t += 32)
        s += cv[t] * (lc[t] >= 0 ? xw[lc[t]] : xe[t]);
    } else {
      for (int t = rp[i] + lane; t < rp[i + 1]; t += 32) {
        const int j = ci[t];
        s += val[t] * ((j >= k0 && j < k1) ? xw[j - k0] : xin[j]);
      }
    }
    s = warp_sum(s);
    if (lane == 0) xw[i - k0] = xw[i - k0] + dinv[i] * (b[i] - s);
    __syncwarp();
  }
  if (k0 + lane < k1) xout[k0 + lane] = xw[lane];
}

template <class T>
__global__ void k_copy_vec(int n, const T* __restrict__ in, T* __restrict__ out,
                           const int* active) {
  if (!*active) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i];
}

// x = Cinv b: dense FP64 coarsest solve, one warp per row.
template <class T>
__global__ void k_coarse(int n, const double* __restrict__ Cinv, const T* __restrict__ b,
                         T* __restrict__ x, const int* active) {
  if (!*active) return;
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s += Cinv[(size_t)row * n + c] * (double)b[c];
  s = warp_sum(s);
  if (lane == 0) x[row] = (T)s;
}

// ------------------------------------------------------------------ correction
// r2_i = v_i - sum_j A_ij[:, e] zc_j (P = injection into e), and the forward
// solve's output is reset to the "not yet written" sentinel.
template <class T, class TIN = double>
__global__ void k_correction(int N, int ne, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ ci, const T* __restrict__ ae,
                             const TIN* vbase, const int* jptr, size_t stride,
                             const T* __restrict__ zc, T* r2, T* __restrict__ u,
                             const int* active) {
  if (!*active) return;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i = (int)(g >> 2), r = (int)(g & 3);
  if (i >= N) return;
  T acc = 0;
  int t1 = rp[i + 1];
  if (ne == 2) {
    for (int t = rp[i]; t < t1; ++t) {
      int j = ci[t];
      const T* a = ae + 8 * (size_t)t + 2 * r;
      acc += a[0] * zc[2 * (size_t)j] + a[1] * zc[2 * (size_t)j + 1];
    }
  } else {
    for (int t = rp[i]; t < t1; ++t) acc += ae[8 * (size_t)t + 2 * r] * zc[ci[t]];
  }
  const TIN* v = vbase + (size_t)(*jptr) * stride;
  r2[4 * (size_t)i + r] = (T)v[4 * (size_t)i + r] - acc;  // (in place when v is r2)
  u[4 * (size_t)i + r] = sentinel_of(T(0));
}

// z_i[a] += za_i and z_i[b] += zb_i: CPTR3's two first-stage corrections added
// to the ILU(0) output (one elliptic unknown each).
template <class T>
__global__ void k_add_stages(int N, const T* __restrict__ za, int a, const T* __restrict__ zb,
                             int b, T* __restrict__ zbase, const int* jptr, size_t stride,
                             const int* active) {
  if (!*active) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  T* z = zbase + (size_t)(*jptr) * stride + 4 * (size_t)i;
  z[a] += za[i];
  z[b] += zb[i];
}

// r2 = v (second stage alone) with the same sentinel reset.
template <class T>
__global__ void k_copy_in(int N, const double* __restrict__ vbase, const int* jptr, size_t stride,
                          T* __restrict__ r2, T* __restrict__ u, const int* active, Ctl* ctl) {
  if (!*active) return;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0) { ctl->fwd_ctr = 0u; ctl->bwd_ctr = 0u; }
  if (g >= 4ll * N) return;
  const double* v = vbase + (size_t)(*jptr) * stride;
  r2[g] = (T)v[g];
  u[g] = sentinel_of(T(0));
}

// z = P zc (first stage alone) or z = v (no preconditioner).
template <class T>
__global__ void k_inject(int N, const T* __restrict__ zc, int e0, int e1, T* __restrict__ zbase,
                         const int* jptr, size_t stride, const int* active) {
  if (!*active) return;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 4ll * N) return;
  int i = (int)(g >> 2), r = (int)(g & 3);
  T v = 0;
  const int ne = e1 < 0 ? 1 : 2;
  if (r == e0) v = zc[ne * (size_t)i];
  else if (r == e1) v = zc[ne * (size_t)i + 1];
  zbase[(size_t)(*jptr) * stride + g] = v;
}

template <class T>
__global__ void k_identity(long long n, const double* __restrict__ vbase, T* __restrict__ zbase,
                           const int* jptr, size_t stride, const int* active) {
  if (!*active) return;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  zbase[(size_t)(*jptr) * stride + g] = (T)vbase[(size_t)(*jptr) * stride + g];
}

// ------------------------------------------------------------------ ILU(0) solves
// Sync-free level-scheduled block triangular solves.  The schedule lists the
// rows level by level, each level padded to a multiple of 8 rows; a warp claims
// the next group of 8 schedule positions from a counter (so a group never mixes
// levels and only waits on groups claimed earlier by running warps) and
// handles one row per 4-lane quad, lane r computing component r.  A row's
// dependencies are read through their values, which start as a sentinel NaN:
// a 4-vector that holds no sentinel is final.  Waits are bounded.
template <class T>
__device__ __forceinline__ bool wait_vec(const T* p, T* o, int* status, unsigned limit) {
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

// acc minus, in the row's order, F_k y_{j_k} over its dependencies k in
// [kb, ke), waiting for each y: the indices and factor blocks of the first
// kPre dependencies are loaded before the first wait, so that when one
// dependency arrives the next one's index and block are already in registers.
template <class T>
__device__ __forceinline__ T dep_chain(T acc, int kb, int ke, const int32_t* __restrict__ ci,
                                       const T* __restrict__ F, const T* y, int r, int* status,
                                       unsigned lim) {
  constexpr int kPre = 4;
  int j[kPre];
  T f[kPre][4];
  const int np = ke - kb < kPre ? ke - kb : kPre;
#pragma unroll
  for (int q = 0; q < kPre; ++q)
    if (q < np) {
      j[q] = ci[kb + q];
      ld4(F + 16 * (size_t)(kb + q) + 4 * r, f[q]);
    }
#pragma unroll
  for (int q = 0; q < kPre; ++q)
    if (q < np) {
      T yj[4];
      wait_vec(y + 4 * (size_t)j[q], yj, status, lim);
      acc = sub_rn(acc, dot4(f[q], yj));
    }
  for (int k = kb + kPre; k < ke; ++k) {
    const int jj = ci[k];
    T a[4], yj[4];
    ld4(F + 16 * (size_t)k + 4 * r, a);
    wait_vec(y + 4 * (size_t)jj, yj, status, lim);
    acc = sub_rn(acc, dot4(a, yj));
  }
  return acc;
}

template <class T>
__global__ void __launch_bounds__(256) k_ilu_fwd(int npos, const int32_t* __restrict__ ord,
                                                 const int32_t* __restrict__ Lrp,
                                                 const int32_t* __restrict__ Lci,
                                                 const T* __restrict__ Lv, const T* __restrict__ r2,
                                                 T* u, T* __restrict__ y2, Ctl* ctl,
                                                 const int* active) {
  if (!*active) return;
  int lane = threadIdx.x & 31, sub = lane >> 2, r = lane & 3;
  unsigned ngroups = (unsigned)((npos + 7) >> 3);
  const unsigned lim = ctl->spin;
  for (;;) {
    unsigned gq = 0;
    if (lane == 0) gq = atomicAdd(&ctl->fwd_ctr, 1u);
    gq = __shfl_sync(0xffffffffu, gq, 0);
    if (gq >= ngroups) return;
    int pos = (int)(gq * 8 + sub);
    int i = (pos < npos) ? ord[pos] : -1;
    if (i < 0) continue;
    T acc = dep_chain<T>(r2[4 * (size_t)i + r], Lrp[pos], Lrp[pos + 1], Lci, Lv, u, r,
                         &ctl->status, lim);
    st_volatile(u + 4 * (size_t)i + r, desentinel(acc));
    y2[4 * (size_t)i + r] = sentinel_of(T(0));
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_ilu_bwd(int npos, const int32_t* __restrict__ ord,
                                                 const int32_t* __restrict__ Urp,
                                                 const int32_t* __restrict__ Uci,
                                                 const T* __restrict__ Uv,
                                                 const T* __restrict__ Dinv,
                                                 const T* __restrict__ u, T* y2,
                                                 const T* __restrict__ zc, int e0, int e1,
                                                 T* __restrict__ zbase, const int* jptr,
                                                 size_t stride, Ctl* ctl, const int* active) {
  if (!*active) return;
  int lane = threadIdx.x & 31, sub = lane >> 2, r = lane & 3;
  unsigned ngroups = (unsigned)((npos + 7) >> 3);
  const unsigned lim = ctl->spin;
  T* z = zbase + (size_t)(*jptr) * stride;
  for (;;) {
    unsigned gq = 0;
    if (lane == 0) gq = atomicAdd(&ctl->bwd_ctr, 1u);
    gq = __shfl_sync(0xffffffffu, gq, 0);
    if (gq >= ngroups) return;
    int pos = (int)(gq * 8 + sub);
    int i = (pos < npos) ? ord[pos] : -1;
    if (i < 0) continue;
    // everything that does not depend on other rows is loaded before the
    // dependency waits, so that only the waits and the arithmetic chain the
    // levels (inv(U_ii) loaded after them cost one more memory latency per level)
    T acc = u[4 * (size_t)i + r];
    T d[4];
    ld4(Dinv + 16 * (size_t)pos + 4 * r, d);
    T y1 = 0;
    if (zc) {
      const int ne = e1 < 0 ? 1 : 2;
      if (r == e0) y1 = zc[ne * (size_t)i];
      else if (r == e1) y1 = zc[ne * (size_t)i + 1];
    }
    acc = dep_chain<T>(acc, Urp[pos], Urp[pos + 1], Uci, Uv, y2, r, &ctl->status, lim);
    unsigned mask = 0xFu << (lane & ~3);
    int q0 = lane & ~3;
    T s0 = __shfl_sync(mask, acc, q0 + 0);
    T s1 = __shfl_sync(mask, acc, q0 + 1);
    T s2 = __shfl_sync(mask, acc, q0 + 2);
    T s3 = __shfl_sync(mask, acc, q0 + 3);
    T sv4[4] = {s0, s1, s2, s3};
    T y = dot4(d, sv4);
    st_volatile(y2 + 4 * (size_t)i + r, desentinel(y));
    z[4 * (size_t)i + r] = y1 + y;
  }
}

// ------------------------------------------------------------------ launchers
template <class T>
void launch_rowkernel_pre(int lanes, int n, const Level& L, const T* b, T* x, T* r,
                          const int* active, cptr_ctx* c) {
  cudaStream_t s = c->stream;
  const T* av = (const T*)L.Av;
  const T* dv = (const T*)L.dinv;
  long long thr = (long long)n * lanes;
  switch (lanes) {
    case 2: KL(c, k_vc_pre<2, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, dv, b, x, r, active)); break;
    case 4: KL(c, k_vc_pre<4, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, dv, b, x, r, active)); break;
    case 8: KL(c, k_vc_pre<8, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, dv, b, x, r, active)); break;
    case 16: KL(c, k_vc_pre<16, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, dv, b, x, r, active)); break;
    default: KL(c, k_vc_pre<32, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, dv, b, x, r, active)); break;
  }
}

template <class T>
void launch_rowkernel_post(int lanes, int n, const Level& L, const T* b, const T* xin, T* xout,
                           const int* active, cptr_ctx* c) {
  cudaStream_t s = c->stream;
  const T* av = (const T*)L.Av;
  const T* dv = (const T*)L.dinv;
  long long thr = (long long)n * lanes;
  switch (lanes) {
    case 2: KL(c, k_vc_post<2, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, dv, b, xin, xout, active)); break;
    case 4: KL(c, k_vc_post<4, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, dv, b, xin, xout, active)); break;
    case 8: KL(c, k_vc_post<8, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, dv, b, xin, xout, active)); break;
    case 16: KL(c, k_vc_post<16, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, dv, b, xin, xout, active)); break;
    default: KL(c, k_vc_post<32, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, dv, b, xin, xout, active)); break;
  }
}

template <class T>
void launch_csr_mv(int lanes, const DCSR& M, const T* val, const T* x, T* y, const int* active,
                   cptr_ctx* c) {
  cudaStream_t s = c->stream;
  long long thr = (long long)M.n * lanes;
  switch (lanes) {
    case 2: KL(c, k_csr_mv<2, T><<<nblk(thr), kT, 0, s>>>(M.n, M.rp, M.ci, val, x, y, active)); break;
    case 4: KL(c, k_csr_mv<4, T><<<nblk(thr), kT, 0, s>>>(M.n, M.rp, M.ci, val, x, y, active)); break;
    case 8: KL(c, k_csr_mv<8, T><<<nblk(thr), kT, 0, s>>>(M.n, M.rp, M.ci, val, x, y, active)); break;
    case 16: KL(c, k_csr_mv<16, T><<<nblk(thr), kT, 0, s>>>(M.n, M.rp, M.ci, val, x, y, active)); break;
    default: KL(c, k_csr_mv<32, T><<<nblk(thr), kT, 0, s>>>(M.n, M.rp, M.ci, val, x, y, active)); break;
  }
}

template <class T>
void launch_resid(int lanes, int n, const Level& L, const T* b, const T* x, T* r,
                  const int* active, cptr_ctx* c) {
  cudaStream_t s = c->stream;
  const T* av = (const T*)L.Av;
  long long thr = (long long)n * lanes;
  switch (lanes) {
    case 2: KL(c, k_vc_resid<2, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, b, x, r, active)); break;
    case 4: KL(c, k_vc_resid<4, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, b, x, r, active)); break;
    case 8: KL(c, k_vc_resid<8, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, b, x, r, active)); break;
    case 16: KL(c, k_vc_resid<16, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, b, x, r, active)); break;
    default: KL(c, k_vc_resid<32, T><<<nblk(thr), kT, 0, s>>>(n, L.A.rp, L.A.ci, av, b, x, r, active)); break;
  }
}

// one smoothing sweep xin -> xout (distinct buffers) with the context's smoother
template <class T>
void launch_sweep(cptr_ctx* c, const Level& L, const T* b, const T* xin, T* xout, bool backward,
                  const int* active) {
  const int n = L.A.n;
  if (c->p.smoother == CPTR_SMOOTH_HYBRID_GS) {
    const int blocks = ceil_div(ceil_div(n, kHgsBlock), kHgsWarps);
    KL(c, k_hgs<T><<<blocks > 0 ? blocks : 1, 32 * kHgsWarps, 0, c->stream>>>(
              n, L.A.rp, L.A.ci, (const T*)L.Av, (const T*)L.dinv, b, xin, xout,
              backward ? 1 : 0, active));
  } else {
    launch_rowkernel_post<T>(L.lanes, n, L, b, xin, xout, active, c);
  }
}

// output vector of level l after its V-cycle
template <class T>
T* level_out(cptr_ctx* c, int l) {
  int last = (int)c->lev.size() - 1;
  if (l == 0) return (T*)c->zc;
  if (l == last) return (T*)c->lev[l].x;
  return (T*)c->lev[l].x2;
}

template <class T>
void launch_vcycle(cptr_ctx* c, const T* b0, const int* active) {
  cudaStream_t s = c->stream;
  int last = (int)c->lev.size() - 1;
  const int nu1 = c->p.nu_pre, nu2 = c->p.nu_post;
  const bool fused_pre = nu1 == 1 && c->p.smoother == CPTR_SMOOTH_L1_JACOBI;
  for (int l = 0; l < last; ++l) {
    Level& L = c->lev[l];
    const T* b = (l == 0) ? b0 : (const T*)L.b;
    if (fused_pre) {
      // one l1-Jacobi sweep from zero (x = D^-1 b) fused with the residual
      launch_rowkernel_pre<T>(L.lanes, L.A.n, L, b, (T*)L.x, (T*)L.r, active, c);
    } else {
      // nu1 sweeps from x = 0 (zero start in r), alternating between t and x
      // so that the last one writes x, then r = b - A x
      const size_t nb = sizeof(T) * (size_t)(L.A.n + 1);
      if (nu1 == 0) {
        CTX_CUDA_V(c, cudaMemsetAsync(L.x, 0, nb, s));
      } else {
        CTX_CUDA_V(c, cudaMemsetAsync(L.r, 0, nb, s));
        const T* src = (const T*)L.r;
        for (int k = 0; k < nu1; ++k) {
          T* dst = ((nu1 - 1 - k) % 2 == 0) ? (T*)L.x : (T*)L.t;
          launch_sweep<T>(c, L, b, src, dst, false, active);
          src = dst;
        }
      }
      launch_resid<T>(L.lanes, L.A.n, L, b, (const T*)L.x, (T*)L.r, active, c);
    }
    double ravg = L.R.n ? (double)L.R.nnz / L.R.n : 1.0;
    int rl = ravg <= 8 ? 2 : ravg <= 20 ? 4 : ravg <= 48 ? 8 : 16;
    launch_csr_mv<T>(rl, L.R, (const T*)L.Rv, (const T*)L.r, (T*)c->lev[l + 1].b, active, c);
  }
  {
    Level& Lc = c->lev[last];
    const T* b = (last == 0) ? b0 : (const T*)Lc.b;
    int n = Lc.A.n;
    KL(c, k_coarse<T><<<nblk((long long)n * 32), kT, 0, s>>>(n, c->Cinv, b, level_out<T>(c, last),
                                                       active));
  }
  for (int l = last - 1; l >= 0; --l) {
    Level& L = c->lev[l];
    const T* b = (l == 0) ? b0 : (const T*)L.b;
    KL(c, k_prolong<T><<<nblk(L.A.n), kT, 0, s>>>(L.A.n, L.P.rp, L.P.ci, (const T*)L.Pv,
                                            level_out<T>(c, l + 1), (T*)L.x, active));
    // nu2 sweeps (backward for the hybrid smoother) ending in the level's output
    T* out = level_out<T>(c, l);
    if (nu2 == 0) {
      KL(c, k_copy_vec<T><<<nblk(L.A.n), kT, 0, s>>>(L.A.n, (const T*)L.x, out, active));
    } else {
      const T* src = (const T*)L.x;
      for (int k = 0; k < nu2; ++k) {
        T* dst = (k == nu2 - 1) ? out : (src == (const T*)L.x ? (T*)L.t : (T*)L.x);
        launch_sweep<T>(c, L, b, src, dst, true, active);
        src = dst;
      }
    }
  }
}

template <class T>
void launch_ilu_levels(cptr_ctx* c, const T* zc, void* zbase, const int* jptr, size_t stride,
                       const int* active, int which) {
  cudaStream_t s = c->stream;
  // warps claim groups of 8 rows in level order; the grid bounds how many rows
  // are in flight (a few levels' worth: more only adds warps spinning on rows
  // far ahead of the wavefront, whose polls compete for L2 with the solve)
  // (measured on GB300: 3 blocks of 8 warps per SM beat 8 per SM by 3-8% on the
  // 64x64x32, 1M-point kNN and 200x200x100 systems; fewer lose throughput)
  int grid = c->lvl_grid_forced ? c->lvl_grid_forced : c->lvl_grid ? c->lvl_grid : c->nsm * 3;
  if (which != 2)
    KL(c, k_ilu_fwd<T><<<grid, 256, 0, s>>>(c->npos_f, c->ord_f, c->Lrp, c->Lci, (const T*)c->Lv,
                                            (const T*)c->r2, (T*)c->u, (T*)c->y2, c->ctl, active));
  if (which != 1)
    KL(c, k_ilu_bwd<T><<<grid, 256, 0, s>>>(c->npos_b, c->ord_b, c->Urp, c->Uci, (const T*)c->Uv,
                                            (const T*)c->Dinv, (const T*)c->u, (T*)c->y2, zc,
                                            c->se0, c->se1, (T*)zbase, jptr, stride, c->ctl,
                                            active));
}

// which: 0 = forward and backward, 1 = forward only, 2 = backward only
template <class T>
void launch_ilu(cptr_ctx* c, const T* zc, void* zbase, const int* jptr, size_t stride,
                const int* active, int which = 0) {
  if (c->cluster) launch_tri_cluster(c, zc, zbase, jptr, stride, active, which);
  else if (c->strip) launch_tri_strip(c, zc, zbase, jptr, stride, active, which);
  else if (c->chain) launch_tri_chain(c, zc, zbase, jptr, stride, active, which);
  else if (c->chunked) launch_tri_chunked(c, zc, zbase, jptr, stride, active, which);
  else launch_ilu_levels<T>(c, zc, zbase, jptr, stride, active, which);
}

// elliptic unknowns per cell: 2 (CPTR) or 1 (CPR, e1 < 0)
inline int nell(const cptr_ctx* c) { return c->se1 < 0 ? 1 : 2; }

// k-th hyperbolic unknown (-1 past the last one)
int hidx(const cptr_ctx* c, int k) {
  int h[3] = {-1, -1, -1}, q = 0;
  for (int u = 0; u < 4; ++u)
    if (u != c->se0 && u != c->se1) h[q++] = u;
  return h[k];
}

template <class T>
void launch_precond_t(cptr_ctx* c, const double* vbase, void* zbase, const int* jptr,
                      const int* active) {
  cudaStream_t s = c->stream;
  int N = c->N;
  size_t stride = 4 * (size_t)N;
  switch (c->p.precond) {
    case CPTR_PREC_NONE:
      KL(c, k_identity<T><<<nblk(4ll * N), kT, 0, s>>>(4ll * N, vbase, (T*)zbase, jptr, stride, active));
      return;
    case CPTR_PREC_ILU:
      KL(c, k_copy_in<T><<<nblk(4ll * N), kT, 0, s>>>(N, vbase, jptr, stride, (T*)c->r2, (T*)c->u,
                                                active, c->ctl));
      launch_ilu<T>(c, nullptr, zbase, jptr, stride, active);
      return;
    default:
      break;
  }
  KL(c, k_restrict<T><<<nblk(N), kT, 0, s>>>(N, vbase, jptr, stride, (const T*)c->Wt, c->se0, c->se1,
                                       hidx(c, 0), hidx(c, 1), hidx(c, 2), (T*)c->rhat, active, c->ctl));
  launch_vcycle<T>(c, (const T*)c->rhat, active);
  if (c->p.precond == CPTR_PREC_FIRST) {
    KL(c, k_inject<T><<<nblk(4ll * N), kT, 0, s>>>(N, (const T*)c->zc, c->se0, c->se1, (T*)zbase,
                                             jptr, stride, active));
    return;
  }
  KL(c, k_correction<T><<<nblk(4ll * N), kT, 0, s>>>(N, nell(c), c->rp, c->ci, (const T*)c->AE, vbase, jptr,
                                               stride, (const T*)c->zc, (T*)c->r2, (T*)c->u,
                                               active));
  if (c->p.precond != CPTR_PREC_CPTR3) {
    launch_ilu<T>(c, (const T*)c->zc, zbase, jptr, stride, active);
    return;
  }
  // CPTR3 (Section 3.3): the temperature stage on the residual the pressure
  // stage leaves, r2 <- r2 - A P_T Vcycle_T(R_T r2), then ILU(0) on r2 and the
  // two stage corrections added to its output
  const int* zero = &c->ctl->zero;
  swap_stage(c);
  KL(c, k_restrict<T, T><<<nblk(N), kT, 0, s>>>(N, (const T*)c->r2, zero, 0, (const T*)c->Wt,
                                                c->se0, c->se1, hidx(c, 0), hidx(c, 1),
                                                hidx(c, 2), (T*)c->rhat, active, c->ctl));
  launch_vcycle<T>(c, (const T*)c->rhat, active);
  KL(c, k_correction<T, T><<<nblk(4ll * N), kT, 0, s>>>(N, nell(c), c->rp, c->ci,
                                                        (const T*)c->AE, (const T*)c->r2, zero,
                                                        0, (const T*)c->zc, (T*)c->r2,
                                                        (T*)c->u, active));
  const T* zcT = (const T*)c->zc;
  const int eT = c->se0;
  swap_stage(c);
  launch_ilu<T>(c, nullptr, zbase, jptr, stride, active);
  KL(c, k_add_stages<T><<<nblk(N), kT, 0, s>>>(N, (const T*)c->zc, c->se0, zcT, eT, (T*)zbase,
                                              jptr, stride, active));
}

template <class T>
cptr_status setup_buffers_t(cptr_ctx* c) {
  cudaStream_t s = c->stream;
  int N = c->N;
  if (c->W64) {  // first-stage data exists only when the first stage was built
    CTX_ALLOC(c, c->Wt, T, 4 * (size_t)N, true);
    KL(c, k_convert<T><<<nblk(4ll * N), kT, 0, s>>>(4ll * N, c->W64, (T*)c->Wt));
    CTX_ALLOC(c, c->AE, T, 8 * (size_t)c->nnzb, true);
    KL(c, k_extract_ae<T><<<nblk(c->nnzb), kT, 0, s>>>(c->nnzb, c->v, c->se0, c->se1, (T*)c->AE));
  }
  CTX_ALLOC(c, c->rhat, T, (size_t)nell(c) * N, true);
  CTX_ALLOC(c, c->zc, T, (size_t)nell(c) * N, true);
  if (!c->r2) CTX_ALLOC(c, c->r2, T, 4 * (size_t)N, true);  // may exist from the solve tuning
  if (!c->u) CTX_ALLOC(c, c->u, T, 4 * (size_t)N, true);
  if (!c->y2) CTX_ALLOC(c, c->y2, T, 4 * (size_t)N, true);
  if (!c->zt) CTX_ALLOC(c, c->zt, T, 4 * (size_t)N, true);
  int last = (int)c->lev.size() - 1;
  for (int l = 0; l <= last; ++l) {
    Level& L = c->lev[l];
    int n = L.A.n;
    double avg = n ? (double)L.A.nnz / n : 1.0;
    L.lanes = avg <= 8 ? 2 : avg <= 20 ? 4 : avg <= 48 ? 8 : avg <= 128 ? 16 : 32;
    CTX_ALLOC(c, L.b, T, n + 1, true);
    CTX_ALLOC(c, L.x, T, n + 1, true);
    CTX_ALLOC(c, L.r, T, n + 1, true);
    CTX_ALLOC(c, L.x2, T, n + 1, true);
    CTX_ALLOC(c, L.t, T, n + 1, true);
    if (l == last) continue;
    CTX_ALLOC(c, L.Av, T, L.A.nnz + 1, true);
    KL(c, k_convert<T><<<nblk(L.A.nnz), kT, 0, s>>>(L.A.nnz, L.A.v, (T*)L.Av));
    CTX_ALLOC(c, L.Pv, T, L.P.nnz + 1, true);
    KL(c, k_convert<T><<<nblk(L.P.nnz), kT, 0, s>>>(L.P.nnz, L.P.v, (T*)L.Pv));
    CTX_ALLOC(c, L.Rv, T, L.R.nnz + 1, true);
    KL(c, k_convert<T><<<nblk(L.R.nnz), kT, 0, s>>>(L.R.nnz, L.R.v, (T*)L.Rv));
    CTX_ALLOC(c, L.dinv, T, n + 1, true);
    KL(c, k_inverse<T><<<nblk(n), kT, 0, s>>>(n, L.dl1, (T*)L.dinv));
  }
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

template <class T>
__global__ void k_from_t(long long n, const T* __restrict__ in, double* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

template <class T>
cptr_status apply_piece_t(cptr_ctx* c, int which, const double* in, double* out) {
  cudaStream_t s = c->stream;
  int N = c->N;
  const int* zero = &c->ctl->zero;
  const int* one = &c->ctl->one;
  size_t stride = 4 * (size_t)N;
  switch (which) {
    case CPTR_APPLY_PRECOND:
      launch_precond_t<T>(c, in, c->zt, zero, one);
      KL(c, k_from_t<T><<<nblk(4ll * N), kT, 0, s>>>(4ll * N, (const T*)c->zt, out));
      break;
    case CPTR_APPLY_RESTRICT:
      KL(c, k_restrict<T><<<nblk(N), kT, 0, s>>>(N, in, zero, stride, (const T*)c->Wt, c->se0, c->se1,
                                           hidx(c, 0), hidx(c, 1), hidx(c, 2), (T*)c->rhat, one, c->ctl));
      KL(c, k_from_t<T><<<nblk((long long)nell(c) * N), kT, 0, s>>>((long long)nell(c) * N, (const T*)c->rhat, out));
      break;
    case CPTR_APPLY_VCYCLE:
      KL(c, k_convert<T><<<nblk((long long)nell(c) * N), kT, 0, s>>>((long long)nell(c) * N, in, (T*)c->rhat));
      launch_vcycle<T>(c, (const T*)c->rhat, one);
      KL(c, k_from_t<T><<<nblk((long long)nell(c) * N), kT, 0, s>>>((long long)nell(c) * N, (const T*)c->zc, out));
      break;
    case CPTR_APPLY_FIRST:
    case CPTR_APPLY_CORRECTION:
      KL(c, k_restrict<T><<<nblk(N), kT, 0, s>>>(N, in, zero, stride, (const T*)c->Wt, c->se0, c->se1,
                                           hidx(c, 0), hidx(c, 1), hidx(c, 2), (T*)c->rhat, one, c->ctl));
      launch_vcycle<T>(c, (const T*)c->rhat, one);
      if (which == CPTR_APPLY_FIRST) {
        KL(c, k_inject<T><<<nblk(4ll * N), kT, 0, s>>>(N, (const T*)c->zc, c->se0, c->se1,
                                                 (T*)c->zt, zero, stride, one));
        KL(c, k_from_t<T><<<nblk(4ll * N), kT, 0, s>>>(4ll * N, (const T*)c->zt, out));
      } else {
        KL(c, k_correction<T><<<nblk(4ll * N), kT, 0, s>>>(N, nell(c), c->rp, c->ci, (const T*)c->AE, in, zero,
                                                     stride, (const T*)c->zc, (T*)c->r2,
                                                     (T*)c->u, one));
        KL(c, k_from_t<T><<<nblk(4ll * N), kT, 0, s>>>(4ll * N, (const T*)c->r2, out));
      }
      break;
    case CPTR_APPLY_ILU:
      KL(c, k_copy_in<T><<<nblk(4ll * N), kT, 0, s>>>(N, in, zero, stride, (T*)c->r2, (T*)c->u, one,
                                                c->ctl));
      launch_ilu<T>(c, nullptr, c->zt, zero, stride, one);
      KL(c, k_from_t<T><<<nblk(4ll * N), kT, 0, s>>>(4ll * N, (const T*)c->zt, out));
      break;
    default:
      ctx_set_err(c, "unknown apply selector");
      return CPTR_ERR_INVALID;
  }
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

}  // namespace

cptr_status setup_apply_buffers(cptr_ctx* c) {
  return c->mixed ? setup_buffers_t<float>(c) : setup_buffers_t<double>(c);
}

void launch_precond(cptr_ctx* c, const double* vbase, void* zbase, const int* jptr,
                    const int* active) {
  if (c->mixed) launch_precond_t<float>(c, vbase, zbase, jptr, active);
  else launch_precond_t<double>(c, vbase, zbase, jptr, active);
}

namespace {
template <class T>
__global__ void k_reset_sentinel(long long n, T* __restrict__ u, Ctl* ctl) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) { ctl->fwd_ctr = 0u; ctl->bwd_ctr = 0u; }
  if (i < n) u[i] = sentinel_of(T(0));
}

template <class T>
cptr_status profile_apply_t(cptr_ctx* c, int kernel, bool prepare) {
  cudaStream_t s = c->stream;
  const int* zero = &c->ctl->zero;
  const int* one = &c->ctl->one;
  long long n4 = 4ll * c->N;
  size_t stride = (size_t)n4;
  bool first = !c->lev.empty();
  switch (kernel) {
    case CPTR_KERNEL_ILU_FWD:
    case CPTR_KERNEL_ILU_BWD:
      if (!c->LU64) return CPTR_ERR_INVALID;
      if (prepare) {
        KL(c, k_reset_sentinel<T><<<nblk(n4), kT, 0, s>>>(n4, (T*)c->u, c->ctl));
        if (kernel == CPTR_KERNEL_ILU_BWD) launch_ilu<T>(c, nullptr, c->zt, zero, stride, one, 1);
      } else {
        launch_ilu<T>(c, first ? (const T*)c->zc : nullptr, c->zt, zero, stride, one,
                      kernel == CPTR_KERNEL_ILU_FWD ? 1 : 2);
      }
      break;
    case CPTR_KERNEL_VC_PRE0:
      if (!first || c->lev.size() < 2) return CPTR_ERR_INVALID;
      if (!prepare)
        launch_rowkernel_pre<T>(c->lev[0].lanes, c->lev[0].A.n, c->lev[0], (const T*)c->rhat,
                                (T*)c->lev[0].x, (T*)c->lev[0].r, one, c);
      break;
    case CPTR_KERNEL_CORRECTION:
      if (!first || !c->LU64) return CPTR_ERR_INVALID;
      if (!prepare)
        KL(c, k_correction<T><<<nblk(n4), kT, 0, s>>>(c->N, nell(c), c->rp, c->ci, (const T*)c->AE, c->V,
                                                     zero, stride, (const T*)c->zc, (T*)c->r2,
                                                     (T*)c->u, one));
      break;
    default:
      return CPTR_ERR_INVALID;
  }
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}
}  // namespace

void launch_level_solves(cptr_ctx* c, void* zbase) {
  size_t stride = 4 * (size_t)c->N;
  if (c->mixed)
    launch_ilu_levels<float>(c, nullptr, zbase, &c->ctl->zero, stride, &c->ctl->one, 0);
  else
    launch_ilu_levels<double>(c, nullptr, zbase, &c->ctl->zero, stride, &c->ctl->one, 0);
}

cptr_status profile_apply_kernel(cptr_ctx* c, int kernel, bool prepare) {
  return c->mixed ? profile_apply_t<float>(c, kernel, prepare)
                  : profile_apply_t<double>(c, kernel, prepare);
}

cptr_status launch_apply_piece(cptr_ctx* c, int which, const double* in, double* out) {
  if ((which == CPTR_APPLY_RESTRICT || which == CPTR_APPLY_VCYCLE || which == CPTR_APPLY_FIRST ||
       which == CPTR_APPLY_CORRECTION) && c->lev.empty()) {
    ctx_set_err(c, "no first stage in this preconditioner configuration");
    return CPTR_ERR_INVALID;
  }
  return c->mixed ? apply_piece_t<float>(c, which, in, out)
                  : apply_piece_t<double>(c, which, in, out);
}
