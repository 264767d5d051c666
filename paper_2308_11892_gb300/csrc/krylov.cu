// Flexible GMRES(m) on the device (paper Section 3: right-preconditioned GMRES,
// 200 iterations, relative tolerance 1e-6), FP64 throughout:
//   per step j:  z_j = M^-1 v_j;  w = A z_j;
//                CGS2: h = V^T w, w -= V h (twice, h accumulated);
//                h_{j+1,j} = ||w||; Givens rotation of the new column; v_{j+1} = w / h_{j+1,j}
//   per cycle:   y = H^-1 g (back substitution), x += Z y, true residual.
// All reductions are deterministic: each block writes a partial and the block
// holding the last ticket combines the partials in block order.
#include <cmath>

#include "common.cuh"
#include "ctx.h"

namespace {

constexpr int kT = 256;
inline int nblk(long long n, int per = kT) { return n > 0 ? ceil_div(n, per) : 1; }

// ------------------------------------------------------------------ BSR SpMV
// Four lanes per block row, lane r computing y_i[r]; each lane streams its
// 32-byte row slice of every 128-byte block (the quad reads whole blocks).
template <class TX>
__global__ void __launch_bounds__(256) k_bsr_spmv(int N, const int32_t* __restrict__ rp,
                                                  const int32_t* __restrict__ ci,
                                                  const double* __restrict__ v,
                                                  const TX* __restrict__ xbase, const int* jptr,
                                                  size_t stride, const double* __restrict__ b,
                                                  double* __restrict__ y, const int* active) {
  if (!*active) return;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i = (int)(g >> 2), r = (int)(g & 3);
  if (i >= N) return;
  const TX* x = xbase + (size_t)(*jptr) * stride;
  int t0 = rp[i], t1 = rp[i + 1];
  const double* a = v + 16 * (size_t)t0 + 4 * r;
  double acc = 0.0;
#pragma unroll 2
  for (int t = t0; t < t1; ++t, a += 16) {
    int j = __ldg(ci + t);
    double2 a01 = __ldg(reinterpret_cast<const double2*>(a));
    double2 a23 = __ldg(reinterpret_cast<const double2*>(a) + 1);
    double xj[4];
    ld4(x + 4 * (size_t)j, xj);
    // one FMA chain: four FP64 operations per block and lane (the FP64 pipe,
    // not HBM, bounds this kernel on GB300)
    acc = fma(a01.x, xj[0], acc);
    acc = fma(a01.y, xj[1], acc);
    acc = fma(a23.x, xj[2], acc);
    acc = fma(a23.y, xj[3], acc);
  }
  size_t o = 4 * (size_t)i + r;
  y[o] = b ? b[o] - acc : acc;
}

// ------------------------------------------------------------------ reductions
struct Range {
  long long lo, hi;
};
__device__ __forceinline__ Range block_range(long long n) {
  long long per = (n + gridDim.x - 1) / gridDim.x;
  per = (per + 1) & ~1ll;
  long long lo = per * blockIdx.x;
  long long hi = lo + per < n ? lo + per : n;
  return {lo < n ? lo : n, hi};
}

// Deterministic block reduction of one value (valid in thread 0).
__device__ double block_sum(double s) {
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
  __syncthreads();
  return t;
}

// Sum of part[0..nb) in a fixed tree order by the whole block (valid in thread 0).
__device__ double block_sum_parts(const double* part, int nb) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[b];
  return block_sum(s);
}

// Combines per-block partials part[l*gridDim.x + b] into out[l] (last block,
// one warp per column, fixed order).
__device__ void combine_columns(const double* part, double* out, int nc) {
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int l = warp; l < nc; l += nw) {
    double s = 0.0;
    for (unsigned b = lane; b < gridDim.x; b += 32) s += part[(size_t)l * gridDim.x + b];
    s = warp_sum(s);
    if (lane == 0) out[l] = s;
  }
}

// CGS2 pass 1: out[l] = V_l . w for l <= j.  Columns are taken eight at a time
// so that every thread keeps eight independent loads in flight.
__global__ void __launch_bounds__(256) k_cgs_dot(long long n, const double* __restrict__ V,
                                                 const double* __restrict__ w, double* part,
                                                 double* out, Ctl* ctl) {
  if (!ctl->active) return;
  __shared__ double red[64 * 8];
  int nc = ctl->j + 1;
  Range R = block_range(n);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int lg = 0; lg < nc; lg += 8) {
    double acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = 0.0;
    for (long long i = R.lo + threadIdx.x; i < R.hi; i += blockDim.x) {
      double wi = w[i];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (lg + u < nc) acc[u] += V[(size_t)(lg + u) * n + i] * wi;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      double s = warp_sum(acc[u]);
      if (lane == 0 && lg + u < nc) red[(lg + u) * 8 + warp] = s;
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < nc; l += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += red[l * 8 + q];
    part[(size_t)l * gridDim.x + blockIdx.x] = s;
  }
  if (last_block_ticket(&ctl->red_ctr[0])) {
    combine_columns(part, out, nc);
    if (threadIdx.x == 0) ctl->red_ctr[0] = 0u;
  }
}

// CGS2 pass 2: w -= V h1, then out[l] = V_l . w, with the dot accumulators
// in registers: every thread only ever uses its own rows of V, so the second
// read of V_l[i] comes from L1, and the block needs no shared-memory tile
// (several blocks per SM).  The update uses all (at most MAXH) columns; the
// dots are formed here for the first MAXC of them (the rest, if any, by
// k_cgs_dot_from on the updated w).
template <int MAXC, int MAXH>
__global__ void __launch_bounds__(256) k_cgs_upd_dot_reg(long long n,
                                                         const double* __restrict__ V,
                                                         double* __restrict__ w,
                                                         const double* __restrict__ h1,
                                                         double* part, double* out, Ctl* ctl) {
  if (!ctl->active) return;
  __shared__ double hs[MAXH];
  __shared__ double red[MAXC * 8];
  const int nh = ctl->j + 1;
  const int nc = nh < MAXC ? nh : MAXC;
  for (int l = threadIdx.x; l < nh; l += blockDim.x) hs[l] = h1[l];
  double acc[MAXC];
#pragma unroll
  for (int l = 0; l < MAXC; ++l) acc[l] = 0.0;
  __syncthreads();
  Range R = block_range(n);
  for (long long i = R.lo + threadIdx.x; i < R.hi; i += blockDim.x) {
    double wi = w[i];
#pragma unroll 8
    for (int l = 0; l < nh; ++l) wi -= hs[l] * V[(size_t)l * n + i];
    w[i] = wi;
#pragma unroll
    for (int l = 0; l < MAXC; ++l)
      if (l < nc) acc[l] += V[(size_t)l * n + i] * wi;
  }
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int l = 0; l < MAXC; ++l) {
    if (l >= nc) break;
    double s = warp_sum(acc[l]);
    if (lane == 0) red[l * 8 + warp] = s;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < nc; l += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[l * 8 + q];
    part[(size_t)l * gridDim.x + blockIdx.x] = s;
  }
  if (last_block_ticket(&ctl->red_ctr[1])) {
    combine_columns(part, out, nc);
    if (threadIdx.x == 0) ctl->red_ctr[1] = 0u;
  }
}

// out[l] = V_l . w for the columns c0 <= l <= j (nothing when j < c0): the
// second-pass dots beyond the register kernel's first MAXC columns, in
// k_cgs_dot's arrangement (eight columns at a time, fixed reduction order).
__global__ void __launch_bounds__(256) k_cgs_dot_from(long long n, const double* __restrict__ V,
                                                      const double* __restrict__ w, int c0,
                                                      double* part, double* out, Ctl* ctl) {
  if (!ctl->active) return;
  const int nc = ctl->j + 1;
  if (nc <= c0) return;
  __shared__ double red[64 * 8];
  Range R = block_range(n);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int lg = c0; lg < nc; lg += 8) {
    double acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = 0.0;
    for (long long i = R.lo + threadIdx.x; i < R.hi; i += blockDim.x) {
      double wi = w[i];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (lg + u < nc) acc[u] += V[(size_t)(lg + u) * n + i] * wi;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      double s = warp_sum(acc[u]);
      if (lane == 0 && lg + u < nc) red[(lg + u - c0) * 8 + warp] = s;
    }
  }
  __syncthreads();
  for (int l = c0 + (int)threadIdx.x; l < nc; l += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += red[(l - c0) * 8 + q];
    part[(size_t)l * gridDim.x + blockIdx.x] = s;
  }
  if (last_block_ticket(&ctl->red_ctr[0])) {
    combine_columns(part + (size_t)c0 * gridDim.x, out + c0, nc - c0);
    if (threadIdx.x == 0) ctl->red_ctr[0] = 0u;
  }
}

// CGS2 pass 3: w -= V h2 and ||w||^2; the last block forms column j of the
// Hessenberg matrix (h1 + h2, ||w||), applies the previous Givens rotations,
// creates the new one and updates g (inputs staged in shared memory first).
__global__ void __launch_bounds__(256) k_cgs_upd_norm(long long n, const double* __restrict__ V,
                                                      double* __restrict__ w,
                                                      const double* __restrict__ h1,
                                                      const double* __restrict__ h2, double* part,
                                                      double* H, double* cs, double* sn,
                                                      double* g, Ctl* ctl, int* hflag) {
  if (!ctl->active) return;
  __shared__ double hs[64], col[66], css[64], sns[64];
  int j = ctl->j, m = ctl->m;
  int nc = j + 1;
  for (int l = threadIdx.x; l < nc; l += blockDim.x) hs[l] = h2[l];
  __syncthreads();
  Range R = block_range(n);
  double s = 0.0;
  for (long long i = R.lo + threadIdx.x; i < R.hi; i += blockDim.x) {
    double wi = w[i];
    for (int l = 0; l < nc; ++l) wi -= hs[l] * V[(size_t)l * n + i];
    w[i] = wi;
    s += wi * wi;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block_ticket(&ctl->red_ctr[2])) return;
  double ss = block_sum_parts(part, gridDim.x);
  for (int l = threadIdx.x; l < nc; l += blockDim.x) {
    col[l] = h1[l] + h2[l];
    css[l] = cs[l];
    sns[l] = sn[l];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  ctl->red_ctr[2] = 0u;
  double hn = sqrt(ss);
  col[j + 1] = hn;
  for (int l = 0; l < j; ++l) {
    double a = col[l], bb = col[l + 1];
    col[l] = css[l] * a + sns[l] * bb;
    col[l + 1] = -sns[l] * a + css[l] * bb;
  }
  double a = col[j], bb = col[j + 1];
  double d = hypot(a, bb);
  double cj = 1.0, sj = 0.0;
  if (d != 0.0) { cj = a / d; sj = bb / d; }
  cs[j] = cj;
  sn[j] = sj;
  col[j] = cj * a + sj * bb;
  col[j + 1] = 0.0;
  double gj = g[j];
  double gn = -sj * gj;
  g[j + 1] = gn;
  g[j] = cj * gj;
  double* Hc = H + (size_t)j * (m + 1);
  for (int l = 0; l <= j + 1; ++l) Hc[l] = col[l];
  ctl->iters += 1;
  ctl->k = j + 1;
  ctl->hn = hn;
  bool conv = fabs(gn) <= ctl->tol_abs;
  bool stop = !isfinite(gn) || !isfinite(hn) || conv || ctl->iters >= ctl->maxit || hn == 0.0 ||
              j + 1 == m;
  if (conv) ctl->conv = 1;
  if (stop) {
    ctl->active = 0;
    *hflag = 0;
    __threadfence_system();
  }
}

// v_{j+1} = w / h_{j+1,j}; the last block advances j.
__global__ void __launch_bounds__(256) k_scale_next(long long n, double* __restrict__ V,
                                                    const double* __restrict__ w, Ctl* ctl) {
  if (!ctl->active) return;
  int j = ctl->j;
  double hn = ctl->hn;
  Range R = block_range(n);
  double* vn = V + (size_t)(j + 1) * n;
  const double rinv = 1.0 / hn;  // one division, then products (FP64 division is slow here)
  for (long long i = R.lo + threadIdx.x; i < R.hi; i += blockDim.x) vn[i] = w[i] * rinv;
  if (last_block_ticket(&ctl->red_ctr[3]) && threadIdx.x == 0) {
    ctl->red_ctr[3] = 0u;
    ctl->j = j + 1;
  }
}

// ||b|| -> bnorm, tol_abs
__global__ void k_rhs_norm(long long n, const double* __restrict__ b, double* part, double tol,
                           Ctl* ctl) {
  Range R = block_range(n);
  double s = 0.0;
  for (long long i = R.lo + threadIdx.x; i < R.hi; i += blockDim.x) s += b[i] * b[i];
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block_ticket(&ctl->red_ctr[4])) return;
  double ss = block_sum_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    ctl->red_ctr[4] = 0u;
    ctl->bnorm = sqrt(ss);
    ctl->tol_abs = tol * ctl->bnorm;
  }
}

// Start of a restart cycle: beta = ||r|| (r already in V_0); decide whether
// to iterate; g = beta e_1.
__global__ void k_cycle_start(long long n, const double* __restrict__ r, double* part, double* g,
                              int m, Ctl* ctl, int* hflag) {
  Range R = block_range(n);
  double s = 0.0;
  for (long long i = R.lo + threadIdx.x; i < R.hi; i += blockDim.x) s += r[i] * r[i];
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block_ticket(&ctl->red_ctr[5])) return;
  double ss = block_sum_parts(part, gridDim.x);
  for (int l = threadIdx.x + 1; l <= m; l += blockDim.x) g[l] = 0.0;
  if (threadIdx.x == 0) {
    ctl->red_ctr[5] = 0u;
    double beta = sqrt(ss);
    ctl->beta = beta;
    ctl->j = 0;
    ctl->k = 0;
    ctl->conv = 0;
    g[0] = beta;
    bool go = isfinite(beta) && beta > ctl->tol_abs && ctl->iters < ctl->maxit;
    ctl->active = go ? 1 : 0;
    *hflag = go ? 1 : 0;
    __threadfence_system();
  }
}

__global__ void k_scale0(long long n, double* __restrict__ V, Ctl* ctl) {
  if (!ctl->active) return;
  double beta = ctl->beta;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) V[i] = V[i] / beta;
}

// y = H(0:k,0:k)^-1 g (upper triangular after the rotations)
__global__ void k_backsolve(const double* H, const double* g, double* y, Ctl* ctl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int k = ctl->k, m = ctl->m;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= H[(size_t)l * (m + 1) + i] * y[l];
    y[i] = s / H[(size_t)i * (m + 1) + i];
  }
}

// x += Z y
template <class TZ>
__global__ void k_xupdate(long long n, double* __restrict__ x, const TZ* __restrict__ Z,
                          const double* __restrict__ y, const Ctl* ctl) {
  __shared__ double ys[64];
  int k = ctl->k;
  for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = y[l];
  __syncthreads();
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double xi = x[i];
  for (int l = 0; l < k; ++l) xi += ys[l] * (double)Z[(size_t)l * n + i];
  x[i] = xi;
}

template <class TX>
void spmv_t(cptr_ctx* c, const TX* xbase, const int* jptr, size_t stride, double* y,
            const double* b, const int* active) {
  KL(c, k_bsr_spmv<TX><<<nblk(4ll * c->N), kT, 0, c->stream>>>(c->N, c->rp, c->ci, c->v, xbase, jptr,
                                                         stride, b, y, active));
}

void launch_step(cptr_ctx* c) {
  long long n = 4ll * c->N;
  size_t stride = (size_t)n;
  cudaStream_t s = c->stream;
  Ctl* ctl = c->ctl;
  launch_precond(c, c->V, c->Z, &ctl->j, &ctl->active);
  if (c->mixed)
    spmv_t<float>(c, (const float*)c->Z, &ctl->j, stride, c->w, nullptr, &ctl->active);
  else
    spmv_t<double>(c, (const double*)c->Z, &ctl->j, stride, c->w, nullptr, &ctl->active);
  KL(c, k_cgs_dot<<<c->NBd, kT, 0, s>>>(n, c->V, c->w, c->part, c->h1, ctl));
  if (c->p.restart + 1 <= 32) {
    KL(c, k_cgs_upd_dot_reg<32, 32><<<c->NB, kT, 0, s>>>(n, c->V, c->w, c->h1, c->part,
                                                                 c->h2, ctl));
  } else {  // restart <= 63: the update and the first 32 dots, then the other dots
    KL(c, k_cgs_upd_dot_reg<32, 64><<<c->NB, kT, 0, s>>>(n, c->V, c->w, c->h1, c->part,
                                                                 c->h2, ctl));
    KL(c, k_cgs_dot_from<<<c->NBd, kT, 0, s>>>(n, c->V, c->w, 32, c->part, c->h2, ctl));
  }
  KL(c, k_cgs_upd_norm<<<c->NBd, kT, 0, s>>>(n, c->V, c->w, c->h1, c->h2, c->part, c->H, c->cs,
                                            c->sn, c->g, ctl, c->hflag_dev));
  KL(c, k_scale_next<<<c->NB, kT, 0, s>>>(n, c->V, c->w, ctl));
}

}  // namespace

namespace {
__global__ void k_set_step(Ctl* ctl, int j) {
  ctl->j = j;
  ctl->active = 1;
}
}  // namespace

cptr_status profile_krylov_kernel(cptr_ctx* c, int kernel, bool prepare) {
  long long n = 4ll * c->N;
  switch (kernel) {
    case CPTR_KERNEL_SPMV:
      if (!prepare) spmv_t<double>(c, c->xd, &c->ctl->zero, 0, c->w, nullptr, &c->ctl->one);
      break;
    case CPTR_KERNEL_MDOT:
      if (prepare)
        KL(c, k_set_step<<<1, 1, 0, c->stream>>>(c->ctl, mdot_profile_column(c->info, c->p.restart)));
      else KL(c, k_cgs_dot<<<c->NBd, kT, 0, c->stream>>>(n, c->V, c->w, c->part, c->h1, c->ctl));
      break;
    default:
      return CPTR_ERR_INVALID;
  }
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

void launch_spmv(cptr_ctx* c, const void* x, bool x_f32, double* y, const double* b) {
  if (x_f32) spmv_t<float>(c, (const float*)x, &c->ctl->zero, 0, y, b, &c->ctl->one);
  else spmv_t<double>(c, (const double*)x, &c->ctl->zero, 0, y, b, &c->ctl->one);
}

cptr_status krylov_alloc(cptr_ctx* c) {
  if (c->V) return CPTR_OK;
  int m = c->p.restart;
  long long n = 4ll * c->N;
  size_t zb = c->mixed ? sizeof(float) : sizeof(double);
  // one block per 1024 rows at most, and no more blocks than the
  // register-accumulator CGS pass keeps resident (a single wave)
  int occ = 8;
  {
    int b = 0;
    cudaError_t e = m + 1 <= 32
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cgs_upd_dot_reg<32, 32>, kT, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cgs_upd_dot_reg<32, 64>, kT, 0);
    if (e == cudaSuccess && b > 0) occ = b;
    cudaGetLastError();
  }
  c->NB = (int)std::min<long long>(std::max<long long>(1, (n + 1023) / 1024),
                                   (long long)occ * c->nsm);
  // the dot and norm passes hold far fewer registers than the register-
  // accumulator pass: one wave of their own keeps more loads in flight
  int occd = occ;
  {
    const void* light[3] = {(const void*)k_cgs_dot, (const void*)k_cgs_dot_from,
                            (const void*)k_cgs_upd_norm};
    int lo = 1 << 30;
    for (const void* f : light) {
      int b = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kT, 0) == cudaSuccess && b > 0)
        lo = std::min(lo, b);
    }
    cudaGetLastError();
    if (lo < (1 << 30)) occd = std::max(occ, lo);
  }
  c->NBd = (int)std::min<long long>(std::max<long long>(1, (n + 1023) / 1024),
                                    (long long)occd * c->nsm);
  CTX_ALLOC(c, c->V, double, (size_t)(m + 1) * n, false);
  c->Z = ctx_alloc(c, zb * (size_t)m * n + 16, false);
  if (!c->Z) return CPTR_ERR_NOMEM;
  CTX_ALLOC(c, c->w, double, n, false);
  CTX_ALLOC(c, c->xd, double, n, false);
  CTX_ALLOC(c, c->bd, double, n, false);
  CTX_ALLOC(c, c->H, double, (size_t)(m + 1) * (m + 1), false);
  CTX_ALLOC(c, c->cs, double, m + 1, false);
  CTX_ALLOC(c, c->sn, double, m + 1, false);
  CTX_ALLOC(c, c->g, double, m + 2, false);
  CTX_ALLOC(c, c->yv, double, m + 1, false);
  CTX_ALLOC(c, c->h1, double, m + 2, false);
  CTX_ALLOC(c, c->h2, double, m + 2, false);
  CTX_ALLOC(c, c->part, double, (size_t)(m + 2) * std::max(c->NB, c->NBd), false);
  CTX_CUDA(c, cudaMemsetAsync(c->H, 0, sizeof(double) * (m + 1) * (m + 1), c->stream));
  return CPTR_OK;
}

void krylov_release_graph(cptr_ctx* c) {
  if (c->step_exec) {
    cudaGraphExecDestroy(c->step_exec);
    c->step_exec = nullptr;
  }
}

static cptr_status ensure_graph(cptr_ctx* c) {
  if (c->step_exec || !c->p.use_graphs) return CPTR_OK;
  cudaGraph_t graph = nullptr;
  long long before = c->nlaunch;
  CTX_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  launch_step(c);
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  c->step_kernels = c->nlaunch - before;  // capturing launches nothing; replays do
  c->nlaunch = before;
  if (e != cudaSuccess || !graph) {
    cudaGetLastError();
    c->p.use_graphs = 0;  // fall back to direct launches of the same kernels
    return CPTR_OK;
  }
  e = cudaGraphInstantiate(&c->step_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->step_exec = nullptr;
    c->p.use_graphs = 0;
  }
  return CPTR_OK;
}

cptr_status krylov_solve(cptr_ctx* c, double tol, int maxit) {
  long long n = 4ll * c->N;
  int m = c->p.restart;
  cudaStream_t s = c->stream;
  Ctl h{};
  h.m = m;
  h.maxit = maxit;
  h.one = 1;
  h.spin = c->spin_limit;
  CTX_CUDA(c, cudaMemcpyAsync(c->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  cptr_status st = ensure_graph(c);
  if (st) return st;
  KL(c, k_rhs_norm<<<c->NB, kT, 0, s>>>(n, c->bd, c->part, tol, c->ctl));
  cudaEvent_t ev[2];
  CTX_CUDA(c, cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
  CTX_CUDA(c, cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
  cptr_status result = CPTR_OK;
  for (int cycle = 0;; ++cycle) {
    // r = b - A x into V_0, beta, decision, v_0 = r / beta
    spmv_t<double>(c, c->xd, &c->ctl->zero, 0, c->V, c->bd, &c->ctl->one);
    KL(c, k_cycle_start<<<c->NB, kT, 0, s>>>(n, c->V, c->part, c->g, m, c->ctl, c->hflag_dev));
    KL(c, k_scale0<<<nblk(n), kT, 0, s>>>(n, c->V, c->ctl));
    CTX_CUDA(c, cudaMemcpyAsync(&h, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CTX_CUDA(c, cudaStreamSynchronize(s));
    if (h.status != DEV_OK) { result = h.status == DEV_TIMEOUT ? CPTR_ERR_TIMEOUT : CPTR_ERR_BREAKDOWN; break; }
    if (!std::isfinite(h.beta)) { result = CPTR_ERR_BREAKDOWN; ctx_set_err(c, "non-finite residual"); break; }
    if (h.bnorm == 0.0) {
      CTX_CUDA(c, cudaMemsetAsync(c->xd, 0, sizeof(double) * n, s));
      h.beta = 0.0;
      result = CPTR_OK;
      break;
    }
    if (!h.active) {
      result = (h.beta <= h.tol_abs) ? CPTR_OK : CPTR_ERR_MAXIT;
      break;
    }
    for (int j = 0; j < m; ++j) {
      if (c->step_exec) {
        CTX_CUDA(c, cudaGraphLaunch(c->step_exec, s));
        c->nlaunch += c->step_kernels;
      } else {
        launch_step(c);
      }
      CTX_CUDA(c, cudaEventRecord(ev[j & 1], s));
      if (j >= 1) {
        CTX_CUDA(c, cudaEventSynchronize(ev[(j - 1) & 1]));
        if (*c->hflag == 0) break;
      }
    }
    KL(c, k_backsolve<<<1, 32, 0, s>>>(c->H, c->g, c->yv, c->ctl));
    if (c->mixed)
      KL(c, k_xupdate<float><<<nblk(n), kT, 0, s>>>(n, c->xd, (const float*)c->Z, c->yv, c->ctl));
    else
      KL(c, k_xupdate<double><<<nblk(n), kT, 0, s>>>(n, c->xd, (const double*)c->Z, c->yv, c->ctl));
    CTX_CUDA(c, cudaGetLastError());
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  c->info.iters = h.iters;
  c->info.rel_resid = h.bnorm > 0.0 ? h.beta / h.bnorm : 0.0;
  return result;
}
