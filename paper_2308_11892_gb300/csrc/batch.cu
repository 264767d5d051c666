// Batched solves of many small systems in one launch.
//
// A small system (thousands of cells) leaves most of the GPU idle in the
// per-system path, whose Krylov loop launches a few dozen kernels per
// iteration and reads a host flag at every restart.  Here one thread block
// runs the whole flexible GMRES(m) loop of one system on the device, with the
// Eq. 3 preconditioner (Quasi-IMPES restriction, the system-AMG V-cycle, the
// correction, the ILU(0) solves level by level, the combination), the outer
// block SpMV, CGS2 with Givens rotations, the back substitution, restarts and
// the true residual, separated by block barriers only; a grid of such blocks
// advances every system of the batch at once.  Each system reads its own
// context's hierarchy, factors and work vectors (built by cptr_setup), and
// every sum has a fixed order that does not depend on the batch: a system's
// result is the same alone and in any batch.
#include <algorithm>
#include <chrono>
#include <string>
#include <cmath>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "ctx.h"

namespace {

constexpr int kBT = 512;        // threads per system
constexpr int kBMaxLev = 25;    // AMG levels
constexpr int kBMaxM = 32;      // restart length

struct BLevel {
  int n;
  const int32_t *Arp, *Aci;
  const void* Av;    // apply precision
  const void* dinv;  // apply precision
  int nc;            // rows of the next level (R: nc x n, P: n x nc)
  const int32_t *Rrp, *Rci;
  const void* Rv;
  const int32_t *Prp, *Pci;
  const void* Pv;
  void *b, *x, *r, *x2, *t;
};

struct alignas(16) BSys {
  int N, m, maxit, nlev, ne, e0, e1, h0, h1, h2, nu_pre, nu_post, nlf, nlb, first;
  double tol;
  const int32_t *rp, *ci;
  const double* v;    // the FP64 operator
  const void* Wt;     // decoupling weights (apply precision)
  const void* AE;     // elliptic columns of A (apply precision)
  const double* Cinv; // dense inverse of the coarsest operator
  void *rhat, *zc, *r2, *u, *y2;
  const int32_t *offf, *ordf, *Lrp, *Lci;
  const void* Lv;
  const int32_t *offb, *ordb, *Urp, *Uci;
  const void *Uv, *Dinv;
  double *V, *w, *x, *b;
  void* Z;
  BLevel lev[kBMaxLev];
};

struct BOut {
  int iters, status;
  double rel_resid;
};

// Sum of v over the block in a fixed order (warps, then warp sums in order);
// every thread returns the total.
__device__ double bsum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();  // red is free (a previous call may still be reading it)
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
  return t;
}

// The row loops below load four entries before summing their products (in
// entry order, the same sums as an entry-by-entry loop).  One SM carries a
// whole system here, so the FP64 parts (the outer SpMV, CGS2, norms) run at
// that SM's FP64 rate, which bounds them; the FP32 preconditioner waits on
// block barriers and memory latency.

// y = A x (4x4 blocks, FP64 accumulation in block order), y = b - A x when b
template <class TX>
__device__ void bspmv(const BSys& S, const TX* __restrict__ x, const double* __restrict__ b,
                      double* __restrict__ y) {
  const int n4 = 4 * S.N;
  const int32_t* __restrict__ rp = S.rp;
  const int32_t* __restrict__ ci = S.ci;
  const double* __restrict__ v = S.v;
  for (int g = threadIdx.x; g < n4; g += blockDim.x) {
    const int i = g >> 2, r = g & 3;
    double acc = 0.0;
    int t = rp[i];
    const int t1 = rp[i + 1];
    for (; t + 4 <= t1; t += 4) {
      int j[4];
      double a[4][4], xv[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) j[u] = ci[t + u];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a[u][q] = v[16 * (size_t)(t + u) + 4 * r + q];
          xv[u][q] = (double)x[4 * (size_t)j[u] + q];
        }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc = fma(a[u][q], xv[u][q], acc);
    }
    for (; t < t1; ++t) {
      const double* a = v + 16 * (size_t)t + 4 * r;
      const TX* xj = x + 4 * (size_t)ci[t];
      acc = fma(a[0], (double)xj[0], acc);
      acc = fma(a[1], (double)xj[1], acc);
      acc = fma(a[2], (double)xj[2], acc);
      acc = fma(a[3], (double)xj[3], acc);
    }
    y[g] = b ? b[g] - acc : acc;
  }
}

// sum over row i of a CSR operator of val * x, in entry order
template <class T>
__device__ __forceinline__ T row_sum(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const T* __restrict__ val, const T* __restrict__ x, int i) {
  T s = 0;
  int t = rp[i];
  const int t1 = rp[i + 1];
  for (; t + 4 <= t1; t += 4) {
    int j[4];
    T a[4], xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      j[u] = ci[t + u];
      a[u] = val[t + u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = x[j[u]];
#pragma unroll
    for (int u = 0; u < 4; ++u) s += a[u] * xv[u];
  }
  for (; t < t1; ++t) s += val[t] * x[ci[t]];
  return s;
}

// r = b - A x on one AMG level (scalar CSR, apply precision)
template <class T>
__device__ void lresid(const BLevel& L, const T* __restrict__ b, const T* __restrict__ x,
                       T* __restrict__ r) {
  const int32_t* __restrict__ rp = L.Arp;
  const int32_t* __restrict__ ci = L.Aci;
  const T* __restrict__ av = (const T*)L.Av;
  const int n = L.n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) r[i] = b[i] - row_sum<T>(rp, ci, av, x, i);
}

// xout = xin + D_l1^-1 (b - A xin): one l1-Jacobi sweep
template <class T>
__device__ void lsweep(const BLevel& L, const T* __restrict__ b, const T* __restrict__ xin,
                       T* __restrict__ xout) {
  const int32_t* __restrict__ rp = L.Arp;
  const int32_t* __restrict__ ci = L.Aci;
  const T* __restrict__ av = (const T*)L.Av;
  const T* __restrict__ dv = (const T*)L.dinv;
  const int n = L.n;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    xout[i] = xin[i] + dv[i] * (b[i] - row_sum<T>(rp, ci, av, xin, i));
}

}  // namespace

namespace {

// One V(nu_pre, nu_post) cycle with l1-Jacobi from a zero guess on the
// system's hierarchy: b0 (level 0 right-hand side) -> zc.
template <class T>
__device__ void bvcycle(const BSys& S, const T* b0) {
  const int last = S.nlev - 1;
  for (int l = 0; l < last; ++l) {
    const BLevel& L = S.lev[l];
    const T* b = l == 0 ? b0 : (const T*)L.b;
    T* x = (T*)L.x;
    T* t = (T*)L.t;
    if (S.nu_pre == 0) {
      for (int i = threadIdx.x; i < L.n; i += blockDim.x) x[i] = 0;
    } else {
      // first sweep from zero: x = D^-1 b; the others alternate so the last writes x
      T* dst = ((S.nu_pre - 1) % 2 == 0) ? x : t;
      const T* dv = (const T*)L.dinv;
      for (int i = threadIdx.x; i < L.n; i += blockDim.x) dst[i] = dv[i] * b[i];
      const T* src = dst;
      for (int k = 1; k < S.nu_pre; ++k) {
        __syncthreads();
        T* d2 = ((S.nu_pre - 1 - k) % 2 == 0) ? x : t;
        lsweep<T>(L, b, src, d2);
        src = d2;
      }
    }
    __syncthreads();
    lresid<T>(L, b, x, (T*)L.r);
    __syncthreads();
    // b_{l+1} = R r
    const T* rv = (const T*)L.Rv;
    const T* r = (const T*)L.r;
    T* bn = (T*)S.lev[l + 1].b;
    for (int i = threadIdx.x; i < L.nc; i += blockDim.x) bn[i] = row_sum<T>(L.Rrp, L.Rci, rv, r, i);
    __syncthreads();
  }
  {
    // coarsest level: x = Cinv b in FP64
    const BLevel& Lc = S.lev[last];
    const T* b = last == 0 ? b0 : (const T*)Lc.b;
    T* xo = last == 0 ? (T*)S.zc : (T*)Lc.x;
    const int n = Lc.n;
    const double* __restrict__ Cinv = S.Cinv;
    const int lane = threadIdx.x & 31;
    // one warp per row, lanes over the columns, then a fixed shuffle tree
    for (int i = threadIdx.x >> 5; i < n; i += blockDim.x >> 5) {
      double s = 0.0;
      for (int q = lane; q < n; q += 32) s += Cinv[(size_t)i * n + q] * (double)b[q];
      s = warp_sum(s);
      if (lane == 0) xo[i] = (T)s;
    }
    __syncthreads();
  }
  for (int l = last - 1; l >= 0; --l) {
    const BLevel& L = S.lev[l];
    const T* b = l == 0 ? b0 : (const T*)L.b;
    const T* xc = (l + 1 == last) ? (const T*)S.lev[l + 1].x : (const T*)S.lev[l + 1].x2;
    T* x = (T*)L.x;
    T* t = (T*)L.t;
    T* out = l == 0 ? (T*)S.zc : (T*)L.x2;
    const T* pv = (const T*)L.Pv;
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) x[i] += row_sum<T>(L.Prp, L.Pci, pv, xc, i);
    __syncthreads();
    if (S.nu_post == 0) {
      for (int i = threadIdx.x; i < L.n; i += blockDim.x) out[i] = x[i];
    } else {
      const T* src = x;
      for (int k = 0; k < S.nu_post; ++k) {
        T* dst = (k == S.nu_post - 1) ? out : (src == x ? t : x);
        lsweep<T>(L, b, src, dst);
        __syncthreads();
        src = dst;
      }
    }
    __syncthreads();
  }
}

// z = M^-1 v (Eq. 3) for the FP64 vector v; z in the apply precision.
template <class T>
__device__ void bprecond(const BSys& S, const double* v, T* z) {
  const int N = S.N;
  T* rhat = (T*)S.rhat;
  T* zc = (T*)S.zc;
  T* r2 = (T*)S.r2;
  T* u = (T*)S.u;
  T* y2 = (T*)S.y2;
  if (S.first) {
    // Quasi-IMPES restriction: rhat_i = v_i[e] - W_i v_i[h]
    const T* W = (const T*)S.Wt;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const double* rv = v + 4 * (size_t)i;
      const T* w = W + 4 * (size_t)i;
      if (S.ne == 2) {
        T re0 = (T)rv[S.e0], re1 = (T)rv[S.e1], rh0 = (T)rv[S.h0], rh1 = (T)rv[S.h1];
        rhat[2 * (size_t)i] = re0 - w[0] * rh0 - w[1] * rh1;
        rhat[2 * (size_t)i + 1] = re1 - w[2] * rh0 - w[3] * rh1;
      } else {
        rhat[i] = (T)rv[S.e0] - w[0] * (T)rv[S.h0] - w[1] * (T)rv[S.h1] - w[2] * (T)rv[S.h2];
      }
    }
    __syncthreads();
    bvcycle<T>(S, rhat);
    // correction: r2 = v - A P zc (elliptic columns of A only)
    const T* __restrict__ ae = (const T*)S.AE;
    const int32_t* __restrict__ rp = S.rp;
    const int32_t* __restrict__ ci = S.ci;
    const int ne = S.ne;
    for (int g = threadIdx.x; g < 4 * N; g += blockDim.x) {
      const int i = g >> 2, r = g & 3;
      T acc = 0;
      int t = rp[i];
      const int t1 = rp[i + 1];
      for (; t + 4 <= t1; t += 4) {
        int j[4];
        T a0[4], a1[4], z0[4], z1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          j[u] = ci[t + u];
          a0[u] = ae[8 * (size_t)(t + u) + 2 * r];
          a1[u] = ae[8 * (size_t)(t + u) + 2 * r + 1];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          z0[u] = ne == 2 ? zc[2 * (size_t)j[u]] : zc[j[u]];
          z1[u] = ne == 2 ? zc[2 * (size_t)j[u] + 1] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (ne == 2) acc += a0[u] * z0[u] + a1[u] * z1[u];
          else acc += a0[u] * z0[u];
        }
      }
      for (; t < t1; ++t) {
        const int jj = ci[t];
        const T* a = ae + 8 * (size_t)t + 2 * r;
        if (ne == 2) acc += a[0] * zc[2 * (size_t)jj] + a[1] * zc[2 * (size_t)jj + 1];
        else acc += a[0] * zc[jj];
      }
      r2[g] = (T)v[g] - acc;
    }
  } else {
    for (int g = threadIdx.x; g < 4 * N; g += blockDim.x) r2[g] = (T)v[g];
  }
  __syncthreads();
  // ILU(0): forward, one level after the other (the library's rounding sequence)
  const int r = threadIdx.x & 3, quad = threadIdx.x >> 2, nquad = blockDim.x >> 2;
  const T* Lv = (const T*)S.Lv;
  for (int lv = 0; lv < S.nlf; ++lv) {
    for (int p = S.offf[lv] + quad; p < S.offf[lv + 1]; p += nquad) {
      const int i = S.ordf[p];
      if (i < 0) continue;
      T acc = r2[4 * (size_t)i + r];
      for (int k = S.Lrp[p]; k < S.Lrp[p + 1]; ++k) {
        T l[4], uj[4];
        const T* lp = Lv + 16 * (size_t)k + 4 * r;
        const T* up = u + 4 * (size_t)S.Lci[k];
        l[0] = lp[0]; l[1] = lp[1]; l[2] = lp[2]; l[3] = lp[3];
        uj[0] = up[0]; uj[1] = up[1]; uj[2] = up[2]; uj[3] = up[3];
        acc = sub_rn(acc, dot4(l, uj));
      }
      u[4 * (size_t)i + r] = acc;
    }
    __syncthreads();
  }
  // backward with inv(U_ii), then z = P zc + y2
  const T* Uv = (const T*)S.Uv;
  const T* Dv = (const T*)S.Dinv;
  const unsigned qmask = 0xFu << ((threadIdx.x & 31) & ~3);
  const int q0 = (threadIdx.x & 31) & ~3;
  for (int lv = 0; lv < S.nlb; ++lv) {
    const int pe = S.offb[lv + 1];
    // uniform rounds: the quads of a warp shuffle together
    for (int pb = S.offb[lv]; pb < pe; pb += nquad) {
      const int p = pb + quad;
      const int i = p < pe ? S.ordb[p] : -1;
      T acc = 0, d[4] = {0, 0, 0, 0}, y1 = 0;
      if (i >= 0) {
        // inv(U_ii) and the first-stage part before the row's sums
        const T* dp = Dv + 16 * (size_t)p + 4 * r;
        d[0] = dp[0]; d[1] = dp[1]; d[2] = dp[2]; d[3] = dp[3];
        if (S.first) {
          if (r == S.e0) y1 = zc[S.ne * (size_t)i];
          else if (S.ne == 2 && r == S.e1) y1 = zc[2 * (size_t)i + 1];
        }
        acc = u[4 * (size_t)i + r];
        for (int k = S.Urp[p]; k < S.Urp[p + 1]; ++k) {
          T a[4], yj[4];
          const T* ap = Uv + 16 * (size_t)k + 4 * r;
          const T* yp = y2 + 4 * (size_t)S.Uci[k];
          a[0] = ap[0]; a[1] = ap[1]; a[2] = ap[2]; a[3] = ap[3];
          yj[0] = yp[0]; yj[1] = yp[1]; yj[2] = yp[2]; yj[3] = yp[3];
          acc = sub_rn(acc, dot4(a, yj));
        }
      }
      T s4[4];
      s4[0] = __shfl_sync(qmask, acc, q0 + 0);
      s4[1] = __shfl_sync(qmask, acc, q0 + 1);
      s4[2] = __shfl_sync(qmask, acc, q0 + 2);
      s4[3] = __shfl_sync(qmask, acc, q0 + 3);
      if (i >= 0) {
        const T y = dot4(d, s4);
        y2[4 * (size_t)i + r] = y;
        z[4 * (size_t)i + r] = y1 + y;
      }
    }
    __syncthreads();
  }
}

}  // namespace

namespace {

// Flexible GMRES(m) with CGS2 and Givens rotations for system blockIdx.x,
// the same algorithm (and stopping rules) as the per-system driver:
// convergence when ||b - A x|| <= tol ||b||, iterations = preconditioner
// applications, a cycle ends at m steps, on convergence of the estimate, at
// maxit or on an exact breakdown, and the true residual decides whether to
// start another.
template <class T>
__global__ void __launch_bounds__(kBT, 1) k_batch_fgmres(const BSys* __restrict__ sys,
                                                      BOut* __restrict__ out) {
  // the system's descriptor in shared memory: its pointers are then read
  // without a global load, and stores to global memory cannot alias them
  __shared__ BSys S;
  {
    const int4* src = reinterpret_cast<const int4*>(sys + blockIdx.x);
    int4* dst = reinterpret_cast<int4*>(&S);
    for (int k = threadIdx.x; k < (int)(sizeof(BSys) / 16); k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  __shared__ double red[kBT / 32];
  __shared__ double sH[(kBMaxM + 1) * kBMaxM];  // column j at j*(m+1), rotated
  __shared__ double scs[kBMaxM], ssn[kBMaxM], sg[kBMaxM + 1], sy[kBMaxM], sh1[kBMaxM + 1],
      sh2[kBMaxM + 1];
  __shared__ int s_stop;
  const int n4 = 4 * S.N, m = S.m;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  T* Z = (T*)S.Z;
  // ||b||
  double s = 0.0;
  for (int i = tid; i < n4; i += blockDim.x) s += S.b[i] * S.b[i];
  const double bnorm = sqrt(bsum(s, red));
  const double tol_abs = S.tol * bnorm;
  int iters = 0, status = CPTR_OK;
  double beta = 0.0;
  if (bnorm == 0.0) {
    for (int i = tid; i < n4; i += blockDim.x) S.x[i] = 0.0;
  } else {
    for (;;) {
      // r = b - A x into V_0, beta = ||r||
      bspmv<double>(S, S.x, S.b, S.V);
      __syncthreads();
      s = 0.0;
      for (int i = tid; i < n4; i += blockDim.x) s += S.V[i] * S.V[i];
      beta = sqrt(bsum(s, red));
      if (!isfinite(beta)) { status = CPTR_ERR_BREAKDOWN; break; }
      if (beta <= tol_abs) break;
      if (iters >= S.maxit) { status = CPTR_ERR_MAXIT; break; }
      for (int i = tid; i < n4; i += blockDim.x) S.V[i] = S.V[i] / beta;
      if (tid == 0) {
        sg[0] = beta;
        for (int l = 1; l <= m; ++l) sg[l] = 0.0;
      }
      __syncthreads();
      int k = 0;
      for (int j = 0; j < m; ++j) {
        const double* vj = S.V + (size_t)j * n4;
        T* zj = Z + (size_t)j * n4;
        bprecond<T>(S, vj, zj);
        bspmv<T>(S, zj, nullptr, S.w);
        __syncthreads();
        // CGS2: h1 = V^T w; w -= V h1; h2 = V^T w; w -= V h2 (one warp per
        // column: the FP64 pipe, not the number of warps, bounds these dots)
        for (int pass = 0; pass < 2; ++pass) {
          double* hh = pass == 0 ? sh1 : sh2;
          const double* __restrict__ wv = S.w;
          for (int l = warp; l <= j; l += nw) {
            const double* __restrict__ vl = S.V + (size_t)l * n4;
            double d = 0.0;
            for (int i = lane; i < n4; i += 32) d += vl[i] * wv[i];
            d = warp_sum(d);
            if (lane == 0) hh[l] = d;
          }
          __syncthreads();
          for (int i = tid; i < n4; i += blockDim.x) {
            double wi = S.w[i];
            for (int l = 0; l <= j; ++l) wi -= hh[l] * S.V[(size_t)l * n4 + i];
            S.w[i] = wi;
          }
          __syncthreads();
        }
        s = 0.0;
        for (int i = tid; i < n4; i += blockDim.x) s += S.w[i] * S.w[i];
        const double hn = sqrt(bsum(s, red));
        if (tid == 0) {
          double* col = sH + (size_t)j * (m + 1);
          for (int l = 0; l <= j; ++l) col[l] = sh1[l] + sh2[l];
          col[j + 1] = hn;
          for (int l = 0; l < j; ++l) {
            const double a = col[l], b = col[l + 1];
            col[l] = scs[l] * a + ssn[l] * b;
            col[l + 1] = -ssn[l] * a + scs[l] * b;
          }
          const double a = col[j], b = col[j + 1];
          const double dd = hypot(a, b);
          double cj = 1.0, sj = 0.0;
          if (dd != 0.0) { cj = a / dd; sj = b / dd; }
          scs[j] = cj;
          ssn[j] = sj;
          col[j] = cj * a + sj * b;
          col[j + 1] = 0.0;
          const double gj = sg[j];
          const double gn = -sj * gj;
          sg[j + 1] = gn;
          sg[j] = cj * gj;
          const bool conv = fabs(gn) <= tol_abs;
          s_stop = (!isfinite(gn) || !isfinite(hn) || conv || iters + 1 >= S.maxit ||
                    hn == 0.0 || j + 1 == m) ? 1 : 0;
        }
        __syncthreads();
        ++iters;
        k = j + 1;
        if (s_stop) break;
        const double rinv = 1.0 / hn;
        double* vn = S.V + (size_t)(j + 1) * n4;
        for (int i = tid; i < n4; i += blockDim.x) vn[i] = S.w[i] * rinv;
        __syncthreads();
      }
      // y = H^-1 g, x += Z y
      if (tid == 0) {
        for (int i = k - 1; i >= 0; --i) {
          double t = sg[i];
          for (int l = i + 1; l < k; ++l) t -= sH[(size_t)l * (m + 1) + i] * sy[l];
          sy[i] = t / sH[(size_t)i * (m + 1) + i];
        }
      }
      __syncthreads();
      for (int i = tid; i < n4; i += blockDim.x) {
        double xi = S.x[i];
        for (int l = 0; l < k; ++l) xi += sy[l] * (double)Z[(size_t)l * n4 + i];
        S.x[i] = xi;
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    out[blockIdx.x].iters = iters;
    out[blockIdx.x].status = status;
    out[blockIdx.x].rel_resid = bnorm > 0.0 ? beta / bnorm : 0.0;
  }
}

}  // namespace

namespace {

int hidx_of(int e0, int e1, int k) {
  int h[3] = {-1, -1, -1}, q = 0;
  for (int u = 0; u < 4; ++u)
    if (u != e0 && u != e1) h[q++] = u;
  return h[k];
}

// Descriptor of one set-up context; CPTR_ERR_INVALID for configurations the
// batched kernel does not run (see cptr.h).
cptr_status describe(cptr_ctx* c, double tol, int maxit, BSys* d, std::string& why) {
  if (!c->setup_done) { why = "context not set up"; return CPTR_ERR_INVALID; }
  const int pc = c->p.precond;
  if (pc != CPTR_PREC_CPTR && pc != CPTR_PREC_ILU) { why = "batched solves run CPTR, CPR or ILU(0) alone"; return CPTR_ERR_INVALID; }
  if (c->p.mgr) { why = "batched solves do not run the MGR reduction"; return CPTR_ERR_INVALID; }
  if (c->p.smoother != CPTR_SMOOTH_L1_JACOBI) { why = "batched solves smooth with l1-Jacobi"; return CPTR_ERR_INVALID; }
  if (c->p.restart > kBMaxM) { why = "batched solves need restart <= 32"; return CPTR_ERR_INVALID; }
  if ((int)c->lev.size() > kBMaxLev) { why = "too many AMG levels"; return CPTR_ERR_INVALID; }
  if (!c->Lrp || !c->Urp || !c->Dinv) {
    // the level-ordered factor arrays (built when the tuner picked another schedule)
    cptr_status st = build_level_solve_arrays(c);
    if (st) return st;
    CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  *d = BSys();
  d->N = c->N;
  d->m = c->p.restart;
  d->maxit = maxit > 0 ? maxit : c->p.maxit;
  d->tol = tol > 0.0 ? tol : c->p.tol;
  d->first = pc == CPTR_PREC_CPTR ? 1 : 0;
  d->ne = c->se1 < 0 ? 1 : 2;
  d->e0 = c->se0;
  d->e1 = c->se1;
  d->h0 = hidx_of(c->se0, c->se1, 0);
  d->h1 = hidx_of(c->se0, c->se1, 1);
  d->h2 = hidx_of(c->se0, c->se1, 2);
  d->nu_pre = c->p.nu_pre;
  d->nu_post = c->p.nu_post;
  d->rp = c->rp; d->ci = c->ci; d->v = c->v;
  d->Wt = c->Wt; d->AE = c->AE; d->Cinv = c->Cinv;
  d->rhat = c->rhat; d->zc = c->zc; d->r2 = c->r2; d->u = c->u; d->y2 = c->y2;
  d->nlf = c->nlev_f; d->nlb = c->nlev_b;
  d->offf = c->loff_f; d->ordf = c->ord_f; d->Lrp = c->Lrp; d->Lci = c->Lci; d->Lv = c->Lv;
  d->offb = c->loff_b; d->ordb = c->ord_b; d->Urp = c->Urp; d->Uci = c->Uci; d->Uv = c->Uv;
  d->Dinv = c->Dinv;
  d->V = c->V; d->w = c->w; d->x = c->xd; d->b = c->bd; d->Z = c->Z;
  d->nlev = (int)c->lev.size();
  for (int l = 0; l < d->nlev; ++l) {
    const Level& L = c->lev[l];
    BLevel& B = d->lev[l];
    B.n = L.A.n;
    B.Arp = L.A.rp; B.Aci = L.A.ci; B.Av = L.Av; B.dinv = L.dinv;
    const bool last = l == d->nlev - 1;
    B.nc = last ? 0 : L.nc;
    B.Rrp = L.R.rp; B.Rci = L.R.ci; B.Rv = L.Rv;
    B.Prp = L.P.rp; B.Pci = L.P.ci; B.Pv = L.Pv;
    B.b = L.b; B.x = L.x; B.r = L.r; B.x2 = L.x2; B.t = L.t;
  }
  return CPTR_OK;
}

}  // namespace

extern "C" cptr_status cptr_solve_batch(cptr_ctx* const* ctxs, int n, const double* const* rhs,
                                        double* const* x, double tol, int maxit,
                                        cptr_info* infos) {
  if (!ctxs || n <= 0 || !rhs || !x) return CPTR_ERR_INVALID;
  cptr_ctx* c0 = ctxs[0];
  if (!c0) return CPTR_ERR_INVALID;
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k] || !rhs[k] || !x[k]) return CPTR_ERR_INVALID;
    if (ctxs[k]->dev != c0->dev || ctxs[k]->mixed != c0->mixed) {
      ctx_set_err(c0, "a batch needs one device and one precision");
      return CPTR_ERR_INVALID;
    }
    for (int q = 0; q < k; ++q)
      if (ctxs[q] == ctxs[k]) { ctx_set_err(c0, "a context appears twice in the batch"); return CPTR_ERR_INVALID; }
  }
  auto t0 = std::chrono::steady_clock::now();
  std::vector<BSys> h(n);
  for (int k = 0; k < n; ++k) {
    std::string why;
    cptr_status st = describe(ctxs[k], tol, maxit, &h[k], why);
    if (st) {
      if (!why.empty()) ctx_set_err(c0, why.c_str());
      return st;
    }
  }
  cudaStream_t s = c0->stream;
  // every context's own work (setup, earlier solves) precedes the batch
  for (int k = 0; k < n; ++k) CTX_CUDA(c0, cudaStreamSynchronize(ctxs[k]->stream));
  for (int k = 0; k < n; ++k) {
    size_t nb = sizeof(double) * 4 * (size_t)ctxs[k]->N;
    CTX_CUDA(c0, cudaMemcpyAsync(ctxs[k]->bd, rhs[k], nb, cudaMemcpyDefault, s));
    CTX_CUDA(c0, cudaMemcpyAsync(ctxs[k]->xd, x[k], nb, cudaMemcpyDefault, s));
  }
  BSys* dsys = nullptr;
  BOut* dout = nullptr;
  CTX_CUDA(c0, cudaMallocAsync((void**)&dsys, sizeof(BSys) * (size_t)n, s));
  cudaError_t e = cudaMallocAsync((void**)&dout, sizeof(BOut) * (size_t)n, s);
  if (e != cudaSuccess) { cudaFreeAsync(dsys, s); return ctx_cuda_fail(c0, e, "batch outputs"); }
  std::vector<BOut> ho(n);
  e = cudaMemcpyAsync(dsys, h.data(), sizeof(BSys) * (size_t)n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    if (c0->mixed) k_batch_fgmres<float><<<n, kBT, 0, s>>>(dsys, dout);
    else k_batch_fgmres<double><<<n, kBT, 0, s>>>(dsys, dout);
    ++c0->nlaunch;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ho.data(), dout, sizeof(BOut) * (size_t)n, cudaMemcpyDeviceToHost, s);
  for (int k = 0; k < n && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(x[k], ctxs[k]->xd, sizeof(double) * 4 * (size_t)ctxs[k]->N,
                        cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(dsys, s);
  cudaFreeAsync(dout, s);
  if (e != cudaSuccess) return ctx_cuda_fail(c0, e, "batched solve");
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  cptr_status worst = CPTR_OK;
  for (int k = 0; k < n; ++k) {
    cptr_ctx* c = ctxs[k];
    c->info.iters = ho[k].iters;
    c->info.rel_resid = ho[k].rel_resid;
    c->info.status = ho[k].status;
    c->info.solve_s = secs;
    c->info.launches = c->nlaunch;
    if (infos) infos[k] = c->info;
    if (ho[k].status != CPTR_OK && (worst == CPTR_OK || ho[k].status != CPTR_ERR_MAXIT))
      worst = (cptr_status)ho[k].status;
  }
  return worst;
}
