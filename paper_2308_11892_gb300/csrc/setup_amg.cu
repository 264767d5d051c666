// Setup of the first stage on the device: BSR validation, Quasi-IMPES
// decoupling to the (p, T) system, and the unknown-based system-AMG hierarchy
// (strength, PMIS, extended+i interpolation truncated to pmax entries,
// Galerkin products, l1 diagonals, dense inverse of the coarsest operator).
//
// This translation unit is compiled with -fmad=false: every product and sum
// is an individually rounded IEEE operation, so the integer decisions that
// depend on floating point (strong connections, PMIS order, truncation) are
// reproducible and independent of the compiler's contraction choices.
#include <algorithm>
#include <cmath>
#include <queue>
#include <utility>
#include <vector>

#include "common.cuh"
#include "ctx.h"

namespace {

constexpr int kT = 256;
enum { ST_U = 0, ST_C = 1, ST_F = -1, ST_CNEW = 2 };

// ------------------------------------------------------------------ validate
__global__ void k_validate(int N, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           int32_t* __restrict__ diag, int* __restrict__ bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int t0 = rp[i], t1 = rp[i + 1];
  int d = -1;
  if (t1 < t0) { atomicExch(bad, 1); return; }
  for (int t = t0; t < t1; ++t) {
    int j = ci[t];
    if (j < 0 || j >= N || (t > t0 && j <= ci[t - 1])) { atomicExch(bad, 1); return; }
    if (j == i) d = t;
  }
  if (d < 0) { atomicExch(bad, 1); return; }
  diag[i] = d;
}

// ------------------------------------------------------------------ decoupling
// W_i = D[e,h] inv(D[h,h]) with D = A_ii; e has ne = 2 unknowns (CPTR) or 1
// (CPR, e1 < 0), h the nh = 4 - ne others.  inv(D[h,h]) is the adjugate over
// the determinant (2x2 or 3x3 cofactor formula), in the oracle's operation order.
__global__ void k_qi_w(int N, const double* __restrict__ v, const int32_t* __restrict__ diag,
                       int e0, int e1, int h0, int h1, int h2, double* __restrict__ W,
                       int* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int ne = e1 < 0 ? 1 : 2, nh = 4 - ne;
  const int e[2] = {e0, e1}, h[3] = {h0, h1, h2};
  const double* D = v + 16 * (size_t)diag[i];
  double inv[9];
  if (nh == 2) {
    double a = D[h0 * 4 + h0], b = D[h0 * 4 + h1];
    double cc = D[h1 * 4 + h0], d = D[h1 * 4 + h1];
    double det = a * d - b * cc;
    double mx = fmax(fmax(fabs(a), fabs(b)), fmax(fabs(cc), fabs(d)));
    if (!(fabs(det) > 1e-300 * mx * mx) || !isfinite(det)) {
      dev_fail(status, DEV_BREAKDOWN);
      return;
    }
    inv[0] = d / det; inv[1] = -b / det; inv[2] = -cc / det; inv[3] = a / det;
  } else {
    double m[9], mx = 0.0;
    for (int r = 0; r < 3; ++r)
      for (int s = 0; s < 3; ++s) {
        m[3 * r + s] = D[h[r] * 4 + h[s]];
        mx = fmax(mx, fabs(m[3 * r + s]));
      }
    double c00 = m[4] * m[8] - m[5] * m[7];
    double c01 = m[5] * m[6] - m[3] * m[8];
    double c02 = m[3] * m[7] - m[4] * m[6];
    double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    if (!(fabs(det) > 1e-300 * mx * mx * mx) || !isfinite(det)) {
      dev_fail(status, DEV_BREAKDOWN);
      return;
    }
    inv[0] = c00 / det;
    inv[1] = (m[2] * m[7] - m[1] * m[8]) / det;
    inv[2] = (m[1] * m[5] - m[2] * m[4]) / det;
    inv[3] = c01 / det;
    inv[4] = (m[0] * m[8] - m[2] * m[6]) / det;
    inv[5] = (m[2] * m[3] - m[0] * m[5]) / det;
    inv[6] = c02 / det;
    inv[7] = (m[1] * m[6] - m[0] * m[7]) / det;
    inv[8] = (m[0] * m[4] - m[1] * m[3]) / det;
  }
  for (int r = 0; r < ne; ++r)
    for (int s = 0; s < nh; ++s) {
      double acc = 0.0;
      for (int t = 0; t < nh; ++t) acc += D[e[r] * 4 + h[t]] * inv[t * nh + s];
      W[4 * (size_t)i + nh * r + s] = acc;
    }
}

// Ahat_ij = A_ij[e,e] - W_i A_ij[h,e], scattered into the ne N scalar CSR whose
// row ne i + r holds, for each block column j, the entries ne j .. ne j + ne - 1.
__global__ void k_qi_ahat(int N, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ v, const double* __restrict__ W, int e0,
                          int e1, int h0, int h1, int h2, int32_t* __restrict__ Arp,
                          int32_t* __restrict__ Aci, double* __restrict__ Av) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int ne = e1 < 0 ? 1 : 2, nh = 4 - ne;
  const int e[2] = {e0, e1}, h[3] = {h0, h1, h2};
  int t0 = rp[i], t1 = rp[i + 1], nb = t1 - t0;
  int base = ne * ne * t0;
  for (int r = 0; r < ne; ++r) Arp[ne * i + r] = base + r * ne * nb;
  if (i == N - 1) Arp[ne * N] = ne * ne * t1;
  const double* Wi = W + 4 * (size_t)i;
  for (int r = 0; r < ne; ++r) {
    int pos = base + r * ne * nb;
    for (int t = t0; t < t1; ++t) {
      const double* B = v + 16 * (size_t)t;
      for (int s = 0; s < ne; ++s) {
        double acc = B[e[r] * 4 + e[s]];
        for (int q = 0; q < nh; ++q) acc -= Wi[nh * r + q] * B[h[q] * 4 + e[s]];
        Aci[pos] = ne * ci[t] + s;
        Av[pos] = acc;
        ++pos;
      }
    }
  }
}

// function (elliptic unknown) of every row of Ahat: they alternate over the ne unknowns
__global__ void k_func_alternating(int n, int ne, int32_t* f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = i % ne;
}

// ------------------------------------------------------------------ strength
__device__ __forceinline__ double row_diag(const int32_t* rp, const int32_t* ci, const double* v,
                                           int i) {
  for (int t = rp[i]; t < rp[i + 1]; ++t)
    if (ci[t] == i) return v[t];
  return 0.0;
}

// Strength, one warp per row (the row maximum does not depend on the order in
// which it is taken, so the strong flags equal the sequential definition's).
// L lanes per row (8, 16 or 32, by the level's mean row length; the flags and
// counts do not depend on it).  Every lane of the warp reaches the collectives
// (lanes of rows past n included), which work on each row's L lanes.
template <int L>
__global__ void k_strength(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ v, const int32_t* __restrict__ func,
                           double theta, uint8_t* __restrict__ S, int32_t* __restrict__ cnt) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = (int)(g / L), lane = (int)(g % L);
  const bool valid = i < n;
  const unsigned base = (threadIdx.x & 31) & ~(unsigned)(L - 1);
  const unsigned smask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << base);
  const int t0 = valid ? rp[i] : 0, t1 = valid ? rp[i + 1] : 0, fi = valid ? func[i] : 0;
  double d = 0.0;
  int has = 0;
  for (int t = t0 + lane; t < t1; t += L)
    if (ci[t] == i && !has) { d = v[t]; has = 1; }
  unsigned m = __ballot_sync(0xffffffffu, has) & smask;
  d = __shfl_sync(0xffffffffu, d, m ? __ffs(m) - 1 : 0);
  if (!m) d = 0.0;
  // -s a_ij with s = sign(a_ii): a_ij itself when a_ii < 0, else its negation
  // (exact either way); the comparisons run on integer keys (same results)
  const bool dneg = d_lt0(d);
  double mx = 0.0;
  int any = 0;
  for (int t = t0 + lane; t < t1; t += L) {
    int j = ci[t];
    S[t] = 0;
    if (j == i || func[j] != fi) continue;
    const double val = dneg ? v[t] : d_neg_of(v[t]);
    if (!any || d_gt(val, mx)) { mx = val; any = 1; }
  }
  for (int o = L / 2; o > 0; o >>= 1) {
    double omx = __shfl_xor_sync(0xffffffffu, mx, o, L);
    int oany = __shfl_xor_sync(0xffffffffu, any, o, L);
    if (oany && (!any || d_gt(omx, mx))) { mx = omx; any = 1; }
  }
  if (!valid || !any || !d_gt0(mx)) return;
  const double thr = theta * mx;
  for (int t = t0 + lane; t < t1; t += L) {
    int j = ci[t];
    if (j == i || func[j] != fi) continue;
    if (d_ge(dneg ? v[t] : d_neg_of(v[t]), thr)) {
      S[t] = 1;
      atomicAdd(&cnt[j], 1);
    }
  }
}

// S^T lists, L lanes per row of S (the order within a list is not used:
// PMIS only tests conditions over all of it)
template <int L>
__global__ void k_st_fill(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const uint8_t* __restrict__ S, const int32_t* __restrict__ tp,
                          int32_t* __restrict__ cur, int32_t* __restrict__ tj) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = (int)(g / L), lane = (int)(g % L);
  if (i >= n) return;
  for (int t = rp[i] + lane; t < rp[i + 1]; t += L)
    if (S[t]) {
      const int j = ci[t];
      tj[tp[j] + atomicAdd(&cur[j], 1)] = i;
    }
}

// ------------------------------------------------------------------ PMIS
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  // SplitMix64 (Steele, Lea & Flood 2014): add the golden gamma, then mix.
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_pmis_init(int n, const int32_t* __restrict__ cnt, uint64_t seed, int level,
                            double* __restrict__ lam, int32_t* __restrict__ st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t x = seed ^ ((uint64_t)(uint32_t)level << 32) ^ (uint64_t)(uint32_t)i;
  double rho = (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0);
  lam[i] = (double)cnt[i] + rho;
  st[i] = (cnt[i] == 0) ? ST_F : ST_U;
}

// lambda_i > lambda_j, ties broken by index.  lambda = count + rho >= 0, and
// non-negative doubles order exactly as their bit patterns (integer compare).
__device__ __forceinline__ bool lam_greater(const double* lam, int i, int j) {
  const long long a = __double_as_longlong(lam[i]), b = __double_as_longlong(lam[j]);
  return a > b || (a == b && i > j);
}

__global__ void k_pmis_select(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const uint8_t* __restrict__ S, const int32_t* __restrict__ tp,
                              const int32_t* __restrict__ tj, const double* __restrict__ lam,
                              int32_t* st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (ld_volatile_i32(st + i) != ST_U) return;
  bool ok = true;
  for (int t = rp[i]; t < rp[i + 1] && ok; ++t) {
    if (!S[t]) continue;
    int j = ci[t];
    int sj = ld_volatile_i32(st + j);
    if ((sj == ST_U || sj == ST_CNEW) && !lam_greater(lam, i, j)) ok = false;
  }
  for (int t = tp[i]; t < tp[i + 1] && ok; ++t) {
    int j = tj[t];
    int sj = ld_volatile_i32(st + j);
    if ((sj == ST_U || sj == ST_CNEW) && !lam_greater(lam, i, j)) ok = false;
  }
  if (ok) st[i] = ST_CNEW;
}

__global__ void k_pmis_update(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const uint8_t* __restrict__ S, int32_t* st, int* remaining) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int si = ld_volatile_i32(st + i);
  if (si == ST_CNEW) { st[i] = ST_C; return; }
  if (si != ST_U) return;
  for (int t = rp[i]; t < rp[i + 1]; ++t) {
    if (!S[t]) continue;
    int sk = ld_volatile_i32(st + ci[t]);
    if (sk == ST_C || sk == ST_CNEW) { st[i] = ST_F; return; }
  }
  atomicAdd(remaining, 1);
}

// The same two PMIS phases with one warp per point, for levels whose rows are
// long (the lanes scan the strong neighbours and vote; the decisions are those
// of the thread-per-point kernels).
__global__ void k_pmis_select_warp(int n, const int32_t* __restrict__ rp,
                                   const int32_t* __restrict__ ci, const uint8_t* __restrict__ S,
                                   const int32_t* __restrict__ tp, const int32_t* __restrict__ tj,
                                   const double* __restrict__ lam, int32_t* st) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i = (int)(g >> 5), lane = (int)(g & 31);
  if (i >= n) return;
  if (ld_volatile_i32(st + i) != ST_U) return;  // the same value for the whole warp
  bool bad = false;
  for (int t = rp[i] + lane; t < rp[i + 1] && !bad; t += 32) {
    if (!S[t]) continue;
    int j = ci[t];
    int sj = ld_volatile_i32(st + j);
    if ((sj == ST_U || sj == ST_CNEW) && !lam_greater(lam, i, j)) bad = true;
  }
  for (int t = tp[i] + lane; t < tp[i + 1] && !bad; t += 32) {
    int j = tj[t];
    int sj = ld_volatile_i32(st + j);
    if ((sj == ST_U || sj == ST_CNEW) && !lam_greater(lam, i, j)) bad = true;
  }
  if (!__any_sync(0xffffffffu, bad) && lane == 0) st[i] = ST_CNEW;
}

__global__ void k_pmis_update_warp(int n, const int32_t* __restrict__ rp,
                                   const int32_t* __restrict__ ci, const uint8_t* __restrict__ S,
                                   int32_t* st, int* remaining) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i = (int)(g >> 5), lane = (int)(g & 31);
  if (i >= n) return;
  int si = ld_volatile_i32(st + i);
  if (si == ST_CNEW) {
    if (lane == 0) st[i] = ST_C;
    return;
  }
  if (si != ST_U) return;
  bool f = false;
  for (int t = rp[i] + lane; t < rp[i + 1] && !f; t += 32) {
    if (!S[t]) continue;
    int sk = ld_volatile_i32(st + ci[t]);
    if (sk == ST_C || sk == ST_CNEW) f = true;
  }
  f = __any_sync(0xffffffffu, f);
  if (lane == 0) {
    if (f) st[i] = ST_F;
    else atomicAdd(remaining, 1);
  }
}

__global__ void k_pmis_final(int n, const int32_t* __restrict__ st, int32_t* __restrict__ cf,
                             int32_t* __restrict__ isc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = (st[i] == ST_C) ? 1 : -1;
  cf[i] = c;
  isc[i] = (c == 1);
}

__device__ __forceinline__ int find_sorted(const int32_t* a, int n, int key) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int x = a[mid];
    if (x == key) return mid;
    if (x < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// abar_kl: a_kl if its sign is opposite to that of a_kk (a_kk >= 0 counts as
// positive), else 0; the sign tests run on the bit pattern (same results).
__device__ __forceinline__ double abar(double akk, double akl) {
  const bool keep = d_ge0(akk) ? d_lt0(akl) : d_gt0(akl);
  return keep ? akl : 0.0;
}

// Extended+i weights for one fine row; same loop order and arithmetic as the
// definition: a_ii and the direct a_ij first, weak same-function connections
// outside Chat lumped into the diagonal, then the strong F neighbours k
// distributed through abar_kl / sum_{l in Chat u {i}} abar_kl.
__global__ void k_interp(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const double* __restrict__ v, const uint8_t* __restrict__ S,
                         const int32_t* __restrict__ cf, const int32_t* __restrict__ func,
                         const int32_t* __restrict__ cidx, const long long* __restrict__ off,
                         int32_t* __restrict__ sc_col, double* __restrict__ sc_num,
                         int32_t* __restrict__ sc_ord, int pmax, int32_t* __restrict__ pcnt,
                         int32_t* __restrict__ pcol, double* __restrict__ pval) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (cf[i] == 1) {
    pcnt[i] = 1;
    pcol[(size_t)i * pmax] = cidx[i];
    pval[(size_t)i * pmax] = 1.0;
    return;
  }
  int32_t* chat = sc_col + off[i];
  double* num = sc_num + off[i];
  int32_t* ord = sc_ord + off[i];
  int q = 0;
  for (int t = rp[i]; t < rp[i + 1]; ++t) {
    if (!S[t]) continue;
    int j = ci[t];
    if (cf[j] == 1) {
      chat[q++] = j;
    } else {
      for (int t2 = rp[j]; t2 < rp[j + 1]; ++t2)
        if (S[t2] && cf[ci[t2]] == 1) chat[q++] = ci[t2];
    }
  }
  if (q == 0) { pcnt[i] = 0; return; }
  for (int a = 1; a < q; ++a) {  // insertion sort
    int key = chat[a], b = a - 1;
    while (b >= 0 && chat[b] > key) { chat[b + 1] = chat[b]; --b; }
    chat[b + 1] = key;
  }
  int u = 0;
  for (int t = 0; t < q; ++t)
    if (t == 0 || chat[t] != chat[u - 1]) chat[u++] = chat[t];
  q = u;
  for (int t = 0; t < q; ++t) num[t] = 0.0;
  double dg = 0.0;
  int fi = func[i];
  for (int t = rp[i]; t < rp[i + 1]; ++t) {
    int j = ci[t];
    if (j == i) { dg += v[t]; continue; }
    if (func[j] != fi) continue;
    int pos = find_sorted(chat, q, j);
    if (pos >= 0) { num[pos] += v[t]; continue; }
    if (!S[t]) dg += v[t];
  }
  for (int t = rp[i]; t < rp[i + 1]; ++t) {
    int k = ci[t];
    if (!S[t] || cf[k] == 1) continue;
    double aik = v[t];
    double akk = row_diag(rp, ci, v, k);
    int fk = func[k];
    double den = 0.0;
    for (int t2 = rp[k]; t2 < rp[k + 1]; ++t2) {
      int l = ci[t2];
      if (l == k || func[l] != fk) continue;
      if (l == i || find_sorted(chat, q, l) >= 0) den += abar(akk, v[t2]);
    }
    if (den == 0.0) { dg += aik; continue; }
    double f = aik / den;
    for (int t2 = rp[k]; t2 < rp[k + 1]; ++t2) {
      int l = ci[t2];
      if (l == k || func[l] != fk) continue;
      double ab = abar(akk, v[t2]);
      if (ab == 0.0) continue;
      if (l == i) { dg += f * ab; continue; }
      int pos = find_sorted(chat, q, l);
      if (pos >= 0) num[pos] += f * ab;
    }
  }
  if (dg == 0.0 || !isfinite(dg)) { pcnt[i] = 0; return; }
  int m = 0;
  for (int t = 0; t < q; ++t) {
    double w = -num[t] / dg;
    if (w != 0.0) { chat[m] = chat[t]; num[m] = w; ++m; }
  }
  if (m > pmax) {
    double sum_all = 0.0;
    for (int t = 0; t < m; ++t) sum_all += num[t];
    for (int t = 0; t < m; ++t) ord[t] = t;
    for (int a = 0; a < pmax; ++a) {
      int best = a;
      for (int b2 = a + 1; b2 < m; ++b2) {
        double wb = fabs(num[ord[b2]]), wa = fabs(num[ord[best]]);
        if (wb > wa || (wb == wa && ord[b2] < ord[best])) best = b2;
      }
      int tmp = ord[a]; ord[a] = ord[best]; ord[best] = tmp;
    }
    for (int a = 1; a < pmax; ++a) {  // kept entries in column order
      int key = ord[a], b = a - 1;
      while (b >= 0 && ord[b] > key) { ord[b + 1] = ord[b]; --b; }
      ord[b + 1] = key;
    }
    double sum_kept = 0.0;
    for (int a = 0; a < pmax; ++a) sum_kept += num[ord[a]];
    double scale = (sum_kept != 0.0) ? sum_all / sum_kept : 1.0;
    for (int a = 0; a < pmax; ++a) {
      pcol[(size_t)i * pmax + a] = cidx[chat[ord[a]]];
      pval[(size_t)i * pmax + a] = num[ord[a]] * scale;
    }
    pcnt[i] = pmax;
  } else {
    for (int a = 0; a < m; ++a) {
      pcol[(size_t)i * pmax + a] = cidx[chat[a]];
      pval[(size_t)i * pmax + a] = num[a];
    }
    pcnt[i] = m;
  }
}

__global__ void k_compact_rows(int n, int pmax, const int32_t* __restrict__ prp,
                               const int32_t* __restrict__ pcol, const double* __restrict__ pval,
                               int32_t* __restrict__ ci, double* __restrict__ v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = prp[i], c = prp[i + 1] - b;
  for (int a = 0; a < c; ++a) {
    ci[b + a] = pcol[(size_t)i * pmax + a];
    v[b + a] = pval[(size_t)i * pmax + a];
  }
}

// ------------------------------------------------------------------ transpose
__global__ void k_count_cols(int nnz, const int32_t* __restrict__ ci, int32_t* __restrict__ cnt) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nnz) atomicAdd(&cnt[ci[t]], 1);
}

__global__ void k_transpose_fill(int n, const int32_t* __restrict__ rp,
                                 const int32_t* __restrict__ ci, const double* __restrict__ v,
                                 const int32_t* __restrict__ trp, int32_t* __restrict__ cur,
                                 int32_t* __restrict__ tci, double* __restrict__ tv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int t = rp[i]; t < rp[i + 1]; ++t) {
    int j = ci[t];
    int pos = trp[j] + atomicAdd(&cur[j], 1);
    tci[pos] = i;
    tv[pos] = v[t];
  }
}

// Sorts each row of a transpose by column (its keys are distinct), one warp
// per row: the row is copied to shared memory and every entry is written to
// the position given by its rank.  Rows longer than kSortRow are sorted by one
// lane in place.
constexpr int kSortRow = 256;
constexpr int kSortWarps = 8;
__global__ void __launch_bounds__(32 * kSortWarps) k_sort_rows(int n,
                                                               const int32_t* __restrict__ rp,
                                                               int32_t* __restrict__ ci,
                                                               double* __restrict__ v) {
  __shared__ int sk[kSortWarps][kSortRow];
  __shared__ double sv[kSortWarps][kSortRow];
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31,
            w = threadIdx.x >> 5;
  if (r >= n) return;
  const int b = rp[r], len = rp[r + 1] - b;
  if (len <= kSortRow) {
    for (int q = lane; q < len; q += 32) {
      sk[w][q] = ci[b + q];
      sv[w][q] = v[b + q];
    }
    __syncwarp();
    for (int q = lane; q < len; q += 32) {
      const int key = sk[w][q];
      int rank = 0;
      for (int o = 0; o < len; ++o) rank += sk[w][o] < key;
      ci[b + rank] = key;
      v[b + rank] = sv[w][q];
    }
    return;
  }
  if (lane != 0) return;
  for (int a = b + 1; a < b + len; ++a) {
    int key = ci[a];
    double kv = v[a];
    int c = a - 1;
    while (c >= b && ci[c] > key) { ci[c + 1] = ci[c]; v[c + 1] = v[c]; --c; }
    ci[c + 1] = key;
    v[c + 1] = kv;
  }
}

// ------------------------------------------------------------------ SpGEMM
__global__ void k_spgemm_ub(int n, const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                            const int32_t* __restrict__ brp, int32_t* __restrict__ hs,
                            int32_t* __restrict__ prods, int bcols, int* mx3 = nullptr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long u = 0;
  for (int t = arp[i]; t < arp[i + 1]; ++t) u += brp[aci[t] + 1] - brp[aci[t]];
  const int np = (int)(u < (1ll << 30) ? u : (1ll << 30));
  if (prods) prods[i] = np;
  if (bcols > 0 && u > bcols) u = bcols;  // distinct columns never exceed B's columns
  int h = 0;
  if (u > 0) {
    h = 1;
    while (h < 2 * u && h < (1 << 30)) h <<= 1;
  }
  hs[i] = h;
  if (mx3) {  // largest table, product count and A-row length (atomics only for a new maximum)
    const int na = arp[i + 1] - arp[i];
    if (h > ld_volatile_i32(&mx3[0])) atomicMax(&mx3[0], h);
    if (np > ld_volatile_i32(&mx3[1])) atomicMax(&mx3[1], np);
    if (na > ld_volatile_i32(&mx3[2])) atomicMax(&mx3[2], na);
  }
}
// rows of C from their product-count slots to their final place
__global__ void k_spgemm_compact(int n, const long long* __restrict__ toff,
                                 const int32_t* __restrict__ cnt, const int32_t* __restrict__ tci,
                                 const double* __restrict__ tv, const int32_t* __restrict__ crp,
                                 int32_t* __restrict__ cci, double* __restrict__ cv) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i = (int)(g >> 5), lane = (int)(g & 31);
  if (i >= n) return;
  const long long s = toff[i];
  const int o = crp[i], m = cnt[i];
  for (int q = lane; q < m; q += 32) {
    cci[o + q] = tci[s + q];
    cv[o + q] = tv[s + q];
  }
}

// Row i of A*B accumulated in an open-addressing table; each entry sums its
// products in the loop order (A row ascending, then B row ascending), starting
// from 0.0 at first touch.  The occupied entries are then moved to the front
// and sorted by column.
__global__ void k_spgemm_hash(int r0, int r1, const int32_t* __restrict__ arp,
                              const int32_t* __restrict__ aci, const double* __restrict__ av,
                              const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                              const double* __restrict__ bv, const long long* __restrict__ hoff,
                              int32_t* __restrict__ hcol, double* __restrict__ hval,
                              int32_t* __restrict__ cnt, int* status) {
  int i = r0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r1) return;
  long long base = hoff[i] - hoff[r0];
  int hs = (int)(hoff[i + 1] - hoff[i]);
  int32_t* hc = hcol + base;
  double* hv = hval + base;
  for (int h = 0; h < hs; ++h) hc[h] = -1;
  unsigned mask = (unsigned)hs - 1u;
  for (int t = arp[i]; t < arp[i + 1]; ++t) {
    int k = aci[t];
    double a = av[t];
    for (int t2 = brp[k]; t2 < brp[k + 1]; ++t2) {
      int j = bci[t2];
      double prod = a * bv[t2];
      unsigned h = ((unsigned)j * 2654435761u) & mask;
      int probes = 0;
      while (hc[h] != j && hc[h] != -1 && probes < hs) { h = (h + 1u) & mask; ++probes; }
      if (probes >= hs) {  // table full: cannot happen with hs >= 2 * products
        dev_fail(status, DEV_BREAKDOWN);
        cnt[i] = 0;
        return;
      }
      if (hc[h] == -1) { hc[h] = j; hv[h] = 0.0; }
      hv[h] += prod;
    }
  }
  int u = 0;
  for (int h = 0; h < hs; ++h)
    if (hc[h] != -1) {
      int cj = hc[h];
      double cv = hv[h];
      // insertion into the sorted front [0, u)
      int b = u - 1;
      while (b >= 0 && hc[b] > cj) { hc[b + 1] = hc[b]; hv[b + 1] = hv[b]; --b; }
      hc[b + 1] = cj;
      hv[b + 1] = cv;
      ++u;
    }
  cnt[i] = u;
}

__global__ void k_spgemm_gather(int r0, int r1, const long long* __restrict__ hoff,
                                const int32_t* __restrict__ hcol, const double* __restrict__ hval,
                                const int32_t* __restrict__ boff, int32_t* __restrict__ oc,
                                double* __restrict__ ov) {
  int i = r0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r1) return;
  long long base = hoff[i] - hoff[r0];
  int o = boff[i - r0], u = boff[i - r0 + 1] - o;
  for (int a = 0; a < u; ++a) {
    oc[o + a] = hcol[base + a];
    ov[o + a] = hval[base + a];
  }
}

// ------------------------------------------------------------------ block-per-row setup
// One thread block per output row.  The row's column set is built in a
// shared-memory hash set (no floating point involved), sorted with a bitonic
// network, and every output entry then sums its own contributions in the
// definition's loop order (so results equal the sequential Gustavson / ext+i
// accumulation bit for bit).  Rows whose set does not fit set *overflow and
// the caller falls back to the thread-per-row kernels above.
// Keys are never removed, so a slot seen holding the key needs no atomic: the
// slot is read first and claimed by compare-and-swap only while it is empty
// (candidate lists repeat a few keys many times).
__device__ __forceinline__ bool set_insert(int* tab, int hs, int key, int* count) {
  unsigned h = ((unsigned)key * 2654435761u) & (unsigned)(hs - 1);
  for (int p = 0; p < hs; ++p) {
    int cur = *reinterpret_cast<volatile int*>(&tab[h]);
    if (cur == -1) {
      cur = atomicCAS(&tab[h], -1, key);
      if (cur == -1) { atomicAdd(count, 1); return true; }
    }
    if (cur == key) return true;
    h = (h + 1u) & (unsigned)(hs - 1);
  }
  return false;
}

// Moves the set into list[0..u) sorted ascending.  Small sets (u <= 128) are
// copied to tmp[0..u) and each key is written at its rank (two barriers);
// larger ones are padded to a power of two and bitonic-sorted in list.
// tmp (u ints) may alias nothing else in use.
constexpr int kRankSortMax = 128;
__device__ int set_to_sorted(const int* tab, int hs, int* list, int* tmp, int u, int* cursor) {
  if (u <= kRankSortMax) {
    for (int h = threadIdx.x; h < hs; h += blockDim.x)
      if (tab[h] != -1) tmp[atomicAdd(cursor, 1)] = tab[h];
    __syncthreads();
    for (int q = threadIdx.x; q < u; q += blockDim.x) {
      const int key = tmp[q];
      int rank = 0;
      for (int o = 0; o < u; ++o) rank += tmp[o] < key;
      list[rank] = key;
    }
    __syncthreads();
    return u;
  }
  for (int h = threadIdx.x; h < hs; h += blockDim.x)
    if (tab[h] != -1) list[atomicAdd(cursor, 1)] = tab[h];
  int P = 1;
  while (P < u) P <<= 1;
  __syncthreads();
  for (int q = u + threadIdx.x; q < P; q += blockDim.x) list[q] = 0x7fffffff;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1)
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int idx = threadIdx.x; idx < P; idx += blockDim.x) {
        int ixj = idx ^ jj;
        if (ixj > idx) {
          bool up = (idx & k) == 0;
          int a = list[idx], b = list[ixj];
          if ((a > b) == up) { list[idx] = b; list[ixj] = a; }
        }
      }
      __syncthreads();
    }
  return P;
}

__device__ __forceinline__ int bsearch_row(const int32_t* ci, int lo, int hi, int key) {
  hi -= 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int x = ci[mid];
    if (x == key) return mid;
    if (x < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// Position of a key in the sorted list built from a hash set (-1 if absent),
// through the hash table and its slot -> position map.
__device__ __forceinline__ int chat_pos(const int* tab, const int* tabpos, int hs, int key) {
  unsigned h = ((unsigned)key * 2654435761u) & (unsigned)(hs - 1);
  for (int p = 0; p < hs; ++p) {
    int k = tab[h];
    if (k == key) return tabpos[h];
    if (k == -1) return -1;
    h = (h + 1u) & (unsigned)(hs - 1);
  }
  return -1;
}

constexpr int kSpgemmSeg = 256;  // products staged per segment
struct SpgSmem {
  size_t tab, tabpos, list, acc, sbv, sbc, spos, stt, sav, sak, soff, tbl, total;
  int tcap;  // doubles of the product table
};
__host__ __device__ inline SpgSmem spgemm_layout(int hsmax, int maxa) {
  SpgSmem L;
  size_t o = 0;
  auto take = [&](size_t b) { size_t at = o; o += (b + 15) & ~(size_t)15; return at; };
  L.tcap = hsmax / 2 > 1024 ? hsmax / 2 : 1024;
  L.tab = take(4 * (size_t)hsmax);
  L.tabpos = take(4 * (size_t)hsmax);
  L.list = take(4 * (size_t)hsmax);
  L.acc = take(8 * (size_t)(hsmax / 2));
  L.sbv = take(8 * (size_t)kSpgemmSeg);
  L.sbc = take(4 * (size_t)kSpgemmSeg);
  L.spos = take(4 * (size_t)kSpgemmSeg);
  L.stt = take(4 * (size_t)kSpgemmSeg);
  L.sav = take(8 * (size_t)maxa);
  L.sak = take(4 * (size_t)maxa);
  L.soff = take(4 * ((size_t)maxa + 1));
  L.tbl = take(8 * (size_t)L.tcap);
  L.total = o;
  return L;
}
__host__ __device__ inline size_t spgemm_smem(int hsmax, int maxa) {
  return spgemm_layout(hsmax, maxa).total;
}
// absent entry of an ordered-sum table (a NaN that no computation produces)
__device__ __forceinline__ double tbl_absent() { return __longlong_as_double((long long)SENT_F64); }
__device__ __forceinline__ bool tbl_present(double x) {
  return (unsigned long long)__double_as_longlong(x) != SENT_F64;
}

// mode 0: count the columns of row i of A*B; mode 1: write them (sorted) and
// their values into C at crp[i].  Every output entry sums its products in
// the order of the entries of A (the definition's loop order).
__global__ void k_i64_to_i32(int n, const long long* __restrict__ in, int32_t* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)in[i];
}
// rows deferred by the shared-memory pass, and the global scratch each needs
__global__ void k_spgemm_deferred(int n, const int32_t* __restrict__ cnt,
                                  const int32_t* __restrict__ arp,
                                  const int32_t* __restrict__ hrow, int32_t* __restrict__ rows,
                                  long long* __restrict__ bytes, int* nrows) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cnt[i] != -1) return;
  int k = atomicAdd(nrows, 1);
  rows[k] = i;
  int hs = hrow[i] < 32 ? 32 : hrow[i];
  int na = arp[i + 1] - arp[i];
  bytes[k] = (long long)((spgemm_smem(hs, na < 1 ? 1 : na) + 255) & ~(size_t)255);
}

// Rows of C = A B with at most kSpwProd products, one warp per row: the
// products are staged in shared memory, ranked by (column, product index) and
// each output column is summed by one lane over its products in that order,
// i.e. in the order of the entries of A, starting from 0.0 (the same sums as
// k_spgemm_row).  Other rows are appended to rows[] for the block kernel.
constexpr int kSpwProd = 64;
constexpr int kSpwWarps = 8;
struct SpwSmem {
  int soff[kSpwProd + 1];  // first product of each A entry
  int bst[kSpwProd];       // start of each A entry's B row
  double sa[kSpwProd];     // A values
  int key[kSpwProd];       // product columns, then sorted columns
  int skey[kSpwProd];
  double val[kSpwProd];    // products, then in sorted order
  double sval[kSpwProd];
};
__global__ void __launch_bounds__(32 * kSpwWarps) k_spgemm_warp(
    int n, const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
    const double* __restrict__ av, const int32_t* __restrict__ brp,
    const int32_t* __restrict__ bci, const double* __restrict__ bv,
    const int32_t* __restrict__ prods, const long long* __restrict__ toff,
    int32_t* __restrict__ cci, double* __restrict__ cv, int32_t* __restrict__ cnt,
    int32_t* __restrict__ rows, int* nrows) {
  __shared__ SpwSmem sm_all[kSpwWarps];
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  SpwSmem& W = sm_all[threadIdx.x >> 5];
  const int t0 = arp[i], nA = arp[i + 1] - t0, T = prods[i];
  if (T > kSpwProd || nA > kSpwProd) {
    if (lane == 0) rows[atomicAdd(nrows, 1)] = i;
    return;
  }
  // A entries: B-row starts and lengths, offsets by an inclusive warp scan
  int carry = 0;
  if (lane == 0) W.soff[0] = 0;
  for (int e0 = 0; e0 < nA; e0 += 32) {
    const int e = e0 + lane;
    int len = 0;
    if (e < nA) {
      const int k = aci[t0 + e];
      const int b = brp[k];
      len = brp[k + 1] - b;
      W.bst[e] = b;
      W.sa[e] = av[t0 + e];
    }
    int x = len;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (e < nA) W.soff[e + 1] = carry + x;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  __syncwarp();
  // products: column and value a_ik b_kj
  for (int p = lane; p < T; p += 32) {
    int lo = 0, hi = nA - 1;  // entry e with soff[e] <= p < soff[e+1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (W.soff[mid] <= p) lo = mid; else hi = mid - 1;
    }
    const int src = W.bst[lo] + (p - W.soff[lo]);
    W.key[p] = bci[src];
    W.val[p] = W.sa[lo] * bv[src];
  }
  __syncwarp();
  // rank by (column, product index)
  for (int p = lane; p < T; p += 32) {
    const int k = W.key[p];
    int r = 0;
    for (int q = 0; q < T; ++q) {
      const int kq = W.key[q];
      r += kq < k || (kq == k && q < p);
    }
    W.skey[r] = k;
    W.sval[r] = W.val[p];
  }
  __syncwarp();
  // one lane per distinct column sums its run
  int u = 0;
  const long long o = toff[i];
  for (int r0 = 0; r0 < T; r0 += 32) {
    const int r = r0 + lane;
    const bool head = r < T && (r == 0 || W.skey[r] != W.skey[r - 1]);
    const unsigned hb = __ballot_sync(0xffffffffu, head);
    if (head) {
      const int col = W.skey[r];
      double sum = 0.0;
      for (int q = r; q < T && W.skey[q] == col; ++q) sum += W.sval[q];
      const int qo = u + __popc(hb & ((1u << lane) - 1u));
      cci[o + qo] = col;
      cv[o + qo] = sum;
    }
    u += __popc(hb);
  }
  if (lane == 0) cnt[i] = u;
}

// Rows of C = A B with at most tprod products, one block per row (rows[] when
// given).  Every product is formed once; the distinct columns are collected
// in a hash set and sorted; the products are bucketed by output column in
// product-index order, which is the order of the entries of A, and each
// bucket is summed by one thread from 0.0 (the same sums as k_spgemm_row).  A row that does not fit is deferred (cnt = -1, *overflow).
struct SpsSmem {
  size_t tab, tabpos, list, ccnt, cfill, cstart, pcol, pv, ppos, sidx, sav, soff, bst, total;
};
__host__ __device__ inline SpsSmem sps_layout(int hsmax, int tprod, int maxa) {
  SpsSmem L;
  size_t o = 0;
  auto take = [&](size_t b) { size_t at = o; o += (b + 15) & ~(size_t)15; return at; };
  L.tab = take(4 * (size_t)hsmax);
  L.tabpos = take(4 * (size_t)hsmax);
  L.list = take(4 * (size_t)(hsmax / 2));
  L.ccnt = take(4 * (size_t)(hsmax / 2));
  L.cfill = take(4 * (size_t)(hsmax / 2));
  L.cstart = take(4 * ((size_t)hsmax / 2 + 1));
  L.pcol = take(4 * (size_t)tprod);
  L.pv = take(8 * (size_t)tprod);
  L.ppos = take(4 * (size_t)tprod);
  L.sidx = take(4 * (size_t)tprod);
  L.sav = take(8 * (size_t)maxa);
  L.soff = take(4 * ((size_t)maxa + 1));
  L.bst = take(4 * (size_t)maxa);
  L.total = o;
  return L;
}
// inclusive scan of a[1..n] in place by warp 0 (a[0] = 0)
__device__ __forceinline__ void warp0_scan(int* a, int n) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  int carry = 0;
  if (lane == 0) a[0] = 0;
  for (int b = 1; b <= n; b += 32) {
    const int idx = b + lane;
    int x = idx <= n ? a[idx] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (idx <= n) a[idx] = x + carry;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
}
__global__ void k_spgemm_sorted(int hsmax, int tprod, int maxa, const int32_t* __restrict__ hrow,
                                const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                const double* __restrict__ av, const int32_t* __restrict__ brp,
                                const int32_t* __restrict__ bci, const double* __restrict__ bv,
                                const int32_t* __restrict__ prods,
                                const long long* __restrict__ toff, int32_t* __restrict__ cci,
                                double* __restrict__ cv, int32_t* __restrict__ cnt, int* overflow,
                                const int32_t* __restrict__ rows) {
  extern __shared__ __align__(16) unsigned char sps_dyn[];
  const int i = rows ? rows[blockIdx.x] : (int)blockIdx.x;
  const int t0 = arp[i], nA = arp[i + 1] - t0, T = prods[i];
  const SpsSmem Ly = sps_layout(hsmax, tprod, maxa);
  int* tab = reinterpret_cast<int*>(sps_dyn + Ly.tab);
  int* tabpos = reinterpret_cast<int*>(sps_dyn + Ly.tabpos);
  int* list = reinterpret_cast<int*>(sps_dyn + Ly.list);
  int* ccnt = reinterpret_cast<int*>(sps_dyn + Ly.ccnt);
  int* cfill = reinterpret_cast<int*>(sps_dyn + Ly.cfill);
  int* cstart = reinterpret_cast<int*>(sps_dyn + Ly.cstart);
  int* pcol = reinterpret_cast<int*>(sps_dyn + Ly.pcol);
  double* pv = reinterpret_cast<double*>(sps_dyn + Ly.pv);
  int* ppos = reinterpret_cast<int*>(sps_dyn + Ly.ppos);
  int* sidx = reinterpret_cast<int*>(sps_dyn + Ly.sidx);
  double* sav = reinterpret_cast<double*>(sps_dyn + Ly.sav);
  int* soff = reinterpret_cast<int*>(sps_dyn + Ly.soff);
  int* bst = reinterpret_cast<int*>(sps_dyn + Ly.bst);
  __shared__ int count, cursor, bad;
  if (T > tprod || nA > maxa) {
    if (threadIdx.x == 0) { atomicAdd(overflow, 1); cnt[i] = -1; }
    return;
  }
  int hs = hrow[i];
  hs = hs < 32 ? 32 : (hs > hsmax ? hsmax : hs);
  for (int h = threadIdx.x; h < hs; h += blockDim.x) tab[h] = -1;
  for (int e = threadIdx.x; e < nA; e += blockDim.x) {
    const int k = aci[t0 + e];
    const int b = brp[k];
    sav[e] = av[t0 + e];
    bst[e] = b;
    soff[e + 1] = brp[k + 1] - b;
  }
  if (threadIdx.x == 0) { count = 0; cursor = 0; bad = 0; }
  __syncthreads();
  warp0_scan(soff, nA);
  __syncthreads();
  // products: column and value a_ik b_kj, the column into the set
  for (int p0 = threadIdx.x; p0 < T; p0 += 4 * blockDim.x) {
    int src[4], ent[4], col[4];
    double b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int p = p0 + u * blockDim.x;
      src[u] = -1;
      if (p < T) {
        int lo = 0, hi = nA - 1;  // entry e with soff[e] <= p < soff[e+1]
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (soff[mid] <= p) lo = mid; else hi = mid - 1;
        }
        src[u] = bst[lo] + (p - soff[lo]);
        ent[u] = lo;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (src[u] >= 0) {
        col[u] = bci[src[u]];
        b[u] = bv[src[u]];
      }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (src[u] >= 0) {
        const int p = p0 + u * blockDim.x;
        pcol[p] = col[u];
        pv[p] = sav[ent[u]] * b[u];
        if (!set_insert(tab, hs, col[u], &count)) bad = 1;
      }
  }
  __syncthreads();
  const int nu = count;
  if (bad || 2 * nu > hs) {
    if (threadIdx.x == 0) { atomicAdd(overflow, 1); cnt[i] = -1; }
    return;
  }
  if (threadIdx.x == 0) cnt[i] = nu;
  if (nu == 0) return;
  set_to_sorted(tab, hs, list, tabpos, nu, &cursor);
  for (int q = threadIdx.x; q < nu; q += blockDim.x) {
    unsigned h = ((unsigned)list[q] * 2654435761u) & (unsigned)(hs - 1);
    while (tab[h] != list[q]) h = (h + 1u) & (unsigned)(hs - 1);
    tabpos[h] = q;
    ccnt[q] = 0;
    cfill[q] = 0;
  }
  __syncthreads();
  // bucket sizes per output column, then their starts
  for (int p = threadIdx.x; p < T; p += blockDim.x) {
    const int q = chat_pos(tab, tabpos, hs, pcol[p]);
    ppos[p] = q;
    atomicAdd(&ccnt[q], 1);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nu; q += blockDim.x) cstart[q + 1] = ccnt[q];
  __syncthreads();
  warp0_scan(cstart, nu);
  __syncthreads();
  // stable placement by warp 0, 32 products at a time in index order: equal
  // columns within a chunk are ranked by lane, and each column's leader lane
  // advances its fill count, so every bucket lists its products in order
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int p0 = 0; p0 < T; p0 += 32) {
      const int p = p0 + lane;
      const int q = p < T ? ppos[p] : -1;
      const unsigned same = __match_any_sync(0xffffffffu, q);
      const int fill = p < T ? cfill[q] : 0;
      __syncwarp();
      if (p < T) {
        const int rank = __popc(same & ((1u << lane) - 1u));
        sidx[cstart[q] + fill + rank] = p;
        if (rank == 0) cfill[q] = fill + __popc(same);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // each column: its products in index order, summed from 0.0
  const long long o = toff[i];
  for (int q = threadIdx.x; q < nu; q += blockDim.x) {
    double sum = 0.0;
    for (int a = cstart[q]; a < cstart[q + 1]; ++a) sum += pv[sidx[a]];
    cci[o + q] = list[q];
    cv[o + q] = sum;
  }
}

// GLOBAL = false: one block per row (rows[blockIdx.x] when rows is given),
//   tables in shared memory sized for hsmax and maxa; a row that does not fit is deferred (cnt = -1, *overflow counts it).
// GLOBAL = true: one block per deferred row (rows[blockIdx.x]), its tables in
//   global scratch at gscr + goff[blockIdx.x], sized for the row itself.
template <bool GLOBAL>
__global__ void k_spgemm_row(int hsmax, int maxa, const int32_t* __restrict__ hrow,
                             const int32_t* __restrict__ arp,
                             const int32_t* __restrict__ aci, const double* __restrict__ av,
                             const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                             const double* __restrict__ bv, const long long* __restrict__ toff,
                             int32_t* __restrict__ cci, double* __restrict__ cv,
                             int32_t* __restrict__ cnt, int* overflow,
                             const int32_t* __restrict__ rows, const long long* __restrict__ goff,
                             unsigned char* __restrict__ gscr) {
  extern __shared__ __align__(16) unsigned char gsm_dyn[];
  const int i = rows ? rows[blockIdx.x] : (int)blockIdx.x;
  const int t0 = arp[i], t1 = arp[i + 1], nA = t1 - t0;
  if (GLOBAL) {
    hsmax = hrow[i] < 32 ? 32 : hrow[i];
    maxa = nA < 1 ? 1 : nA;
  }
  unsigned char* gsm = GLOBAL ? gscr + goff[blockIdx.x] : gsm_dyn;
  const SpgSmem Ly = spgemm_layout(hsmax, maxa);
  int* tab = reinterpret_cast<int*>(gsm + Ly.tab);
  int* tabpos = reinterpret_cast<int*>(gsm + Ly.tabpos);
  int* list = reinterpret_cast<int*>(gsm + Ly.list);
  double* acc = reinterpret_cast<double*>(gsm + Ly.acc);
  double* sbv = reinterpret_cast<double*>(gsm + Ly.sbv);
  int* sbc = reinterpret_cast<int*>(gsm + Ly.sbc);
  int* spos = reinterpret_cast<int*>(gsm + Ly.spos);
  int* stt = reinterpret_cast<int*>(gsm + Ly.stt);
  double* sav = reinterpret_cast<double*>(gsm + Ly.sav);
  int* sak = reinterpret_cast<int*>(gsm + Ly.sak);
  int* soff = reinterpret_cast<int*>(gsm + Ly.soff);
  double* tbl = reinterpret_cast<double*>(gsm + Ly.tbl);
  __shared__ int count, cursor, bad;
  if (nA > maxa) {  // (shared-memory pass only)
    if (threadIdx.x == 0) { atomicAdd(overflow, 1); cnt[i] = -1; }
    return;
  }
  // this row's table: a power of two >= 2 x its product count (hrow), capped
  int hs = hrow[i];
  hs = hs < 32 ? 32 : (hs > hsmax ? hsmax : hs);
  for (int h = threadIdx.x; h < hs; h += blockDim.x) tab[h] = -1;
  for (int e = threadIdx.x; e < nA; e += blockDim.x) {
    int k = aci[t0 + e];
    sak[e] = k;
    sav[e] = av[t0 + e];
    soff[e + 1] = brp[k + 1] - brp[k];
  }
  if (threadIdx.x == 0) { count = 0; cursor = 0; bad = 0; }
  __syncthreads();
  if (threadIdx.x < 32) {  // inclusive scan of the B-row lengths by one warp
    int lane = threadIdx.x, carry = 0;
    if (lane == 0) soff[0] = 0;
    for (int base = 1; base <= nA; base += 32) {
      int idx = base + lane;
      int x = idx <= nA ? soff[idx] : 0;
      for (int o2 = 1; o2 < 32; o2 <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o2);
        if (lane >= o2) x += y;
      }
      if (idx <= nA) soff[idx] = x + carry;
      carry += __shfl_sync(0xffffffffu, x, 31);
    }
  }
  __syncthreads();
  const int total = soff[nA];
  // column set, one product per thread-iteration
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int lo = 0, hi = nA - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (soff[mid] <= e) lo = mid; else hi = mid - 1;
    }
    if (!set_insert(tab, hs, bci[brp[sak[lo]] + (e - soff[lo])], &count)) bad = 1;
  }
  __syncthreads();
  const int u = count;
  if (bad || 2 * u > hs) {  // (shared-memory pass only: the global tables hold every row)
    if (threadIdx.x == 0) { atomicAdd(overflow, 1); cnt[i] = -1; }
    return;
  }
  if (threadIdx.x == 0) cnt[i] = u;
  if (u == 0) return;  // no products: an empty output row
  set_to_sorted(tab, hs, list, tabpos, u, &cursor);
  for (int q = threadIdx.x; q < u; q += blockDim.x) {
    unsigned h = ((unsigned)list[q] * 2654435761u) & (unsigned)(hs - 1);
    while (tab[h] != list[q]) h = (h + 1u) & (unsigned)(hs - 1);
    tabpos[h] = q;
    acc[q] = 0.0;
  }
  __syncthreads();
  const int tsub = Ly.tcap / u;  // A entries per product table (1 <= u <= tcap)
  // products staged in segments of consecutive A entries; every product finds
  // its output column in the hash table, lands in tbl[A entry][column], and
  // each column adds its products in the order of the entries of A (absent
  // cells are skipped, as the definition skips them).  A single B row longer
  // than a segment is read from global memory by the column-owner loop.
  for (int ts = 0; ts < nA;) {
    int te = ts + 1;
    while (te < nA && soff[te + 1] - soff[ts] <= kSpgemmSeg) ++te;
    const int base = soff[ts];
    const bool fits = soff[te] - base <= kSpgemmSeg;
    if (fits) {
      for (int e = base + threadIdx.x; e < soff[te]; e += blockDim.x) {
        int lo = ts, hi = te - 1;
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (soff[mid] <= e) lo = mid; else hi = mid - 1;
        }
        int src = brp[sak[lo]] + (e - soff[lo]);
        int col = bci[src];
        sbc[e - base] = col;
        sbv[e - base] = bv[src];
        stt[e - base] = lo;
        spos[e - base] = chat_pos(tab, tabpos, hs, col);
      }
      __syncthreads();
      for (int tb = ts; tb < te; tb += tsub) {
        const int tbe = min(te, tb + tsub);
        for (int x = threadIdx.x; x < (tbe - tb) * u; x += blockDim.x) tbl[x] = tbl_absent();
        __syncthreads();
        for (int e = soff[tb] - base + threadIdx.x; e < soff[tbe] - base; e += blockDim.x)
          tbl[(size_t)(stt[e] - tb) * u + spos[e]] = sav[stt[e]] * sbv[e];
        __syncthreads();
        for (int q = threadIdx.x; q < u; q += blockDim.x) {
          double sum = acc[q];
          for (int t = tb; t < tbe; ++t) {
            const double x = tbl[(size_t)(t - tb) * u + q];
            if (tbl_present(x)) sum += x;
          }
          acc[q] = sum;
        }
        __syncthreads();
      }
    } else {
      for (int q = threadIdx.x; q < u; q += blockDim.x) {
        const int J = list[q];
        double sum = acc[q];
        for (int t = ts; t < te; ++t) {
          int k = sak[t];
          int pos = bsearch_row(bci, brp[k], brp[k + 1], J);
          if (pos >= 0) sum += sav[t] * bv[pos];
        }
        acc[q] = sum;
      }
      __syncthreads();
    }
    ts = te;
  }
  const long long o = toff[i];  // this row's slot: as many entries as it has products
  for (int q = threadIdx.x; q < u; q += blockDim.x) {
    cci[o + q] = list[q];
    cv[o + q] = acc[q];
  }
}

// Extended+i row of P for fine point i (same arithmetic and order as the
// thread-per-row kernel k_interp).  Row i and the rows of its strong F
// neighbours are staged in shared memory first (one parallel load round);
// the Chat set is built in a shared hash set and sorted; each neighbour's
// denominator is summed by one thread over its staged row; the weights are
// accumulated in push form, neighbour by neighbour in row order with a barrier
// in between (within one neighbour every target column is distinct), which
// reproduces the sequential order of the definition.
struct InterpSmem {
  size_t tab, tabpos, list, num, ri_c, ri_v, ri_f, inc, koff, kst, fk, akk, denz, abki, st_c,
      st_v, st_f, st_e, t_den, spos, tbl, total;
  int tcap;  // doubles of the distribution table
};
// tmin: smallest table of ordered sums (1024 doubles for wide blocks; the
// one-warp configuration for short rows uses a smaller one)
__host__ __device__ inline InterpSmem interp_layout(int hs, int rl, int kcap, int tmin = 1024) {
  InterpSmem L;
  size_t o = 0;
  auto take = [&](size_t b) { size_t at = o; o += (b + 15) & ~(size_t)15; return at; };
  L.tcap = hs / 2 + 1 > tmin ? hs / 2 + 1 : tmin;  // > nq (2 nq <= hs)
  L.tab = take(4 * (size_t)hs);
  L.tabpos = take(4 * (size_t)hs);
  L.list = take(4 * (size_t)(hs / 2));  // nq <= hs / 2 keys (bitonic padding included)
  L.num = take(8 * (size_t)(hs / 2));
  L.inc = take(4 * (size_t)rl);
  L.ri_c = take(4 * (size_t)rl);
  L.ri_v = take(8 * (size_t)rl);
  L.ri_f = take(4 * (size_t)rl);
  L.koff = take(4 * ((size_t)rl + 1));
  L.kst = take(4 * (size_t)rl);
  L.fk = take(8 * (size_t)rl);
  L.akk = take(8 * (size_t)rl);
  L.denz = take(4 * (size_t)rl);
  L.abki = take(8 * (size_t)rl);
  L.st_c = take(4 * (size_t)kcap);
  L.st_v = take(8 * (size_t)kcap);
  L.st_f = take(4 * (size_t)kcap);
  L.st_e = take(4 * (size_t)kcap);
  L.t_den = take(8 * (size_t)kcap);
  L.spos = take(4 * (size_t)kcap);
  L.tbl = take(8 * (size_t)L.tcap);
  L.total = o;
  return L;
}
enum { IF_S = 1, IF_SAME = 2, IF_C = 4, IF_DIAG = 8 };

// Per matrix entry (row r, column l) of one level, the facts ext+i looks up:
// strong (IF_S), func[l] == func[r] (IF_SAME), l a C point (IF_C), l == r
// (IF_DIAG).  One warp per row, coalesced.
template <int L>
__global__ void k_entry_flags(int n, const int32_t* __restrict__ rp,
                              const int32_t* __restrict__ ci, const uint8_t* __restrict__ S,
                              const int32_t* __restrict__ cf, const int32_t* __restrict__ func,
                              uint8_t* __restrict__ ef) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = (int)(g / L), lane = (int)(g % L);
  if (r >= n) return;
  const int fr = func[r];
  for (int t = rp[r] + lane; t < rp[r + 1]; t += L) {
    const int l = ci[t];
    ef[t] = (uint8_t)((S[t] ? IF_S : 0) | (func[l] == fr ? IF_SAME : 0) |
                      (cf[l] == 1 ? IF_C : 0) | (l == r ? IF_DIAG : 0));
  }
}

// L lanes per fine point (8, 16 or 32): ub[i] = candidate count of Chat_i
// (strong C neighbours plus the strong C of each strong F neighbour, with
// repeats) and the largest sum of the strong F neighbours' row lengths
// (*stage); integer counts, the same for any L.  A row's collectives use its
// own L lanes; every lane reaches the final sums.
template <int L>
__global__ void k_interp_sizes(int n, const int32_t* __restrict__ rp,
                               const int32_t* __restrict__ ci, const uint8_t* __restrict__ ef,
                               const int32_t* __restrict__ cf, int32_t* __restrict__ ub,
                               int* stage) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = (int)(g / L), lane = (int)(g % L);
  const bool valid = i < n;
  const unsigned base = (threadIdx.x & 31) & ~(unsigned)(L - 1);
  const unsigned smask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << base);
  if (valid && lane == 0) {  // longest row (the atomic only for a new maximum)
    const int len = rp[i + 1] - rp[i];
    if (len > ld_volatile_i32(stage + 2)) atomicMax(stage + 2, len);
  }
  int u = 0, sz = 0;
  if (valid && cf[i] != 1) {
    const int t1 = rp[i + 1];
    for (int t0 = rp[i]; t0 < t1; t0 += L) {
      const int t = t0 + lane;
      int j = -1;
      bool sf = false;  // strong F neighbour
      if (t < t1 && (ef[t] & IF_S)) {
        if (ef[t] & IF_C) ++u;
        else { j = ci[t]; sf = true; }
      }
      // the row's lanes scan each strong F neighbour's row together
      for (unsigned m = __ballot_sync(smask, sf); m; m &= m - 1) {
        const int k = __shfl_sync(smask, j, __ffs(m) - 1);
        const int b = rp[k], e = rp[k + 1];
        if (lane == 0) sz += e - b;
        for (int t2 = b + lane; t2 < e; t2 += L)
          if ((ef[t2] & (IF_S | IF_C)) == (IF_S | IF_C)) ++u;
      }
    }
  }
  for (int o = L / 2; o > 0; o >>= 1) {
    u += __shfl_xor_sync(0xffffffffu, u, o, L);
    sz += __shfl_xor_sync(0xffffffffu, sz, o, L);
  }
  if (valid && lane == 0) {
    ub[i] = u;
    if (sz > ld_volatile_i32(stage)) atomicMax(stage, sz);
    if (u > ld_volatile_i32(stage + 1)) atomicMax(stage + 1, u);  // largest candidate count
  }
}

// rows deferred by the shared-memory ext+i pass and the scratch each needs
__global__ void k_interp_deferred(int n, const int32_t* __restrict__ pcnt,
                                  const int32_t* __restrict__ rp, const int32_t* __restrict__ ub,
                                  int kcap, int32_t* __restrict__ rows,
                                  int32_t* __restrict__ bytes, int* nrows);
// Row and per-row scratch sizes of an F point's ext+i computation (GLOBAL
// pass): table >= 2 x its Chat candidates, arrays for its own row length.
__host__ __device__ inline int interp_hs(int ub) {
  int h = 64;
  while (h < 2 * ub) h <<= 1;
  return h;
}

// GLOBAL = false: one block per row, tables in shared memory sized for hsmax,
//   rl and kcap; a row that does not fit is deferred (pcnt = -1, *overflow
//   counts it).
// GLOBAL = true: one block per deferred row (rows[blockIdx.x]), its tables in
//   global scratch at gscr + goff[blockIdx.x], sized for that row.
__global__ void k_interp_deferred(int n, const int32_t* __restrict__ pcnt,
                                  const int32_t* __restrict__ rp, const int32_t* __restrict__ ub,
                                  int kcap, int32_t* __restrict__ rows,
                                  int32_t* __restrict__ bytes, int* nrows) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || pcnt[i] != -1) return;
  int k = atomicAdd(nrows, 1);
  rows[k] = i;
  size_t b = interp_layout(interp_hs(ub[i]), rp[i + 1] - rp[i], kcap).total;
  bytes[k] = (int32_t)((b + 255) & ~(size_t)255);
}

template <bool GLOBAL>
__global__ void k_interp_row(int n, int hsmax, const int32_t* __restrict__ ubrow, int rl,
                             int kcap, int tmin, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ ci, const double* __restrict__ v,
                             const uint8_t* __restrict__ ef, const int32_t* __restrict__ cf,
                             const int32_t* __restrict__ func, const int32_t* __restrict__ cidx,
                             int pmax, int32_t* __restrict__ pcnt, int32_t* __restrict__ pcol,
                             double* __restrict__ pval, int* overflow,
                             const int32_t* __restrict__ rows, const long long* __restrict__ goff,
                             unsigned char* __restrict__ gscr) {
  extern __shared__ __align__(16) unsigned char ism_dyn[];
  const int i = GLOBAL ? rows[blockIdx.x] : (int)blockIdx.x;
  if (i >= n) return;
  if (GLOBAL) {
    hsmax = interp_hs(ubrow[i]);
    rl = rp[i + 1] - rp[i];
  }
  unsigned char* ism = GLOBAL ? gscr + goff[blockIdx.x] : ism_dyn;
  const InterpSmem Ly = interp_layout(hsmax, rl, kcap, GLOBAL ? 1024 : tmin);
  int* tab = reinterpret_cast<int*>(ism + Ly.tab);
  int* list = reinterpret_cast<int*>(ism + Ly.list);
  double* num = reinterpret_cast<double*>(ism + Ly.num);
  int* ri_c = reinterpret_cast<int*>(ism + Ly.ri_c);
  double* ri_v = reinterpret_cast<double*>(ism + Ly.ri_v);
  int* ri_f = reinterpret_cast<int*>(ism + Ly.ri_f);
  int* koff = reinterpret_cast<int*>(ism + Ly.koff);
  int* kst = reinterpret_cast<int*>(ism + Ly.kst);
  double* fk = reinterpret_cast<double*>(ism + Ly.fk);
  double* akk = reinterpret_cast<double*>(ism + Ly.akk);
  int* denz = reinterpret_cast<int*>(ism + Ly.denz);
  double* abki = reinterpret_cast<double*>(ism + Ly.abki);
  int* st_c = reinterpret_cast<int*>(ism + Ly.st_c);
  double* st_v = reinterpret_cast<double*>(ism + Ly.st_v);
  int* st_f = reinterpret_cast<int*>(ism + Ly.st_f);
  int* tabpos = reinterpret_cast<int*>(ism + Ly.tabpos);
  int* inc = reinterpret_cast<int*>(ism + Ly.inc);
  int* st_e = reinterpret_cast<int*>(ism + Ly.st_e);
  double* t_den = reinterpret_cast<double*>(ism + Ly.t_den);
  int* spos = reinterpret_cast<int*>(ism + Ly.spos);
  double* tbl = reinterpret_cast<double*>(ism + Ly.tbl);
  __shared__ int count, cursor, bad;
  __shared__ double dg_s;
  if (cf[i] == 1) {
    if (threadIdx.x == 0) {
      pcnt[i] = 1;
      pcol[(size_t)i * pmax] = cidx[i];
      pval[(size_t)i * pmax] = 1.0;
    }
    return;
  }
  const int t0 = rp[i], t1 = rp[i + 1], ni = t1 - t0;
  if (ni > rl) {  // (shared-memory pass only)
    if (threadIdx.x == 0) { pcnt[i] = -1; atomicAdd(overflow, 1); }
    return;
  }
  int hs = 32;
  while (hs < 2 * ubrow[i] && hs < hsmax) hs <<= 1;
  // ---- stage row i: columns, values, flags; staged-row lengths of strong F neighbours
  for (int e = threadIdx.x; e < ni; e += blockDim.x) {
    const int j = ci[t0 + e];
    const int f = ef[t0 + e] & (IF_S | IF_SAME | IF_C);
    ri_c[e] = j;
    ri_v[e] = v[t0 + e];
    ri_f[e] = f;
    int len = 0;
    if ((f & IF_S) && !(f & IF_C)) {  // strong F neighbour: its row start and length
      const int b = rp[j];
      len = rp[j + 1] - b;
      kst[e] = b;
    }
    koff[e + 1] = len;
  }
  for (int h = threadIdx.x; h < hs; h += blockDim.x) tab[h] = -1;
  if (threadIdx.x == 0) { count = 0; cursor = 0; bad = 0; }
  __syncthreads();
  if (threadIdx.x < 32) {  // offsets of the staged rows (inclusive warp scan)
    int lane = threadIdx.x, carry = 0;
    if (lane == 0) koff[0] = 0;
    for (int base = 1; base <= ni; base += 32) {
      int idx = base + lane;
      int x = idx <= ni ? koff[idx] : 0;
      for (int o2 = 1; o2 < 32; o2 <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o2);
        if (lane >= o2) x += y;
      }
      if (idx <= ni) koff[idx] = x + carry;
      carry += __shfl_sync(0xffffffffu, x, 31);
    }
  }
  __syncthreads();
  const int K = koff[ni];
  // ---- Chat: strong C neighbours and the strong C of the strong F neighbours
  for (int e = threadIdx.x; e < ni; e += blockDim.x)
    if ((ri_f[e] & IF_S) && (ri_f[e] & IF_C))
      if (!set_insert(tab, hs, ri_c[e], &count)) bad = 1;
  // (four candidates per thread at a time, so that their loads overlap)
  for (int q0 = threadIdx.x; q0 < K; q0 += 4 * blockDim.x) {
    int src[4], col[4], fl[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = q0 + u * blockDim.x;
      src[u] = -1;
      if (q < K) {
        int lo = 0, hi = ni - 1;  // entry e with koff[e] <= q < koff[e+1]
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (koff[mid] <= q) lo = mid; else hi = mid - 1;
        }
        src[u] = kst[lo] + (q - koff[lo]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (src[u] >= 0) {
        fl[u] = ef[src[u]];
        col[u] = ci[src[u]];
      }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (src[u] >= 0 && (fl[u] & (IF_S | IF_C)) == (IF_S | IF_C))
        if (!set_insert(tab, hs, col[u], &count)) bad = 1;
  }
  __syncthreads();
  const int nq = count;
  if (bad || 2 * nq > hs) {  // (shared-memory pass only: a global table fits every row)
    if (threadIdx.x == 0) { pcnt[i] = -1; atomicAdd(overflow, 1); }
    return;
  }
  if (nq == 0) {
    if (threadIdx.x == 0) pcnt[i] = 0;
    return;
  }
  set_to_sorted(tab, hs, list, tabpos, nq, &cursor);
  for (int p = threadIdx.x; p < nq; p += blockDim.x) {
    unsigned h = ((unsigned)list[p] * 2654435761u) & (unsigned)(hs - 1);
    while (tab[h] != list[p]) h = (h + 1u) & (unsigned)(hs - 1);
    tabpos[h] = p;
  }
  // ---- direct terms a_ij, j in Chat (each column once per row)
  for (int p = threadIdx.x; p < nq; p += blockDim.x) num[p] = 0.0;
  __syncthreads();
  for (int e = threadIdx.x; e < ni; e += blockDim.x) {
    int j = ri_c[e];
    int pos = chat_pos(tab, tabpos, hs, j);
    inc[e] = pos >= 0;
    if (j == i || !(ri_f[e] & IF_SAME)) continue;
    if (pos >= 0) num[pos] += ri_v[e];
  }
  __syncthreads();
  // position of i among the sorted Chat columns (i is an F point, not in Chat)
  int ipos = 0;
  for (int hi = nq; ipos < hi;) {
    const int mid = (ipos + hi) >> 1;
    if (list[mid] < i) ipos = mid + 1; else hi = mid;
  }
  const int dw = nq + 1;          // positions of Chat u {i}
  const int dsub = Ly.tcap / dw;  // neighbours per denominator table (>= 1)
  // ---- strong F neighbours, staged in segments of at most kcap entries
  for (int es = 0; es < ni;) {
    int ee = es + 1;
    while (ee < ni && koff[ee + 1] - koff[es] <= kcap) ++ee;
    const int base = koff[es], kend = koff[ee];
    if (kend - base > kcap) {  // a neighbour row longer than the stage: deferred
      if (threadIdx.x == 0) { pcnt[i] = -1; atomicAdd(overflow, 1); }
      return;
    }
    for (int q0 = base + threadIdx.x; q0 < kend; q0 += 4 * blockDim.x) {
      int src[4], ent[4], col[4], fl[4];
      double val[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * blockDim.x;
        src[u] = -1;
        if (q < kend) {
          int lo = es, hi = ee - 1;
          while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (koff[mid] <= q) lo = mid; else hi = mid - 1;
          }
          src[u] = kst[lo] + (q - koff[lo]);
          ent[u] = lo;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (src[u] >= 0) {
          col[u] = ci[src[u]];
          val[u] = v[src[u]];
          fl[u] = ef[src[u]];  // relative to the neighbour's own row
        }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (src[u] >= 0) {
          const int q = q0 + u * blockDim.x - base;
          st_c[q] = col[u];
          st_v[q] = val[u];
          st_f[q] = fl[u];
          st_e[q] = ent[u];
        }
    }
    for (int e = es + threadIdx.x; e < ee; e += blockDim.x) {
      fk[e] = 0.0; denz[e] = 0; akk[e] = 0.0; abki[e] = 0.0;
    }
    __syncthreads();
    // a_kk of each strong F neighbour (its row holds one diagonal entry)
    for (int q = threadIdx.x; q < kend - base; q += blockDim.x) {
      const int e = st_e[q], fe = ri_f[e];
      if ((st_f[q] & IF_DIAG) && (fe & IF_S) && !(fe & IF_C)) akk[e] = st_v[q];
    }
    __syncthreads();
    // per staged entry: its term of the denominator sum_{l in Chat u {i}} abar_kl,
    // abar_ki, and the Chat position of l
    for (int q = threadIdx.x; q < kend - base; q += blockDim.x) {
      const int e = st_e[q], fe = ri_f[e], f = st_f[q], l = st_c[q];
      double td = 0.0;
      int sp = -1;
      if ((fe & IF_S) && !(fe & IF_C) && !(f & IF_DIAG) && (f & IF_SAME)) {
        const double ab = abar(akk[e], st_v[q]);
        if (l == i) {
          td = ab;
          abki[e] = ab;
        } else {
          const int pos = chat_pos(tab, tabpos, hs, l);
          if (pos >= 0) { td = ab; sp = pos; }
        }
      }
      t_den[q] = td;
      spos[q] = sp;
    }
    __syncthreads();
    // denominators in row order.  Only entries with l in Chat u {i} give a
    // nonzero term, and abar never returns -0.0, so the zero terms leave the
    // sum unchanged and are skipped.  Rows are sorted, so row order is the
    // order of l in the sorted set Chat u {i}: each batch of neighbours fills
    // a [neighbour][position] table with its nonzero terms and sums its row
    // of it, a chain of at most nq + 1 additions instead of the row length.
    // The same table then gives the distribution: column p of Chat adds
    // fk_e abar_kl of each neighbour e in row order, skipping absent cells
    // (and neighbours with a zero denominator) as the definition skips them.
    for (int eb = es; eb < ee; eb += dsub) {
      const int ebe = min(ee, eb + dsub);
      for (int x = threadIdx.x; x < (ebe - eb) * dw; x += blockDim.x) tbl[x] = tbl_absent();
      __syncthreads();
      for (int q = koff[eb] - base + threadIdx.x; q < koff[ebe] - base; q += blockDim.x) {
        const double td = t_den[q];
        if (d_eq0(td)) continue;
        const int sp = spos[q];  // < 0 with a nonzero term only for l == i
        const int pp = sp < 0 ? ipos : sp + (sp >= ipos ? 1 : 0);
        tbl[(size_t)(st_e[q] - eb) * dw + pp] = td;
      }
      __syncthreads();
      for (int e = eb + threadIdx.x; e < ebe; e += blockDim.x) {
        if (!(ri_f[e] & IF_S) || (ri_f[e] & IF_C)) continue;
        double den = 0.0;
        for (int p = 0; p < dw; ++p) {
          const double x = tbl[(size_t)(e - eb) * dw + p];
          if (tbl_present(x)) den += x;
        }
        if (d_eq0(den)) denz[e] = 1;
        else fk[e] = ri_v[e] / den;
      }
      __syncthreads();
      for (int p = threadIdx.x; p < nq; p += blockDim.x) {
        const int pp = p + (p >= ipos ? 1 : 0);
        double sum = num[p];
        for (int e = eb; e < ebe; ++e) {
          const double x = tbl[(size_t)(e - eb) * dw + pp];
          if (tbl_present(x) && !denz[e]) sum += fk[e] * x;
        }
        num[p] = sum;
      }
      __syncthreads();
    }
    es = ee;
  }
  // ---- diagonal: each entry's terms decided in parallel (inc[e] bit 0: the
  // first loop's term ri_v[e], bit 1: the second loop's term, kept in abki[e]),
  // then added by one thread in definition order
  for (int e = threadIdx.x; e < ni; e += blockDim.x) {
    const int j = ri_c[e], f = ri_f[e];
    int bits = 0;
    if (j == i || ((f & IF_SAME) && !inc[e] && !(f & IF_S))) bits |= 1;
    if ((f & IF_S) && !(f & IF_C)) {
      if (denz[e]) {
        abki[e] = ri_v[e];
        bits |= 2;
      } else if (!d_eq0(abki[e])) {
        abki[e] = fk[e] * abki[e];
        bits |= 2;
      }
    }
    inc[e] = bits;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double dgt = 0.0;
    for (int e = 0; e < ni; ++e)
      if (inc[e] & 1) dgt += ri_v[e];
    for (int e = 0; e < ni; ++e)
      if (inc[e] & 2) dgt += abki[e];
    dg_s = dgt;
  }
  __syncthreads();
  const double dg = dg_s;
  if (d_eq0(dg) || dmag(dg) >= 0x7ff0000000000000ull) {  // zero or not finite
    if (threadIdx.x == 0) pcnt[i] = 0;
    return;
  }
  for (int p = threadIdx.x; p < nq; p += blockDim.x) num[p] = -num[p] / dg;
  __syncthreads();
  if (threadIdx.x >= 32) return;
  // ---- one warp: drop exact zeros, then truncate to the pmax largest |w|
  const int lane = threadIdx.x;
  double* wv = num;
  int m = 0;
  for (int p0 = 0; p0 < nq; p0 += 32) {
    const int p = p0 + lane;
    const bool nz = p < nq && !d_eq0(wv[p]);
    const double w = nz ? wv[p] : 0.0;
    const int col = nz ? list[p] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, nz);
    __syncwarp();
    if (nz) {
      const int d = m + __popc(bal & ((1u << lane) - 1u));
      list[d] = col;
      wv[d] = w;
    }
    m += __popc(bal);
    __syncwarp();
  }
  if (m <= pmax) {
    for (int a = lane; a < m; a += 32) {
      pcol[(size_t)i * pmax + a] = cidx[list[a]];
      pval[(size_t)i * pmax + a] = wv[a];
    }
    if (lane == 0) pcnt[i] = m;
    return;
  }
  const int keep = pmax < 64 ? pmax : 64;
  int* ord = tabpos;  // free now; keep < m <= nq < hs entries
  bool anynan = false;
  for (int p = lane; p < m; p += 32) anynan |= d_isnan(wv[p]);
  if (!__any_sync(0xffffffffu, anynan)) {
    // the picks in order of (|w| descending, index ascending): each round
    // takes the largest entry below the previous pick, by |w| bit patterns
    unsigned long long pm = 0;
    int pi = -1;
    for (int a = 0; a < keep; ++a) {
      unsigned long long bm = 0;
      int bi = -1;
      for (int p = lane; p < m; p += 32) {
        const unsigned long long mg = dmag(wv[p]);
        if (a > 0 && !(mg < pm || (mg == pm && p > pi))) continue;
        if (bi < 0 || mg > bm) { bm = mg; bi = p; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long om = __shfl_xor_sync(0xffffffffu, bm, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (bi < 0 || om > bm || (om == bm && oi < bi))) { bm = om; bi = oi; }
      }
      pm = bm;
      pi = bi;
      if (lane == 0) ord[a] = bi;
    }
  } else if (lane == 0) {
    // a NaN weight: the definition's comparisons, one by one
    for (int a = 0; a < keep; ++a) {
      int best = -1;
      for (int b2 = 0; b2 < m; ++b2) {
        bool taken = false;
        for (int c2 = 0; c2 < a; ++c2) taken |= (ord[c2] == b2);
        if (taken) continue;
        if (best < 0) { best = b2; continue; }
        double wb = fabs(wv[b2]), wa = fabs(wv[best]);
        if (wb > wa || (wb == wa && b2 < best)) best = b2;
      }
      ord[a] = best;
    }
  }
  __syncwarp();
  double scale = 1.0;
  if (lane == 0) {
    for (int a = 1; a < keep; ++a) {
      int key = ord[a], b = a - 1;
      while (b >= 0 && ord[b] > key) { ord[b + 1] = ord[b]; --b; }
      ord[b + 1] = key;
    }
    // both sums in index order, as one walk (ord is ascending), so that the
    // two dependent chains overlap
    double sum_all = 0.0, sum_kept = 0.0;
    for (int t = 0, a = 0; t < m; ++t) {
      const double w = wv[t];
      if (a < keep && ord[a] == t) { sum_kept += w; ++a; }
      sum_all += w;
    }
    scale = d_eq0(sum_kept) ? 1.0 : sum_all / sum_kept;
    pcnt[i] = keep;
  }
  scale = __shfl_sync(0xffffffffu, scale, 0);
  __syncwarp();
  for (int a = lane; a < keep; a += 32) {
    pcol[(size_t)i * pmax + a] = cidx[list[ord[a]]];
    pval[(size_t)i * pmax + a] = wv[ord[a]] * scale;
  }
}

// ------------------------------------------------------------------ l1, coarse
__global__ void k_l1(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                     const double* __restrict__ v, double* __restrict__ d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double aii = 0.0, off = 0.0;
  for (int t = rp[i]; t < rp[i + 1]; ++t) {
    if (ci[t] == i) aii = v[t];
    else off += fabs(v[t]);
  }
  d[i] = (aii < 0.0) ? aii - off : aii + off;
}

// ---- one aggregate level: truncation of P = P1 P2 and the final split ----
// Per row, the ext+i truncation rule in the order of the oracle's truncate_rows:
// exact zeros dropped, the sum of all entries, the pmax largest |w| (ties: the
// smaller column) by selection, kept entries in column order, their sum, and
// the rescaling by sum_all / sum_kept (one thread per row; rows are short).
__global__ void k_trunc_count(int n, const int32_t* __restrict__ rp, const double* __restrict__ v,
                              int pmax, int32_t* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int m = 0;
  for (int t = rp[i]; t < rp[i + 1]; ++t) m += !d_eq0(v[t]);
  cnt[i] = m < pmax ? m : pmax;
}

__global__ void k_trunc_fill(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ v, int pmax, int32_t* __restrict__ ord,
                             const int32_t* __restrict__ orp, int32_t* __restrict__ oci,
                             double* __restrict__ ov) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int t0 = rp[i];
  int* o = ord + t0;
  int m = 0;
  for (int t = t0; t < rp[i + 1]; ++t)
    if (!d_eq0(v[t])) o[m++] = t;
  const int q = orp[i];
  if (m <= pmax) {
    for (int a = 0; a < m; ++a) {
      oci[q + a] = ci[o[a]];
      ov[q + a] = v[o[a]];
    }
    return;
  }
  double sum_all = 0.0;
  for (int k = 0; k < m; ++k) sum_all += v[o[k]];
  for (int a = 0; a < pmax; ++a) {
    int best = a;
    for (int b = a + 1; b < m; ++b) {
      double wb = fabs(v[o[b]]), wa = fabs(v[o[best]]);
      if (wb > wa || (wb == wa && o[b] < o[best])) best = b;
    }
    int tmp = o[a];
    o[a] = o[best];
    o[best] = tmp;
  }
  for (int a = 1; a < pmax; ++a) {  // kept entries back in column (position) order
    int x = o[a], b = a - 1;
    while (b >= 0 && o[b] > x) {
      o[b + 1] = o[b];
      --b;
    }
    o[b + 1] = x;
  }
  double sum_kept = 0.0;
  for (int a = 0; a < pmax; ++a) sum_kept += v[o[a]];
  const double scale = d_eq0(sum_kept) ? 1.0 : sum_all / sum_kept;
  for (int a = 0; a < pmax; ++a) {
    oci[q + a] = ci[o[a]];
    ov[q + a] = v[o[a]] * scale;
  }
}

// A first-stage C point stays C only if the second stage keeps it.
__global__ void k_agg_cf(int n, int32_t* __restrict__ cf0, const int32_t* __restrict__ cidx0,
                         const int32_t* __restrict__ cf1) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && cf0[i] == 1 && cf1[cidx0[i]] != 1) cf0[i] = -1;
}

// ---- aggressive first level (agg = 2): distance-two strength among the C
// points, and multipass interpolation ----
__global__ void k_strong_count(int n, const int32_t* __restrict__ rp, const uint8_t* __restrict__ S,
                               int32_t* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int m = 0;
  for (int t = rp[i]; t < rp[i + 1]; ++t) m += S[t] ? 1 : 0;
  cnt[i] = m;
}

// B: the strong pattern with unit values
__global__ void k_strong_fill(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const uint8_t* __restrict__ S, const int32_t* __restrict__ brp,
                              int32_t* __restrict__ bci, double* __restrict__ bv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int q = brp[i];
  for (int t = rp[i]; t < rp[i + 1]; ++t)
    if (S[t]) { bci[q] = ci[t]; bv[q] = 1.0; ++q; }
}

// Row i of G (C point i): the C points j != i in the union of the sorted
// rows i of B and of B B (distance one or two in the strength graph), in
// column order; counted (gci == nullptr) or written in C numbering.
__global__ void k_g2_row(int n, const int32_t* __restrict__ cf, const int32_t* __restrict__ cidx,
                         const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                         const int32_t* __restrict__ b2rp, const int32_t* __restrict__ b2ci,
                         const int32_t* __restrict__ grp, int32_t* __restrict__ gcnt,
                         int32_t* __restrict__ gci) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cf[i] != 1) return;
  int a = brp[i], ae = brp[i + 1], b = b2rp[i], be = b2rp[i + 1];
  int q = gci ? grp[cidx[i]] : 0, m = 0;
  while (a < ae || b < be) {
    int j;
    if (b >= be || (a < ae && bci[a] < b2ci[b])) j = bci[a++];
    else if (a >= ae || b2ci[b] < bci[a]) j = b2ci[b++];
    else { j = bci[a]; ++a; ++b; }
    if (j == i || cf[j] != 1) continue;
    if (gci) gci[q + m] = cidx[j];
    ++m;
  }
  if (!gci) gcnt[cidx[i]] = m;
}

__global__ void k_col_count(int nnz, const int32_t* __restrict__ ci, int32_t* __restrict__ cnt) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nnz) atomicAdd(&cnt[ci[t]], 1);
}

__global__ void k_isc_from_cf(int n, const int32_t* __restrict__ cf, int32_t* __restrict__ isc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) isc[i] = cf[i] == 1;
}

// Multipass: pass 0 for C points, -1 for points not yet interpolated; rows
// of C points are unit rows.
__global__ void k_mp_init(int n, const int32_t* __restrict__ cf, const int32_t* __restrict__ cidx,
                          int32_t* __restrict__ pass, int32_t* __restrict__ qcnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  pass[i] = cf[i] == 1 ? 0 : -1;
  qcnt[i] = cf[i] == 1 ? 1 : 0;
}

__global__ void k_unit_rows(int n, const int32_t* __restrict__ cf, const int32_t* __restrict__ cidx,
                            const int32_t* __restrict__ qrp, int32_t* __restrict__ qci,
                            double* __restrict__ qv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cf[i] != 1) return;
  qci[qrp[i]] = cidx[i];
  qv[qrp[i]] = 1.0;
}

// The points pass ps reaches: not yet interpolated, with strong dependencies
// interpolated in earlier passes (their number is the row's weight count).
__global__ void k_mp_count(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const uint8_t* __restrict__ S, const int32_t* __restrict__ pass, int ps,
                           int32_t* __restrict__ newp, int32_t* __restrict__ wcnt, int* reached) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int nk = 0;
  if (pass[i] < 0)
    for (int t = rp[i]; t < rp[i + 1]; ++t) nk += (S[t] && pass[ci[t]] >= 0) ? 1 : 0;
  wcnt[i] = nk;
  newp[i] = nk > 0 ? ps : pass[i];
  if (nk > 0) atomicAdd(reached, 1);
}

// The pass's weights, in the oracle's order: sumK over the interpolated
// strong dependencies, sumN over the same-function couplings of sign
// opposite to a_ii, d = a_ii plus those of the same sign (column order each);
// w_ik = -(alpha a_ik) / d with alpha = sumN / sumK.
__global__ void k_mp_fill(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ v, const uint8_t* __restrict__ S,
                          const int32_t* __restrict__ func, const int32_t* __restrict__ pass,
                          const int32_t* __restrict__ wrp, int32_t* __restrict__ wci,
                          double* __restrict__ wv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || wrp[i + 1] == wrp[i]) return;
  const int t0 = rp[i], t1 = rp[i + 1], fi = func[i];
  double aii = 0.0;
  for (int t = t0; t < t1; ++t)
    if (ci[t] == i) { aii = v[t]; break; }
  const bool neg = aii < 0.0;
  double sumK = 0.0, sumN = 0.0, d = aii;
  for (int t = t0; t < t1; ++t)
    if (S[t] && pass[ci[t]] >= 0) sumK += v[t];
  for (int t = t0; t < t1; ++t) {
    int j = ci[t];
    if (j == i || func[j] != fi) continue;
    double sa = neg ? -v[t] : v[t];
    if (sa < 0.0) sumN += v[t];
  }
  for (int t = t0; t < t1; ++t) {
    int j = ci[t];
    if (j == i || func[j] != fi) continue;
    double sa = neg ? -v[t] : v[t];
    if (sa > 0.0) d += v[t];
  }
  const double alpha = sumN / sumK;
  int q = wrp[i];
  for (int t = t0; t < t1; ++t)
    if (S[t] && pass[ci[t]] >= 0) {
      wci[q] = ci[t];
      wv[q] = -(alpha * v[t]) / d;
      ++q;
    }
}

// The rows after the pass: the pass's new rows from W Q, the others from Q.
__global__ void k_mp_merge(int n, int ps, const int32_t* __restrict__ pass,
                           const int32_t* __restrict__ newp, const int32_t* __restrict__ qrp,
                           const int32_t* __restrict__ qci, const double* __restrict__ qv,
                           const int32_t* __restrict__ wqrp, const int32_t* __restrict__ wqci,
                           const double* __restrict__ wqv, const int32_t* __restrict__ orp,
                           int32_t* __restrict__ ocnt, int32_t* __restrict__ oci,
                           double* __restrict__ ov) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool fresh = newp[i] == ps && pass[i] < 0;
  const int32_t* rp = fresh ? wqrp : qrp;
  const int32_t* ci = fresh ? wqci : qci;
  const double* v = fresh ? wqv : qv;
  if (!oci) { ocnt[i] = rp[i + 1] - rp[i]; return; }
  int q = orp[i];
  for (int t = rp[i]; t < rp[i + 1]; ++t, ++q) {
    oci[q] = ci[t];
    ov[q] = v[t];
  }
}

__global__ void k_coarse_func(int n, const int32_t* __restrict__ cf, const int32_t* __restrict__ cidx,
                              const int32_t* __restrict__ f, int32_t* __restrict__ fc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && cf[i] == 1) fc[cidx[i]] = f[i];
}

__global__ void k_dense_fill(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ v, double* __restrict__ M) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  size_t w = 2 * (size_t)n;
  for (int c = 0; c < 2 * n; ++c) M[i * w + c] = (c == n + i) ? 1.0 : 0.0;
  for (int t = rp[i]; t < rp[i + 1]; ++t) M[i * w + ci[t]] += v[t];
}

// Gauss-Jordan inversion with partial pivoting on [M | I] (one block of 1024
// threads, seen as 32 rows x 32 columns of threads).  At step k the columns
// left of k are unit columns already, so only columns k..2n-1 are updated; the
// normalised pivot row and the column factors are staged in shared memory.
__global__ void __launch_bounds__(1024) k_gauss_jordan(int n, double* __restrict__ M,
                                                       double* __restrict__ inv, int* status) {
  extern __shared__ double gj_sh[];  // pivot row [2n] | column factors [n]
  double* prow = gj_sh;
  double* fcol = gj_sh + 2 * n;
  __shared__ double bval[1024];
  __shared__ int bidx[1024];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int w = 2 * n;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = n;
    for (int r = k + tid; r < n; r += blockDim.x) {
      double a = fabs(M[(size_t)r * w + k]);
      if (a > best) { best = a; bi = r; }
    }
    bval[tid] = best;
    bidx[tid] = bi;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (tid < st) {
        double o = bval[tid + st];
        int oi = bidx[tid + st];
        if (o > bval[tid] || (o == bval[tid] && oi < bidx[tid])) {
          bval[tid] = o;
          bidx[tid] = oi;
        }
      }
      __syncthreads();
    }
    const int p = bidx[0];
    const double pb = bval[0];
    __syncthreads();
    if (!(pb > 0.0) || !isfinite(pb) || p >= n) {
      if (tid == 0) dev_fail(status, DEV_BREAKDOWN);
      return;
    }
    // rows k..n-1 hold zeros left of column k: swap and scale from column k on
    const double piv = M[(size_t)p * w + k];
    __syncthreads();
    for (int c = k + tid; c < w; c += blockDim.x) {
      double vk = M[(size_t)k * w + c], vp = M[(size_t)p * w + c];
      if (p != k) M[(size_t)p * w + c] = vk;
      double v = vp / piv;
      prow[c] = v;
      M[(size_t)k * w + c] = v;
    }
    __syncthreads();
    for (int r = tid; r < n; r += blockDim.x) fcol[r] = (r == k) ? 0.0 : M[(size_t)r * w + k];
    __syncthreads();
    for (int r = ty; r < n; r += 32) {
      const double f = fcol[r];
      if (f != 0.0) {
        double* Mr = M + (size_t)r * w;
        for (int c = k + tx; c < w; c += 32) Mr[c] -= f * prow[c];
      }
    }
    __syncthreads();
  }
  for (int r = ty; r < n; r += 32)
    for (int c = tx; c < n; c += 32) inv[(size_t)r * n + c] = M[(size_t)r * w + n + c];
}

// Gauss-Jordan on one cluster of kGjCtas CTAs, the augmented matrix [M | I]
// held in their shared memory: CTA q owns columns [q w, q w + w) of the n x 2n
// matrix (row-major slice).  Step k: the owner of column k finds the pivot in
// its slice; after a cluster barrier every CTA reads the pivot row index and
// the column-k factors through DSMEM; after a second barrier every CTA swaps,
// scales and updates its own columns.  Same operations per element as
// k_gauss_jordan, so the inverse is bit-identical to it.
constexpr int kGjCtas = 16;
constexpr int kGjThreads = 512;
__device__ __forceinline__ void gj_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ unsigned gj_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
template <class V>
__device__ __forceinline__ V gj_remote(const V* local_ptr, unsigned rank) {
  unsigned la = (unsigned)__cvta_generic_to_shared(local_ptr), ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
  V v;
  if (sizeof(V) == 8) {
    unsigned long long x;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(x) : "r"(ra) : "memory");
    memcpy(&v, &x, 8);
  } else {
    unsigned x;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(x) : "r"(ra) : "memory");
    memcpy(&v, &x, 4);
  }
  return v;
}
template <class V>
__device__ __forceinline__ void gj_push(V* local_ptr, unsigned rank, V v) {
  unsigned la = (unsigned)__cvta_generic_to_shared(local_ptr), ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
  if (sizeof(V) == 8) {
    unsigned long long x;
    memcpy(&x, &v, 8);
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(ra), "l"(x) : "memory");
  } else {
    unsigned x;
    memcpy(&x, &v, 4);
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(ra), "r"(x) : "memory");
  }
}
// Gauss-Jordan with partial pivoting of [M | I] on one cluster, each CTA
// holding a slice of w columns in shared memory.  At step k the CTA owning
// column k picks the pivot with one warp (largest |a_rk|, ties to the smaller
// row), and pushes the pivot row index, the pivot and the column-k factors of
// the swapped matrix into every CTA's double-buffered arrays; one cluster
// barrier publishes them (passing step k-1's barrier means every CTA has
// finished step k-2, so buffer k & 1 is free).  Each CTA then swaps, scales
// and eliminates its own slice.
__global__ void __launch_bounds__(kGjThreads) k_gauss_jordan_cluster(int n, int w,
                                                                     const double* __restrict__ M,
                                                                     double* __restrict__ inv,
                                                                     int* status) {
  extern __shared__ __align__(16) double gjs[];
  double* S = gjs;                      // n x w slice
  double* fcolb = gjs + (size_t)n * w;  // 2 x n pushed column-k factors
  __shared__ int s_p[2];
  __shared__ double s_piv[2];
  __shared__ int own_p;
  const unsigned q = gj_rank();
  const int tid = threadIdx.x;
  const int c0 = (int)q * w, W = 2 * n;
  const int wq = max(0, min(w, W - c0));
  for (size_t x = tid; x < (size_t)n * w; x += blockDim.x) {
    int r = (int)(x / w), cc = (int)(x % w);
    S[x] = cc < wq ? M[(size_t)r * W + c0 + cc] : 0.0;
  }
  __syncthreads();
  gj_cluster_sync();  // every slice filled before any push or DSMEM access
  bool failed = false;
  for (int k = 0; k < n; ++k) {
    const unsigned o = (unsigned)(k / w);  // owner of column k
    const int b = k & 1;
    if (q == o) {
      const int kc = k - c0;
      if (tid < 32) {
        double best = -1.0;
        int bi = n;
        for (int r = k + tid; r < n; r += 32) {
          const double a = fabs(S[(size_t)r * w + kc]);
          if (a > best) { best = a; bi = r; }
        }
        for (int off = 16; off > 0; off >>= 1) {
          const double ov = __shfl_xor_sync(0xffffffffu, best, off);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
          if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (tid == 0) own_p = (best > 0.0 && isfinite(best) && bi < n) ? bi : -1;
      }
      __syncthreads();
      const int p = own_p;
      // column k of the matrix with rows k and p swapped, with 0 at row k
      for (int x = tid; x < kGjCtas * n; x += blockDim.x) {
        const int dst = x / n, r = x % n;
        const int src = (r == k) ? p : (r == p ? k : r);
        const double f = (r == k || p < 0) ? 0.0 : S[(size_t)src * w + kc];
        gj_push(&fcolb[(size_t)b * n + r], (unsigned)dst, f);
      }
      if (tid < kGjCtas) {
        gj_push(&s_p[b], (unsigned)tid, p);
        gj_push(&s_piv[b], (unsigned)tid, p >= 0 ? S[(size_t)p * w + kc] : 0.0);
      }
    }
    gj_cluster_sync();
    const int p = s_p[b];
    if (p < 0) { failed = true; break; }  // every CTA reads the same value
    const double piv = s_piv[b];
    const double* fcol = fcolb + (size_t)b * n;
    // swap rows k and p, scale row k (the pivot row), from column k on
    const int cstart = max(0, k - c0);
    for (int cc = cstart + tid; cc < wq; cc += blockDim.x) {
      double vk = S[(size_t)k * w + cc], vp = S[(size_t)p * w + cc];
      if (p != k) S[(size_t)p * w + cc] = vk;
      S[(size_t)k * w + cc] = vp / piv;
    }
    __syncthreads();
    const int nc = wq - cstart;
    if (nc > 0) {
      for (size_t x = tid; x < (size_t)n * nc; x += blockDim.x) {
        const int r = (int)(x / nc), cc = cstart + (int)(x % nc);
        const double f = fcol[r];
        if (f != 0.0) S[(size_t)r * w + cc] -= f * S[(size_t)k * w + cc];
      }
    }
    __syncthreads();
  }
  if (failed && q == 0 && tid == 0) dev_fail(status, DEV_BREAKDOWN);
  gj_cluster_sync();  // no CTA leaves while another may still write into it
  if (failed) return;
  for (size_t x = tid; x < (size_t)n * wq; x += blockDim.x) {
    const int r = (int)(x / wq), cc = (int)(x % wq);
    const int col = c0 + cc;
    if (col >= n) inv[(size_t)r * n + (col - n)] = S[(size_t)r * w + cc];
  }
}

inline int nblk(long long n) { return n > 0 ? ceil_div(n, kT) : 1; }

// A product's distinct column count is at most its product count `bound`;
// where that passes 2^31 - 1 the 32-bit row pointers could wrap, so the exact
// count is taken in 64 bits first and a total past the limit is refused (the
// buffers sized from a wrapped total would be too small).
cptr_status check_count_fits(cptr_ctx* c, const int32_t* cnt, int n, long long bound) {
  if (bound <= INT32_MAX) return CPTR_OK;
  long long* wide_off;
  CTX_ALLOC(c, wide_off, long long, n + 1, true);
  long long wide = 0;
  cptr_status st = scan_i64(c, cnt, wide_off, n, &wide);
  if (st) return st;
  if (wide > INT32_MAX) {
    ctx_set_err(c, "a sparse product of the AMG setup has more than 2^31 - 1 entries");
    return CPTR_ERR_NOMEM;
  }
  return CPTR_OK;
}

// C = A * B with bounded scratch: rows are processed in batches whose hash
// tables fit in kCap slots.
cptr_status spgemm_fallback(cptr_ctx* c, const DCSR& A, const DCSR& B, DCSR& C);

// C = A * B: block-per-row symbolic count, row pointers, block-per-row fill;
// falls back to the batched thread-per-row hash kernel when a row's column
// set does not fit in shared memory.
cptr_status spgemm(cptr_ctx* c, const DCSR& A, const DCSR& B, DCSR& C) {
  if (c->force_fallback) return spgemm_fallback(c, A, B, C);
  int n = A.n;
  int32_t *hs, *cnt;
  int* flags;
  int32_t* prods;
  CTX_ALLOC(c, hs, int32_t, n + 1, true);
  CTX_ALLOC(c, cnt, int32_t, n + 1, true);
  CTX_ALLOC(c, prods, int32_t, n + 1, true);
  CTX_ALLOC(c, flags, int, 8, true);
  CTX_CUDA(c, cudaMemsetAsync(flags, 0, 8 * sizeof(int), c->stream));
  KL(c, k_spgemm_ub<<<nblk(n), kT, 0, c->stream>>>(n, A.rp, A.ci, B.rp, hs, prods, B.m,
                                                    flags + 4));
  cptr_status st;
  // product offsets; the maxima and the product total come back in one read
  long long* toff;
  CTX_ALLOC(c, toff, long long, n + 1, true);
  st = scan_i64(c, prods, toff, n, nullptr);
  if (st) return st;
  struct {
    int mx3[3];
    int pad;
    long long nprod;
  } hv;
  CTX_CUDA(c, cudaMemcpyAsync(hv.mx3, flags + 4, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                              c->stream));
  CTX_CUDA(c, cudaMemcpyAsync(&hv.nprod, toff + n, sizeof(long long), cudaMemcpyDeviceToHost,
                              c->stream));
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  const int* mx3 = hv.mx3;
  const long long nprod = hv.nprod;
  const int kSmemHs = 4096, kSmemRow = 1024, kSmemProd = 1024;  // shared-memory pass limits
  const int mx = mx3[0];
  int hsz = mx < 64 ? 64 : (mx > kSmemHs ? kSmemHs : mx);
  int thr = hsz >= 2048 ? 256 : 128;
  int tprod = 64;
  while (tprod < mx3[1] && tprod < kSmemProd) tprod <<= 1;
  int maxa = mx3[2] < 1 ? 1 : (mx3[2] > kSmemRow ? kSmemRow : mx3[2]);
  const size_t ssm = sps_layout(hsz, tprod, maxa).total;
  // one pass: every row writes its sorted columns into a slot as long as its
  // product count, then the rows are compacted behind the row pointers
  int32_t* tci;
  double* tv;
  CTX_ALLOC(c, tci, int32_t, nprod + 1, true);
  CTX_ALLOC(c, tv, double, nprod + 1, true);
  // rows with few products: one warp per row, the others one block per row
  // (the warp pass runs when the average row has at most kSpwProd products);
  // rows too large for shared memory are deferred (flags[0] counts them)
  // Bucketing pays where the ordered-product table wastes the most: long A
  // rows (the table's column sums scan every A entry) or few products per
  // row; short A rows with many products (R (AP) on coarse levels) keep the
  // table kernel, whose shared memory does not grow with the product count.
  const bool bucketed = c->spgemm_path == 2 ||
                        (c->spgemm_path == 0 && (A.nnz >= 16ll * n || nprod <= 256ll * n));
  size_t tsm = 0;
  if (!bucketed) {
    tsm = spgemm_smem(hsz, maxa);
    CTX_CUDA(c, cudaFuncSetAttribute(k_spgemm_row<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  }
  int32_t* brows = nullptr;
  int nb = c->spgemm_path == 3 ? 0 : n;
  if (c->spgemm_path == 3) {  // every row to the global-scratch pass
    CTX_CUDA(c, cudaMemsetAsync(cnt, 0xff, sizeof(int32_t) * n, c->stream));
    CTX_CUDA(c, cudaMemcpyAsync(flags, &n, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  } else if (c->spgemm_path == 0 && nprod <= (long long)kSpwProd * n) {
    CTX_ALLOC(c, brows, int32_t, n + 1, true);
    KL(c, k_spgemm_warp<<<nblk((long long)n * 32), 32 * kSpwWarps, 0, c->stream>>>(
              n, A.rp, A.ci, A.v, B.rp, B.ci, B.v, prods, toff, tci, tv, cnt, brows, flags + 3));
    CTX_CUDA(c, cudaMemcpyAsync(&nb, flags + 3, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  if (bucketed)
    CTX_CUDA(c, raise_smem_limit(c, (const void*)k_spgemm_sorted));
  if (nb > 0 && bucketed)
    KL(c, k_spgemm_sorted<<<nb, thr, ssm, c->stream>>>(hsz, tprod, maxa, hs, A.rp, A.ci, A.v,
                                                       B.rp, B.ci, B.v, prods, toff, tci, tv, cnt,
                                                       flags, brows));
  else if (nb > 0)
    KL(c, k_spgemm_row<false><<<nb, thr, tsm, c->stream>>>(hsz, maxa, hs, A.rp, A.ci, A.v, B.rp,
                                                            B.ci, B.v, toff, tci, tv, cnt, flags,
                                                            brows, nullptr, nullptr));
  int ndef = 0;
  CTX_CUDA(c, cudaMemcpyAsync(&ndef, flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  if (ndef > 0) {
    // rows too wide for shared memory: the same algorithm, tables in global scratch
    int32_t *rows, *rbytes;
    long long *goff, *rb64;
    CTX_ALLOC(c, rows, int32_t, ndef + 1, true);
    CTX_ALLOC(c, rb64, long long, ndef + 1, true);
    CTX_ALLOC(c, rbytes, int32_t, ndef + 1, true);
    CTX_ALLOC(c, goff, long long, ndef + 1, true);
    CTX_CUDA(c, cudaMemsetAsync(flags + 2, 0, sizeof(int), c->stream));
    KL(c, k_spgemm_deferred<<<nblk(n), kT, 0, c->stream>>>(n, cnt, A.rp, hs, rows, rb64,
                                                            flags + 2));
    KL(c, k_i64_to_i32<<<nblk(ndef), kT, 0, c->stream>>>(ndef, rb64, rbytes));
    long long gtot = 0;
    st = scan_i64(c, rbytes, goff, ndef, &gtot);
    if (st) return st;
    unsigned char* gscr = (unsigned char*)ctx_alloc(c, (size_t)gtot + 256, true);
    if (!gscr) return CPTR_ERR_NOMEM;
    CTX_CUDA(c, cudaMemsetAsync(flags + 1, 0, sizeof(int), c->stream));
    KL(c, k_spgemm_row<true><<<ndef, 256, 0, c->stream>>>(0, 0, hs, A.rp, A.ci, A.v, B.rp, B.ci,
                                                          B.v, toff, tci, tv, cnt, flags + 1,
                                                          rows, goff, gscr));
    int left = 0;  // a deferred row that overflowed again would leave cnt = -1
    CTX_CUDA(c, cudaMemcpyAsync(&left, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CTX_CUDA(c, cudaStreamSynchronize(c->stream));
    if (left) return spgemm_fallback(c, A, B, C);
    CTX_CUDA(c, cudaGetLastError());
  }
  C.n = n;
  C.m = B.m;
  st = check_count_fits(c, cnt, n, nprod);
  if (st) return st;
  CTX_ALLOC(c, C.rp, int32_t, n + 1, true);
  int total = 0;
  st = scan_i32(c, cnt, C.rp, n, &total);
  if (st) return st;
  C.nnz = total;
  CTX_ALLOC(c, C.ci, int32_t, total + 1, true);
  CTX_ALLOC(c, C.v, double, total + 1, true);
  KL(c, k_spgemm_compact<<<nblk((long long)n * 32), kT, 0, c->stream>>>(n, toff, cnt, tci, tv,
                                                                        C.rp, C.ci, C.v));
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

cptr_status spgemm_fallback(cptr_ctx* c, const DCSR& A, const DCSR& B, DCSR& C) {
  const long long kCap = 1ll << 26;
  int n = A.n;
  int32_t* hs;
  long long* hoff;
  int32_t* cnt;
  CTX_ALLOC(c, hs, int32_t, n + 1, true);
  CTX_ALLOC(c, hoff, long long, n + 1, true);
  CTX_ALLOC(c, cnt, int32_t, n + 1, true);
  KL(c, k_spgemm_ub<<<nblk(n), kT, 0, c->stream>>>(n, A.rp, A.ci, B.rp, hs, nullptr, 0));
  long long tot = 0;
  cptr_status st = scan_i64(c, hs, hoff, n, &tot);
  if (st) return st;
  std::vector<long long> ho(n + 1);
  CTX_CUDA(c, cudaMemcpyAsync(ho.data(), hoff, sizeof(long long) * (n + 1),
                              cudaMemcpyDeviceToHost, c->stream));
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  long long maxrow = 0;
  for (int i = 0; i < n; ++i) maxrow = std::max(maxrow, ho[i + 1] - ho[i]);
  long long cap = std::max(std::min(tot, kCap), maxrow);
  int32_t* hcol;
  double* hval;
  CTX_ALLOC(c, hcol, int32_t, cap + 1, true);
  CTX_ALLOC(c, hval, double, cap + 1, true);
  struct Batch { int r0, r1; int32_t* oc; double* ov; int cnt; };
  std::vector<Batch> batches;
  int r0 = 0;
  while (r0 < n) {
    int r1 = r0;
    while (r1 < n && ho[r1 + 1] - ho[r0] <= cap) ++r1;
    if (r1 == r0) r1 = r0 + 1;
    int nb = r1 - r0;
    KL(c, k_spgemm_hash<<<nblk(nb), kT, 0, c->stream>>>(r0, r1, A.rp, A.ci, A.v, B.rp, B.ci, B.v, hoff,
                                                  hcol, hval, cnt, &c->ctl->status));
    int32_t* boff;
    CTX_ALLOC(c, boff, int32_t, nb + 1, true);
    int bt = 0;
    st = scan_i32(c, cnt + r0, boff, nb, &bt);
    if (st) return st;
    Batch b{r0, r1, nullptr, nullptr, bt};
    CTX_ALLOC(c, b.oc, int32_t, bt + 1, true);
    CTX_ALLOC(c, b.ov, double, bt + 1, true);
    KL(c, k_spgemm_gather<<<nblk(nb), kT, 0, c->stream>>>(r0, r1, hoff, hcol, hval, boff, b.oc, b.ov));
    batches.push_back(b);
    r0 = r1;
  }
  C.n = n;
  C.m = B.m;
  st = check_count_fits(c, cnt, n, tot);
  if (st) return st;
  CTX_ALLOC(c, C.rp, int32_t, n + 1, true);
  int total = 0;
  st = scan_i32(c, cnt, C.rp, n, &total);
  if (st) return st;
  C.nnz = total;
  CTX_ALLOC(c, C.ci, int32_t, total + 1, true);
  CTX_ALLOC(c, C.v, double, total + 1, true);
  long long o = 0;
  for (auto& b : batches) {
    if (b.cnt > 0) {
      CTX_CUDA(c, cudaMemcpyAsync(C.ci + o, b.oc, sizeof(int32_t) * b.cnt,
                                  cudaMemcpyDeviceToDevice, c->stream));
      CTX_CUDA(c, cudaMemcpyAsync(C.v + o, b.ov, sizeof(double) * b.cnt, cudaMemcpyDeviceToDevice,
                                  c->stream));
    }
    o += b.cnt;
  }
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

cptr_status transpose(cptr_ctx* c, const DCSR& P, DCSR& R) {
  R.n = P.m;
  R.m = P.n;
  R.nnz = P.nnz;
  int32_t *cnt, *cur;
  CTX_ALLOC(c, cnt, int32_t, R.n + 1, true);
  CTX_ALLOC(c, cur, int32_t, R.n + 1, true);
  CTX_ALLOC(c, R.rp, int32_t, R.n + 1, true);
  CTX_ALLOC(c, R.ci, int32_t, R.nnz + 1, true);
  CTX_ALLOC(c, R.v, double, R.nnz + 1, true);
  CTX_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (R.n + 1), c->stream));
  CTX_CUDA(c, cudaMemsetAsync(cur, 0, sizeof(int32_t) * (R.n + 1), c->stream));
  KL(c, k_count_cols<<<nblk(P.nnz), kT, 0, c->stream>>>(P.nnz, P.ci, cnt));
  cptr_status st = scan_i32(c, cnt, R.rp, R.n, nullptr);
  if (st) return st;
  KL(c, k_transpose_fill<<<nblk(P.n), kT, 0, c->stream>>>(P.n, P.rp, P.ci, P.v, R.rp, cur, R.ci, R.v));
  KL(c, k_sort_rows<<<nblk((long long)R.n * 32), 32 * kSortWarps, 0, c->stream>>>(R.n, R.rp, R.ci, R.v));
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

}  // namespace

// ====================================================================== host
cptr_status setup_validate(cptr_ctx* c) {
  int* bad;
  CTX_ALLOC(c, bad, int, 1, false);
  CTX_CUDA(c, cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
  KL(c, k_validate<<<nblk(c->N), kT, 0, c->stream>>>(c->N, c->rp, c->ci, c->diag, bad));
  int h = 0;
  CTX_CUDA(c, cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  if (h) {
    ctx_set_err(c, "malformed BSR: index out of range, unsorted row, or missing diagonal block");
    return CPTR_ERR_INVALID;
  }
  return CPTR_OK;
}

cptr_status setup_decouple(cptr_ctx* c) {
  int N = c->N;
  const int ne = c->se1 < 0 ? 1 : 2;
  int h[3] = {-1, -1, -1}, k = 0;
  for (int u = 0; u < 4; ++u)
    if (u != c->se0 && u != c->se1) h[k++] = u;
  CTX_ALLOC(c, c->W64, double, 4 * (size_t)N, true);
  KL(c, k_qi_w<<<nblk(N), kT, 0, c->stream>>>(N, c->v, c->diag, c->se0, c->se1, h[0], h[1], h[2],
                                               c->W64, &c->ctl->status));
  c->lev.clear();
  c->lev.emplace_back();
  Level& L0 = c->lev[0];
  L0.A.n = L0.A.m = ne * N;
  L0.A.nnz = ne * ne * c->nnzb;
  CTX_ALLOC(c, L0.A.rp, int32_t, (size_t)ne * N + 1, true);
  CTX_ALLOC(c, L0.A.ci, int32_t, L0.A.nnz, true);
  CTX_ALLOC(c, L0.A.v, double, L0.A.nnz, true);
  CTX_ALLOC(c, L0.func, int32_t, (size_t)ne * N, true);
  KL(c, k_qi_ahat<<<nblk(N), kT, 0, c->stream>>>(N, c->rp, c->ci, c->v, c->W64, c->se0, c->se1,
                                                  h[0], h[1], h[2], L0.A.rp, L0.A.ci, L0.A.v));
  KL(c, k_func_alternating<<<nblk((long long)ne * N), kT, 0, c->stream>>>(ne * N, ne, L0.func));
  CTX_CUDA(c, cudaGetLastError());
  return ctx_check_device_status(c);
}

// HMIS on one domain (coarsen = CPTR_COARSEN_HMIS): the first pass of
// classical Ruge-Stueben coarsening decides every point, so the PMIS pass
// that HMIS runs after it has nothing left.  The pass is a sequential greedy
// walk, so it runs on the host over a copy of the strength graph:
// lambda_i = |S_i^T| (the points that depend strongly on i); while an
// undecided point has lambda > 0, the undecided point with the largest lambda
// (ties: the smaller index) becomes C, its undecided strong dependents become
// F and raise by one the lambda of each undecided point they depend on
// strongly, and the new C point lowers by one the lambda of each undecided
// point it depends on strongly; what is left becomes F.  A max-heap keyed by
// (lambda, -index) with stale entries skipped finds the next point.  The
// outcome does not depend on the order of the S^T lists.
cptr_status hmis_first_pass(cptr_ctx* c, int n, int nnz, const int32_t* drp, const int32_t* dci,
                            const uint8_t* dS, const int32_t* dtp, const int32_t* dtj,
                            int32_t* dstt) {
  std::vector<int32_t> rp(n + 1), ci(nnz), tp(n + 1);
  std::vector<uint8_t> S(nnz);
  CTX_CUDA(c, cudaMemcpyAsync(rp.data(), drp, sizeof(int32_t) * (n + 1),
                              cudaMemcpyDeviceToHost, c->stream));
  CTX_CUDA(c, cudaMemcpyAsync(ci.data(), dci, sizeof(int32_t) * (size_t)nnz,
                              cudaMemcpyDeviceToHost, c->stream));
  CTX_CUDA(c, cudaMemcpyAsync(S.data(), dS, (size_t)nnz, cudaMemcpyDeviceToHost, c->stream));
  CTX_CUDA(c, cudaMemcpyAsync(tp.data(), dtp, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost,
                              c->stream));
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<int32_t> tj((size_t)tp[n] + 1);
  if (tp[n] > 0)
    CTX_CUDA(c, cudaMemcpyAsync(tj.data(), dtj, sizeof(int32_t) * (size_t)tp[n],
                                cudaMemcpyDeviceToHost, c->stream));
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<int32_t> lam(n), st(n, ST_U);
  std::priority_queue<std::pair<int32_t, int32_t>> heap;  // (lambda, -index)
  for (int i = 0; i < n; ++i) {
    lam[i] = tp[i + 1] - tp[i];
    heap.emplace(lam[i], -i);
  }
  while (!heap.empty()) {
    const auto top = heap.top();
    heap.pop();
    const int i = -top.second;
    if (st[i] != ST_U || top.first != lam[i]) continue;  // decided, or an old lambda
    if (lam[i] == 0) break;
    st[i] = ST_C;
    for (int q = tp[i]; q < tp[i + 1]; ++q) {
      const int j = tj[q];
      if (st[j] != ST_U) continue;
      st[j] = ST_F;
      for (int t = rp[j]; t < rp[j + 1]; ++t) {
        const int k = ci[t];
        if (S[t] && st[k] == ST_U) heap.emplace(++lam[k], -k);
      }
    }
    for (int t = rp[i]; t < rp[i + 1]; ++t) {
      const int k = ci[t];
      if (S[t] && st[k] == ST_U) heap.emplace(--lam[k], -k);
    }
  }
  for (int i = 0; i < n; ++i)
    if (st[i] == ST_U) st[i] = ST_F;
  CTX_CUDA(c, cudaMemcpyAsync(dstt, st.data(), sizeof(int32_t) * (size_t)n,
                              cudaMemcpyHostToDevice, c->stream));
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));  // st goes out of scope
  return CPTR_OK;
}

// Lanes per row of the setup's row kernels (strength, flags, sizes, S^T):
// 8, 16 or 32 by the mean row length (their results do not depend on it).
inline int row_lanes(int n, long long nnz) {
  const double a = n > 0 ? (double)nnz / n : 1.0;
  return a <= 12.0 ? 8 : a <= 24.0 ? 16 : 32;
}
#define ROW_LAUNCH(c, lanes, n, kern, ...)                                                   \
  do {                                                                                       \
    if ((lanes) == 8)                                                                        \
      KL(c, kern<8><<<nblk((long long)(n) * 8), kT, 0, (c)->stream>>>(__VA_ARGS__));        \
    else if ((lanes) == 16)                                                                  \
      KL(c, kern<16><<<nblk((long long)(n) * 16), kT, 0, (c)->stream>>>(__VA_ARGS__));      \
    else                                                                                     \
      KL(c, kern<32><<<nblk((long long)(n) * 32), kT, 0, (c)->stream>>>(__VA_ARGS__));      \
  } while (0)

// C/F splitting of a strength graph (rows rp/ci, strong flags S, cnt[j] =
// the points that depend strongly on j): S^T, then PMIS in rounds (weights of
// `level`) or the HMIS first pass; cf = +1 / -1, isc = 1 for C points.
cptr_status split_graph(cptr_ctx* c, int n, int nnz, const int32_t* rp, const int32_t* ci,
                        const uint8_t* S, const int32_t* cnt, int level, int32_t* cf,
                        int32_t* isc) {
  cptr_status st;
  int32_t *tp, *cur, *tj, *stt;
  double* lam;
  int* remaining;
  CTX_ALLOC(c, tp, int32_t, n + 1, true);
  CTX_ALLOC(c, cur, int32_t, n + 1, true);
  CTX_ALLOC(c, stt, int32_t, n + 1, true);
  CTX_ALLOC(c, lam, double, n + 1, true);
  CTX_ALLOC(c, remaining, int, 1, true);
  CTX_CUDA(c, cudaMemsetAsync(cur, 0, sizeof(int32_t) * (n + 1), c->stream));
  // S^T offsets on the device; the lists are sized by the graph's entries
  // (an upper bound of the strong couplings), which spares a host read
  st = scan_i32(c, cnt, tp, n, nullptr);
  if (st) return st;
  CTX_ALLOC(c, tj, int32_t, (size_t)nnz + 1, true);
  ROW_LAUNCH(c, row_lanes(n, nnz), n, k_st_fill, n, rp, ci, S, tp, cur, tj);
  if (c->p.coarsen == CPTR_COARSEN_HMIS) {
    st = hmis_first_pass(c, n, nnz, rp, ci, S, tp, tj, stt);
    if (st) return st;
  } else {
    KL(c, k_pmis_init<<<nblk(n), kT, 0, c->stream>>>(n, cnt, c->p.seed, level, lam, stt));
  }
  for (int round = 0; c->p.coarsen != CPTR_COARSEN_HMIS; ++round) {
    if (round > 100000) {
      ctx_set_err(c, "PMIS did not terminate");
      return CPTR_ERR_BREAKDOWN;
    }
    // four rounds per host check: a round with no undecided point is a no-op
    // long rows: one warp per point
    const bool warp_pts = nnz >= 16ll * n;
    for (int q = 0; q < 4; ++q) {
      if (warp_pts)
        KL(c, k_pmis_select_warp<<<nblk(32ll * n), kT, 0, c->stream>>>(n, rp, ci, S, tp, tj, lam,
                                                                      stt));
      else
        KL(c, k_pmis_select<<<nblk(n), kT, 0, c->stream>>>(n, rp, ci, S, tp, tj, lam, stt));
      CTX_CUDA(c, cudaMemsetAsync(remaining, 0, sizeof(int), c->stream));
      if (warp_pts)
        KL(c, k_pmis_update_warp<<<nblk(32ll * n), kT, 0, c->stream>>>(n, rp, ci, S, stt,
                                                                      remaining));
      else
        KL(c, k_pmis_update<<<nblk(n), kT, 0, c->stream>>>(n, rp, ci, S, stt, remaining));
    }
    int rem = 0;
    CTX_CUDA(c, cudaMemcpyAsync(&rem, remaining, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CTX_CUDA(c, cudaStreamSynchronize(c->stream));
    if (rem == 0) break;
  }
  KL(c, k_pmis_final<<<nblk(n), kT, 0, c->stream>>>(n, stt, cf, isc));
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

// The aggressive first level's second split (agg = 2): among the first
// split's C points, j is a distance-two strong dependency of i when j is a
// strong dependency of i or of one of i's strong dependencies (the union of
// the rows of B and B B, B the strong pattern); those C points are split
// again by the same algorithm (level 1's PMIS weights), and a C point stays C
// only if the second split keeps it.  Updates L->cf and isc.
cptr_status aggressive_split(cptr_ctx* c, Level* L, const uint8_t* S, int32_t* isc) {
  const int n = L->A.n;
  cptr_status st;
  int32_t* cidx1;
  CTX_ALLOC(c, cidx1, int32_t, n + 1, true);
  int nc1 = 0;
  st = scan_i32(c, isc, cidx1, n, &nc1);
  if (st) return st;
  if (nc1 == 0) return CPTR_OK;
  DCSR B, B2, G;
  B.n = B.m = n;
  int32_t* bcnt;
  CTX_ALLOC(c, bcnt, int32_t, n + 1, true);
  KL(c, k_strong_count<<<nblk(n), kT, 0, c->stream>>>(n, L->A.rp, S, bcnt));
  CTX_ALLOC(c, B.rp, int32_t, n + 1, true);
  st = scan_i32(c, bcnt, B.rp, n, &B.nnz);
  if (st) return st;
  CTX_ALLOC(c, B.ci, int32_t, (size_t)B.nnz + 1, true);
  CTX_ALLOC(c, B.v, double, (size_t)B.nnz + 1, true);
  KL(c, k_strong_fill<<<nblk(n), kT, 0, c->stream>>>(n, L->A.rp, L->A.ci, S, B.rp, B.ci, B.v));
  st = spgemm(c, B, B, B2);
  if (st) return st;
  int32_t* gcnt;
  CTX_ALLOC(c, gcnt, int32_t, nc1 + 1, true);
  KL(c, k_g2_row<<<nblk(n), kT, 0, c->stream>>>(n, L->cf, cidx1, B.rp, B.ci, B2.rp, B2.ci,
                                                 nullptr, gcnt, nullptr));
  G.n = G.m = nc1;
  CTX_ALLOC(c, G.rp, int32_t, nc1 + 1, true);
  st = scan_i32(c, gcnt, G.rp, nc1, &G.nnz);
  if (st) return st;
  CTX_ALLOC(c, G.ci, int32_t, (size_t)G.nnz + 1, true);
  KL(c, k_g2_row<<<nblk(n), kT, 0, c->stream>>>(n, L->cf, cidx1, B.rp, B.ci, B2.rp, B2.ci, G.rp,
                                                 nullptr, G.ci));
  uint8_t* S2;
  int32_t *cnt2, *cf2, *isc2;
  CTX_ALLOC(c, S2, uint8_t, (size_t)G.nnz + 1, true);
  CTX_ALLOC(c, cnt2, int32_t, nc1 + 1, true);
  CTX_ALLOC(c, cf2, int32_t, nc1 + 1, true);
  CTX_ALLOC(c, isc2, int32_t, nc1 + 1, true);
  CTX_CUDA(c, cudaMemsetAsync(S2, 1, (size_t)G.nnz + 1, c->stream));
  CTX_CUDA(c, cudaMemsetAsync(cnt2, 0, sizeof(int32_t) * (nc1 + 1), c->stream));
  if (G.nnz > 0) KL(c, k_col_count<<<nblk(G.nnz), kT, 0, c->stream>>>(G.nnz, G.ci, cnt2));
  st = split_graph(c, nc1, G.nnz, G.rp, G.ci, S2, cnt2, 1, cf2, isc2);
  if (st) return st;
  KL(c, k_agg_cf<<<nblk(n), kT, 0, c->stream>>>(n, L->cf, cidx1, cf2));
  KL(c, k_isc_from_cf<<<nblk(n), kT, 0, c->stream>>>(n, L->cf, isc));
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

// Multipass interpolation for the aggressive first level (agg = 2): C points
// take unit rows (pass 0); pass ps = 1, 2, ... gives every point not yet
// interpolated that has strong dependencies interpolated in earlier passes
// the row W_ps Q, W_ps its weights (k_mp_fill) and Q the rows built before
// it, until a pass reaches no point; the rows are then truncated like
// ext+i's (k_trunc_*).
cptr_status multipass_interp(cptr_ctx* c, Level* L, const uint8_t* S, const int32_t* cidx,
                             int nc, DCSR& P) {
  const int n = L->A.n, pmax = c->p.pmax;
  cptr_status st;
  int32_t *pass, *newp, *cnt;
  int* reached;
  CTX_ALLOC(c, pass, int32_t, n + 1, true);
  CTX_ALLOC(c, newp, int32_t, n + 1, true);
  CTX_ALLOC(c, cnt, int32_t, n + 1, true);
  CTX_ALLOC(c, reached, int, 1, true);
  DCSR Q;
  Q.n = n;
  Q.m = nc;
  KL(c, k_mp_init<<<nblk(n), kT, 0, c->stream>>>(n, L->cf, cidx, pass, cnt));
  CTX_ALLOC(c, Q.rp, int32_t, n + 1, true);
  st = scan_i32(c, cnt, Q.rp, n, &Q.nnz);
  if (st) return st;
  CTX_ALLOC(c, Q.ci, int32_t, (size_t)Q.nnz + 1, true);
  CTX_ALLOC(c, Q.v, double, (size_t)Q.nnz + 1, true);
  KL(c, k_unit_rows<<<nblk(n), kT, 0, c->stream>>>(n, L->cf, cidx, Q.rp, Q.ci, Q.v));
  for (int ps = 1;; ++ps) {
    if (ps > n + 1) {
      ctx_set_err(c, "multipass interpolation did not terminate");
      return CPTR_ERR_BREAKDOWN;
    }
    CTX_CUDA(c, cudaMemsetAsync(reached, 0, sizeof(int), c->stream));
    KL(c, k_mp_count<<<nblk(n), kT, 0, c->stream>>>(n, L->A.rp, L->A.ci, S, pass, ps, newp, cnt,
                                                     reached));
    int r = 0;
    CTX_CUDA(c, cudaMemcpyAsync(&r, reached, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CTX_CUDA(c, cudaStreamSynchronize(c->stream));
    if (r == 0) break;
    DCSR W, WQ, N2;
    W.n = W.m = n;
    CTX_ALLOC(c, W.rp, int32_t, n + 1, true);
    st = scan_i32(c, cnt, W.rp, n, &W.nnz);
    if (st) return st;
    CTX_ALLOC(c, W.ci, int32_t, (size_t)W.nnz + 1, true);
    CTX_ALLOC(c, W.v, double, (size_t)W.nnz + 1, true);
    KL(c, k_mp_fill<<<nblk(n), kT, 0, c->stream>>>(n, L->A.rp, L->A.ci, L->A.v, S, L->func, pass,
                                                    W.rp, W.ci, W.v));
    st = spgemm(c, W, Q, WQ);
    if (st) return st;
    KL(c, k_mp_merge<<<nblk(n), kT, 0, c->stream>>>(n, ps, pass, newp, Q.rp, Q.ci, Q.v, WQ.rp,
                                                     WQ.ci, WQ.v, nullptr, cnt, nullptr,
                                                     nullptr));
    N2.n = n;
    N2.m = nc;
    CTX_ALLOC(c, N2.rp, int32_t, n + 1, true);
    st = scan_i32(c, cnt, N2.rp, n, &N2.nnz);
    if (st) return st;
    CTX_ALLOC(c, N2.ci, int32_t, (size_t)N2.nnz + 1, true);
    CTX_ALLOC(c, N2.v, double, (size_t)N2.nnz + 1, true);
    KL(c, k_mp_merge<<<nblk(n), kT, 0, c->stream>>>(n, ps, pass, newp, Q.rp, Q.ci, Q.v, WQ.rp,
                                                     WQ.ci, WQ.v, N2.rp, nullptr, N2.ci, N2.v));
    Q = N2;
    CTX_CUDA(c, cudaMemcpyAsync(pass, newp, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice,
                                c->stream));
  }
  int32_t* tord;
  CTX_ALLOC(c, tord, int32_t, (size_t)Q.nnz + 1, true);
  KL(c, k_trunc_count<<<nblk(n), kT, 0, c->stream>>>(n, Q.rp, Q.v, pmax, cnt));
  P.n = n;
  P.m = nc;
  CTX_ALLOC(c, P.rp, int32_t, n + 1, true);
  st = scan_i32(c, cnt, P.rp, n, &P.nnz);
  if (st) return st;
  CTX_ALLOC(c, P.ci, int32_t, (size_t)P.nnz + 1, true);
  CTX_ALLOC(c, P.v, double, (size_t)P.nnz + 1, true);
  KL(c, k_trunc_fill<<<nblk(n), kT, 0, c->stream>>>(n, Q.rp, Q.ci, Q.v, pmax, tord, P.rp, P.ci,
                                                     P.v));
  CTX_CUDA(c, cudaGetLastError());
  return CPTR_OK;
}

cptr_status setup_amg(cptr_ctx* c) {
  const int kMaxDense = 4096;
  cptr_status st;
  bool collapsed = false;  // one aggregate level: the second stage has been folded in
  for (int l = 0;; ++l) {
    Level* L = &c->lev[l];
    int n = L->A.n, nnz = L->A.nnz;
    bool coarsest = (n <= c->p.max_coarse) || (l + 1 >= c->p.max_levels);
    if (!coarsest) {
      uint8_t* S;
      int32_t *cnt, *isc, *cidx;
      CTX_ALLOC(c, S, uint8_t, nnz + 1, true);
      CTX_ALLOC(c, cnt, int32_t, n + 1, true);
      CTX_ALLOC(c, isc, int32_t, n + 1, true);
      CTX_ALLOC(c, cidx, int32_t, n + 1, true);
      CTX_ALLOC(c, L->cf, int32_t, n + 1, true);
      CTX_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), c->stream));
      ROW_LAUNCH(c, row_lanes(n, nnz), n, k_strength, n, L->A.rp, L->A.ci, L->A.v, L->func,
                 c->p.theta, S, cnt);
      ctx_phase(c, "  strength");
      st = split_graph(c, n, nnz, L->A.rp, L->A.ci, S, cnt, l, L->cf, isc);
      if (st) return st;
      if (l == 0 && c->p.agg == 2) {
        // BoomerAMG-style aggressive first level: a second split of the C
        // points on distance-two strength
        st = aggressive_split(c, L, S, isc);
        if (st) return st;
      }
      int nc = 0;
      st = scan_i32(c, isc, cidx, n, &nc);
      if (st) return st;
      L->cidx = cidx;
      ctx_phase(c, "  pmis");
      if (nc == 0 || (double)nc > 0.9 * (double)n) {
        coarsest = true;
        L->cf = nullptr;
      } else {
        // ---- interpolation
        if (l == 0 && c->p.agg == 2) {
          st = multipass_interp(c, L, S, cidx, nc, L->P);
          if (st) return st;
          L->nc = nc;
          ctx_phase(c, "  interp");
        } else {
        int32_t *ub, *pcnt, *pcol, *sc_col, *sc_ord;
        long long* off;
        double *pval, *sc_num;
        int pmax = c->p.pmax;
        CTX_ALLOC(c, ub, int32_t, n + 1, true);
        CTX_ALLOC(c, off, long long, n + 1, true);
        CTX_ALLOC(c, pcnt, int32_t, n + 1, true);
        CTX_ALLOC(c, pcol, int32_t, (size_t)n * pmax + 1, true);
        CTX_ALLOC(c, pval, double, (size_t)n * pmax + 1, true);
        // block-per-row ext+i (shared memory, then global scratch for the rows
        // that do not fit); the thread-per-row kernel is the last resort
        int* flags;
        CTX_ALLOC(c, flags, int, 5, true);
        CTX_CUDA(c, cudaMemsetAsync(flags, 0, 5 * sizeof(int), c->stream));
        uint8_t* ef;
        CTX_ALLOC(c, ef, uint8_t, nnz + 1, true);
        ROW_LAUNCH(c, row_lanes(n, L->A.nnz), n, k_entry_flags, n, L->A.rp, L->A.ci, S, L->cf,
                   L->func, ef);
        ROW_LAUNCH(c, row_lanes(n, L->A.nnz), n, k_interp_sizes, n, L->A.rp, L->A.ci, ef, L->cf,
                   ub, flags + 2);
        // largest staging size, candidate count and row length, in one read
        int mx3[3] = {0, 0, 0};
        CTX_CUDA(c, cudaMemcpyAsync(mx3, flags + 2, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                                    c->stream));
        CTX_CUDA(c, cudaStreamSynchronize(c->stream));
        const int mstage = mx3[0], mub = mx3[1], mrl = mx3[2];
        const int kMaxHs = 8192;
        const size_t kMaxSmem = 200 * 1024;
        int hsz = 64;
        while (hsz < 2 * mub && hsz < kMaxHs) hsz <<= 1;
        int rl = 32;
        while (rl < mrl) rl <<= 1;
        int kcap = 32;  // staged neighbour entries per segment: <= 256, >= the longest row
        while (kcap < std::min(mstage, 256)) kcap <<= 1;
        while (kcap < mrl) kcap <<= 1;
        // shared-memory pass for the rows that fit modest tables; the others
        // (long rows, large Chat sets, long neighbour rows) are deferred to the
        // same kernel with per-row tables in global scratch
        // (the hash table is sized by candidates counted with repeats; Chat sets
        // hold a few dozen columns, and a row whose set exceeds the table is
        // deferred like any row that does not fit)
        const int hs_s = std::min(hsz, 512), rl_s = std::min(rl, 512), kc_s = std::min(kcap, 512);
        // short rows (every phase fits one warp's lanes a few times): one warp
        // per row with a small ordered-sum table, so that more rows are resident
        const bool narrow = c->interp_path == 0 && rl_s <= 32 && kc_s <= 128;
        const int tmin = 256;  // the table holds |Chat|+1 terms per strong F neighbour
        const int ithr = narrow ? 32 : (hs_s >= 2048 ? 256 : 128);
        size_t smem = interp_layout(hs_s, rl_s, kc_s, tmin).total;
        int over = (smem > kMaxSmem || c->force_fallback) ? 1 : 0;
        if (!over) {
          CTX_CUDA(c, cudaFuncSetAttribute(k_interp_row<false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kMaxSmem));
          int* dfl;
          CTX_ALLOC(c, dfl, int, 3, true);
          CTX_CUDA(c, cudaMemsetAsync(dfl, 0, 3 * sizeof(int), c->stream));
          if (c->interp_path == 2) {  // every row to the global-scratch pass
            CTX_CUDA(c, cudaMemsetAsync(pcnt, 0xff, sizeof(int32_t) * n, c->stream));
            CTX_CUDA(c, cudaMemcpyAsync(dfl, &n, sizeof(int), cudaMemcpyHostToDevice, c->stream));
          } else
            KL(c, k_interp_row<false><<<n, ithr, smem, c->stream>>>(
                    n, hs_s, ub, rl_s, kc_s, tmin, L->A.rp, L->A.ci, L->A.v, ef, L->cf, L->func, cidx,
                    pmax, pcnt, pcol, pval, dfl, nullptr, nullptr, nullptr));
          int ndef = 0;
          CTX_CUDA(c, cudaMemcpyAsync(&ndef, dfl, sizeof(int), cudaMemcpyDeviceToHost,
                                      c->stream));
          CTX_CUDA(c, cudaStreamSynchronize(c->stream));
          if (ndef > 0) {
            int32_t *drows, *dbytes;
            long long* goff;
            CTX_ALLOC(c, drows, int32_t, ndef + 1, true);
            CTX_ALLOC(c, dbytes, int32_t, ndef + 1, true);
            CTX_ALLOC(c, goff, long long, ndef + 1, true);
            KL(c, k_interp_deferred<<<nblk(n), kT, 0, c->stream>>>(n, pcnt, L->A.rp, ub, kcap,
                                                                    drows, dbytes, dfl + 1));
            long long gtot = 0;
            st = scan_i64(c, dbytes, goff, ndef, &gtot);
            if (st) return st;
            unsigned char* gscr = (unsigned char*)ctx_alloc(c, (size_t)gtot + 256, true);
            if (!gscr) return CPTR_ERR_NOMEM;
            KL(c, k_interp_row<true><<<ndef, 256, 0, c->stream>>>(
                      n, 0, ub, 0, kcap, 1024, L->A.rp, L->A.ci, L->A.v, ef, L->cf, L->func, cidx, pmax,
                      pcnt, pcol, pval, dfl + 2, drows, goff, gscr));
            CTX_CUDA(c, cudaMemcpyAsync(&over, dfl + 2, sizeof(int), cudaMemcpyDeviceToHost,
                                        c->stream));
            CTX_CUDA(c, cudaStreamSynchronize(c->stream));
          }
        }
        if (over || c->force_fallback) {
          // ub sizes the per-row scratch of the thread-per-row kernel
          long long tot = 0;
          st = scan_i64(c, ub, off, n, &tot);
          if (st) return st;
          CTX_ALLOC(c, sc_col, int32_t, tot + 1, true);
          CTX_ALLOC(c, sc_ord, int32_t, tot + 1, true);
          CTX_ALLOC(c, sc_num, double, tot + 1, true);
          KL(c, k_interp<<<nblk(n), kT, 0, c->stream>>>(n, L->A.rp, L->A.ci, L->A.v, S, L->cf,
                                                        L->func, cidx, off, sc_col, sc_num, sc_ord,
                                                        pmax, pcnt, pcol, pval));
        }
        L->P.n = n;
        L->P.m = nc;
        CTX_ALLOC(c, L->P.rp, int32_t, n + 1, true);
        int pnnz = 0;
        st = scan_i32(c, pcnt, L->P.rp, n, &pnnz);
        if (st) return st;
        L->P.nnz = pnnz;
        CTX_ALLOC(c, L->P.ci, int32_t, pnnz + 1, true);
        CTX_ALLOC(c, L->P.v, double, pnnz + 1, true);
        KL(c, k_compact_rows<<<nblk(n), kT, 0, c->stream>>>(n, pmax, L->P.rp, pcol, pval, L->P.ci,
                                                      L->P.v));
        L->nc = nc;
        ctx_phase(c, "  interp");
        }
        if (l == 1 && c->p.agg == 1 && !collapsed) {
          // one aggregate level: level 1 was the Galerkin operator of the first
          // split and L->P its interpolation; the first level interpolates in
          // two stages, P = trunc(P1 P2), its coarse operator is P^T A P, and
          // the intermediate operator is dropped from the hierarchy
          Level& L0 = c->lev[0];
          const int n0 = L0.A.n;
          DCSR Pq, P, R, AP, Ac;
          st = spgemm(c, L0.P, L->P, Pq);
          if (st) return st;
          int32_t *tcnt, *tord;
          CTX_ALLOC(c, tcnt, int32_t, n0 + 1, true);
          CTX_ALLOC(c, tord, int32_t, (size_t)Pq.nnz + 1, true);
          KL(c, k_trunc_count<<<nblk(n0), kT, 0, c->stream>>>(n0, Pq.rp, Pq.v, c->p.pmax, tcnt));
          P.n = n0;
          P.m = nc;
          CTX_ALLOC(c, P.rp, int32_t, n0 + 1, true);
          int pn = 0;
          st = scan_i32(c, tcnt, P.rp, n0, &pn);
          if (st) return st;
          P.nnz = pn;
          CTX_ALLOC(c, P.ci, int32_t, pn + 1, true);
          CTX_ALLOC(c, P.v, double, pn + 1, true);
          KL(c, k_trunc_fill<<<nblk(n0), kT, 0, c->stream>>>(n0, Pq.rp, Pq.ci, Pq.v, c->p.pmax, tord,
                                                              P.rp, P.ci, P.v));
          st = transpose(c, P, R);
          if (st) return st;
          st = spgemm(c, L0.A, P, AP);
          if (st) return st;
          st = spgemm(c, R, AP, Ac);
          if (st) return st;
          KL(c, k_agg_cf<<<nblk(n0), kT, 0, c->stream>>>(n0, L0.cf, L0.cidx, L->cf));
          Level nx;
          nx.A = Ac;
          CTX_ALLOC(c, nx.func, int32_t, nc + 1, true);
          KL(c, k_coarse_func<<<nblk(n), kT, 0, c->stream>>>(n, L->cf, cidx, L->func, nx.func));
          CTX_CUDA(c, cudaGetLastError());
          L0.P = P;
          L0.R = R;
          L0.nc = nc;
          c->lev[1] = nx;  // the intermediate level's arrays are setup-lifetime memory
          collapsed = true;
          ctx_phase(c, "  aggregate level");
          --l;  // the new level 1 is coarsened by the next pass
          continue;
        }
        st = transpose(c, L->P, L->R);
        if (st) return st;
        ctx_phase(c, "  transpose");
        DCSR AP, Ac;
        st = spgemm(c, L->A, L->P, AP);
        if (st) return st;
        ctx_phase(c, "  spgemm A*P");
        st = spgemm(c, L->R, AP, Ac);
        if (st) return st;
        ctx_phase(c, "  spgemm R*(AP)");
        CTX_ALLOC(c, L->dl1, double, n + 1, true);
        KL(c, k_l1<<<nblk(n), kT, 0, c->stream>>>(n, L->A.rp, L->A.ci, L->A.v, L->dl1));
        Level nx;
        nx.A = Ac;
        CTX_ALLOC(c, nx.func, int32_t, nc + 1, true);
        KL(c, k_coarse_func<<<nblk(n), kT, 0, c->stream>>>(n, L->cf, cidx, L->func, nx.func));
        CTX_CUDA(c, cudaGetLastError());
        c->lev.push_back(nx);  // invalidates L
      }
    }
    if (coarsest) {
      Level* Lc = &c->lev[l];
      int nn = Lc->A.n;
      c->lev.resize(l + 1);
      if (nn > kMaxDense) {
        ctx_set_err(c, "AMG coarsening stalled above the dense coarse-solve limit");
        return CPTR_ERR_BREAKDOWN;
      }
      c->ncoarse = nn;
      double* M;
      CTX_ALLOC(c, M, double, 2 * (size_t)nn * nn + 1, true);
      CTX_ALLOC(c, c->Cinv, double, (size_t)nn * nn + 1, true);
      KL(c, k_dense_fill<<<nblk(nn), kT, 0, c->stream>>>(nn, Lc->A.rp, Lc->A.ci, Lc->A.v, M));
      // one cluster holding the whole augmented matrix when it fits, else one block
      bool clustered = false;
      {
        const int w = (2 * nn + kGjCtas - 1) / kGjCtas;
        const size_t csmem = sizeof(double) * ((size_t)nn * w + 2 * (size_t)nn);
        if (csmem <= 200 * 1024) {
          CTX_CUDA(c, cudaFuncSetAttribute(k_gauss_jordan_cluster,
                                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
          CTX_CUDA(c, raise_smem_limit(c, (const void*)k_gauss_jordan_cluster));
          cudaLaunchConfig_t cfg = {};
          cfg.gridDim = dim3(kGjCtas);
          cfg.blockDim = dim3(kGjThreads);
          cfg.dynamicSmemBytes = csmem;
          cfg.stream = c->stream;
          cudaLaunchAttribute at[1];
          at[0].id = cudaLaunchAttributeClusterDimension;
          at[0].val.clusterDim.x = kGjCtas;
          at[0].val.clusterDim.y = 1;
          at[0].val.clusterDim.z = 1;
          cfg.attrs = at;
          cfg.numAttrs = 1;
          int ncl = 0;
          if (cudaOccupancyMaxActiveClusters(&ncl, k_gauss_jordan_cluster, &cfg) != cudaSuccess) {
            cudaGetLastError();
            ncl = 0;
          }
          if (ncl >= 1) {
            const double* Mc = M;
            KL(c, cudaLaunchKernelEx(&cfg, k_gauss_jordan_cluster, nn, w, Mc, c->Cinv,
                                     &c->ctl->status));
            clustered = true;
          }
        }
      }
      const size_t gj_smem = sizeof(double) * 3 * (size_t)nn;
      if (!clustered && gj_smem > 48 * 1024)
        CTX_CUDA(c, raise_smem_limit(c, (const void*)k_gauss_jordan));
      if (!clustered)
      KL(c, k_gauss_jordan<<<1, 1024, gj_smem, c->stream>>>(nn, M, c->Cinv,
                                                                   &c->ctl->status));
      CTX_CUDA(c, cudaGetLastError());
      st = ctx_check_device_status(c);
      if (st) return st;
      ctx_phase(c, "  coarse inverse");
      break;
    }
  }
  long long tot = 0;
  for (auto& L : c->lev) tot += L.A.nnz;
  c->op_complexity = c->lev[0].A.nnz ? (double)tot / c->lev[0].A.nnz : 0.0;
  return CPTR_OK;
}
