/*
 * FP64 CPU oracle for CPTR-preconditioned flexible GMRES.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the benchmark's
 * CPU baseline.  Plain, single-threaded, unblocked loops in the order the
 * method states them.  Compile with -ffp-contract=off (no fused multiply-add)
 * so that every product and sum is an individually rounded IEEE operation.
 *
 * Readings of points the paper leaves open are marked READING; each one is
 * also listed in the design notes of the repository.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define BS 4
#define MAXLEV 32
#define MAX_DENSE_COARSE 4096

typedef struct {
  int n, m, nnz;   /* n rows, m columns */
  int32_t *rp, *ci;
  double* v;
} ocsr;

typedef struct {
  ocsr A;
  int32_t* func;
  int32_t* cf;     /* +1 C, -1 F (only on non-coarsest levels) */
  ocsr P, R;       /* P: n x nc, R = P^T */
  double* dl1;
  int nc;
  double *b, *x, *r, *x2;   /* work vectors */
} olevel;

struct orc_amg {
  int nlev;
  int nu_pre, nu_post, smoother;  /* the V-cycle's smoothing (orc_params) */
  olevel lev[MAXLEV];
  int ncoarse;
  double* LU;
  int32_t* piv;
  double* work;
};

/* One decoupled first stage: the elliptic unknowns it keeps, W_i and Ahat of the
 * Quasi-IMPES decoupling onto them, and the AMG hierarchy of Ahat (or, in the
 * exact-stage test modes, a dense LU of Ahat). */
typedef struct {
  int ne, nh;        /* elliptic unknowns: 2 (CPTR, {e0, e1}) or 1 ({e0}); nh = 4 - ne */
  int ee[2];         /* elliptic unknowns */
  int hh[3];         /* the other unknowns, increasing */
  double* W;         /* N x 4 */
  ocsr Ahat;         /* ne N x ne N scalar, interleaved elliptic unknowns */
  orc_amg* amg;
  double* AhLU;      /* dense LU of Ahat (exact stage, tests only) */
  int32_t* AhPiv;
} ostage;

struct orc_ctx {
  int N, nnzb;
  int32_t *rp, *ci, *diag;
  double* v;         /* the operator GMRES works on (the reduced one with mgr) */
  double* vfull;     /* mgr: the given matrix, before the reduction */
  orc_params p;
  ostage st[2];      /* [0] the first stage; [1] the temperature stage of CPTR3 */
  int nst;           /* stages in use: 1, or 2 for CPTR3 */
  double* LU;        /* nnzb x 16 */
  int32_t* ilu_level;
  int ilu_nlev;
  int setup_done;
  /* last Arnoldi cycle */
  int last_k;
  double *lastV, *lastZ, *lastH;
  int last_cap;
  double *t4a, *t4b, *t4c, *t2a, *t2b;
};

/* the unknown (and equation row) that the first MGR reduction eliminates:
 * rho_H2O, the last density, with the volume constraint (Section 3.4) */
enum { MGR_U = 2 };

/* ------------------------------------------------------------------ */
uint64_t orc_splitmix64(uint64_t x) {
  /* SplitMix64 (Steele, Lea & Flood 2014) finaliser applied to x + golden gamma */
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static double pmis_rho(uint64_t seed, int level, int i) {
  uint64_t x = seed ^ ((uint64_t)(uint32_t)level << 32) ^ (uint64_t)(uint32_t)i;
  return (double)(orc_splitmix64(x) >> 11) * (1.0 / 9007199254740992.0);
}

void orc_params_default(orc_params* p) {
  p->restart = 30;
  p->maxit = 200;     /* Section 3: 200 maximum iterations */
  p->tol = 1e-6;      /* Section 3: relative tolerance 1e-6 */
  p->theta = 0.25;    /* READING: strength threshold (paper: HYPRE defaults) */
  p->pmax = 4;        /* Section 3.1: ext+i truncated to 4 elements per row */
  p->max_coarse = 256;
  p->max_levels = 25;
  p->precond = ORC_PREC_CPTR;
  p->seed = 0x5eed;
  p->e0 = 0;
  p->e1 = 3;
  p->mgr = 0;
  p->agg = 0;
  p->coarsen = ORC_COARSEN_PMIS;
  p->nu_pre = 1;      /* Section 3.1: one V-cycle; READING: V(1,1) */
  p->nu_post = 1;
  p->smoother = ORC_SMOOTH_L1_JACOBI;
}

static void csr_free(ocsr* a) {
  free(a->rp); free(a->ci); free(a->v);
  memset(a, 0, sizeof(*a));
}

static double dnrm2(int n, const double* x) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += x[i] * x[i];
  return sqrt(s);
}
static double ddot(int n, const double* x, const double* y) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

/* y = A x for scalar CSR */
static void csr_mv(const ocsr* A, const double* x, double* y) {
  for (int i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) s += A->v[t] * x[A->ci[t]];
    y[i] = s;
  }
}

/* ------------------------------------------------------------------ */
/* dense LU with partial pivoting (row of largest |a|, first on ties)  */
static int dense_lu(int n, double* A, int32_t* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(A[(size_t)k * n + k]);
    for (int r = k + 1; r < n; ++r) {
      double a = fabs(A[(size_t)r * n + k]);
      if (a > best) { best = a; p = r; }
    }
    piv[k] = p;
    if (!(best > 0.0) || !isfinite(best)) return ORC_BREAKDOWN;
    if (p != k)
      for (int c = 0; c < n; ++c) {
        double t = A[(size_t)k * n + c];
        A[(size_t)k * n + c] = A[(size_t)p * n + c];
        A[(size_t)p * n + c] = t;
      }
    double d = A[(size_t)k * n + k];
    for (int r = k + 1; r < n; ++r) {
      double l = A[(size_t)r * n + k] / d;
      A[(size_t)r * n + k] = l;
      for (int c = k + 1; c < n; ++c) A[(size_t)r * n + c] -= l * A[(size_t)k * n + c];
    }
  }
  return ORC_OK;
}

static void dense_lu_solve(int n, const double* LU, const int32_t* piv, const double* b, double* x) {
  for (int i = 0; i < n; ++i) x[i] = b[i];
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
  }
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int c = 0; c < i; ++c) s -= LU[(size_t)i * n + c] * x[c];
    x[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int c = i + 1; c < n; ++c) s -= LU[(size_t)i * n + c] * x[c];
    x[i] = s / LU[(size_t)i * n + i];
  }
}

/* 4x4 inverse by Gauss-Jordan elimination with partial pivoting */
static int inv4(const double* M, double* out) {
  double a[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 8; ++c) a[r][c] = (c < 4) ? M[r * 4 + c] : (c - 4 == r ? 1.0 : 0.0);
  for (int c = 0; c < 4; ++c) {
    int p = c;
    double best = fabs(a[c][c]);
    for (int r = c + 1; r < 4; ++r)
      if (fabs(a[r][c]) > best) { best = fabs(a[r][c]); p = r; }
    if (!(best > 0.0) || !isfinite(best)) return ORC_BREAKDOWN;
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
  return ORC_OK;
}

/* C = A * B for 4x4 row-major */
static void mul4(const double* A, const double* B, double* C) {
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += A[r * 4 + k] * B[k * 4 + c];
      C[r * 4 + c] = s;
    }
}

/* ================================================================== */
/* AMG setup (unknown-based system AMG on a scalar CSR with function tags) */
/* ================================================================== */

static double row_diag(const ocsr* A, int i) {
  for (int t = A->rp[i]; t < A->rp[i + 1]; ++t)
    if (A->ci[t] == i) return A->v[t];
  return 0.0;
}

/* Strength of connection, same-function couplings only.
 * READING: j is a strong dependency of i when -s*a_ij >= theta * max_k(-s*a_ik),
 * s = sign(a_ii), k over off-diagonal same-function entries; no strong
 * dependencies when that maximum is <= 0. */
static void strength(const ocsr* A, const int32_t* func, double theta, char* S) {
  for (int i = 0; i < A->n; ++i) {
    double s = row_diag(A, i) < 0.0 ? -1.0 : 1.0;
    double mx = 0.0;
    int any = 0;
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      int j = A->ci[t];
      S[t] = 0;
      if (j == i || func[j] != func[i]) continue;
      double val = -s * A->v[t];
      if (!any || val > mx) { mx = val; any = 1; }
    }
    if (!any || !(mx > 0.0)) continue;
    double thr = theta * mx;
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      int j = A->ci[t];
      if (j == i || func[j] != func[i]) continue;
      if (-s * A->v[t] >= thr) S[t] = 1;
    }
  }
}

enum { ST_U = 0, ST_C = 1, ST_F = -1, ST_CNEW = 2 };

static int lam_greater(const double* lam, int i, int j) {
  return lam[i] > lam[j] || (lam[i] == lam[j] && i > j);
}

/* PMIS coarsening (De Sterck, Yang & Heys 2006), in rounds.
 * READING: the paper names HMIS; PMIS is the default of both codes (a
 * deviation) and HMIS the option coarsen = ORC_COARSEN_HMIS (rs_first_pass).
 * lambda_i = |{j : i in S_j}| + rho_i.  Points with lambda_i < 1 start as F.
 * Each round: an undecided i becomes C when (lambda_i, i) exceeds (lambda_j, j)
 * for every undecided j in S_i u S_i^T (undecided as of the start of the round);
 * then each undecided j that depends strongly on a C point becomes F. */
static int pmis(const ocsr* A, const char* S, uint64_t seed, int level, const double* rho0,
                int32_t* cf) {
  int n = A->n;
  int* cnt = (int*)calloc((size_t)n + 1, sizeof(int));
  double* lam = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  int* st = (int*)malloc(sizeof(int) * (size_t)(n + 1));
  for (int i = 0; i < n; ++i)
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t)
      if (S[t]) cnt[A->ci[t]]++;
  /* transpose of S */
  int* tp = (int*)calloc((size_t)n + 1, sizeof(int));
  for (int i = 0; i < n; ++i) tp[i + 1] = tp[i] + cnt[i];
  int* tj = (int*)malloc(sizeof(int) * (size_t)(tp[n] + 1));
  int* fill = (int*)malloc(sizeof(int) * (size_t)(n + 1));
  for (int i = 0; i < n; ++i) fill[i] = tp[i];
  for (int i = 0; i < n; ++i)
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t)
      if (S[t]) tj[fill[A->ci[t]]++] = i;
  for (int i = 0; i < n; ++i) {
    double rho = rho0 ? rho0[i] : pmis_rho(seed, level, i);
    lam[i] = (double)cnt[i] + rho;
    st[i] = (cnt[i] == 0) ? ST_F : ST_U;
  }
  /* every round decides at least the undecided point of largest (lambda, i),
   * so more than n rounds means a fault: reported, not looped on */
  int rounds = 0, ok_all = 1;
  for (;;) {
    int undecided = 0;
    for (int i = 0; i < n; ++i) undecided += (st[i] == ST_U);
    if (!undecided) break;
    if (++rounds > n + 1) { ok_all = 0; break; }
    for (int i = 0; i < n; ++i) {
      if (st[i] != ST_U) continue;
      int ok = 1;
      for (int t = A->rp[i]; t < A->rp[i + 1] && ok; ++t) {
        if (!S[t]) continue;
        int j = A->ci[t];
        if ((st[j] == ST_U || st[j] == ST_CNEW) && !lam_greater(lam, i, j)) ok = 0;
      }
      for (int t = tp[i]; t < tp[i + 1] && ok; ++t) {
        int j = tj[t];
        if ((st[j] == ST_U || st[j] == ST_CNEW) && !lam_greater(lam, i, j)) ok = 0;
      }
      if (ok) st[i] = ST_CNEW;
    }
    for (int i = 0; i < n; ++i)
      if (st[i] == ST_CNEW) st[i] = ST_C;
    for (int j = 0; j < n; ++j) {
      if (st[j] != ST_U) continue;
      for (int t = A->rp[j]; t < A->rp[j + 1]; ++t)
        if (S[t] && st[A->ci[t]] == ST_C) { st[j] = ST_F; break; }
    }
  }
  for (int i = 0; i < n; ++i) cf[i] = (st[i] == ST_C) ? 1 : -1;
  free(cnt); free(lam); free(st); free(tp); free(tj); free(fill);
  return ok_all ? ORC_OK : ORC_BREAKDOWN;
}

/* The first pass of classical Ruge-Stueben coarsening (HMIS on one domain).
 * lambda_i = |{j : i in S_j}|, the number of points that depend strongly on i.
 * While an undecided point has lambda > 0, the undecided point with the
 * largest lambda (ties: the smaller index) becomes C; every undecided point
 * that depends strongly on it becomes F, and each such new F point raises by
 * one the lambda of every undecided point it depends on strongly; the new C
 * point lowers by one the lambda of every undecided point it depends on
 * strongly.  The points left undecided (lambda 0) become F.
 * The largest lambda is found with a binary heap of (lambda, index) entries;
 * an entry whose lambda is out of date, or whose point is decided, is skipped
 * when it reaches the top. */
typedef struct { int lam, i; } rs_entry;

static int rs_before(rs_entry a, rs_entry b) {   /* a leaves the heap before b */
  return a.lam > b.lam || (a.lam == b.lam && a.i < b.i);
}

static void rs_push(rs_entry* h, int* size, rs_entry e) {
  int k = (*size)++;
  h[k] = e;
  while (k > 0) {
    int parent = (k - 1) / 2;
    if (!rs_before(h[k], h[parent])) break;
    rs_entry t = h[k]; h[k] = h[parent]; h[parent] = t;
    k = parent;
  }
}

static rs_entry rs_pop(rs_entry* h, int* size) {
  rs_entry top = h[0];
  h[0] = h[--(*size)];
  int k = 0;
  for (;;) {
    int l = 2 * k + 1, r = l + 1, m = k;
    if (l < *size && rs_before(h[l], h[m])) m = l;
    if (r < *size && rs_before(h[r], h[m])) m = r;
    if (m == k) break;
    rs_entry t = h[k]; h[k] = h[m]; h[m] = t;
    k = m;
  }
  return top;
}

static int rs_first_pass(const ocsr* A, const char* S, int32_t* cf) {
  int n = A->n;
  int* lam = (int*)calloc((size_t)n + 1, sizeof(int));
  int* st = (int*)malloc(sizeof(int) * (size_t)(n + 1));
  for (int i = 0; i < n; ++i)
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t)
      if (S[t]) lam[A->ci[t]]++;
  /* transpose of S: the points that depend strongly on each point */
  int* tp = (int*)calloc((size_t)n + 1, sizeof(int));
  for (int i = 0; i < n; ++i) tp[i + 1] = tp[i] + lam[i];
  int* tj = (int*)malloc(sizeof(int) * (size_t)(tp[n] + 1));
  int* fill = (int*)malloc(sizeof(int) * (size_t)(n + 1));
  for (int i = 0; i < n; ++i) fill[i] = tp[i];
  for (int i = 0; i < n; ++i)
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t)
      if (S[t]) tj[fill[A->ci[t]]++] = i;
  /* every lambda change pushes one entry: at most n + 2 nnz(S) of them */
  size_t cap = (size_t)n + 2 * (size_t)tp[n] + 1;
  rs_entry* heap = (rs_entry*)malloc(sizeof(rs_entry) * cap);
  int size = 0;
  for (int i = 0; i < n; ++i) {
    st[i] = ST_U;
    rs_entry e = {lam[i], i};
    rs_push(heap, &size, e);
  }
  while (size > 0) {
    rs_entry e = rs_pop(heap, &size);
    int i = e.i;
    if (st[i] != ST_U || e.lam != lam[i]) continue;   /* out of date */
    if (lam[i] == 0) break;                           /* the rest become F */
    st[i] = ST_C;
    for (int q = tp[i]; q < tp[i + 1]; ++q) {
      int j = tj[q];
      if (st[j] != ST_U) continue;
      st[j] = ST_F;
      for (int t = A->rp[j]; t < A->rp[j + 1]; ++t) {
        int k = A->ci[t];
        if (!S[t] || st[k] != ST_U) continue;
        lam[k]++;
        rs_entry u = {lam[k], k};
        rs_push(heap, &size, u);
      }
    }
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      int k = A->ci[t];
      if (!S[t] || st[k] != ST_U) continue;
      lam[k]--;
      rs_entry u = {lam[k], k};
      rs_push(heap, &size, u);
    }
  }
  for (int i = 0; i < n; ++i) cf[i] = (st[i] == ST_C) ? 1 : -1;
  free(lam); free(st); free(tp); free(tj); free(fill); free(heap);
  return ORC_OK;
}

static int cmp_int(const void* a, const void* b) {
  int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

static int find_sorted(const int* a, int n, int key) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] == key) return mid;
    if (a[mid] < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* sign-opposite part of a_kl relative to the diagonal a_kk */
static double abar(double akk, double akl) {
  if (akk >= 0.0) return akl < 0.0 ? akl : 0.0;
  return akl > 0.0 ? akl : 0.0;
}

/* Extended+i interpolation (De Sterck, Falgout, Nolting & Yang 2008), same-function
 * couplings only, truncated to pmax entries per row (Section 3.1).
 * For an F point i with strong C set C_i, strong F set F_i, the interpolatory set is
 * Chat_i = C_i u (union over k in F_i of the strong C points of k).  With
 * abar_kl = a_kl when its sign differs from a_kk (else 0) and
 * d_k = sum over l in Chat_i u {i} of abar_kl:
 *   atilde_ii = a_ii + sum(weak same-function a_in, n not in Chat_i)
 *             + sum_{k in F_i} a_ik abar_ki / d_k
 *   w_ij = -(a_ij + sum_{k in F_i} a_ik abar_kj / d_k) / atilde_ii,  j in Chat_i.
 * READING: when d_k == 0 the connection a_ik is lumped into atilde_ii.
 * READING: truncation keeps the pmax largest |w_ij| (ties: smaller column) and
 * rescales them by (sum of all w)/(sum of kept w) when the kept sum is nonzero. */
static int build_interp(const ocsr* A, const int32_t* func, const char* S, const int32_t* cf,
                        int pmax, ocsr* P, int* nc_out) {
  int n = A->n;
  int32_t* cidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int nc = 0;
  for (int i = 0; i < n; ++i) cidx[i] = (cf[i] == 1) ? nc++ : -1;
  int32_t* prow_cnt = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
  int32_t* pcol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n * pmax + 1));
  double* pval = (double*)malloc(sizeof(double) * (size_t)(n * pmax + 1));
  int cap = 64;
  int* chat = (int*)malloc(sizeof(int) * (size_t)cap);
  double* num = (double*)malloc(sizeof(double) * (size_t)cap);
  int* ord = (int*)malloc(sizeof(int) * (size_t)cap);
  for (int i = 0; i < n; ++i) {
    if (cf[i] == 1) {
      prow_cnt[i] = 1; pcol[(size_t)i * pmax] = cidx[i]; pval[(size_t)i * pmax] = 1.0;
      continue;
    }
    /* gather Chat_i */
    int q = 0;
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      if (!S[t]) continue;
      int j = A->ci[t];
      if (cf[j] == 1) {
        if (q == cap) { cap *= 2; chat = realloc(chat, sizeof(int) * cap); num = realloc(num, sizeof(double) * cap); ord = realloc(ord, sizeof(int) * cap); }
        chat[q++] = j;
      } else {
        for (int t2 = A->rp[j]; t2 < A->rp[j + 1]; ++t2) {
          if (!S[t2]) continue;
          int l = A->ci[t2];
          if (cf[l] != 1) continue;
          if (q == cap) { cap *= 2; chat = realloc(chat, sizeof(int) * cap); num = realloc(num, sizeof(double) * cap); ord = realloc(ord, sizeof(int) * cap); }
          chat[q++] = l;
        }
      }
    }
    if (q == 0) { prow_cnt[i] = 0; continue; }
    qsort(chat, (size_t)q, sizeof(int), cmp_int);
    int u = 0;
    for (int t = 0; t < q; ++t)
      if (t == 0 || chat[t] != chat[u - 1]) chat[u++] = chat[t];
    q = u;
    for (int t = 0; t < q; ++t) num[t] = 0.0;
    double dg = 0.0;
    /* direct terms: a_ii, a_ij for j in Chat, weak lumping */
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      int j = A->ci[t];
      if (j == i) { dg += A->v[t]; continue; }
      if (func[j] != func[i]) continue;
      int pos = find_sorted(chat, q, j);
      if (pos >= 0) { num[pos] += A->v[t]; continue; }
      if (!S[t]) dg += A->v[t];
    }
    /* distribution of strong F neighbours */
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      int k = A->ci[t];
      if (!S[t] || cf[k] == 1) continue;
      double aik = A->v[t];
      double akk = row_diag(A, k);
      double den = 0.0;
      for (int t2 = A->rp[k]; t2 < A->rp[k + 1]; ++t2) {
        int l = A->ci[t2];
        if (l == k || func[l] != func[k]) continue;
        if (l == i || find_sorted(chat, q, l) >= 0) den += abar(akk, A->v[t2]);
      }
      if (den == 0.0) { dg += aik; continue; }
      double f = aik / den;
      for (int t2 = A->rp[k]; t2 < A->rp[k + 1]; ++t2) {
        int l = A->ci[t2];
        if (l == k || func[l] != func[k]) continue;
        double ab = abar(akk, A->v[t2]);
        if (ab == 0.0) continue;
        if (l == i) { dg += f * ab; continue; }
        int pos = find_sorted(chat, q, l);
        if (pos >= 0) num[pos] += f * ab;
      }
    }
    if (dg == 0.0 || !isfinite(dg)) { prow_cnt[i] = 0; continue; }
    /* weights, dropping exact zeros */
    int m = 0;
    for (int t = 0; t < q; ++t) {
      double w = -num[t] / dg;
      if (w != 0.0) { chat[m] = chat[t]; num[m] = w; ++m; }
    }
    if (m > pmax) {
      double sum_all = 0.0;
      for (int t = 0; t < m; ++t) sum_all += num[t];
      for (int t = 0; t < m; ++t) ord[t] = t;
      /* selection of the pmax largest |w| (ties: smaller column index == smaller t) */
      for (int a = 0; a < pmax; ++a) {
        int best = a;
        for (int b2 = a + 1; b2 < m; ++b2) {
          double wb = fabs(num[ord[b2]]), wa = fabs(num[ord[best]]);
          if (wb > wa || (wb == wa && ord[b2] < ord[best])) best = b2;
        }
        int tmp = ord[a]; ord[a] = ord[best]; ord[best] = tmp;
      }
      qsort(ord, (size_t)pmax, sizeof(int), cmp_int);  /* kept entries in column order */
      double sum_kept = 0.0;
      for (int a = 0; a < pmax; ++a) sum_kept += num[ord[a]];
      double scale = (sum_kept != 0.0) ? sum_all / sum_kept : 1.0;
      for (int a = 0; a < pmax; ++a) {
        pcol[(size_t)i * pmax + a] = cidx[chat[ord[a]]];
        pval[(size_t)i * pmax + a] = num[ord[a]] * scale;
      }
      prow_cnt[i] = pmax;
    } else {
      for (int a = 0; a < m; ++a) {
        pcol[(size_t)i * pmax + a] = cidx[chat[a]];
        pval[(size_t)i * pmax + a] = num[a];
      }
      prow_cnt[i] = m;
    }
  }
  P->n = n; P->m = nc;
  P->rp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  P->rp[0] = 0;
  for (int i = 0; i < n; ++i) P->rp[i + 1] = P->rp[i] + prow_cnt[i];
  P->nnz = P->rp[n];
  P->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P->nnz + 1));
  P->v = (double*)malloc(sizeof(double) * (size_t)(P->nnz + 1));
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < prow_cnt[i]; ++a) {
      P->ci[P->rp[i] + a] = pcol[(size_t)i * pmax + a];
      P->v[P->rp[i] + a] = pval[(size_t)i * pmax + a];
    }
  free(cidx); free(prow_cnt); free(pcol); free(pval); free(chat); free(num); free(ord);
  *nc_out = nc;
  return ORC_OK;
}

/* transpose of a CSR (rows of the result list source rows in increasing order) */
static void csr_transpose(const ocsr* A, ocsr* T) {
  T->n = A->m; T->m = A->n; T->nnz = A->nnz;
  T->rp = (int32_t*)calloc((size_t)T->n + 1, sizeof(int32_t));
  T->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(A->nnz + 1));
  T->v = (double*)malloc(sizeof(double) * (size_t)(A->nnz + 1));
  for (int t = 0; t < A->nnz; ++t) T->rp[A->ci[t] + 1]++;
  for (int i = 0; i < T->n; ++i) T->rp[i + 1] += T->rp[i];
  int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)(T->n + 1));
  for (int i = 0; i < T->n; ++i) fill[i] = T->rp[i];
  for (int i = 0; i < A->n; ++i)
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      int pos = fill[A->ci[t]]++;
      T->ci[pos] = i;
      T->v[pos] = A->v[t];
    }
  free(fill);
}

/* C = A * B (Gustavson; each output entry accumulates in the loop order
 * k ascending over row i of A, then along row k of B; columns sorted) */
static void csr_matmul(const ocsr* A, const ocsr* B, ocsr* C) {
  int n = A->n, m = B->m;
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
  double* acc = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  for (int j = 0; j < m; ++j) mark[j] = -1;
  C->n = n; C->m = m;
  C->rp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  C->rp[0] = 0;
  for (int i = 0; i < n; ++i) {
    int cnt = 0;
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      int k = A->ci[t];
      for (int t2 = B->rp[k]; t2 < B->rp[k + 1]; ++t2) {
        int j = B->ci[t2];
        if (mark[j] != i) { mark[j] = i; ++cnt; }
      }
    }
    C->rp[i + 1] = C->rp[i] + cnt;
  }
  C->nnz = C->rp[n];
  C->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(C->nnz + 1));
  C->v = (double*)malloc(sizeof(double) * (size_t)(C->nnz + 1));
  for (int j = 0; j < m; ++j) mark[j] = -1;
  for (int i = 0; i < n; ++i) {
    int base = C->rp[i], cnt = 0;
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      int k = A->ci[t];
      double a = A->v[t];
      for (int t2 = B->rp[k]; t2 < B->rp[k + 1]; ++t2) {
        int j = B->ci[t2];
        if (mark[j] != i) { mark[j] = i; C->ci[base + cnt++] = j; acc[j] = 0.0; }
        acc[j] += a * B->v[t2];
      }
    }
    qsort(C->ci + base, (size_t)cnt, sizeof(int32_t), cmp_int);
    for (int t = 0; t < cnt; ++t) C->v[base + t] = acc[C->ci[base + t]];
  }
  free(mark); free(acc);
}

static void truncate_rows(ocsr* P, int pmax);

/* Aggressive coarsening of the first level, second pass (agg = 2, READING
 * R19): among the first split's C points, j is a distance-two strong
 * dependency of i when j is a strong dependency of i, or of a strong
 * dependency k of i (any k, C or F); the C points are split again, by the
 * same algorithm, on that graph (its PMIS weights are level 1's), and a C
 * point stays C only if this second split keeps it.  cf: in the first split,
 * out the final one. */
static int aggressive_split(const ocsr* A, const char* S, const orc_params* p, int32_t* cf) {
  int n = A->n, nc1 = 0;
  int32_t* c1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  for (int i = 0; i < n; ++i) c1[i] = (cf[i] == 1) ? nc1++ : -1;
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  for (int i = 0; i < n; ++i) mark[i] = -1;
  ocsr G;
  G.n = G.m = nc1;
  G.rp = (int32_t*)calloc((size_t)nc1 + 1, sizeof(int32_t));
  int cap = 16, nnz = 0;
  G.ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  for (int i = 0; i < n; ++i) {
    if (cf[i] != 1) continue;
    int q = 0;
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      if (!S[t]) continue;
      int k = A->ci[t];
      if (cf[k] == 1 && k != i && mark[k] != i) { mark[k] = i; list[q++] = k; }
      for (int t2 = A->rp[k]; t2 < A->rp[k + 1]; ++t2) {
        if (!S[t2]) continue;
        int j = A->ci[t2];
        if (cf[j] == 1 && j != i && mark[j] != i) { mark[j] = i; list[q++] = j; }
      }
    }
    qsort(list, (size_t)q, sizeof(int32_t), cmp_int);
    if (nnz + q > cap) {
      while (nnz + q > cap) cap *= 2;
      G.ci = (int32_t*)realloc(G.ci, sizeof(int32_t) * (size_t)cap);
    }
    for (int a = 0; a < q; ++a) G.ci[nnz++] = c1[list[a]];
    G.rp[c1[i] + 1] = nnz;
  }
  G.nnz = nnz;
  G.v = (double*)malloc(sizeof(double) * (size_t)(nnz + 1));
  char* S2 = (char*)malloc((size_t)nnz + 1);
  for (int t = 0; t < nnz; ++t) { G.v[t] = 1.0; S2[t] = 1; }
  int32_t* cf2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nc1 + 1));
  int st = (p->coarsen == ORC_COARSEN_HMIS) ? rs_first_pass(&G, S2, cf2)
                                             : pmis(&G, S2, p->seed, 1, NULL, cf2);
  for (int i = 0; i < n; ++i)
    if (cf[i] == 1 && cf2[c1[i]] != 1) cf[i] = -1;
  free(c1); free(mark); free(list); free(S2); free(cf2);
  free(G.rp); free(G.ci); free(G.v);
  return st;
}

/* Multipass interpolation (Stueben 2001; READING R19).  C points interpolate
 * themselves (pass 0).  In pass p = 1, 2, ... every F point not yet
 * interpolated that has strong dependencies interpolated in earlier passes
 * (the set K_i, C points included) gets
 *   P_i = sum_{k in K_i} w_ik P_k,   w_ik = -(alpha_i a_ik) / d_i,
 *   alpha_i = (sum of its same-function couplings of sign opposite to a_ii)
 *             / (sum_{k in K_i} a_ik),
 *   d_i = a_ii + (its same-function couplings of the same sign as a_ii),
 * sums in column order; pass 1 is direct interpolation from the strong C
 * neighbours.  The rows of a pass are the product W_p P of the pass's weights
 * and the rows built before it.  F points that no pass reaches interpolate
 * from nothing.  Rows are then truncated as build_interp's (truncate_rows). */
static void multipass_interp(const ocsr* A, const int32_t* func, const char* S, const int32_t* cf,
                             int pmax, ocsr* P, int* nc_out) {
  int n = A->n, nc = 0;
  int32_t* cidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t* pass = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  for (int i = 0; i < n; ++i) {
    cidx[i] = (cf[i] == 1) ? nc++ : -1;
    pass[i] = (cf[i] == 1) ? 0 : -1;
  }
  ocsr Q;  /* the rows built so far (empty for points not yet reached) */
  Q.n = n; Q.m = nc; Q.nnz = nc;
  Q.rp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  Q.ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nc + 1));
  Q.v = (double*)malloc(sizeof(double) * (size_t)(nc + 1));
  Q.rp[0] = 0;
  for (int i = 0; i < n; ++i) {
    int q = Q.rp[i];
    if (cf[i] == 1) { Q.ci[q] = cidx[i]; Q.v[q] = 1.0; ++q; }
    Q.rp[i + 1] = q;
  }
  int32_t* newp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  for (int ps = 1;; ++ps) {
    /* the pass's weights W (n x n), rows only for the points it reaches */
    ocsr W;
    W.n = W.m = n;
    W.rp = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    int cap = 16, wn = 0, reached = 0;
    W.ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    W.v = (double*)malloc(sizeof(double) * (size_t)cap);
    for (int i = 0; i < n; ++i) {
      newp[i] = pass[i];
      if (pass[i] < 0) {
        double sumK = 0.0;
        int nk = 0;
        for (int t = A->rp[i]; t < A->rp[i + 1]; ++t)
          if (S[t] && pass[A->ci[t]] >= 0) { sumK += A->v[t]; ++nk; }
        if (nk > 0) {
          double aii = row_diag(A, i), s = aii < 0.0 ? -1.0 : 1.0;
          double sumN = 0.0, d = aii;
          for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
            int j = A->ci[t];
            if (j == i || func[j] != func[i]) continue;
            if (s * A->v[t] < 0.0) sumN += A->v[t];
          }
          for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
            int j = A->ci[t];
            if (j == i || func[j] != func[i]) continue;
            if (s * A->v[t] > 0.0) d += A->v[t];
          }
          double alpha = sumN / sumK;
          if (wn + nk > cap) {
            while (wn + nk > cap) cap *= 2;
            W.ci = (int32_t*)realloc(W.ci, sizeof(int32_t) * (size_t)cap);
            W.v = (double*)realloc(W.v, sizeof(double) * (size_t)cap);
          }
          for (int t = A->rp[i]; t < A->rp[i + 1]; ++t)
            if (S[t] && pass[A->ci[t]] >= 0) {
              W.ci[wn] = A->ci[t];
              W.v[wn] = -(alpha * A->v[t]) / d;
              ++wn;
            }
          newp[i] = ps;
          ++reached;
        }
      }
      W.rp[i + 1] = wn;
    }
    W.nnz = wn;
    if (reached == 0) { csr_free(&W); break; }
    ocsr WQ;
    csr_matmul(&W, &Q, &WQ);
    /* Q takes the new rows of WQ (those rows of Q are empty) */
    ocsr N2;
    N2.n = n; N2.m = nc;
    N2.rp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
    N2.rp[0] = 0;
    for (int i = 0; i < n; ++i) {
      int len = (newp[i] == ps && pass[i] < 0) ? WQ.rp[i + 1] - WQ.rp[i] : Q.rp[i + 1] - Q.rp[i];
      N2.rp[i + 1] = N2.rp[i] + len;
    }
    N2.nnz = N2.rp[n];
    N2.ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N2.nnz + 1));
    N2.v = (double*)malloc(sizeof(double) * (size_t)(N2.nnz + 1));
    for (int i = 0; i < n; ++i) {
      const ocsr* src = (newp[i] == ps && pass[i] < 0) ? &WQ : &Q;
      int q = N2.rp[i];
      for (int t = src->rp[i]; t < src->rp[i + 1]; ++t, ++q) {
        N2.ci[q] = src->ci[t];
        N2.v[q] = src->v[t];
      }
    }
    csr_free(&Q); csr_free(&W); csr_free(&WQ);
    Q = N2;
    for (int i = 0; i < n; ++i) pass[i] = newp[i];
  }
  truncate_rows(&Q, pmax);
  *P = Q;
  *nc_out = nc;
  free(cidx); free(pass); free(newp);
}

static void level_alloc_work(olevel* L) {
  int n = L->A.n;
  L->b = (double*)calloc((size_t)n + 1, sizeof(double));
  L->x = (double*)calloc((size_t)n + 1, sizeof(double));
  L->r = (double*)calloc((size_t)n + 1, sizeof(double));
  L->x2 = (double*)calloc((size_t)n + 1, sizeof(double));
}

static void csr_copy(ocsr* dst, int n, int m, const int32_t* rp, const int32_t* ci, const double* v) {
  dst->n = n; dst->m = m; dst->nnz = rp[n];
  dst->rp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  dst->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(dst->nnz + 1));
  dst->v = (double*)malloc(sizeof(double) * (size_t)(dst->nnz + 1));
  memcpy(dst->rp, rp, sizeof(int32_t) * (size_t)(n + 1));
  memcpy(dst->ci, ci, sizeof(int32_t) * (size_t)dst->nnz);
  memcpy(dst->v, v, sizeof(double) * (size_t)dst->nnz);
}

void orc_amg_destroy(orc_amg* a) {
  if (!a) return;
  for (int l = 0; l < a->nlev; ++l) {
    olevel* L = &a->lev[l];
    csr_free(&L->A); csr_free(&L->P); csr_free(&L->R);
    free(L->func); free(L->cf); free(L->dl1); free(L->b); free(L->x); free(L->r); free(L->x2);
  }
  free(a->LU); free(a->piv); free(a->work);
  free(a);
}

/* l1 diagonal. READING: "first order relaxation" (Section 3.1) is taken as
 * l1-Jacobi, d_i = a_ii + sign(a_ii) * sum_{j != i} |a_ij| over the full row. */
static void l1_diag(const ocsr* A, double* d) {
  for (int i = 0; i < A->n; ++i) {
    double aii = 0.0, off = 0.0;
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      if (A->ci[t] == i) aii = A->v[t]; else off += fabs(A->v[t]);
    }
    d[i] = (aii < 0.0) ? aii - off : aii + off;
  }
}

/* Truncation of one interpolation operator's rows to pmax entries by the rule
 * of build_interp (READING R7): exact zeros dropped, the pmax largest |w| kept
 * (ties: smaller column), rescaled by (sum of all w) / (sum of kept w) when the
 * kept sum is nonzero, kept entries in column order. */
static void truncate_rows(ocsr* P, int pmax) {
  int32_t* rp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P->n + 1));
  int32_t* ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P->nnz + 1));
  double* v = (double*)malloc(sizeof(double) * (size_t)(P->nnz + 1));
  int* ord = (int*)malloc(sizeof(int) * (size_t)(P->nnz + 1));
  int q = 0;
  rp[0] = 0;
  for (int i = 0; i < P->n; ++i) {
    int t0 = P->rp[i], m = 0;
    for (int t = t0; t < P->rp[i + 1]; ++t)
      if (P->v[t] != 0.0) ord[t0 + m++] = t;     /* positions of the nonzeros */
    int* o = ord + t0;
    if (m > pmax) {
      double sum_all = 0.0;
      for (int k = 0; k < m; ++k) sum_all += P->v[o[k]];
      for (int a = 0; a < pmax; ++a) {
        int best = a;
        for (int b2 = a + 1; b2 < m; ++b2) {
          double wb = fabs(P->v[o[b2]]), wa = fabs(P->v[o[best]]);
          if (wb > wa || (wb == wa && o[b2] < o[best])) best = b2;
        }
        int tmp = o[a]; o[a] = o[best]; o[best] = tmp;
      }
      qsort(o, (size_t)pmax, sizeof(int), cmp_int);
      double sum_kept = 0.0;
      for (int a = 0; a < pmax; ++a) sum_kept += P->v[o[a]];
      double scale = (sum_kept != 0.0) ? sum_all / sum_kept : 1.0;
      for (int a = 0; a < pmax; ++a) { ci[q] = P->ci[o[a]]; v[q] = P->v[o[a]] * scale; ++q; }
    } else {
      for (int a = 0; a < m; ++a) { ci[q] = P->ci[o[a]]; v[q] = P->v[o[a]]; ++q; }
    }
    rp[i + 1] = q;
  }
  free(P->rp); free(P->ci); free(P->v); free(ord);
  P->rp = rp; P->ci = ci; P->v = v; P->nnz = q;
}

static orc_amg* amg_build(ocsr* A0 /* taken */, int32_t* func0 /* taken */, const orc_params* p,
                          const int32_t* forced_cf0, const int32_t* forced_cf1,
                          const double* rho0, int* status) {
  orc_amg* a = (orc_amg*)calloc(1, sizeof(orc_amg));
  a->nu_pre = p->nu_pre;
  a->nu_post = p->nu_post;
  a->smoother = p->smoother;
  a->lev[0].A = *A0;
  a->lev[0].func = func0;
  a->nlev = 1;
  *status = ORC_OK;
  int collapsed = 0;
  for (int l = 0;; ++l) {
    olevel* L = &a->lev[l];
    level_alloc_work(L);
    int n = L->A.n;
    int coarsest = (n <= p->max_coarse) || (l + 1 >= p->max_levels);
    if (!coarsest) {
      char* S = (char*)malloc((size_t)L->A.nnz + 1);
      strength(&L->A, L->func, p->theta, S);
      L->cf = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
      if (l == 0 && forced_cf0) memcpy(L->cf, forced_cf0, sizeof(int32_t) * (size_t)n);
      else if (l == 1 && p->agg == 1 && !collapsed && forced_cf1)
        memcpy(L->cf, forced_cf1, sizeof(int32_t) * (size_t)n);
      else if ((p->coarsen == ORC_COARSEN_HMIS ? rs_first_pass(&L->A, S, L->cf)
                : pmis(&L->A, S, p->seed, l, (l == 0) ? rho0 : NULL, L->cf)) != ORC_OK) {
        free(S);
        *status = ORC_BREAKDOWN;
        a->nlev = l + 1;
        return a;
      }
      if (l == 0 && p->agg == 2 && aggressive_split(&L->A, S, p, L->cf) != ORC_OK) {
        free(S);
        *status = ORC_BREAKDOWN;
        a->nlev = l + 1;
        return a;
      }
      int nc = 0;
      for (int i = 0; i < n; ++i) nc += (L->cf[i] == 1);
      if (nc == 0 || (double)nc > 0.9 * (double)n) {
        coarsest = 1;            /* coarsening stalled: this level is solved directly */
        free(L->cf); L->cf = NULL;
      } else if (l == 1 && p->agg == 1 && !collapsed) {
        /* "One aggregate level" (READING R8): the first level is coarsened a
         * second time, on the Galerkin operator of its first split, and
         * interpolates in two stages, P = trunc(P1 P2); its coarse operator is
         * P^T A P.  The intermediate operator is not kept as a level. */
        olevel* L0 = &a->lev[0];
        ocsr P2, P, R, AP, Ac;
        int nc2 = 0;
        build_interp(&L->A, L->func, S, L->cf, p->pmax, &P2, &nc2);
        csr_matmul(&L0->P, &P2, &P);
        truncate_rows(&P, p->pmax);
        csr_transpose(&P, &R);
        csr_matmul(&L0->A, &P, &AP);
        csr_matmul(&R, &AP, &Ac);
        csr_free(&AP); csr_free(&P2);
        for (int i = 0, c1 = 0; i < L0->A.n; ++i)     /* C points of both stages */
          if (L0->cf[i] == 1) { if (L->cf[c1] != 1) L0->cf[i] = -1; ++c1; }
        csr_free(&L0->P); csr_free(&L0->R);
        L0->P = P; L0->R = R; L0->nc = nc2;
        int32_t* f2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nc2 + 1));
        for (int i = 0, c2 = 0; i < n; ++i)
          if (L->cf[i] == 1) f2[c2++] = L->func[i];
        csr_free(&L->A);
        free(L->func); free(L->cf); free(L->b); free(L->x); free(L->r);
        memset(L, 0, sizeof(*L));
        L->A = Ac;
        L->func = f2;
        collapsed = 1;
        a->nlev = 2;
        free(S);
        --l;        /* the new level 1 is processed by the next pass */
        continue;
      } else {
        if (l == 0 && p->agg == 2)
          multipass_interp(&L->A, L->func, S, L->cf, p->pmax, &L->P, &L->nc);
        else
          build_interp(&L->A, L->func, S, L->cf, p->pmax, &L->P, &L->nc);
        csr_transpose(&L->P, &L->R);
        ocsr AP, Ac;
        csr_matmul(&L->A, &L->P, &AP);
        csr_matmul(&L->R, &AP, &Ac);
        csr_free(&AP);
        L->dl1 = (double*)malloc(sizeof(double) * (size_t)(n + 1));
        l1_diag(&L->A, L->dl1);
        olevel* Nx = &a->lev[l + 1];
        Nx->A = Ac;
        Nx->func = (int32_t*)malloc(sizeof(int32_t) * (size_t)(L->nc + 1));
        for (int i = 0, c = 0; i < n; ++i)
          if (L->cf[i] == 1) Nx->func[c++] = L->func[i];
        a->nlev = l + 2;
      }
      free(S);
    }
    if (coarsest) {
      if (n > MAX_DENSE_COARSE) { *status = ORC_BREAKDOWN; a->nlev = l + 1; return a; }
      a->nlev = l + 1;
      a->ncoarse = n;
      a->LU = (double*)calloc((size_t)n * n + 1, sizeof(double));
      a->piv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
      a->work = (double*)malloc(sizeof(double) * (size_t)(n + 1));
      for (int i = 0; i < n; ++i)
        for (int t = L->A.rp[i]; t < L->A.rp[i + 1]; ++t)
          a->LU[(size_t)i * n + L->A.ci[t]] += L->A.v[t];
      if (n > 0 && dense_lu(n, a->LU, a->piv) != ORC_OK) *status = ORC_BREAKDOWN;
      break;
    }
  }
  return a;
}

orc_amg* orc_amg_create(int n, const int32_t* rp, const int32_t* ci, const double* v,
                        const int32_t* func, const orc_params* p, const int32_t* forced_cf0,
                        const int32_t* forced_cf1, const double* rho0, int* status) {
  ocsr A;
  csr_copy(&A, n, n, rp, ci, v);
  int32_t* f = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
  if (func) memcpy(f, func, sizeof(int32_t) * (size_t)n);
  int st = 0;
  orc_amg* a = amg_build(&A, f, p, forced_cf0, forced_cf1, rho0, &st);
  if (status) *status = st;
  return a;
}

/* One l1-Jacobi sweep: x += D_l1^-1 (b - A x). */
static void l1_jacobi_sweep(const olevel* L, const double* b, double* x) {
  int n = L->A.n;
  csr_mv(&L->A, x, L->r);
  for (int i = 0; i < n; ++i) L->r[i] = b[i] - L->r[i];
  for (int i = 0; i < n; ++i) x[i] += L->r[i] / L->dl1[i];
}

/* One hybrid l1-Gauss-Seidel sweep (see ORC_SMOOTH_HYBRID_GS): each block of
 * ORC_HGS_BLOCK rows relaxes its rows one after the other, forward or backward,
 * x_i += (b_i - sum_j a_ij x_j) / d_i with the newest values of its own rows and
 * the sweep's starting values (xs) of every other row. */
static void hybrid_gs_sweep(const olevel* L, const double* b, double* x, double* xs, int backward) {
  int n = L->A.n;
  memcpy(xs, x, sizeof(double) * (size_t)n);
  for (int k0 = 0; k0 < n; k0 += ORC_HGS_BLOCK) {
    int k1 = k0 + ORC_HGS_BLOCK < n ? k0 + ORC_HGS_BLOCK : n;
    for (int q = 0; q < k1 - k0; ++q) {
      int i = backward ? k1 - 1 - q : k0 + q;
      double s = 0.0;
      for (int t = L->A.rp[i]; t < L->A.rp[i + 1]; ++t) {
        int j = L->A.ci[t];
        s += L->A.v[t] * ((j >= k0 && j < k1) ? x[j] : xs[j]);
      }
      x[i] += (b[i] - s) / L->dl1[i];
    }
  }
}

static void smooth(const orc_amg* a, const olevel* L, const double* b, double* x, int sweeps,
                   int backward) {
  for (int k = 0; k < sweeps; ++k) {
    if (a->smoother == ORC_SMOOTH_HYBRID_GS) hybrid_gs_sweep(L, b, x, L->x2, backward);
    else l1_jacobi_sweep(L, b, x);
  }
}

/* One V(nu_pre, nu_post) cycle from a zero initial guess (Section 3.1: one
 * V-cycle): pre-smoothing, residual, restriction, the coarser cycle,
 * prolongation, post-smoothing; the coarsest level is solved exactly. */
static void vcycle_rec(const orc_amg* a, int l, const double* b, double* x) {
  const olevel* L = &a->lev[l];
  int n = L->A.n;
  if (l == a->nlev - 1) {
    if (n > 0) dense_lu_solve(n, a->LU, a->piv, b, x);
    return;
  }
  const olevel* Nx = &a->lev[l + 1];
  for (int i = 0; i < n; ++i) x[i] = 0.0;
  smooth(a, L, b, x, a->nu_pre, 0);                                /* pre-smooth */
  csr_mv(&L->A, x, L->r);
  for (int i = 0; i < n; ++i) L->r[i] = b[i] - L->r[i];           /* residual */
  csr_mv(&L->R, L->r, Nx->b);                                      /* restrict */
  vcycle_rec(a, l + 1, Nx->b, Nx->x);
  for (int i = 0; i < n; ++i) {                                    /* prolong */
    double s = 0.0;
    for (int t = L->P.rp[i]; t < L->P.rp[i + 1]; ++t) s += L->P.v[t] * Nx->x[L->P.ci[t]];
    x[i] += s;
  }
  smooth(a, L, b, x, a->nu_post, 1);                               /* post-smooth */
}

void orc_amg_vcycle(const orc_amg* a, const double* b, double* x) { vcycle_rec(a, 0, b, x); }
/* `sweeps` smoothing sweeps on level l from the given x (tests of the smoothers) */
void orc_amg_smooth(const orc_amg* a, int l, const double* b, double* x, int sweeps, int backward) {
  smooth(a, &a->lev[l], b, x, sweeps, backward);
}
int orc_amg_nlevels(const orc_amg* a) { return a->nlev; }
void orc_amg_level_info(const orc_amg* a, int l, int32_t* info) {
  const olevel* L = &a->lev[l];
  info[0] = L->A.n; info[1] = L->A.nnz;
  info[2] = (l < a->nlev - 1) ? L->nc : 0;
  info[3] = (l < a->nlev - 1) ? L->P.nnz : 0;
}
void orc_amg_level_A(const orc_amg* a, int l, int32_t* rp, int32_t* ci, double* v) {
  const ocsr* A = &a->lev[l].A;
  memcpy(rp, A->rp, sizeof(int32_t) * (size_t)(A->n + 1));
  memcpy(ci, A->ci, sizeof(int32_t) * (size_t)A->nnz);
  memcpy(v, A->v, sizeof(double) * (size_t)A->nnz);
}
/* The coarsest level (solved directly) has no split, no P and no smoother:
 * there these accessors write zeros (an empty P, cf = 0, dl1 = 0). */
void orc_amg_level_P(const orc_amg* a, int l, int32_t* rp, int32_t* ci, double* v) {
  if (l >= a->nlev - 1) {
    memset(rp, 0, sizeof(int32_t) * (size_t)(a->lev[l].A.n + 1));
    return;
  }
  const ocsr* P = &a->lev[l].P;
  memcpy(rp, P->rp, sizeof(int32_t) * (size_t)(P->n + 1));
  memcpy(ci, P->ci, sizeof(int32_t) * (size_t)P->nnz);
  memcpy(v, P->v, sizeof(double) * (size_t)P->nnz);
}
void orc_amg_level_cf(const orc_amg* a, int l, int32_t* cf) {
  if (l >= a->nlev - 1) {
    memset(cf, 0, sizeof(int32_t) * (size_t)a->lev[l].A.n);
    return;
  }
  memcpy(cf, a->lev[l].cf, sizeof(int32_t) * (size_t)a->lev[l].A.n);
}
void orc_amg_level_func(const orc_amg* a, int l, int32_t* f) {
  memcpy(f, a->lev[l].func, sizeof(int32_t) * (size_t)a->lev[l].A.n);
}
void orc_amg_level_dl1(const orc_amg* a, int l, double* d) {
  if (l >= a->nlev - 1) {
    memset(d, 0, sizeof(double) * (size_t)a->lev[l].A.n);
    return;
  }
  memcpy(d, a->lev[l].dl1, sizeof(double) * (size_t)a->lev[l].A.n);
}
double orc_amg_op_complexity(const orc_amg* a) {
  double s = 0.0;
  for (int l = 0; l < a->nlev; ++l) s += a->lev[l].A.nnz;
  return a->lev[0].A.nnz ? s / a->lev[0].A.nnz : 0.0;
}

/* ================================================================== */
/* full system                                                         */
/* ================================================================== */
/* elliptic unknowns {e0} (e1 < 0) or {e0, e1} of a stage, the others in increasing order */
static void stage_unknowns(ostage* s, int e0, int e1) {
  s->ne = e1 < 0 ? 1 : 2;
  s->nh = 4 - s->ne;
  s->ee[0] = e0;
  s->ee[1] = e1;
  int k = 0;
  for (int u = 0; u < 4; ++u)
    if (u != e0 && u != e1) s->hh[k++] = u;
}

orc_ctx* orc_create(int n_cells, const int32_t* rowptr, const int32_t* col, const double* vals,
                    const orc_params* p) {
  if (n_cells <= 0 || !rowptr || !col || !vals) return NULL;
  orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
  c->N = n_cells;
  c->nnzb = rowptr[n_cells];
  c->rp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_cells + 1));
  c->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(c->nnzb + 1));
  c->v = (double*)malloc(sizeof(double) * 16 * (size_t)(c->nnzb + 1));
  c->diag = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_cells + 1));
  memcpy(c->rp, rowptr, sizeof(int32_t) * (size_t)(n_cells + 1));
  memcpy(c->ci, col, sizeof(int32_t) * (size_t)c->nnzb);
  memcpy(c->v, vals, sizeof(double) * 16 * (size_t)c->nnzb);
  if (p) c->p = *p; else orc_params_default(&c->p);
  for (int i = 0; i < n_cells; ++i) {
    c->diag[i] = -1;
    for (int t = c->rp[i]; t < c->rp[i + 1]; ++t) {
      if (c->ci[t] < 0 || c->ci[t] >= n_cells || (t > c->rp[i] && c->ci[t] <= c->ci[t - 1])) {
        orc_destroy(c); return NULL;
      }
      if (c->ci[t] == i) c->diag[i] = t;
    }
    if (c->diag[i] < 0) { orc_destroy(c); return NULL; }
  }
  if (c->p.nu_pre < 0 || c->p.nu_post < 0 || c->p.nu_pre > 8 || c->p.nu_post > 8 ||
      (c->p.smoother != ORC_SMOOTH_L1_JACOBI && c->p.smoother != ORC_SMOOTH_HYBRID_GS) ||
      (c->p.coarsen != ORC_COARSEN_PMIS && c->p.coarsen != ORC_COARSEN_HMIS) ||
      c->p.agg < 0 || c->p.agg > 2) {
    orc_destroy(c);
    return NULL;
  }
  if (c->p.e0 < 0 || c->p.e0 > 3 || c->p.e1 < -1 || c->p.e1 > 3 || c->p.e1 == c->p.e0 ||
      (c->p.mgr && (c->p.e0 == MGR_U || c->p.e1 == MGR_U))) {
    orc_destroy(c);
    return NULL;
  }
  if (c->p.mgr) {
    c->vfull = (double*)malloc(sizeof(double) * 16 * (size_t)(c->nnzb + 1));
    memcpy(c->vfull, vals, sizeof(double) * 16 * (size_t)c->nnzb);
  }
  if (c->p.precond == ORC_PREC_CPTR3 || c->p.precond == ORC_PREC_CPTR3_EXACT) {
    /* CPTR3 (Section 3.3): pressure and temperature each decoupled on its own,
     * stage 0 keeps e0 (p), stage 1 keeps e1 (T) */
    if (c->p.e1 < 0) { orc_destroy(c); return NULL; }
    c->nst = 2;
    stage_unknowns(&c->st[0], c->p.e0, -1);
    stage_unknowns(&c->st[1], c->p.e1, -1);
  } else {
    c->nst = 1;
    stage_unknowns(&c->st[0], c->p.e0, c->p.e1);
  }
  size_t n4 = (size_t)4 * n_cells;
  c->t4a = (double*)calloc(n4, sizeof(double));
  c->t4b = (double*)calloc(n4, sizeof(double));
  c->t4c = (double*)calloc(n4, sizeof(double));
  c->t2a = (double*)calloc(n4 / 2, sizeof(double));
  c->t2b = (double*)calloc(n4 / 2, sizeof(double));
  return c;
}

void orc_destroy(orc_ctx* c) {
  if (!c) return;
  free(c->rp); free(c->ci); free(c->v); free(c->vfull); free(c->diag);
  for (int k = 0; k < 2; ++k) {
    free(c->st[k].W);
    csr_free(&c->st[k].Ahat);
    orc_amg_destroy(c->st[k].amg);
    free(c->st[k].AhLU); free(c->st[k].AhPiv);
  }
  free(c->LU); free(c->ilu_level);
  free(c->lastV); free(c->lastZ); free(c->lastH);
  free(c->t4a); free(c->t4b); free(c->t4c); free(c->t2a); free(c->t2b);
  free(c);
}

/* Quasi-IMPES decoupling (Section 3 first stage; Section 5.2 "Quasi-IMPES").
 * READING: R_i = [I_e, -W_i] with W_i = D_i[e,h] * inv(D_i[h,h]) from the
 * diagonal block D_i = A_ii only; prolongation is injection into e.
 * Ahat_ij = A_ij[e,e] - W_i A_ij[h,e] = (R A P)_ij.  CPTR (Section 3.2) has
 * e = {p, T} and a 2x2 D[h,h]; CPR (Section 3.1) has e = {p} and a 3x3 D[h,h].
 * inv(D[h,h]) is the adjugate divided by the determinant (cofactor formula). */
static int decouple(orc_ctx* c, ostage* sg) {
  int N = c->N, ne = sg->ne, nh = sg->nh, *e = sg->ee, *h = sg->hh;
  sg->W = (double*)malloc(sizeof(double) * 4 * (size_t)N);
  for (int i = 0; i < N; ++i) {
    const double* D = c->v + 16 * (size_t)c->diag[i];
    double inv[9];
    if (nh == 2) {
      double a = D[h[0] * 4 + h[0]], b = D[h[0] * 4 + h[1]];
      double cc = D[h[1] * 4 + h[0]], d = D[h[1] * 4 + h[1]];
      double det = a * d - b * cc;
      double mx = fmax(fmax(fabs(a), fabs(b)), fmax(fabs(cc), fabs(d)));
      if (!(fabs(det) > 1e-300 * mx * mx) || !isfinite(det)) return ORC_BREAKDOWN;
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
      if (!(fabs(det) > 1e-300 * mx * mx * mx) || !isfinite(det)) return ORC_BREAKDOWN;
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
        sg->W[4 * (size_t)i + nh * r + s] = acc;
      }
  }
  ocsr* Ah = &sg->Ahat;
  Ah->n = Ah->m = ne * N;
  Ah->nnz = ne * ne * c->nnzb;
  Ah->rp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ne * N + 1));
  Ah->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(Ah->nnz + 1));
  Ah->v = (double*)malloc(sizeof(double) * (size_t)(Ah->nnz + 1));
  int pos = 0;
  for (int i = 0; i < N; ++i) {
    const double* W = sg->W + 4 * (size_t)i;
    for (int r = 0; r < ne; ++r) {
      Ah->rp[ne * i + r] = pos;
      for (int t = c->rp[i]; t < c->rp[i + 1]; ++t) {
        const double* B = c->v + 16 * (size_t)t;
        for (int s = 0; s < ne; ++s) {
          double acc = B[e[r] * 4 + e[s]];
          for (int q = 0; q < nh; ++q) acc -= W[nh * r + q] * B[h[q] * 4 + e[s]];
          Ah->ci[pos] = ne * c->ci[t] + s;
          Ah->v[pos] = acc;
          ++pos;
        }
      }
    }
  }
  Ah->rp[ne * N] = pos;
  return ORC_OK;
}

/* Block ILU(0) in natural order, IKJ form, no pivoting (Section 3.1: zero fill-in).
 * Stores L_ik (unit block-lower), U_ij and inv(U_ii) in place of A's blocks. */
static int ilu0_factor(orc_ctx* c) {
  int N = c->N;
  c->LU = (double*)malloc(sizeof(double) * 16 * (size_t)(c->nnzb + 1));
  memcpy(c->LU, c->v, sizeof(double) * 16 * (size_t)c->nnzb);
  double tmp[16];
  for (int i = 0; i < N; ++i) {
    for (int t = c->rp[i]; t < c->rp[i + 1]; ++t) {
      int k = c->ci[t];
      if (k >= i) break;
      double* Aik = c->LU + 16 * (size_t)t;
      mul4(Aik, c->LU + 16 * (size_t)c->diag[k], tmp);     /* L_ik = A_ik inv(U_kk) */
      memcpy(Aik, tmp, sizeof(tmp));
      int t2 = c->diag[k] + 1;                               /* U_kj, j > k */
      for (int t3 = t + 1; t3 < c->rp[i + 1]; ++t3) {
        int j = c->ci[t3];
        while (t2 < c->rp[k + 1] && c->ci[t2] < j) ++t2;
        if (t2 < c->rp[k + 1] && c->ci[t2] == j) {
          mul4(Aik, c->LU + 16 * (size_t)t2, tmp);
          double* Aij = c->LU + 16 * (size_t)t3;
          for (int q = 0; q < 16; ++q) Aij[q] -= tmp[q];
        }
      }
    }
    double* Dii = c->LU + 16 * (size_t)c->diag[i];
    if (inv4(Dii, tmp) != ORC_OK) return ORC_BREAKDOWN;
    memcpy(Dii, tmp, sizeof(tmp));
  }
  /* level sets of the lower triangle (reported; the oracle solves sequentially) */
  c->ilu_level = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N + 1));
  int mx = 0;
  for (int i = 0; i < N; ++i) {
    int lv = 0;
    for (int t = c->rp[i]; t < c->diag[i]; ++t) {
      int q = c->ilu_level[c->ci[t]] + 1;
      if (q > lv) lv = q;
    }
    c->ilu_level[i] = lv;
    if (lv > mx) mx = lv;
  }
  c->ilu_nlev = mx + 1;
  return ORC_OK;
}

/* First MGR reduction (Section 3.4): equation row MGR_U of every cell is a
 * volume constraint that involves only the cell's own unknowns, so unknown
 * MGR_U of cell j is x_j[u] = (b_j[u] - sum_{s != u} A_jj[u,s] x_j[s]) / A_jj[u,u]
 * exactly.  Substituting it into every other row gives the reduced operator
 *   At_ij[r,s] = A_ij[r,s] - A_ij[r,u] * (A_jj[u,s] / A_jj[u,u]),  r, s != u,
 * the Schur complement of the constraint block, with no approximation.
 * READING: the reduced system keeps the 4x4 block layout; row and column u
 * become the identity row and column (zero right-hand side), so CPTR on it is
 * CPTR on the remaining (p, rho, T) unknowns. */
static int mgr_reduce(orc_ctx* c) {
  const int u = MGR_U;
  for (int i = 0; i < c->N; ++i) {
    double q = c->vfull[16 * (size_t)c->diag[i] + 5 * u];
    if (q == 0.0 || !isfinite(q)) return ORC_BREAKDOWN;
    for (int t = c->rp[i]; t < c->rp[i + 1]; ++t) {
      if (t == c->diag[i]) continue;
      const double* B = c->vfull + 16 * (size_t)t;
      for (int s = 0; s < 4; ++s)
        if (B[4 * u + s] != 0.0) return ORC_INVALID;   /* the constraint is not local */
    }
  }
  for (int i = 0; i < c->N; ++i)
    for (int t = c->rp[i]; t < c->rp[i + 1]; ++t) {
      const double* B = c->vfull + 16 * (size_t)t;
      const double* Dj = c->vfull + 16 * (size_t)c->diag[c->ci[t]];
      double* R = c->v + 16 * (size_t)t;
      for (int r = 0; r < 4; ++r)
        for (int s = 0; s < 4; ++s) {
          if (r == u || s == u) R[4 * r + s] = (r == s && c->ci[t] == i) ? 1.0 : 0.0;
          else R[4 * r + s] = B[4 * r + s] - B[4 * r + u] * (Dj[4 * u + s] / Dj[5 * u]);
        }
    }
  return ORC_OK;
}

/* reduced right-hand side bt_i[r] = b_i[r] - sum_j A_ij[r,u] * (b_j[u] / A_jj[u,u]), bt_i[u] = 0 */
static void mgr_rhs(const orc_ctx* c, const double* b, double* bt) {
  const int u = MGR_U;
  for (int i = 0; i < c->N; ++i)
    for (int r = 0; r < 4; ++r) {
      if (r == u) { bt[4 * (size_t)i + r] = 0.0; continue; }
      double acc = b[4 * (size_t)i + r];
      for (int t = c->rp[i]; t < c->rp[i + 1]; ++t) {
        int j = c->ci[t];
        const double* B = c->vfull + 16 * (size_t)t;
        acc -= B[4 * r + u] * (b[4 * (size_t)j + u] / c->vfull[16 * (size_t)c->diag[j] + 5 * u]);
      }
      bt[4 * (size_t)i + r] = acc;
    }
}

/* eliminated unknown from the constraint row: x_i[u] = (b_i[u] - sum_{s != u} A_ii[u,s] x_i[s]) / A_ii[u,u] */
static void mgr_recover(const orc_ctx* c, const double* b, double* x) {
  const int u = MGR_U;
  for (int i = 0; i < c->N; ++i) {
    const double* D = c->vfull + 16 * (size_t)c->diag[i];
    double acc = b[4 * (size_t)i + u];
    for (int s = 0; s < 4; ++s)
      if (s != u) acc -= D[4 * u + s] * x[4 * (size_t)i + s];
    x[4 * (size_t)i + u] = acc / D[5 * u];
  }
}

/* Decoupling, then the system AMG on Ahat (functions alternate over the
 * elliptic unknowns: one function, i.e. scalar AMG, for a single unknown), or a
 * dense LU of Ahat in the exact-stage test modes. */
static int build_stage(orc_ctx* c, ostage* sg) {
  int st = decouple(c, sg);
  if (st) return st;
  const int pc = c->p.precond;
  if (pc == ORC_PREC_CPTR_EXACT1 || pc == ORC_PREC_CPTR3_EXACT) {
    int n = sg->Ahat.n;
    sg->AhLU = (double*)calloc((size_t)n * n, sizeof(double));
    sg->AhPiv = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int i = 0; i < n; ++i)
      for (int t = sg->Ahat.rp[i]; t < sg->Ahat.rp[i + 1]; ++t)
        sg->AhLU[(size_t)i * n + sg->Ahat.ci[t]] += sg->Ahat.v[t];
    return dense_lu(n, sg->AhLU, sg->AhPiv);
  }
  if (pc == ORC_PREC_CPTR || pc == ORC_PREC_FIRST || pc == ORC_PREC_CPTR3) {
    ocsr Acopy;
    csr_copy(&Acopy, sg->Ahat.n, sg->Ahat.m, sg->Ahat.rp, sg->Ahat.ci, sg->Ahat.v);
    int32_t* func = (int32_t*)malloc(sizeof(int32_t) * (size_t)(sg->Ahat.n + 1));
    for (int i = 0; i < sg->Ahat.n; ++i) func[i] = i % sg->ne;
    sg->amg = amg_build(&Acopy, func, &c->p, NULL, NULL, NULL, &st);
  }
  return st;
}

int orc_setup(orc_ctx* c) {
  if (!c) return ORC_INVALID;
  if (c->p.mgr) {
    int sr = mgr_reduce(c);
    if (sr) return sr;
  }
  int st = 0;
  for (int k = 0; k < c->nst; ++k) {
    st = build_stage(c, &c->st[k]);
    if (st) return st;
  }
  st = ilu0_factor(c);
  if (st) return st;
  c->setup_done = 1;
  return ORC_OK;
}

void orc_spmv(const orc_ctx* c, const double* x, double* y) {
  for (int i = 0; i < c->N; ++i) {
    double s[4] = {0, 0, 0, 0};
    for (int t = c->rp[i]; t < c->rp[i + 1]; ++t) {
      const double* B = c->v + 16 * (size_t)t;
      const double* xj = x + 4 * (size_t)c->ci[t];
      for (int r = 0; r < 4; ++r)
        for (int q = 0; q < 4; ++q) s[r] += B[r * 4 + q] * xj[q];
    }
    for (int r = 0; r < 4; ++r) y[4 * (size_t)i + r] = s[r];
  }
}

/* restriction rhat_i = r_i[e] - W_i r_i[h] of one stage */
static void stage_restrict(const orc_ctx* c, const ostage* sg, const double* r, double* rhat) {
  for (int i = 0; i < c->N; ++i) {
    const double* ri = r + 4 * (size_t)i;
    const double* W = sg->W + 4 * (size_t)i;
    for (int q = 0; q < sg->ne; ++q) {
      double e = ri[sg->ee[q]];
      for (int t = 0; t < sg->nh; ++t) e -= W[sg->nh * q + t] * ri[sg->hh[t]];
      rhat[sg->ne * (size_t)i + q] = e;
    }
  }
}

static void stage_vcycle(const ostage* sg, const double* b, double* x) {
  if (sg->AhLU) { dense_lu_solve(sg->Ahat.n, sg->AhLU, sg->AhPiv, b, x); return; }
  vcycle_rec(sg->amg, 0, b, x);
}

/* one stage's M^-1 r = P Vcycle(Ahat, R r), P = injection into its elliptic unknowns */
static void stage_apply(const orc_ctx* c, const ostage* sg, const double* r, double* y1) {
  stage_restrict(c, sg, r, c->t2a);
  stage_vcycle(sg, c->t2a, c->t2b);
  for (int i = 0; i < c->N; ++i) {
    double* y = y1 + 4 * (size_t)i;
    y[0] = y[1] = y[2] = y[3] = 0.0;
    for (int q = 0; q < sg->ne; ++q) y[sg->ee[q]] = c->t2b[sg->ne * (size_t)i + q];
  }
}

void orc_restrict(const orc_ctx* c, const double* r, double* rhat) {
  stage_restrict(c, &c->st[0], r, rhat);
}

void orc_vcycle(const orc_ctx* c, const double* b, double* x) { stage_vcycle(&c->st[0], b, x); }

/* M1^-1 r = P Vcycle(Ahat, R r) of the first stage */
void orc_first_stage(const orc_ctx* c, const double* r, double* y1) {
  stage_apply(c, &c->st[0], r, y1);
}

/* CPTR3's first two stages (Section 3.3), composed like Eq. 3:
 * y = yA + yB with yA = M_p r (pressure stage) and yB = M_T (r - A yA)
 * (temperature stage), i.e. M_pT = M_p + M_T (I - A M_p).
 * READING: the paper names the three-stage split and that pressure and
 * temperature each go to a monolithic AMG, and refers to an earlier paper for
 * the algorithm; the stages are taken in the order p, T, ILU(0), each applied
 * to the residual the previous ones leave, like the two stages of Eq. 3. */
void orc_cptr3_first_two(const orc_ctx* c, const double* r, double* y) {
  size_t n4 = 4 * (size_t)c->N;
  double* yB = (double*)malloc(sizeof(double) * n4);
  double* r1 = (double*)malloc(sizeof(double) * n4);
  stage_apply(c, &c->st[0], r, y);
  orc_spmv(c, y, r1);
  for (size_t i = 0; i < n4; ++i) r1[i] = r[i] - r1[i];
  stage_apply(c, &c->st[1], r1, yB);
  for (size_t i = 0; i < n4; ++i) y[i] += yB[i];
  free(yB); free(r1);
}

/* the temperature stage of CPTR3 alone: M_T r = P_T Vcycle(Ahat_T, R_T r) */
void orc_cptr3_stage_t(const orc_ctx* c, const double* r, double* y) {
  stage_apply(c, &c->st[1], r, y);
}

/* r2 = r - A y1 */
void orc_correction(const orc_ctx* c, const double* r, const double* y1, double* r2) {
  orc_spmv(c, y1, r2);
  for (size_t i = 0; i < 4 * (size_t)c->N; ++i) r2[i] = r[i] - r2[i];
}

/* y = (LU)^-1 r: forward u_i = r_i - sum_{k<i} L_ik u_k, backward
 * y_i = inv(U_ii) (u_i - sum_{j>i} U_ij y_j) */
void orc_ilu_apply(const orc_ctx* c, const double* r, double* y) {
  int N = c->N;
  for (int i = 0; i < N; ++i) {
    double u[4];
    for (int q = 0; q < 4; ++q) u[q] = r[4 * (size_t)i + q];
    for (int t = c->rp[i]; t < c->diag[i]; ++t) {
      const double* L = c->LU + 16 * (size_t)t;
      const double* uk = y + 4 * (size_t)c->ci[t];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) u[a] -= L[a * 4 + b] * uk[b];
    }
    for (int q = 0; q < 4; ++q) y[4 * (size_t)i + q] = u[q];
  }
  for (int i = N - 1; i >= 0; --i) {
    double u[4];
    for (int q = 0; q < 4; ++q) u[q] = y[4 * (size_t)i + q];
    for (int t = c->diag[i] + 1; t < c->rp[i + 1]; ++t) {
      const double* U = c->LU + 16 * (size_t)t;
      const double* yj = y + 4 * (size_t)c->ci[t];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) u[a] -= U[a * 4 + b] * yj[b];
    }
    const double* Di = c->LU + 16 * (size_t)c->diag[i];
    for (int a = 0; a < 4; ++a) {
      double s = 0.0;
      for (int b = 0; b < 4; ++b) s += Di[a * 4 + b] * u[b];
      y[4 * (size_t)i + a] = s;
    }
  }
}

/* Eq. 3: z = M1^-1 r + M2^-1 (r - A M1^-1 r) */
void orc_precond(const orc_ctx* c, const double* r, double* z) {
  size_t n4 = 4 * (size_t)c->N;
  switch (c->p.precond) {
    case ORC_PREC_NONE:
      memcpy(z, r, sizeof(double) * n4);
      return;
    case ORC_PREC_ILU:
      orc_ilu_apply(c, r, z);
      return;
    case ORC_PREC_FIRST:
      orc_first_stage(c, r, z);
      return;
    default: break;
  }
  double* y1 = c->t4a;
  double* r2 = c->t4b;
  double* y2 = c->t4c;
  if (c->nst == 2) orc_cptr3_first_two(c, r, y1);  /* CPTR3: z = M_pT r + M_ILU (r - A M_pT r) */
  else orc_first_stage(c, r, y1);
  orc_correction(c, r, y1, r2);
  orc_ilu_apply(c, r2, y2);
  for (size_t i = 0; i < n4; ++i) z[i] = y1[i] + y2[i];
}

/* Flexible GMRES(m), right preconditioned (Section 3), classical Gram-Schmidt
 * with one full re-orthogonalisation (CGS2), Givens rotations.
 * READING: convergence is ||b - A x||_2 <= tol ||b||_2; the iteration count is
 * the number of preconditioner applications. */
static int gmres(orc_ctx* c, const double* b, double* x, double tol, int maxit, orc_info* info) {
  int n = 4 * c->N, m = c->p.restart;
  if (m < 1) return ORC_INVALID;
  double* V = (double*)calloc((size_t)(m + 1) * n, sizeof(double));
  double* Z = (double*)calloc((size_t)m * n, sizeof(double));
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));   /* H[row*m + col] */
  double* Hraw = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double *cs = (double*)calloc((size_t)m, sizeof(double)), *sn = (double*)calloc((size_t)m, sizeof(double));
  double* g = (double*)calloc((size_t)m + 1, sizeof(double));
  double* y = (double*)calloc((size_t)m + 1, sizeof(double));
  double* h = (double*)calloc((size_t)m + 1, sizeof(double));
  double* w = (double*)calloc((size_t)n, sizeof(double));
  double* r = (double*)calloc((size_t)n, sizeof(double));
  int status = ORC_MAXIT, iters = 0;
  double bnorm = dnrm2(n, b), beta = 0.0;
  if (bnorm == 0.0) {
    memset(x, 0, sizeof(double) * (size_t)n);
    status = ORC_OK;
    goto done;
  }
  orc_spmv(c, x, r);
  for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
  beta = dnrm2(n, r);
  for (;;) {
    if (!isfinite(beta)) { status = ORC_BREAKDOWN; break; }
    if (beta <= tol * bnorm) { status = ORC_OK; break; }
    if (iters >= maxit) { status = ORC_MAXIT; break; }
    for (int i = 0; i < n; ++i) V[i] = r[i] / beta;
    memset(g, 0, sizeof(double) * (size_t)(m + 1));
    memset(H, 0, sizeof(double) * (size_t)(m + 1) * m);
    memset(Hraw, 0, sizeof(double) * (size_t)(m + 1) * m);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * n;
      double* zj = Z + (size_t)j * n;
      orc_precond(c, vj, zj);
      orc_spmv(c, zj, w);
      for (int pass = 0; pass < 2; ++pass) {
        for (int l = 0; l <= j; ++l) h[l] = ddot(n, V + (size_t)l * n, w);
        for (int l = 0; l <= j; ++l) {
          const double* vl = V + (size_t)l * n;
          for (int i = 0; i < n; ++i) w[i] -= h[l] * vl[i];
        }
        for (int l = 0; l <= j; ++l) H[l * m + j] += h[l];
      }
      double hn = dnrm2(n, w);
      H[(j + 1) * m + j] = hn;
      for (int l = 0; l <= j + 1; ++l) Hraw[l * m + j] = H[l * m + j];
      for (int l = 0; l < j; ++l) {
        double a = H[l * m + j], bb = H[(l + 1) * m + j];
        H[l * m + j] = cs[l] * a + sn[l] * bb;
        H[(l + 1) * m + j] = -sn[l] * a + cs[l] * bb;
      }
      double a = H[j * m + j], bb = H[(j + 1) * m + j];
      double d = hypot(a, bb);
      if (d == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
      else { cs[j] = a / d; sn[j] = bb / d; }
      H[j * m + j] = cs[j] * a + sn[j] * bb;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++iters;
      k = j + 1;
      if (!isfinite(g[j + 1]) || !isfinite(hn)) break;
      if (fabs(g[j + 1]) <= tol * bnorm || iters >= maxit || hn == 0.0) break;
      double* vn = V + (size_t)(j + 1) * n;
      for (int i = 0; i < n; ++i) vn[i] = w[i] / hn;
    }
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int l = i + 1; l < k; ++l) s -= H[i * m + l] * y[l];
      y[i] = s / H[i * m + i];
    }
    for (int l = 0; l < k; ++l) {
      const double* zl = Z + (size_t)l * n;
      for (int i = 0; i < n; ++i) x[i] += y[l] * zl[i];
    }
    /* keep the last cycle's basis for the Arnoldi-relation pin */
    if (c->last_cap < m) {
      free(c->lastV); free(c->lastZ); free(c->lastH);
      c->lastV = (double*)malloc(sizeof(double) * (size_t)(m + 1) * n);
      c->lastZ = (double*)malloc(sizeof(double) * (size_t)m * n);
      c->lastH = (double*)malloc(sizeof(double) * (size_t)(m + 1) * m);
      c->last_cap = m;
    }
    c->last_k = k;
    memcpy(c->lastV, V, sizeof(double) * (size_t)(k + 1) * n);
    /* v_k is only formed when the cycle continues; store w/hn for the relation */
    {
      double hn = Hraw[k * m + (k - 1)];
      double* vk = c->lastV + (size_t)k * n;
      if (hn != 0.0)
        for (int i = 0; i < n; ++i) vk[i] = w[i] / hn;
      else
        memset(vk, 0, sizeof(double) * (size_t)n);
    }
    memcpy(c->lastZ, Z, sizeof(double) * (size_t)k * n);
    for (int row = 0; row <= k; ++row)
      for (int col = 0; col < k; ++col) c->lastH[row * k + col] = Hraw[row * m + col];
    orc_spmv(c, x, r);
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
    beta = dnrm2(n, r);
  }
done:
  if (info) {
    info->iters = iters;
    info->rel_resid = (bnorm > 0.0) ? beta / bnorm : 0.0;
    info->status = status;
    info->amg_levels = c->st[0].amg ? c->st[0].amg->nlev : 0;
    info->ilu_levels = c->ilu_nlev;
    info->op_complexity = c->st[0].amg ? orc_amg_op_complexity(c->st[0].amg) : 0.0;
  }
  free(V); free(Z); free(H); free(Hraw); free(cs); free(sn); free(g); free(y); free(h);
  free(w); free(r);
  return status;
}

/* With mgr the Krylov solve runs on the reduced system (reading: its tolerance
 * is relative to the reduced right-hand side, whose residual equals the full
 * one because the recovered unknowns satisfy the constraint rows exactly). */
int orc_solve(orc_ctx* c, const double* b, double* x, double tol, int maxit, orc_info* info) {
  if (!c || !c->setup_done) return ORC_INVALID;
  if (!c->p.mgr) return gmres(c, b, x, tol, maxit, info);
  size_t n = 4 * (size_t)c->N;
  double* bt = (double*)malloc(sizeof(double) * n);
  double* xt = (double*)malloc(sizeof(double) * n);
  mgr_rhs(c, b, bt);
  memcpy(xt, x, sizeof(double) * n);
  for (int i = 0; i < c->N; ++i) xt[4 * (size_t)i + MGR_U] = 0.0;
  int st = gmres(c, bt, xt, tol, maxit, info);
  mgr_recover(c, b, xt);
  memcpy(x, xt, sizeof(double) * n);
  free(bt); free(xt);
  return st;
}

int orc_last_arnoldi(const orc_ctx* c, double* V, double* Z, double* H) {
  int k = c->last_k, n = 4 * c->N;
  if (k <= 0) return 0;
  if (V) memcpy(V, c->lastV, sizeof(double) * (size_t)(k + 1) * n);
  if (Z) memcpy(Z, c->lastZ, sizeof(double) * (size_t)k * n);
  if (H) memcpy(H, c->lastH, sizeof(double) * (size_t)(k + 1) * k);
  return k;
}

void orc_get_W(const orc_ctx* c, double* W) {
  memcpy(W, c->st[0].W, sizeof(double) * 4 * (size_t)c->N);
}
void orc_get_values(const orc_ctx* c, double* v) {
  memcpy(v, c->v, sizeof(double) * 16 * (size_t)c->nnzb);
}
int orc_ahat_nnz(const orc_ctx* c) { return c->st[0].Ahat.nnz; }
void orc_get_ahat(const orc_ctx* c, int32_t* rp, int32_t* ci, double* v) {
  const ocsr* Ah = &c->st[0].Ahat;
  memcpy(rp, Ah->rp, sizeof(int32_t) * (size_t)(Ah->n + 1));
  memcpy(ci, Ah->ci, sizeof(int32_t) * (size_t)Ah->nnz);
  memcpy(v, Ah->v, sizeof(double) * (size_t)Ah->nnz);
}
void orc_get_ilu(const orc_ctx* c, double* LU) {
  memcpy(LU, c->LU, sizeof(double) * 16 * (size_t)c->nnzb);
}
int orc_ilu_levels(const orc_ctx* c, int32_t* level_of_row) {
  if (level_of_row) memcpy(level_of_row, c->ilu_level, sizeof(int32_t) * (size_t)c->N);
  return c->ilu_nlev;
}
orc_amg* orc_ctx_amg(orc_ctx* c) { return c->st[0].amg; }
orc_amg* orc_ctx_amg_t(orc_ctx* c) { return c->nst == 2 ? c->st[1].amg : NULL; }

/* ================================================================== */
/* Independent scalar ILU(0) on a scalar CSR pattern (IKJ variant, diagonal
 * divisions instead of block inverses).  Used only to cross-check the block
 * ILU(0): both are the unique incomplete factorisation on the same pattern. */
int orc_scalar_ilu0_solve(int n, const int32_t* rp, const int32_t* ci, const double* v,
                          const double* r, double* y) {
  double* a = (double*)malloc(sizeof(double) * (size_t)(rp[n] + 1));
  int32_t* dg = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  memcpy(a, v, sizeof(double) * (size_t)rp[n]);
  for (int i = 0; i < n; ++i) {
    dg[i] = -1;
    for (int t = rp[i]; t < rp[i + 1]; ++t)
      if (ci[t] == i) dg[i] = t;
    if (dg[i] < 0) { free(a); free(dg); free(pos); return ORC_INVALID; }
  }
  for (int j = 0; j < n; ++j) pos[j] = -1;
  for (int i = 0; i < n; ++i) {
    for (int t = rp[i]; t < rp[i + 1]; ++t) pos[ci[t]] = t;
    for (int t = rp[i]; t < rp[i + 1] && ci[t] < i; ++t) {
      int k = ci[t];
      a[t] /= a[dg[k]];
      for (int t2 = dg[k] + 1; t2 < rp[k + 1]; ++t2) {
        int q = pos[ci[t2]];
        if (q >= 0) a[q] -= a[t] * a[t2];
      }
    }
    for (int t = rp[i]; t < rp[i + 1]; ++t) pos[ci[t]] = -1;
    if (a[dg[i]] == 0.0) { free(a); free(dg); free(pos); return ORC_BREAKDOWN; }
  }
  for (int i = 0; i < n; ++i) {
    double s = r[i];
    for (int t = rp[i]; t < dg[i]; ++t) s -= a[t] * y[ci[t]];
    y[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int t = dg[i] + 1; t < rp[i + 1]; ++t) s -= a[t] * y[ci[t]];
    y[i] = s / a[dg[i]];
  }
  free(a); free(dg); free(pos);
  return ORC_OK;
}
