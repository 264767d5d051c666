// First MGR reduction (Section 3.4): the last density (unknown 2) is eliminated
// with equation row 2, a volume constraint that involves only the cell's own
// unknowns, so the elimination is exact and block-local:
//
//   At_ij[r,s] = A_ij[r,s] - A_ij[r,u] * (A_jj[u,s] / A_jj[u,u])   (r, s != u)
//   bt_i[r]    = b_i[r] - sum_j A_ij[r,u] * (b_j[u] / A_jj[u,u])
//   x_i[u]     = (b_i[u] - sum_{s != u} A_ii[u,s] x_i[s]) / A_ii[u,u]
//
// Row and column u of the reduced blocks become the identity row and column
// (zero right-hand side there), so every 4x4 kernel of the library runs CPTR on
// the remaining (p, rho_CO2, T) unknowns unchanged.  The products and
// differences use explicit round-to-nearest operations, in the order written
// above, so the reduced operator is the same bit for bit whatever the
// compiler's contraction choices: the AMG setup on it takes integer decisions.
#include "ctx.h"

namespace {

constexpr int kU = 2;     // the eliminated unknown and its equation row
constexpr int kT = 256;
inline int nblk(long long n) { return (int)((n + kT - 1) / kT); }

enum { MGR_OK = 0, MGR_PIVOT = 1, MGR_NONLOCAL = 2 };

// One warp per block row: lanes walk the row's blocks 16 entries at a time
// (two blocks per warp step, 256 contiguous bytes).
__global__ void k_mgr_reduce(int N, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const int32_t* __restrict__ diag, const double* __restrict__ A,
                             double* __restrict__ At, int* __restrict__ flag) {
  int w = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (w >= N) return;
  const int i = w;
  if (lane == 0) {
    double q = A[16 * (size_t)diag[i] + 5 * kU];
    if (q == 0.0 || !isfinite(q)) atomicMax(flag, MGR_PIVOT);
  }
  long long e0 = 16ll * rp[i], e1 = 16ll * rp[i + 1];
  for (long long e = e0 + lane; e < e1; e += 32) {
    long long t = e >> 4;
    int k = (int)(e & 15), r = k >> 2, s = k & 3;
    int j = ci[t];
    double out;
    if (r == kU || s == kU) {
      if (r == kU && j != i && A[e] != 0.0) atomicMax(flag, MGR_NONLOCAL);
      out = (r == s && j == i) ? 1.0 : 0.0;
    } else {
      const double* Dj = A + 16 * (size_t)diag[j];
      double q = Dj[4 * kU + s] / Dj[5 * kU];
      out = __dsub_rn(A[e], __dmul_rn(A[16 * t + 4 * r + kU], q));
    }
    At[e] = out;
  }
}

// bt = reduced right-hand side, and the eliminated entries of the initial
// guess set to zero; one thread per (cell, equation row).
__global__ void k_mgr_rhs(int N, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const int32_t* __restrict__ diag, const double* __restrict__ A,
                          const double* __restrict__ b, double* __restrict__ bt,
                          double* __restrict__ x) {
  long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= 4ll * N) return;
  int i = (int)(g >> 2), r = (int)(g & 3);
  if (r == kU) {
    bt[g] = 0.0;
    x[g] = 0.0;
    return;
  }
  double acc = b[g];
  for (int t = rp[i]; t < rp[i + 1]; ++t) {
    int j = ci[t];
    double q = b[4 * (size_t)j + kU] / A[16 * (size_t)diag[j] + 5 * kU];
    acc = __dsub_rn(acc, __dmul_rn(A[16 * (size_t)t + 4 * r + kU], q));
  }
  bt[g] = acc;
}

// x_i[u] from the constraint row, one thread per cell
__global__ void k_mgr_recover(int N, const int32_t* __restrict__ diag,
                              const double* __restrict__ A, const double* __restrict__ b,
                              double* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* D = A + 16 * (size_t)diag[i];
  double acc = b[4 * (size_t)i + kU];
  for (int s = 0; s < 4; ++s)
    if (s != kU) acc = __dsub_rn(acc, __dmul_rn(D[4 * kU + s], x[4 * (size_t)i + s]));
  x[4 * (size_t)i + kU] = acc / D[5 * kU];
}

}  // namespace

cptr_status mgr_reduce(cptr_ctx* c) {
  CTX_CUDA(c, cudaMemsetAsync(c->mgr_flag, 0, sizeof(int), c->stream));
  KL(c, k_mgr_reduce<<<nblk(32ll * c->N), kT, 0, c->stream>>>(c->N, c->rp, c->ci, c->diag,
                                                               c->vfull, c->v, c->mgr_flag));
  int flag = 0;
  CTX_CUDA(c, cudaMemcpyAsync(&flag, c->mgr_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CTX_CUDA(c, cudaStreamSynchronize(c->stream));
  if (flag == MGR_NONLOCAL) {
    ctx_set_err(c, "mgr: equation row 2 has entries outside the diagonal block (not a local constraint)");
    return CPTR_ERR_INVALID;
  }
  if (flag == MGR_PIVOT) {
    ctx_set_err(c, "mgr: zero or non-finite pivot A_ii[2,2] of the constraint row");
    return CPTR_ERR_BREAKDOWN;
  }
  return CPTR_OK;
}

void mgr_rhs(cptr_ctx* c) {
  KL(c, k_mgr_rhs<<<nblk(4ll * c->N), kT, 0, c->stream>>>(c->N, c->rp, c->ci, c->diag, c->vfull,
                                                           c->bfull, c->bd, c->xd));
}

void mgr_recover(cptr_ctx* c) {
  KL(c, k_mgr_recover<<<nblk(c->N), kT, 0, c->stream>>>(c->N, c->diag, c->vfull, c->bfull,
                                                         c->xd));
}
