/*
 * FP64 CPU oracle for CPTR-preconditioned flexible GMRES.
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, plain reference that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the library never calls it.  It
 * shares no code, header or constant with the CUDA path.
 *
 * What it computes (paper: Cremon, Franc & Hamon, "Constrained
 * Pressure-Temperature Residual (CPTR) Preconditioner Performance for
 * Large-Scale Thermal CO2 Injection Simulation"):
 *   - Eq. 3 two-stage preconditioner M^-1 = M1^-1 + M2^-1 (I - A M1^-1);
 *   - Section 3 first stage M1^-1 = [[0,0],[0,Mee^-1]] on the elliptic
 *     unknowns e = {p, T} (Section 3.2, CPTR split), built by Quasi-IMPES
 *     decoupling (Section 5.2 names "two-level MGR with Quasi-IMPES");
 *   - Mee^-1: one V-cycle of an unknown-based system AMG (Section 3.1 lists the
 *     AMG defaults; Section 3.2 asks for system AMG);
 *   - M2^-1: ILU(0) of the global matrix (Section 3.1);
 *   - right-preconditioned (flexible) GMRES, 200 iterations max, relative
 *     tolerance 1e-6 (Section 3);
 *   - options: the first MGR reduction, exact elimination of the last density
 *     with a cell-local volume constraint before CPTR (Section 3.4, mgr), and
 *     one aggregate level on the first AMG level (Section 3.1, agg).
 *
 * Parity pins for every function are in tests/test_oracle_pins.py.
 */
#ifndef CPTR_ORACLE_H
#define CPTR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_INVALID = 1, ORC_NOMEM = 2, ORC_MAXIT = 4, ORC_BREAKDOWN = 5 };

/* preconditioner selection (tests use the non-default ones) */
enum { ORC_PREC_NONE = 0, ORC_PREC_CPTR = 1, ORC_PREC_ILU = 2, ORC_PREC_FIRST = 3,
       ORC_PREC_CPTR_EXACT1 = 4,
       /* CPTR3 (Section 3.3): pressure stage, temperature stage, ILU(0), each
          on the residual the previous stages leave; e0 = p, e1 = T */
       ORC_PREC_CPTR3 = 5,
       ORC_PREC_CPTR3_EXACT = 6 /* both first stages solved exactly (dense LU), tests only */ };

typedef struct {
  int restart;       /* FGMRES(m) restart length */
  int maxit;         /* maximum iterations (preconditioner applications) */
  double tol;        /* relative tolerance on ||b - A x|| / ||b|| */
  double theta;      /* AMG strength threshold */
  int pmax;          /* interpolation truncation: max entries per row */
  int max_coarse;    /* stop coarsening at n <= max_coarse */
  int max_levels;    /* maximum number of AMG levels */
  int precond;       /* ORC_PREC_* */
  uint64_t seed;     /* PMIS random weights */
  int e0, e1;        /* elliptic unknowns inside a 4x4 block (default 0 and 3) */
  int mgr;           /* 1: first eliminate unknown 2 with equation row 2, a cell-local
                        volume constraint (Section 3.4), and solve the reduced system */
  int agg;           /* one aggregate level (Section 3.1) on the first AMG level:
                        1: coarsened twice, the second time on the Galerkin operator
                        of the first split, two-stage interpolation (R8);
                        2: the second coarsening on distance-two strength among the
                        first split's C points, multipass interpolation (R19) */
  int nu_pre;        /* smoothing sweeps before the coarse correction (default 1) */
  int nu_post;       /* smoothing sweeps after it (default 1) */
  int smoother;      /* ORC_SMOOTH_L1_JACOBI (default) or ORC_SMOOTH_HYBRID_GS */
  int coarsen;       /* ORC_COARSEN_PMIS (default) or ORC_COARSEN_HMIS (Section 3.1) */
} orc_params;

/* C/F splitting.  ORC_COARSEN_HMIS on one domain: the first pass of classical
 * Ruge-Stueben coarsening decides every point, so the PMIS pass that HMIS runs
 * after it (on the points the subdomain passes leave undecided) has nothing
 * left to do. */
enum { ORC_COARSEN_PMIS = 0, ORC_COARSEN_HMIS = 1 };

/* Smoothers of the V-cycle ("first order relaxation", Section 3.1).
 * ORC_SMOOTH_HYBRID_GS: rows in consecutive blocks of ORC_HGS_BLOCK; inside a
 * block, Gauss-Seidel in row order before the coarse correction and in reverse
 * order after it, with the l1 diagonal as pivot; couplings to other blocks use
 * the values at the start of the sweep. */
enum { ORC_SMOOTH_L1_JACOBI = 0, ORC_SMOOTH_HYBRID_GS = 1 };
enum { ORC_HGS_BLOCK = 32 };

typedef struct {
  int iters;
  double rel_resid;
  int status;
  int amg_levels;
  int ilu_levels;
  double op_complexity;
} orc_info;

typedef struct orc_ctx orc_ctx;
typedef struct orc_amg orc_amg;

void orc_params_default(orc_params* p);

/* ---- full system (4x4 BSR, row-major blocks) ---- */
orc_ctx* orc_create(int n_cells, const int32_t* rowptr, const int32_t* col, const double* vals,
                    const orc_params* p);
int  orc_setup(orc_ctx* c);
void orc_destroy(orc_ctx* c);
int  orc_solve(orc_ctx* c, const double* b, double* x, double tol, int maxit, orc_info* info);

/* ---- individual steps (all FP64, host arrays) ---- */
void orc_spmv(const orc_ctx* c, const double* x, double* y);                 /* y = A x */
/* With mgr, A in orc_spmv and every step below is the reduced operator (after
 * orc_setup), and orc_solve takes and returns the full system's b and x. */
void orc_restrict(const orc_ctx* c, const double* r, double* rhat);          /* 4N -> 2N */
void orc_vcycle(const orc_ctx* c, const double* b, double* x);               /* 2N -> 2N */
void orc_first_stage(const orc_ctx* c, const double* r, double* y1);         /* 4N -> 4N */
void orc_correction(const orc_ctx* c, const double* r, const double* y1, double* r2);
void orc_ilu_apply(const orc_ctx* c, const double* r, double* y);           /* 4N -> 4N */
void orc_precond(const orc_ctx* c, const double* r, double* z);              /* Eq. 3 */
/* CPTR3 only: its first two stages M_pT r, and its temperature stage M_T r */
void orc_cptr3_first_two(const orc_ctx* c, const double* r, double* y);
void orc_cptr3_stage_t(const orc_ctx* c, const double* r, double* y);

/* ---- inspection ---- */
void orc_get_W(const orc_ctx* c, double* W);                 /* N x 4 (2x2 row-major) */
void orc_get_values(const orc_ctx* c, double* v);            /* nnzb x 16: the operator's
                                                                 blocks (reduced with mgr) */
int  orc_ahat_nnz(const orc_ctx* c);
void orc_get_ahat(const orc_ctx* c, int32_t* rp, int32_t* ci, double* v);   /* 2N scalar CSR */
void orc_get_ilu(const orc_ctx* c, double* LU);              /* nnzb x 16: L, U, inv(U_ii) */
int  orc_ilu_levels(const orc_ctx* c, int32_t* level_of_row);
void orc_amg_smooth(const orc_amg* a, int l, const double* b, double* x, int sweeps, int backward);
orc_amg* orc_ctx_amg(orc_ctx* c);
orc_amg* orc_ctx_amg_t(orc_ctx* c);   /* CPTR3's temperature-stage hierarchy (else NULL) */
int  orc_last_arnoldi(const orc_ctx* c, double* V, double* Z, double* H);  /* returns k */

/* ---- standalone scalar / system AMG (for the AMG pins) ---- */
/* forced_cf0 / forced_cf1 (tests): prescribed splits of the first level and,
 * with agg, of its second coarsening; NULL = PMIS */
orc_amg* orc_amg_create(int n, const int32_t* rp, const int32_t* ci, const double* v,
                        const int32_t* func, const orc_params* p, const int32_t* forced_cf0,
                        const int32_t* forced_cf1, const double* rho0, int* status);
void orc_amg_destroy(orc_amg* a);
void orc_amg_vcycle(const orc_amg* a, const double* b, double* x);
int  orc_amg_nlevels(const orc_amg* a);
/* info[0]=n info[1]=nnz(A) info[2]=nc info[3]=nnz(P) */
void orc_amg_level_info(const orc_amg* a, int l, int32_t* info);
void orc_amg_level_A(const orc_amg* a, int l, int32_t* rp, int32_t* ci, double* v);
/* P, cf and dl1 exist below the coarsest level only; on the coarsest level
 * (l = nlevels - 1, solved directly) these three write zeros. */
void orc_amg_level_P(const orc_amg* a, int l, int32_t* rp, int32_t* ci, double* v);
void orc_amg_level_cf(const orc_amg* a, int l, int32_t* cf);
void orc_amg_level_func(const orc_amg* a, int l, int32_t* f);
void orc_amg_level_dl1(const orc_amg* a, int l, double* d);
double orc_amg_op_complexity(const orc_amg* a);

/* ---- independent scalar ILU(0) (pin: block ILU(0) == scalar ILU(0)) ---- */
int orc_scalar_ilu0_solve(int n, const int32_t* rp, const int32_t* ci, const double* v,
                          const double* r, double* y);

/* ---- counter-based generator used for the PMIS weights ---- */
uint64_t orc_splitmix64(uint64_t x);

#ifdef __cplusplus
}
#endif
#endif
