"""GB300-native CPTR-preconditioned flexible GMRES (hand-written CUDA, sm_103a).

The numerical work runs in ``libcptr.so`` (C ABI in ``include/cptr.h``); this
package is the thin Python binding plus a convenience class.  See
``paper_2308_11892_gb300.build.build()`` to compile the library.
"""
from __future__ import annotations

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    APPLY_CORRECTION, APPLY_FIRST, APPLY_ILU, APPLY_PRECOND, APPLY_RESTRICT, APPLY_VCYCLE,
    COPY_A_COL, COPY_A_ROWPTR, COPY_A_VAL, COPY_CF, COPY_DL1, COPY_ILU, COPY_ILU_LEVEL, COPY_P_COL,
    COPY_P_ROWPTR, COPY_P_VAL, COPY_W, CPTRError, EXPORTS, FP64, MIXED, PREC_CPTR, PREC_FIRST,
    PREC_ILU, PREC_NONE, PREC_CPTR3, SMOOTH_L1_JACOBI, SMOOTH_HYBRID_GS, COARSEN_PMIS, COARSEN_HMIS, cptr_amg_levels, cptr_apply, cptr_copy, cptr_create, cptr_destroy,
    cptr_get_info, cptr_level_info, cptr_poll, cptr_server_create, cptr_server_destroy,
    cptr_set_stream, cptr_setup, cptr_solve, cptr_spmv, cptr_submit, cptr_update_values, params,
    cptr_profile_kernel, KERNEL_SPMV, KERNEL_ILU_FWD, KERNEL_ILU_BWD, KERNEL_VC_PRE0,
    KERNEL_CORRECTION, KERNEL_MDOT, cptr_residual_noalloc, NOALLOC_MAX_CELLS,
    cptr_setup_timing, cptr_setup_phases, PHASES, cptr_set_spin_limit, cptr_solve_batch, cptr_server_set_limits,
    cptr_server_last_error, cptr_kernel_flops, cptr_fma_rate,
    OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_MAXIT, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_AGAIN,
)


class Solver:
    """Owns one library context (one BSR system)."""

    def __init__(self, n_cells, rowptr, col, vals, **kw):
        self.N = int(n_cells)
        self.p = params(**kw)
        self.h = cptr_create(self.N, np.ascontiguousarray(rowptr, np.int32) if isinstance(rowptr, np.ndarray) else rowptr,
                             np.ascontiguousarray(col, np.int32) if isinstance(col, np.ndarray) else col,
                             np.ascontiguousarray(vals, np.float64) if isinstance(vals, np.ndarray) else vals,
                             self.p)

    @classmethod
    def from_system(cls, s, **kw):
        return cls(s.n_cells, s.rowptr, s.col, s.vals, **kw)

    def close(self):
        if getattr(self, "h", None):
            cptr_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def setup(self):
        cptr_setup(self.h)
        return self

    def solve(self, rhs, x=None, tol=0.0, maxit=0):
        """Host (numpy) or device (torch) rhs/x; returns (x, info)."""
        if x is None:
            x = np.zeros(4 * self.N) if isinstance(rhs, np.ndarray) else rhs.new_zeros(rhs.shape)
        st, info = cptr_solve(self.h, rhs, x, tol, maxit)
        info["status"] = st
        return x, info

    def levels(self):
        return [cptr_level_info(self.h, l) for l in range(cptr_amg_levels(self.h))]

    def copy(self, level, what, dtype, size):
        out = np.zeros(size, dtype)
        cptr_copy(self.h, level, what, out)
        return out
