"""ctypes binding of libcptr.so (include/cptr.h).

Argument marshalling only: every function forwards to the C ABI of the same
name; all numerical work happens in the library's CUDA kernels.  Pointers may
be host numpy arrays or device addresses (e.g. ``torch.Tensor.data_ptr()``).
Loading fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcptr.so")

OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_MAXIT, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_AGAIN, PENDING = range(9)
PREC_NONE, PREC_CPTR, PREC_ILU, PREC_FIRST = 0, 1, 2, 3
FP64, MIXED = 0, 1
APPLY_PRECOND, APPLY_RESTRICT, APPLY_VCYCLE, APPLY_FIRST, APPLY_CORRECTION, APPLY_ILU = range(6)
(COPY_A_ROWPTR, COPY_A_COL, COPY_A_VAL, COPY_P_ROWPTR, COPY_P_COL, COPY_P_VAL, COPY_CF, COPY_DL1,
 COPY_W, COPY_ILU, COPY_ILU_LEVEL) = range(11)

EXPORTS = (
    "cptr_params_default", "cptr_create", "cptr_update_values", "cptr_set_stream", "cptr_setup",
    "cptr_solve", "cptr_destroy", "cptr_spmv", "cptr_apply", "cptr_amg_levels",
    "cptr_level_info", "cptr_copy", "cptr_get_info", "cptr_server_create", "cptr_submit",
    "cptr_poll", "cptr_server_destroy", "cptr_status_str", "cptr_last_error",
    "cptr_profile_kernel", "cptr_residual_noalloc",
)
KERNEL_SPMV, KERNEL_ILU_FWD, KERNEL_ILU_BWD, KERNEL_VC_PRE0, KERNEL_CORRECTION, KERNEL_MDOT = range(6)


class cptr_params(C.Structure):
    _fields_ = [("restart", C.c_int), ("maxit", C.c_int), ("tol", C.c_double),
                ("precision", C.c_int), ("theta", C.c_double), ("pmax", C.c_int),
                ("max_coarse", C.c_int), ("max_levels", C.c_int), ("precond", C.c_int),
                ("use_graphs", C.c_int), ("seed", C.c_uint64), ("e0", C.c_int), ("e1", C.c_int)]


class cptr_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_resid", C.c_double), ("setup_s", C.c_double),
                ("solve_s", C.c_double), ("amg_levels", C.c_int), ("ilu_levels", C.c_int),
                ("op_complexity", C.c_double), ("status", C.c_int), ("launches", C.c_longlong),
                ("tri_schedule", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load() -> C.CDLL:
    """Loads libcptr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2308_11892_gb300.build.build() "
                           "(nvcc, sm_103a) before using the library")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "cptr_params_default": (None, [C.POINTER(cptr_params)]),
        "cptr_create": (C.c_int, [C.POINTER(vp), i32, i32, vp, vp, vp, C.POINTER(cptr_params)]),
        "cptr_update_values": (C.c_int, [vp, vp]),
        "cptr_set_stream": (C.c_int, [vp, vp]),
        "cptr_setup": (C.c_int, [vp]),
        "cptr_solve": (C.c_int, [vp, vp, vp, dbl, C.c_int, C.POINTER(cptr_info)]),
        "cptr_destroy": (None, [vp]),
        "cptr_spmv": (C.c_int, [vp, vp, vp]),
        "cptr_apply": (C.c_int, [vp, C.c_int, vp, vp]),
        "cptr_amg_levels": (C.c_int, [vp]),
        "cptr_level_info": (C.c_int, [vp, C.c_int, vp]),
        "cptr_copy": (C.c_int, [vp, C.c_int, C.c_int, vp]),
        "cptr_get_info": (C.c_int, [vp, C.POINTER(cptr_info)]),
        "cptr_server_create": (C.c_int, [C.POINTER(vp), C.c_size_t, C.c_int,
                                         C.POINTER(cptr_params)]),
        "cptr_submit": (C.c_int, [vp, i32, vp, vp, vp, vp, dbl, C.c_int, C.POINTER(C.c_uint64)]),
        "cptr_poll": (C.c_int, [vp, C.c_uint64, vp, C.POINTER(cptr_info)]),
        "cptr_server_destroy": (None, [vp]),
        "cptr_status_str": (C.c_char_p, [C.c_int]),
        "cptr_last_error": (C.c_char_p, [vp]),
        "cptr_profile_kernel": (C.c_int, [vp, C.c_int, C.c_int, C.POINTER(dbl),
                                          C.POINTER(dbl)]),
        "cptr_residual_noalloc": (C.c_int, [i32, vp, vp, vp, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def addr(a) -> int:
    """Address of a numpy array (host) or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


class CPTRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def params(**kw) -> cptr_params:
    p = cptr_params()
    load().cptr_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


# ---- same-name thin wrappers -------------------------------------------------
def cptr_create(n_cells, rowptr, col, vals, p: cptr_params | None = None):
    lib = load()
    h = C.c_void_p()
    st = lib.cptr_create(C.byref(h), int(n_cells), 4, addr(rowptr), addr(col), addr(vals),
                         C.byref(p) if p is not None else None)
    if st != OK:
        raise CPTRError(st, f"cptr_create failed: {lib.cptr_status_str(st).decode()}")
    return h


def _check(h, st, what, allow=(OK,)):
    if st not in allow:
        lib = load()
        raise CPTRError(st, f"{what} failed: {lib.cptr_status_str(st).decode()}: "
                            f"{lib.cptr_last_error(h).decode()}")
    return st


def cptr_setup(h):
    return _check(h, load().cptr_setup(h), "cptr_setup")


def cptr_update_values(h, vals):
    return _check(h, load().cptr_update_values(h, addr(vals)), "cptr_update_values")


def cptr_set_stream(h, stream: int | None):
    return _check(h, load().cptr_set_stream(h, stream or None), "cptr_set_stream")


def cptr_solve(h, rhs, x, tol=0.0, maxit=0, allow_maxit=True):
    info = cptr_info()
    st = load().cptr_solve(h, addr(rhs), addr(x), float(tol), int(maxit), C.byref(info))
    _check(h, st, "cptr_solve", (OK, ERR_MAXIT) if allow_maxit else (OK,))
    return st, info.as_dict()


def cptr_destroy(h):
    load().cptr_destroy(h)


def cptr_spmv(h, x, y):
    return _check(h, load().cptr_spmv(h, addr(x), addr(y)), "cptr_spmv")


def cptr_apply(h, which, x, y):
    return _check(h, load().cptr_apply(h, int(which), addr(x), addr(y)), "cptr_apply")


def cptr_amg_levels(h) -> int:
    return load().cptr_amg_levels(h)


def cptr_level_info(h, level):
    info = np.zeros(4, np.int32)
    _check(h, load().cptr_level_info(h, int(level), info.ctypes.data), "cptr_level_info")
    return dict(n=int(info[0]), nnz=int(info[1]), nc=int(info[2]), nnzP=int(info[3]))


def cptr_copy(h, level, what, out: np.ndarray):
    return _check(h, load().cptr_copy(h, int(level), int(what), out.ctypes.data), "cptr_copy")


def cptr_get_info(h):
    info = cptr_info()
    _check(h, load().cptr_get_info(h, C.byref(info)), "cptr_get_info")
    return info.as_dict()


def cptr_profile_kernel(h, kernel: int, reps: int = 10):
    """(mean milliseconds per launch, algorithmic bytes per launch)."""
    ms, nb = C.c_double(), C.c_double()
    _check(h, load().cptr_profile_kernel(h, int(kernel), int(reps), C.byref(ms), C.byref(nb)),
           "cptr_profile_kernel")
    return ms.value, nb.value


NOALLOC_MAX_CELLS = 262144  # CPTR_NOALLOC_MAX_CELLS


def cptr_residual_noalloc(n_cells, rowptr, col, vals, x, b, r, rnorm, stream: int | None = None):
    """r = b - A x and rnorm = ||r||_2 on the device without allocating (device pointers;
    queued on `stream`, returns without waiting).  For callers that must not allocate,
    e.g. while their stream is being captured into a CUDA graph."""
    st = load().cptr_residual_noalloc(int(n_cells), addr(rowptr), addr(col), addr(vals), addr(x),
                                      addr(b), addr(r), addr(rnorm), stream or None)
    if st != OK:
        why = load().cptr_status_str(st).decode()
        if st == ERR_INVALID and int(n_cells) > NOALLOC_MAX_CELLS:
            why = (f"n_cells={int(n_cells)} exceeds the fixed scratch of "
                   f"{NOALLOC_MAX_CELLS} cells")
        raise CPTRError(st, f"cptr_residual_noalloc failed: {why}")
    return st


def cptr_server_create(hbm_budget_bytes: int, max_slots: int, p: cptr_params | None = None):
    h = C.c_void_p()
    st = load().cptr_server_create(C.byref(h), int(hbm_budget_bytes), int(max_slots),
                                   C.byref(p) if p is not None else None)
    if st != OK:
        raise CPTRError(st, "cptr_server_create failed")
    return h


def cptr_submit(s, n_cells, rowptr, col, vals, rhs, tol=0.0, maxit=0) -> int:
    rid = C.c_uint64()
    st = load().cptr_submit(s, int(n_cells), addr(rowptr), addr(col), addr(vals), addr(rhs),
                            float(tol), int(maxit), C.byref(rid))
    if st != OK:
        raise CPTRError(st, "cptr_submit failed")
    return int(rid.value)


def cptr_poll(s, req_id: int, x_out: np.ndarray | None):
    info = cptr_info()
    st = load().cptr_poll(s, C.c_uint64(req_id), addr(x_out), C.byref(info))
    return st, info.as_dict()


def cptr_server_destroy(s):
    load().cptr_server_destroy(s)
