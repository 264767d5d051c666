"""ctypes binding of libcptr.so (include/cptr.h).

Argument marshalling only: every function forwards to the C ABI of the same
name; all numerical work happens in the library's CUDA kernels.  Buffers may
be host numpy arrays, torch tensors (host or device) or raw addresses.  Arrays
and tensors are checked for element type and count against the sizes the call
implies (4N, 16 nnzb, n_e N, the level sizes) before the call, because the C
ABI takes bare pointers and would overrun a short buffer; raw addresses are
the caller's responsibility.  Loading fails loudly when the compiled library
is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcptr.so")

OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_MAXIT, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_AGAIN, PENDING = range(9)
PREC_NONE, PREC_CPTR, PREC_ILU, PREC_FIRST, PREC_CPTR3 = 0, 1, 2, 3, 4
FP64, MIXED = 0, 1
SMOOTH_L1_JACOBI, SMOOTH_HYBRID_GS = 0, 1
COARSEN_PMIS, COARSEN_HMIS = 0, 1
APPLY_PRECOND, APPLY_RESTRICT, APPLY_VCYCLE, APPLY_FIRST, APPLY_CORRECTION, APPLY_ILU = range(6)
(COPY_A_ROWPTR, COPY_A_COL, COPY_A_VAL, COPY_P_ROWPTR, COPY_P_COL, COPY_P_VAL, COPY_CF, COPY_DL1,
 COPY_W, COPY_ILU, COPY_ILU_LEVEL) = range(11)

EXPORTS = (
    "cptr_params_default", "cptr_create", "cptr_update_values", "cptr_set_stream", "cptr_setup",
    "cptr_solve", "cptr_destroy", "cptr_spmv", "cptr_apply", "cptr_amg_levels",
    "cptr_level_info", "cptr_copy", "cptr_get_info", "cptr_server_create", "cptr_submit",
    "cptr_poll", "cptr_server_destroy", "cptr_status_str", "cptr_last_error",
    "cptr_profile_kernel", "cptr_residual_noalloc", "cptr_setup_timing", "cptr_setup_phases",
    "cptr_set_spin_limit", "cptr_solve_batch", "cptr_server_set_limits",
    "cptr_server_last_error", "cptr_kernel_flops", "cptr_fma_rate",
)
PHASES = ("decouple", "strength", "pmis", "interp", "spgemm", "coarse", "ilu", "buffers",
          "ilu_concurrent")  # CPTR_PHASE_* in order
KERNEL_SPMV, KERNEL_ILU_FWD, KERNEL_ILU_BWD, KERNEL_VC_PRE0, KERNEL_CORRECTION, KERNEL_MDOT = range(6)


class cptr_params(C.Structure):
    _fields_ = [("restart", C.c_int), ("maxit", C.c_int), ("tol", C.c_double),
                ("precision", C.c_int), ("theta", C.c_double), ("pmax", C.c_int),
                ("max_coarse", C.c_int), ("max_levels", C.c_int), ("precond", C.c_int),
                ("use_graphs", C.c_int), ("seed", C.c_uint64), ("e0", C.c_int), ("e1", C.c_int),
                ("mgr", C.c_int), ("agg", C.c_int), ("nu_pre", C.c_int), ("nu_post", C.c_int),
                ("smoother", C.c_int), ("tri_tune", C.c_int), ("coarsen", C.c_int)]


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
        "cptr_setup_timing": (C.c_int, [vp, C.c_int]),
        "cptr_set_spin_limit": (C.c_int, [vp, C.c_uint]),
        "cptr_server_set_limits": (C.c_int, [vp, C.c_int, C.c_int]),
        "cptr_server_last_error": (C.c_char_p, [vp]),
        "cptr_solve_batch": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(vp), C.POINTER(vp),
                                       dbl, C.c_int, C.POINTER(cptr_info)]),
        "cptr_setup_phases": (C.c_int, [vp, vp]),
        "cptr_kernel_flops": (C.c_int, [vp, C.c_int, C.POINTER(dbl), C.POINTER(C.c_int)]),
        "cptr_fma_rate": (C.c_int, [C.c_int, C.c_int, C.c_int, vp, C.POINTER(dbl)]),
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


_KINDS = {"f64": (np.dtype(np.float64), "torch.float64"),
          "i32": (np.dtype(np.int32), "torch.int32")}


def buf(a, kind: str, count: int, name: str):
    """Address of `a` after checking that it holds elements of the C type `kind`
    ("f64" or "i32") and at least `count` of them: the library reads or writes
    exactly that many, so a short or mistyped buffer would be overrun (host) or
    read out of bounds (device).  A raw integer address is passed through
    unchecked; None stays None (for arguments the C call allows to be NULL)."""
    if a is None or isinstance(a, int):
        return a
    want_np, want_torch = _KINDS[kind]
    if isinstance(a, np.ndarray):
        if a.dtype != want_np:
            raise TypeError(f"{name} must be {want_np}, got {a.dtype}")
        n = a.size
    elif hasattr(a, "data_ptr"):
        if str(a.dtype) != want_torch:
            raise TypeError(f"{name} must be {want_torch}, got {a.dtype}")
        n = a.numel()
    else:
        raise TypeError(f"unsupported buffer type {type(a)} for {name}")
    if n < count:
        raise ValueError(f"{name} holds {n} elements, the call needs {count}")
    return addr(a)


def _first(a, i: int) -> int:
    """Element i of a host array or a (host or device) tensor, as an int."""
    v = a[i]
    return int(v.item()) if hasattr(v, "item") else int(v)


# sizes of each live context, by handle value: (n_cells, nnzb, ne)
_dims: dict = {}
# cells of each pending serving request, by (server, request id)
_req_cells: dict = {}


def _dims_of(h):
    v = h.value if isinstance(h, C.c_void_p) else h
    return _dims.get(v)


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
def _on_host(a) -> bool:
    return isinstance(a, np.ndarray) or (hasattr(a, "device") and str(a.device) == "cpu")


def _bsr_addrs(n_cells, rowptr, col, vals, device_read=True):
    """Checked addresses of a BSR system's arrays and its block count, read from
    rowptr[n_cells] (None for a raw address, or for a device rowptr when
    device_read is False; col and vals are then checked for their type only)."""
    n = int(n_cells)
    rp = buf(rowptr, "i32", n + 1, "rowptr")
    nnzb = None
    readable = not (rowptr is None or isinstance(rowptr, int)) and (device_read or
                                                                     _on_host(rowptr))
    if readable and n >= 0:
        nnzb = _first(rowptr, n)
    cnt = max(nnzb or 0, 0)
    return rp, buf(col, "i32", cnt, "col"), buf(vals, "f64", 16 * cnt, "vals"), nnzb


def cptr_create(n_cells, rowptr, col, vals, p: cptr_params | None = None):
    lib = load()
    h = C.c_void_p()
    rp, ci, v, nnzb = _bsr_addrs(n_cells, rowptr, col, vals)
    st = lib.cptr_create(C.byref(h), int(n_cells), 4, rp, ci, v,
                         C.byref(p) if p is not None else None)
    if st != OK:
        raise CPTRError(st, f"cptr_create failed: {lib.cptr_status_str(st).decode()}")
    e1 = p.e1 if p is not None else params().e1
    _dims[h.value] = (int(n_cells), nnzb, 1 if e1 < 0 else 2)
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
    d = _dims_of(h)
    need = 16 * d[1] if d and d[1] is not None else 0
    return _check(h, load().cptr_update_values(h, buf(vals, "f64", need, "vals")),
                  "cptr_update_values")


def cptr_set_stream(h, stream: int | None):
    return _check(h, load().cptr_set_stream(h, stream or None), "cptr_set_stream")


def cptr_solve(h, rhs, x, tol=0.0, maxit=0, allow_maxit=True):
    info = cptr_info()
    d = _dims_of(h)
    n4 = 4 * d[0] if d else 0
    st = load().cptr_solve(h, buf(rhs, "f64", n4, "rhs"), buf(x, "f64", n4, "x"), float(tol),
                           int(maxit), C.byref(info))
    _check(h, st, "cptr_solve", (OK, ERR_MAXIT) if allow_maxit else (OK,))
    return st, info.as_dict()


def cptr_destroy(h):
    load().cptr_destroy(h)
    _dims.pop(h.value if isinstance(h, C.c_void_p) else h, None)


def cptr_spmv(h, x, y):
    d = _dims_of(h)
    n4 = 4 * d[0] if d else 0
    return _check(h, load().cptr_spmv(h, buf(x, "f64", n4, "x"), buf(y, "f64", n4, "y")),
                  "cptr_spmv")


def cptr_apply(h, which, x, y):
    d = _dims_of(h)
    n_in = n_out = 4 * d[0] if d else 0
    if d and int(which) == APPLY_RESTRICT:
        n_out = d[2] * d[0]
    elif d and int(which) == APPLY_VCYCLE:
        n_in = n_out = d[2] * d[0]
    return _check(h, load().cptr_apply(h, int(which), buf(x, "f64", n_in, "in"),
                                       buf(y, "f64", n_out, "out")), "cptr_apply")


def cptr_amg_levels(h) -> int:
    return load().cptr_amg_levels(h)


def cptr_level_info(h, level):
    info = np.zeros(4, np.int32)
    _check(h, load().cptr_level_info(h, int(level), info.ctypes.data), "cptr_level_info")
    return dict(n=int(info[0]), nnz=int(info[1]), nc=int(info[2]), nnzP=int(info[3]))


def _copy_size(h, level, what):
    """(element kind, count) that cptr_copy writes for `what` at `level`."""
    what = int(what)
    d = _dims_of(h)
    if what in (COPY_W, COPY_ILU, COPY_ILU_LEVEL):
        if not d:
            return ("i32" if what == COPY_ILU_LEVEL else "f64"), 0
        return {COPY_W: ("f64", 4 * d[0]), COPY_ILU: ("f64", 16 * (d[1] or 0)),
                COPY_ILU_LEVEL: ("i32", d[0])}[what]
    li = cptr_level_info(h, level)
    n, nnz, nnzp = li["n"], li["nnz"], li["nnzP"]
    table = {COPY_A_ROWPTR: ("i32", n + 1), COPY_A_COL: ("i32", nnz), COPY_A_VAL: ("f64", nnz),
             COPY_P_ROWPTR: ("i32", n + 1), COPY_P_COL: ("i32", nnzp),
             COPY_P_VAL: ("f64", nnzp), COPY_CF: ("i32", n), COPY_DL1: ("f64", n)}
    if what not in table:
        raise ValueError(f"unknown copy selector {what}")
    return table[what]


def cptr_copy(h, level, what, out):
    kind, count = _copy_size(h, level, what)
    return _check(h, load().cptr_copy(h, int(level), int(what), buf(out, kind, count, "out")),
                  "cptr_copy")


def cptr_get_info(h):
    info = cptr_info()
    _check(h, load().cptr_get_info(h, C.byref(info)), "cptr_get_info")
    return info.as_dict()


def cptr_solve_batch(handles, rhs_list, x_list, tol=0.0, maxit=0, allow_maxit=True):
    """One launch for all systems: handles of set-up contexts and per-system
    rhs / x buffers (host or device, 4 N_k doubles each).  Returns (status,
    [info dict per system])."""
    n = len(handles)
    if n == 0 or len(rhs_list) != n or len(x_list) != n:
        raise ValueError("one rhs and one x per context")
    hs = (C.c_void_p * n)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    rb = (C.c_void_p * n)()
    xb = (C.c_void_p * n)()
    for k, h in enumerate(handles):
        d = _dims_of(h)
        n4 = 4 * d[0] if d else 0
        rb[k] = buf(rhs_list[k], "f64", n4, f"rhs[{k}]")
        xb[k] = buf(x_list[k], "f64", n4, f"x[{k}]")
    infos = (cptr_info * n)()
    st = load().cptr_solve_batch(hs, n, rb, xb, float(tol), int(maxit), infos)
    _check(handles[0], st, "cptr_solve_batch", (OK, ERR_MAXIT) if allow_maxit else (OK,))
    return st, [i.as_dict() for i in infos]


def cptr_set_spin_limit(h, polls: int = 0):
    return _check(h, load().cptr_set_spin_limit(h, int(polls)), "cptr_set_spin_limit")


def cptr_setup_timing(h, enable: bool = True):
    return _check(h, load().cptr_setup_timing(h, int(bool(enable))), "cptr_setup_timing")


def cptr_setup_phases(h) -> dict:
    """Wall milliseconds per setup phase of the last cptr_setup (timing enabled)."""
    ms = np.zeros(len(PHASES))
    _check(h, load().cptr_setup_phases(h, ms.ctypes.data), "cptr_setup_phases")
    return dict(zip(PHASES, ms.tolist()))


def cptr_profile_kernel(h, kernel: int, reps: int = 10):
    """(mean milliseconds per launch, algorithmic bytes per launch)."""
    ms, nb = C.c_double(), C.c_double()
    _check(h, load().cptr_profile_kernel(h, int(kernel), int(reps), C.byref(ms), C.byref(nb)),
           "cptr_profile_kernel")
    return ms.value, nb.value


def cptr_kernel_flops(h, kernel: int):
    """(algorithmic flops per launch, True when the kernel computes in FP64)."""
    fl, f64 = C.c_double(), C.c_int()
    _check(h, load().cptr_kernel_flops(h, int(kernel), C.byref(fl), C.byref(f64)),
           "cptr_kernel_flops")
    return fl.value, bool(f64.value)


def cptr_fma_rate(fp64: bool, iters: int, reps: int = 5, stream=None):
    """Measured FMA throughput of the current device in TFLOP/s (FP64 or FP32)."""
    tf = C.c_double()
    st = load().cptr_fma_rate(int(bool(fp64)), int(iters), int(reps),
                              None if stream is None else C.c_void_p(int(stream)), C.byref(tf))
    _check(None, st, "cptr_fma_rate")
    return tf.value


NOALLOC_MAX_CELLS = 262144  # CPTR_NOALLOC_MAX_CELLS


def cptr_residual_noalloc(n_cells, rowptr, col, vals, x, b, r, rnorm, stream: int | None = None):
    """r = b - A x and rnorm = ||r||_2 on the device without allocating (device pointers;
    queued on `stream`, returns without waiting).  For callers that must not allocate,
    e.g. while their stream is being captured into a CUDA graph."""
    # no device reads here (the call may be made during stream capture): the block
    # count is not known, so col and vals are checked for their type only
    n, n4 = int(n_cells) + 1, 4 * int(n_cells)
    st = load().cptr_residual_noalloc(int(n_cells), buf(rowptr, "i32", n, "rowptr"),
                                      buf(col, "i32", 0, "col"), buf(vals, "f64", 0, "vals"),
                                      buf(x, "f64", n4, "x"), buf(b, "f64", n4, "b"),
                                      buf(r, "f64", n4, "r"), buf(rnorm, "f64", 1, "rnorm"),
                                      stream or None)
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


def cptr_server_set_limits(s, max_queued: int = 4096, batch_max_cells: int = 0):
    st = load().cptr_server_set_limits(s, int(max_queued), int(batch_max_cells))
    if st != OK:
        raise CPTRError(st, "cptr_server_set_limits failed")
    return st


def cptr_submit(s, n_cells, rowptr, col, vals, rhs, tol=0.0, maxit=0) -> int:
    rid = C.c_uint64()
    rp, ci, v, _ = _bsr_addrs(n_cells, rowptr, col, vals, device_read=False)
    st = load().cptr_submit(s, int(n_cells), rp, ci, v, buf(rhs, "f64", 4 * int(n_cells), "rhs"),
                            float(tol), int(maxit), C.byref(rid))
    if st != OK:
        raise CPTRError(st, "cptr_submit failed")
    _req_cells[(s.value if isinstance(s, C.c_void_p) else s, int(rid.value))] = int(n_cells)
    return int(rid.value)


def cptr_poll(s, req_id: int, x_out: np.ndarray | None):
    info = cptr_info()
    key = (s.value if isinstance(s, C.c_void_p) else s, int(req_id))
    n4 = 4 * _req_cells.get(key, 0)
    st = load().cptr_poll(s, C.c_uint64(req_id), buf(x_out, "f64", n4, "x_out"), C.byref(info))
    if st != PENDING:
        _req_cells.pop(key, None)
    return st, info.as_dict()


def cptr_server_last_error(s) -> str:
    return (load().cptr_server_last_error(s) or b"").decode()


def cptr_server_destroy(s):
    load().cptr_server_destroy(s)
    v = s.value if isinstance(s, C.c_void_p) else s
    for key in [k for k in _req_cells if k[0] == v]:
        del _req_cells[key]
