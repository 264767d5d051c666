"""ctypes binding of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain reference the CUDA library
is checked against; only tests/, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this module.  The library itself never
loads it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

PREC_NONE, PREC_CPTR, PREC_ILU, PREC_FIRST, PREC_CPTR_EXACT1 = 0, 1, 2, 3, 4
PREC_CPTR3, PREC_CPTR3_EXACT = 5, 6
SMOOTH_L1_JACOBI, SMOOTH_HYBRID_GS, HGS_BLOCK = 0, 1, 32
COARSEN_PMIS, COARSEN_HMIS = 0, 1
OK, INVALID, NOMEM, MAXIT, BREAKDOWN = 0, 1, 2, 4, 5


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no fused multiply-add, no fast-math)."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("restart", C.c_int), ("maxit", C.c_int), ("tol", C.c_double),
                ("theta", C.c_double), ("pmax", C.c_int), ("max_coarse", C.c_int),
                ("max_levels", C.c_int), ("precond", C.c_int), ("seed", C.c_uint64),
                ("e0", C.c_int), ("e1", C.c_int), ("mgr", C.c_int), ("agg", C.c_int),
                ("nu_pre", C.c_int), ("nu_post", C.c_int), ("smoother", C.c_int),
                ("coarsen", C.c_int)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_resid", C.c_double), ("status", C.c_int),
                ("amg_levels", C.c_int), ("ilu_levels", C.c_int), ("op_complexity", C.c_double)]


_lib = None
_P = C.c_void_p
_I32 = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_F64 = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    sig = {
        "orc_params_default": (None, [C.POINTER(Params)]),
        "orc_create": (_P, [C.c_int, _I32, _I32, _F64, C.POINTER(Params)]),
        "orc_setup": (C.c_int, [_P]),
        "orc_destroy": (None, [_P]),
        "orc_solve": (C.c_int, [_P, _F64, _F64, C.c_double, C.c_int, C.POINTER(Info)]),
        "orc_spmv": (None, [_P, _F64, _F64]),
        "orc_restrict": (None, [_P, _F64, _F64]),
        "orc_vcycle": (None, [_P, _F64, _F64]),
        "orc_first_stage": (None, [_P, _F64, _F64]),
        "orc_correction": (None, [_P, _F64, _F64, _F64]),
        "orc_ilu_apply": (None, [_P, _F64, _F64]),
        "orc_precond": (None, [_P, _F64, _F64]),
        "orc_cptr3_first_two": (None, [_P, _F64, _F64]),
        "orc_cptr3_stage_t": (None, [_P, _F64, _F64]),
        "orc_ctx_amg_t": (_P, [_P]),
        "orc_get_W": (None, [_P, _F64]),
        "orc_get_values": (None, [_P, _F64]),
        "orc_ahat_nnz": (C.c_int, [_P]),
        "orc_get_ahat": (None, [_P, _I32, _I32, _F64]),
        "orc_get_ilu": (None, [_P, _F64]),
        "orc_ilu_levels": (C.c_int, [_P, C.c_void_p]),
        "orc_ctx_amg": (_P, [_P]),
        "orc_last_arnoldi": (C.c_int, [_P, C.c_void_p, C.c_void_p, C.c_void_p]),
        "orc_amg_create": (_P, [C.c_int, _I32, _I32, _F64, C.c_void_p, C.POINTER(Params),
                                C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
        "orc_amg_destroy": (None, [_P]),
        "orc_amg_vcycle": (None, [_P, _F64, _F64]),
        "orc_amg_smooth": (None, [_P, C.c_int, _F64, _F64, C.c_int, C.c_int]),
        "orc_amg_nlevels": (C.c_int, [_P]),
        "orc_amg_level_info": (None, [_P, C.c_int, _I32]),
        "orc_amg_level_A": (None, [_P, C.c_int, _I32, _I32, _F64]),
        "orc_amg_level_P": (None, [_P, C.c_int, _I32, _I32, _F64]),
        "orc_amg_level_cf": (None, [_P, C.c_int, _I32]),
        "orc_amg_level_func": (None, [_P, C.c_int, _I32]),
        "orc_amg_level_dl1": (None, [_P, C.c_int, _F64]),
        "orc_amg_op_complexity": (C.c_double, [_P]),
        "orc_scalar_ilu0_solve": (C.c_int, [C.c_int, _I32, _I32, _F64, _F64, _F64]),
        "orc_splitmix64": (C.c_uint64, [C.c_uint64]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def default_params(**kw) -> Params:
    lib = _load()
    p = Params()
    lib.orc_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def splitmix64(x: int) -> int:
    return int(_load().orc_splitmix64(C.c_uint64(x & (2**64 - 1))))


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class AMG:
    """Standalone scalar/system AMG hierarchy (oracle)."""

    def __init__(self, handle, owner=None):
        self.h = handle
        self._owner = owner  # keeps a parent context alive; None = owns handle

    @classmethod
    def build(cls, rowptr, col, val, func=None, forced_cf0=None, rho0=None, forced_cf1=None,
              **params):
        lib = _load()
        p = default_params(**params)
        rowptr = np.ascontiguousarray(rowptr, np.int32)
        col = np.ascontiguousarray(col, np.int32)
        val = np.ascontiguousarray(val, np.float64)
        n = rowptr.size - 1
        f = None if func is None else np.ascontiguousarray(func, np.int32)
        cf = None if forced_cf0 is None else np.ascontiguousarray(forced_cf0, np.int32)
        cf1 = None if forced_cf1 is None else np.ascontiguousarray(forced_cf1, np.int32)
        r0 = None if rho0 is None else np.ascontiguousarray(rho0, np.float64)
        st = C.c_int(0)
        h = lib.orc_amg_create(n, rowptr, col, val, _ptr(f), C.byref(p), _ptr(cf), _ptr(cf1),
                               _ptr(r0), C.byref(st))
        if st.value != OK:
            lib.orc_amg_destroy(h)
            raise RuntimeError(f"oracle AMG setup failed with status {st.value}")
        obj = cls(h)
        obj._keep = (f, cf, cf1, r0)
        return obj

    def __del__(self):
        if getattr(self, "_owner", 1) is None and getattr(self, "h", None):
            _load().orc_amg_destroy(self.h)
            self.h = None

    @property
    def nlevels(self) -> int:
        return _load().orc_amg_nlevels(self.h)

    def level_info(self, l: int) -> Dict[str, int]:
        if not 0 <= l < self.nlevels:
            raise ValueError(f"level {l} out of range (levels: {self.nlevels})")
        info = np.zeros(4, np.int32)
        _load().orc_amg_level_info(self.h, l, info)
        return dict(n=int(info[0]), nnz=int(info[1]), nc=int(info[2]), nnzP=int(info[3]))

    def level_A(self, l: int):
        d = self.level_info(l)
        rp = np.zeros(d["n"] + 1, np.int32); ci = np.zeros(max(d["nnz"], 1), np.int32)
        v = np.zeros(max(d["nnz"], 1))
        _load().orc_amg_level_A(self.h, l, rp, ci, v)
        return rp, ci[:d["nnz"]], v[:d["nnz"]]

    def _below_coarsest(self, l: int) -> None:
        if not 0 <= l < self.nlevels - 1:
            raise ValueError(f"level {l} has no split, P or smoother (the coarsest level is "
                             f"{self.nlevels - 1})")

    def level_P(self, l: int):
        self._below_coarsest(l)
        d = self.level_info(l)
        rp = np.zeros(d["n"] + 1, np.int32); ci = np.zeros(max(d["nnzP"], 1), np.int32)
        v = np.zeros(max(d["nnzP"], 1))
        _load().orc_amg_level_P(self.h, l, rp, ci, v)
        return rp, ci[:d["nnzP"]], v[:d["nnzP"]]

    def level_cf(self, l: int) -> np.ndarray:
        self._below_coarsest(l)
        cf = np.zeros(self.level_info(l)["n"], np.int32)
        _load().orc_amg_level_cf(self.h, l, cf)
        return cf

    def level_func(self, l: int) -> np.ndarray:
        f = np.zeros(self.level_info(l)["n"], np.int32)
        _load().orc_amg_level_func(self.h, l, f)
        return f

    def level_dl1(self, l: int) -> np.ndarray:
        self._below_coarsest(l)
        d = np.zeros(self.level_info(l)["n"])
        _load().orc_amg_level_dl1(self.h, l, d)
        return d

    def op_complexity(self) -> float:
        return float(_load().orc_amg_op_complexity(self.h))

    def vcycle(self, b: np.ndarray) -> np.ndarray:
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros_like(b)
        _load().orc_amg_vcycle(self.h, b, x)
        return x

    def smooth(self, l: int, b: np.ndarray, x: np.ndarray, sweeps: int = 1,
               backward: bool = False) -> np.ndarray:
        """`sweeps` sweeps of the hierarchy's smoother on level l from x."""
        self._below_coarsest(l)
        b = np.ascontiguousarray(b, np.float64)
        x = np.ascontiguousarray(x, np.float64).copy()
        _load().orc_amg_smooth(self.h, l, b, x, int(sweeps), int(bool(backward)))
        return x


class Oracle:
    """Plain FP64 CPU CPTR-FGMRES on a 4x4 BSR system."""

    def __init__(self, rowptr, col, vals, **params):
        lib = _load()
        self.p = default_params(**params)
        self.rowptr = np.ascontiguousarray(rowptr, np.int32)
        self.col = np.ascontiguousarray(col, np.int32)
        self.vals = np.ascontiguousarray(vals, np.float64).reshape(-1)
        self.N = self.rowptr.size - 1
        # elliptic unknowns of the first stage: CPR 1, CPTR 2, CPTR3 1 (pressure)
        self.ne = 1 if (self.p.e1 < 0 or self.p.precond in (PREC_CPTR3, PREC_CPTR3_EXACT)) else 2
        self.h = lib.orc_create(self.N, self.rowptr, self.col, self.vals, C.byref(self.p))
        if not self.h:
            raise ValueError("invalid BSR input")
        self._setup = False

    @classmethod
    def from_system(cls, sysm, **params):
        return cls(sysm.rowptr, sysm.col, sysm.vals, **params)

    def __del__(self):
        if getattr(self, "h", None):
            _load().orc_destroy(self.h)
            self.h = None

    def setup(self) -> "Oracle":
        st = _load().orc_setup(self.h)
        if st != OK:
            raise RuntimeError(f"oracle setup failed with status {st}")
        self._setup = True
        return self

    def solve(self, b, x0=None, tol=None, maxit=None):
        n = 4 * self.N
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(n) if x0 is None else np.ascontiguousarray(x0, np.float64).copy()
        info = Info()
        st = _load().orc_solve(self.h, b, x, self.p.tol if tol is None else tol,
                               self.p.maxit if maxit is None else maxit, C.byref(info))
        return x, dict(status=st, iters=info.iters, rel_resid=info.rel_resid,
                       amg_levels=info.amg_levels, ilu_levels=info.ilu_levels,
                       op_complexity=info.op_complexity)

    def _apply(self, fname, x, nout):
        x = np.ascontiguousarray(x, np.float64)
        y = np.zeros(nout)
        getattr(_load(), fname)(self.h, x, y)
        return y

    def spmv(self, x):
        return self._apply("orc_spmv", x, 4 * self.N)

    def restrict(self, r):
        return self._apply("orc_restrict", r, self.ne * self.N)

    def vcycle(self, b):
        return self._apply("orc_vcycle", b, self.ne * self.N)

    def first_stage(self, r):
        return self._apply("orc_first_stage", r, 4 * self.N)

    def correction(self, r, y1):
        out = np.zeros(4 * self.N)
        _load().orc_correction(self.h, np.ascontiguousarray(r, np.float64),
                               np.ascontiguousarray(y1, np.float64), out)
        return out

    def ilu_apply(self, r):
        return self._apply("orc_ilu_apply", r, 4 * self.N)

    def precond(self, r):
        return self._apply("orc_precond", r, 4 * self.N)

    def cptr3_first_two(self, r):
        """CPTR3's pressure and temperature stages, composed like Eq. 3."""
        return self._apply("orc_cptr3_first_two", r, 4 * self.N)

    def cptr3_stage_t(self, r):
        """CPTR3's temperature stage alone."""
        return self._apply("orc_cptr3_stage_t", r, 4 * self.N)

    def W(self):
        """(N, ne, 4 - ne): W_i = D_i[e,h] inv(D_i[h,h])."""
        w = np.zeros(4 * self.N)
        _load().orc_get_W(self.h, w)
        nh = 4 - self.ne
        return w.reshape(self.N, 4)[:, :self.ne * nh].reshape(self.N, self.ne, nh)

    def values(self):
        """(nnzb, 16): the blocks of the operator GMRES works on (after setup with
        mgr=1, the reduced system of the first MGR reduction)."""
        out = np.zeros(self.vals.size)
        _load().orc_get_values(self.h, out)
        return out.reshape(-1, 16)

    def ahat(self):
        nnz = _load().orc_ahat_nnz(self.h)
        rp = np.zeros(self.ne * self.N + 1, np.int32); ci = np.zeros(nnz, np.int32); v = np.zeros(nnz)
        _load().orc_get_ahat(self.h, rp, ci, v)
        return rp, ci, v

    def ilu_factors(self):
        out = np.zeros(self.vals.size)
        _load().orc_get_ilu(self.h, out)
        return out.reshape(-1, 16)

    def ilu_levels(self):
        lv = np.zeros(self.N, np.int32)
        n = _load().orc_ilu_levels(self.h, lv.ctypes.data_as(C.c_void_p))
        return n, lv

    def amg(self) -> AMG:
        h = _load().orc_ctx_amg(self.h)
        return AMG(h, owner=self) if h else None

    def last_arnoldi(self):
        lib = _load()
        k = lib.orc_last_arnoldi(self.h, None, None, None)
        n = 4 * self.N
        V = np.zeros((k + 1, n)); Z = np.zeros((k, n)); H = np.zeros((k + 1, k))
        lib.orc_last_arnoldi(self.h, V.ctypes.data_as(C.c_void_p), Z.ctypes.data_as(C.c_void_p),
                             H.ctypes.data_as(C.c_void_p))
        return V, Z, H


def scalar_ilu0_solve(rowptr, col, val, r):
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    r = np.ascontiguousarray(r, np.float64)
    y = np.zeros_like(r)
    st = _load().orc_scalar_ilu0_solve(rowptr.size - 1, rowptr, col, val, r, y)
    if st != OK:
        raise RuntimeError(f"scalar ILU(0) failed with status {st}")
    return y
