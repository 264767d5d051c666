"""The C-ABI library builds for sm_103a and exports every declared symbol (CPU only)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def libpath():
    from paper_2308_11892_gb300 import build
    return build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "cptr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cptr_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_boundary():
    names = _declared()
    for need in ("cptr_create", "cptr_setup", "cptr_solve", "cptr_submit", "cptr_poll",
                 "cptr_destroy", "cptr_spmv", "cptr_apply"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_export(libpath):
    import paper_2308_11892_gb300 as P
    assert set(_declared()) == set(P.EXPORTS)
    P._lib.load()


def test_host_only_entry_points(libpath):
    """Calls that touch no device: defaults, status strings, argument checks."""
    import paper_2308_11892_gb300 as P
    lib = P._lib.load()
    p = P.params()
    assert p.restart == 30 and p.maxit == 200 and abs(p.tol - 1e-6) < 1e-20
    assert p.e0 == 0 and p.e1 == 3 and p.pmax == 4
    assert lib.cptr_status_str(4) == b"maximum iterations reached"
    h = ctypes.c_void_p()
    assert lib.cptr_create(ctypes.byref(h), 0, 4, None, None, None, None) == P._lib.ERR_INVALID
    assert lib.cptr_create(ctypes.byref(h), 10, 3, None, None, None, None) == P._lib.ERR_INVALID
    # more cells than 32-bit counts of the first AMG level allow: refused before any device call
    one = (ctypes.c_int32 * 1)(0)
    assert lib.cptr_create(ctypes.byref(h), 1 << 29, 4, one, one, one, None) == P._lib.ERR_INVALID
    lib.cptr_destroy(None)
    # the rate and flop calls check their arguments before any device call
    tf, fl, f64 = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    for fp64, iters, reps in ((1, 0, 1), (1, 64, 0), (0, (1 << 21) + 1, 1), (1, (1 << 30) + 1, 1)):
        assert lib.cptr_fma_rate(fp64, iters, reps, None, ctypes.byref(tf)) == P._lib.ERR_INVALID
    assert lib.cptr_fma_rate(1, 64, 1, None, None) == P._lib.ERR_INVALID
    assert lib.cptr_kernel_flops(None, 0, ctypes.byref(fl), ctypes.byref(f64)) == P._lib.ERR_INVALID


def test_binding_checks_buffers_before_the_call(libpath):
    """The binding checks element type and count of every buffer against the
    sizes the C call implies (4N, 16 nnzb, n_e N, level sizes) and raises before
    calling the library, so a short or mistyped array is never overrun.  The
    handles here are fake: every call below must be rejected before it reaches C."""
    import numpy as np
    import torch
    import paper_2308_11892_gb300 as P
    L = P._lib
    # the checker itself
    assert L.buf(None, "f64", 5, "x") is None and L.buf(4096, "f64", 5, "x") == 4096
    a = np.zeros(5)
    assert L.buf(a, "f64", 5, "x") == a.ctypes.data
    with pytest.raises(TypeError):
        L.buf(np.zeros(5, np.float32), "f64", 5, "x")
    with pytest.raises(ValueError):
        L.buf(np.zeros(4), "f64", 5, "x")
    t = torch.zeros(6, dtype=torch.int32)
    assert L.buf(t, "i32", 6, "rp") == t.data_ptr()
    with pytest.raises(TypeError):
        L.buf(torch.zeros(6, dtype=torch.int64), "i32", 6, "rp")
    # cptr_create: rowptr type, then col and vals against rowptr[N]
    rp = np.array([0, 2, 3], np.int32)
    with pytest.raises(TypeError):
        P.cptr_create(2, rp.astype(np.int64), np.zeros(3, np.int32), np.zeros(48))
    with pytest.raises(ValueError, match="col"):
        P.cptr_create(2, rp, np.zeros(2, np.int32), np.zeros(48))
    with pytest.raises(ValueError, match="vals"):
        P.cptr_create(2, rp, np.zeros(3, np.int32), np.zeros(47))
    # calls on a context: sizes recorded at creation (N = 10, nnzb = 30, CPTR n_e = 2)
    fake = 0x7777_0000
    L._dims[fake] = (10, 30, 2)
    try:
        with pytest.raises(ValueError, match="rhs"):
            P.cptr_solve(fake, np.zeros(39), np.zeros(40))
        with pytest.raises(TypeError, match="x"):
            P.cptr_solve(fake, np.zeros(40), np.zeros(40, np.float32))
        with pytest.raises(ValueError, match="y"):
            P.cptr_spmv(fake, np.zeros(40), np.zeros(20))
        with pytest.raises(ValueError, match="out"):
            P.cptr_apply(fake, P.APPLY_RESTRICT, np.zeros(40), np.zeros(19))
        with pytest.raises(ValueError, match="in"):
            P.cptr_apply(fake, P.APPLY_VCYCLE, np.zeros(19), np.zeros(20))
        with pytest.raises(ValueError, match="vals"):
            P.cptr_update_values(fake, np.zeros(16 * 30 - 1))
        with pytest.raises(ValueError, match="out"):
            P.cptr_copy(fake, 0, P.COPY_W, np.zeros(39))
        with pytest.raises(TypeError, match="out"):
            P.cptr_copy(fake, 0, P.COPY_ILU_LEVEL, np.zeros(10))
        with pytest.raises(ValueError, match="out"):
            P.cptr_copy(fake, 0, P.COPY_ILU, np.zeros(16 * 30 - 1))
    finally:
        del L._dims[fake]
    # serving: the request's arrays, and the poll buffer against the request's size
    with pytest.raises(ValueError, match="rhs"):
        P.cptr_submit(fake, 2, rp, np.zeros(3, np.int32), np.zeros(48), np.zeros(7))
    L._req_cells[(fake, 9)] = 10
    try:
        with pytest.raises(ValueError, match="x_out"):
            P.cptr_poll(fake, 9, np.zeros(39))
    finally:
        L._req_cells.pop((fake, 9), None)
    # the allocation-free residual (no device reads: col and vals by type only)
    with pytest.raises(ValueError, match="rnorm"):
        P.cptr_residual_noalloc(10, np.zeros(11, np.int32), np.zeros(1, np.int32), np.zeros(16),
                                np.zeros(40), np.zeros(40), np.zeros(40), np.zeros(0))


def test_mgr_parameter_checks(libpath):
    """mgr defaults to 0; mgr with an elliptic unknown 2, or a value other than
    0/1, is refused by cptr_create before any device work (the pointers are
    never read)."""
    import paper_2308_11892_gb300 as P
    lib = P._lib.load()
    assert P.params().mgr == 0
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(256)
    for kw in (dict(mgr=1, e1=2), dict(mgr=1, e0=2, e1=3), dict(mgr=2)):
        p = P.params(**kw)
        assert lib.cptr_create(ctypes.byref(h), 10, 4, fake, fake, fake,
                               ctypes.byref(p)) == P._lib.ERR_INVALID


def _c_layout(header_dir, header, structs, name):
    """Field offsets and sizes of `structs` as a C compiler lays them out."""
    import subprocess
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", f"#include \"{header}\"",
             "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'  printf("{sname} size %zu\\n", sizeof({sname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{sname} {f} %zu\\n", offsetof({sname}, {f}));')
    lines += ["  return 0;", "}"]
    out_dir = os.path.join(ROOT, "paper_2308_11892_gb300", "_build")
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, f"{name}.c")
    exe = os.path.join(out_dir, name)
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.run([cc, "-I", header_dir, "-o", exe, src], check=True)
    got = {}
    for line in subprocess.run([exe], check=True, capture_output=True,
                               text=True).stdout.splitlines():
        sname, field, val = line.split()
        got[(sname, field)] = int(val)
    return got


def _check_layout(got, structs):
    for sname, cls in structs.items():
        assert got[(sname, "size")] == ctypes.sizeof(cls), sname
        for f, _ in cls._fields_:
            assert got[(sname, f)] == getattr(cls, f).offset, (sname, f)


def test_binding_structs_match_the_header_layout(libpath):
    """The ctypes copies of cptr_params and cptr_info have the C header's field
    offsets and sizes (a mismatch would silently misread parameters)."""
    import paper_2308_11892_gb300 as P
    structs = {"cptr_params": P._lib.cptr_params, "cptr_info": P._lib.cptr_info}
    _check_layout(_c_layout(os.path.join(ROOT, "include"), "cptr.h", structs, "abi_layout"),
                  structs)


def test_oracle_structs_match_its_header_layout():
    import oracle
    structs = {"orc_params": oracle.Params, "orc_info": oracle.Info}
    _check_layout(_c_layout(os.path.join(ROOT, "oracle"), "oracle.h", structs,
                            "oracle_layout"), structs)


def test_every_parameter_check_refuses_before_device_work(libpath):
    """Each out-of-range cptr_params field, changed alone from the defaults, is
    refused by cptr_create with CPTR_ERR_INVALID before any device call (the
    fake matrix pointers are never read)."""
    import paper_2308_11892_gb300 as P
    lib = P._lib.load()
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(256)
    nan = float("nan")
    bad = [("restart", 0), ("restart", 64), ("maxit", -1), ("tol", -1.0), ("tol", nan),
           ("precision", 2), ("precond", P.PREC_NONE - 1), ("precond", P.PREC_CPTR3 + 1),
           ("e0", -1), ("e0", 4), ("e1", -2), ("e1", 4), ("e1", 0), ("pmax", 0),
           ("pmax", 65), ("max_coarse", 0), ("max_levels", 0), ("theta", -0.1),
           ("theta", 1.1), ("theta", nan), ("mgr", 2), ("agg", -1), ("agg", 3),
           ("nu_pre", -1), ("nu_pre", 9), ("nu_post", 9), ("smoother", 2),
           ("tri_tune", 2), ("coarsen", 2)]
    for field, value in bad:
        p = P.params(**{field: value})
        assert lib.cptr_create(ctypes.byref(h), 10, 4, fake, fake, fake,
                               ctypes.byref(p)) == P._lib.ERR_INVALID, (field, value)
    # CPTR3 needs both elliptic unknowns
    p = P.params(precond=P.PREC_CPTR3, e1=-1)
    assert lib.cptr_create(ctypes.byref(h), 10, 4, fake, fake, fake,
                           ctypes.byref(p)) == P._lib.ERR_INVALID
