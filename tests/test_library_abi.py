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
    lib.cptr_destroy(None)
