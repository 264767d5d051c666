"""GPU AMG setup on operators with negative diagonals, positive couplings and
couplings exactly at the strength threshold, against the oracle.

Each scalar operator (tests/amg_cases.py) is the CPR pressure system of a
block system, so the CUDA setup builds its hierarchy on it: the signed
strength test (s = sign(a_ii)), the ext+i distribution over couplings of sign
opposite to a_kk, the inclusive threshold and the signed l1 diagonal all take
their less common branches here.  Same bars as the other parity tests: splits
exact, operator values to 1e-12, preconditioner pieces to 1e-10, the FP64
solve to 1e-8 with iterations within +-1.
"""
import numpy as np
import pytest

from amg_cases import CASES

pytestmark = pytest.mark.gpu

CPR = dict(e0=0, e1=-1)


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_11892_gb300 import build
    build.build()
    import paper_2308_11892_gb300 as P
    return P


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _level(g, P, l):
    info = P.cptr_level_info(g.h, l)
    rp = g.copy(l, P.COPY_A_ROWPTR, np.int32, info["n"] + 1)
    ci = g.copy(l, P.COPY_A_COL, np.int32, info["nnz"])
    v = g.copy(l, P.COPY_A_VAL, np.float64, info["nnz"])
    return info, rp, ci, v


@pytest.mark.parametrize("name", list(CASES))
def test_special_operator_hierarchy_and_solve(P, oracle_mod, name):
    from synth import pressure_embedding
    s = pressure_embedding(*CASES[name](), seed=3)
    n = s.n_cells
    o = oracle_mod.Oracle.from_system(s, **CPR).setup()
    oa = o.amg()
    with P.Solver.from_system(s, **CPR).setup() as g:
        assert P.cptr_amg_levels(g.h) == oa.nlevels
        for l in range(oa.nlevels):
            info, rp, ci, v = _level(g, P, l)
            oi = oa.level_info(l)
            assert (info["n"], info["nnz"]) == (oi["n"], oi["nnz"])
            orp, oci, ov = oa.level_A(l)
            np.testing.assert_array_equal(rp, orp)
            np.testing.assert_array_equal(ci, oci)
            assert _relerr(v, ov) <= 1e-12
            if l == oa.nlevels - 1:
                break
            assert (info["nc"], info["nnzP"]) == (oi["nc"], oi["nnzP"])
            np.testing.assert_array_equal(g.copy(l, P.COPY_CF, np.int32, info["n"]),
                                          oa.level_cf(l))
            orp, oci, ov = oa.level_P(l)
            np.testing.assert_array_equal(g.copy(l, P.COPY_P_ROWPTR, np.int32, info["n"] + 1), orp)
            np.testing.assert_array_equal(g.copy(l, P.COPY_P_COL, np.int32, info["nnzP"]), oci)
            assert _relerr(g.copy(l, P.COPY_P_VAL, np.float64, info["nnzP"]), ov) <= 1e-12
            assert _relerr(g.copy(l, P.COPY_DL1, np.float64, info["n"]), oa.level_dl1(l)) <= 1e-12

        r = np.random.default_rng(7).normal(size=4 * n)

        def run(which, inp, nout):
            out = _dev(np.zeros(nout))
            P.cptr_apply(g.h, which, _dev(inp), out)
            return _host(out)

        rh = o.restrict(r)
        assert _relerr(run(P.APPLY_VCYCLE, rh, n), o.vcycle(rh)) < 1e-10
        assert _relerr(run(P.APPLY_PRECOND, r, 4 * n), o.precond(r)) < 1e-10
        xg, ig = g.solve(s.rhs)
    xo, io = o.solve(s.rhs)
    assert ig["status"] == 0 and io["status"] == 0
    assert abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8


def test_coarsest_inverse_with_row_exchanges(P, oracle_mod):
    """A pressure system small enough to be the coarsest level, whose leading
    diagonal entries (1e-8) are tiny next to their off-diagonal partners: the
    GPU's dense Gauss-Jordan inverse exchanges rows like the oracle's LU (without
    exchanges the elimination would lose about eight digits), and the V-cycle is
    the exact solve."""
    from synth import pressure_embedding
    rng = np.random.default_rng(12)
    n = 9
    M = np.diag(rng.uniform(1.0, 2.0, n)) + 0.1 * rng.normal(size=(n, n))
    M[0, 0] = M[1, 1] = 1e-8
    M[0, 1], M[1, 0] = 3.0, 2.5
    # dense CSR with every entry stored (the zero diagonal entries included)
    rp = np.arange(0, n * n + 1, n, dtype=np.int32)
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    s = pressure_embedding(rp, ci, M.ravel().copy(), seed=3)
    kw = dict(e1=-1, max_coarse=16)
    o = oracle_mod.Oracle.from_system(s, precond=oracle_mod.PREC_FIRST, **kw).setup()
    b = rng.normal(size=n)
    with P.Solver.from_system(s, precond=P.PREC_FIRST, **kw).setup() as g:
        assert P.cptr_amg_levels(g.h) == 1
        out = _dev(np.zeros(n))
        P.cptr_apply(g.h, P.APPLY_VCYCLE, _dev(b), out)
        x = _host(out)
    assert _relerr(x, o.vcycle(b)) < 1e-13
    assert _relerr(x, np.linalg.solve(M, b)) < 1e-13
