"""GPU parity of the first MGR reduction (Section 3.4) against the oracle.

The reduction is computed with explicit round-to-nearest operations in the
oracle's order, so the reduced operator, and therefore the decoupling and the
whole hierarchy, are the same as the oracle's (splits exact, values to 1e-15
for W and the level-0 operator, 1e-12 for the ILU factors); the FP64 solve
matches to 1e-8 with iterations within +-1 and solves the full system (the
constraint rows to rounding); the mixed-precision solve stays within 10% of
the oracle's iterations.  Invalid inputs are refused by cptr_setup.
"""
import numpy as np
import pytest

from synth import config_system, knn, with_volume_constraint

pytestmark = pytest.mark.gpu

SYSTEMS = {
    "c1": lambda: with_volume_constraint(config_system("c1"), seed=4),
    "knn": lambda: with_volume_constraint(knn(10, 8, 4, pe=10.0, seed=31), seed=5),
}


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_11892_gb300 import build
    build.build()
    import paper_2308_11892_gb300 as P
    return P


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_mgr_setup_and_solve_match_oracle(P, oracle_mod, name):
    import torch
    s = SYSTEMS[name]()
    n = s.n_cells
    A = s.to_dense()
    o = oracle_mod.Oracle.from_system(s, mgr=1).setup()
    oa = o.amg()
    with P.Solver.from_system(s, mgr=1) as g:
        with pytest.raises(P.CPTRError):   # the reduced operator does not exist yet
            xd = torch.zeros(4 * n, dtype=torch.float64, device="cuda")
            P.cptr_spmv(g.h, xd, torch.zeros_like(xd))
        g.setup()
        W = g.copy(0, P.COPY_W, np.float64, 4 * n).reshape(-1, 2, 2)
        assert _relerr(W, o.W()) <= 1e-15
        info = P.cptr_level_info(g.h, 0)
        orp, oci, ov = o.ahat()
        np.testing.assert_array_equal(g.copy(0, P.COPY_A_ROWPTR, np.int32, info["n"] + 1), orp)
        np.testing.assert_array_equal(g.copy(0, P.COPY_A_COL, np.int32, info["nnz"]), oci)
        assert _relerr(g.copy(0, P.COPY_A_VAL, np.float64, info["nnz"]), ov) <= 1e-15
        assert P.cptr_amg_levels(g.h) == oa.nlevels
        for l in range(oa.nlevels - 1):
            nl = P.cptr_level_info(g.h, l)["n"]
            np.testing.assert_array_equal(g.copy(l, P.COPY_CF, np.int32, nl), oa.level_cf(l))
        F = g.copy(0, P.COPY_ILU, np.float64, 16 * s.nnzb).reshape(-1, 16)
        assert _relerr(F, o.ilu_factors()) <= 1e-12
        # the public SpMV applies the reduced operator
        x = np.random.default_rng(3).normal(size=4 * n)
        xd = torch.from_numpy(x).cuda()
        yd = torch.zeros_like(xd)
        P.cptr_spmv(g.h, xd, yd)
        torch.cuda.synchronize()
        assert _relerr(yd.cpu().numpy(), o.spmv(x)) <= 1e-14
        xg, ig = g.solve(s.rhs)
    xo, io = o.solve(s.rhs)
    assert ig["status"] == 0 and io["status"] == 0
    assert abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    r = s.rhs - A @ xg
    assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(s.rhs) * 1.01
    assert np.abs(r[2::4]).max() <= 1e-12 * np.abs(A).max() * np.abs(xg).max()
    # mixed precision
    with P.Solver.from_system(s, mgr=1, precision=P.MIXED).setup() as g:
        xm, im = g.solve(s.rhs)
    assert im["status"] == 0
    assert abs(im["iters"] - io["iters"]) <= max(1, int(0.1 * io["iters"]))
    assert np.linalg.norm(s.rhs - A @ xm) <= 1e-6 * np.linalg.norm(s.rhs) * 1.01


def test_mgr_with_the_cpr_split_matches_oracle(P, oracle_mod):
    """mgr with e = {p}: the padded unknown sits inside the 3x3 D[h,h]."""
    s = SYSTEMS["c1"]()
    n = s.n_cells
    o = oracle_mod.Oracle.from_system(s, mgr=1, e1=-1).setup()
    with P.Solver.from_system(s, mgr=1, e1=-1).setup() as g:
        W = g.copy(0, P.COPY_W, np.float64, 4 * n).reshape(n, 4)[:, :3].reshape(n, 1, 3)
        assert _relerr(W, o.W()) <= 1e-15
        oa = o.amg()
        assert P.cptr_amg_levels(g.h) == oa.nlevels
        for l in range(oa.nlevels - 1):
            nl = P.cptr_level_info(g.h, l)["n"]
            np.testing.assert_array_equal(g.copy(l, P.COPY_CF, np.int32, nl), oa.level_cf(l))
        xg, ig = g.solve(s.rhs)
    xo, io = o.solve(s.rhs)
    assert ig["status"] == 0 and abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)


def test_mgr_refuses_invalid_input(P):
    s = SYSTEMS["c1"]()
    v = s.vals.reshape(-1, 4, 4).copy()
    rows = np.repeat(np.arange(s.n_cells), np.diff(s.rowptr))
    off = np.nonzero(rows != s.col)[0]
    d = np.nonzero(rows == s.col)[0]
    bad = v.copy()
    bad[off[7], 2, 3] = 1e-3
    with P.Solver(s.n_cells, s.rowptr, s.col, bad.reshape(-1, 16), mgr=1) as g:
        with pytest.raises(P.CPTRError) as e:
            g.setup()
        assert e.value.status == P._lib.ERR_INVALID
    bad = v.copy()
    bad[d[11], 2, 2] = 0.0
    with P.Solver(s.n_cells, s.rowptr, s.col, bad.reshape(-1, 16), mgr=1) as g:
        with pytest.raises(P.CPTRError) as e:
            g.setup()
        assert e.value.status == P._lib.ERR_BREAKDOWN
        # the same context accepts valid values afterwards
        P.cptr_update_values(g.h, np.ascontiguousarray(s.vals))
        g.setup()
        x, info = g.solve(s.rhs)
        assert info["status"] == 0


def test_mgr_through_the_server(P):
    """A serving request with mgr parameters returns the same solution as the
    direct call, bit for bit."""
    import time
    s = SYSTEMS["knn"]()
    with P.Solver.from_system(s, mgr=1).setup() as g:
        xd, _ = g.solve(s.rhs)
    srv = P.cptr_server_create(4 << 30, 2, P.params(mgr=1))
    try:
        rid = P.cptr_submit(srv, s.n_cells, s.rowptr, s.col, s.vals, s.rhs)
        x = np.zeros(4 * s.n_cells)
        t0 = time.time()
        while True:
            st, info = P.cptr_poll(srv, rid, x)
            if st != P._lib.PENDING:
                break
            assert time.time() - t0 < 120
            time.sleep(0.002)
    finally:
        P.cptr_server_destroy(srv)
    assert st == P._lib.OK
    np.testing.assert_array_equal(x, xd)


def test_mgr_preconditioner_pieces_match_oracle(P, oracle_mod):
    """Every piece of Eq. 3 on the reduced operator, against the oracle's."""
    import torch
    s = SYSTEMS["knn"]()
    n = s.n_cells
    o = oracle_mod.Oracle.from_system(s, mgr=1).setup()
    r = np.random.default_rng(9).normal(size=4 * n)
    r[2::4] = 0.0   # the reduced system's right-hand sides vanish on the eliminated unknown
    with P.Solver.from_system(s, mgr=1).setup() as g:
        def run(which, inp, nout):
            out = torch.zeros(nout, dtype=torch.float64, device="cuda")
            P.cptr_apply(g.h, which, torch.from_numpy(np.ascontiguousarray(inp)).cuda(), out)
            torch.cuda.synchronize()
            return out.cpu().numpy()

        assert _relerr(run(P.APPLY_RESTRICT, r, 2 * n), o.restrict(r)) < 1e-14
        rh = o.restrict(r)
        assert _relerr(run(P.APPLY_VCYCLE, rh, 2 * n), o.vcycle(rh)) < 1e-10
        y1 = o.first_stage(r)
        assert _relerr(run(P.APPLY_FIRST, r, 4 * n), y1) < 1e-10
        assert _relerr(run(P.APPLY_CORRECTION, r, 4 * n), o.correction(r, y1)) < 1e-10
        assert _relerr(run(P.APPLY_ILU, r, 4 * n), o.ilu_apply(r)) < 1e-10
        z = run(P.APPLY_PRECOND, r, 4 * n)
        assert _relerr(z, o.precond(r)) < 1e-10
        assert not z[2::4].any()   # the eliminated unknown stays zero through Eq. 3
