"""GPU parity: every hot-path step of the CUDA library against the FP64 oracle.

Calls go through the C ABI (libcptr.so).  FP64 tolerances: SpMV, decoupling
and ILU factors agree to rounding (<= 1e-13 relative); the AMG hierarchy has
identical C/F splittings (integers, exact) and values to 1e-12; applications
of the preconditioner to 1e-10 (the coarsest level is solved with an explicit
inverse on the GPU and with LU on the CPU); solutions to 1e-8 relative with
iteration counts within +-1.  Mixed precision: iterations within 10% and the
true FP64 residual below the tolerance.
"""
import numpy as np
import pytest

from synth import block_tridiag_chain, cartesian, config_system, knn, random_bsr

pytestmark = pytest.mark.gpu


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


SYSTEMS = {
    "c1": lambda: config_system("c1"),
    "random_ragged": lambda: random_bsr(203, avg_offdiag=5, seed=21, empty_rows=0.2),
    "knn": lambda: knn(12, 10, 5, pe=10.0, seed=31),
    "aniso_cold": lambda: cartesian(13, 11, 9, pe=1.0, seed=41, sigma=2.0, layered=True,
                                    kv_ratio=0.1, cold_dT=40.0),
}


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_spmv(P, oracle_mod, name):
    s = SYSTEMS[name]()
    o = oracle_mod.Oracle.from_system(s)
    x = np.random.default_rng(1).normal(size=4 * s.n_cells)
    with P.Solver.from_system(s) as g:
        xd = _dev(x)
        yd = xd.new_zeros(xd.shape)
        P.cptr_spmv(g.h, xd, yd)
        assert _relerr(_host(yd), o.spmv(x)) < 1e-14


def test_spmv_single_cell_and_empty_rows(P, oracle_mod):
    for s in (cartesian(1, 1, 1, seed=3), random_bsr(17, seed=5, empty_rows=1.0)):
        o = oracle_mod.Oracle.from_system(s)
        x = np.random.default_rng(2).normal(size=4 * s.n_cells)
        with P.Solver.from_system(s) as g:
            xd = _dev(x)
            yd = xd.new_zeros(xd.shape)
            P.cptr_spmv(g.h, xd, yd)
            assert _relerr(_host(yd), o.spmv(x)) < 1e-14


def _hier(g, P, l):
    info = P.cptr_level_info(g.h, l)
    rp = g.copy(l, P.COPY_A_ROWPTR, np.int32, info["n"] + 1)
    ci = g.copy(l, P.COPY_A_COL, np.int32, info["nnz"])
    v = g.copy(l, P.COPY_A_VAL, np.float64, info["nnz"])
    return info, rp, ci, v


# Larger systems for the hierarchy comparison only.  At Pe = 100 the coarse
# operators of the 64x64x32 system reach rows of thousands of columns, which
# the default setup sends to its global-scratch ext+i and SpGEMM passes, and
# the coarsest matrix is inverted on a thread-block cluster.
LARGE = {"c2_pe100": lambda: config_system("c2", pe=100.0)}


@pytest.mark.parametrize("name", ["c1", "knn", "aniso_cold", "c2_pe100"])
def test_setup_hierarchy_matches_oracle(P, oracle_mod, name):
    s = {**SYSTEMS, **LARGE}[name]()
    o = oracle_mod.Oracle.from_system(s).setup()
    oa = o.amg()
    with P.Solver.from_system(s).setup() as g:
        # Quasi-IMPES decoupling
        W = g.copy(0, P.COPY_W, np.float64, 4 * s.n_cells).reshape(-1, 2, 2)
        assert _relerr(W, o.W()) <= 1e-15
        orp, oci, ov = o.ahat()
        info, rp, ci, v = _hier(g, P, 0)
        np.testing.assert_array_equal(rp, orp)
        np.testing.assert_array_equal(ci, oci)
        assert _relerr(v, ov) <= 1e-15
        # AMG levels
        assert P.cptr_amg_levels(g.h) == oa.nlevels
        for l in range(oa.nlevels):
            oi = oa.level_info(l)
            info, rp, ci, v = _hier(g, P, l)
            assert (info["n"], info["nnz"], info["nc"], info["nnzP"]) == \
                (oi["n"], oi["nnz"], oi["nc"], oi["nnzP"])
            orp, oci, ov = oa.level_A(l)
            np.testing.assert_array_equal(rp, orp)
            np.testing.assert_array_equal(ci, oci)
            assert _relerr(v, ov) <= 1e-12
            if l < oa.nlevels - 1:
                cf = g.copy(l, P.COPY_CF, np.int32, info["n"])
                np.testing.assert_array_equal(cf, oa.level_cf(l))
                prp = g.copy(l, P.COPY_P_ROWPTR, np.int32, info["n"] + 1)
                pci = g.copy(l, P.COPY_P_COL, np.int32, info["nnzP"])
                pv = g.copy(l, P.COPY_P_VAL, np.float64, info["nnzP"])
                orp, oci, ov = oa.level_P(l)
                np.testing.assert_array_equal(prp, orp)
                np.testing.assert_array_equal(pci, oci)
                assert _relerr(pv, ov) <= 1e-12
                d = g.copy(l, P.COPY_DL1, np.float64, info["n"])
                assert _relerr(d, oa.level_dl1(l)) <= 1e-12
        # ILU(0)
        F = g.copy(0, P.COPY_ILU, np.float64, 16 * s.nnzb).reshape(-1, 16)
        assert _relerr(F, o.ilu_factors()) <= 1e-12
        nlev, lv = o.ilu_levels()
        np.testing.assert_array_equal(g.copy(0, P.COPY_ILU_LEVEL, np.int32, s.n_cells), lv)


def test_setup_fallback_kernels_match_oracle(P, oracle_mod, monkeypatch):
    """The thread-per-row setup kernels (used when a row's column set does not
    fit in shared memory) build the same hierarchy."""
    monkeypatch.setenv("CPTR_SETUP_FALLBACK", "1")
    test_setup_hierarchy_matches_oracle(P, oracle_mod, "knn")


@pytest.mark.parametrize("var,val", [("CPTR_SPGEMM_PATH", "1"), ("CPTR_SPGEMM_PATH", "2"),
                                     ("CPTR_SPGEMM_PATH", "3"), ("CPTR_INTERP_PATH", "1"),
                                     ("CPTR_INTERP_PATH", "2")])
def test_setup_kernel_paths_match_oracle(P, oracle_mod, monkeypatch, var, val):
    """Each Galerkin SpGEMM path (ordered-table block kernel, bucketed block
    kernel, global-scratch kernel) and each ext+i path (wide blocks, global
    scratch), forced for every row, builds the oracle's hierarchy: the same C/F
    splits and patterns, values within 1e-12.  By default the library picks a
    path per level from its row shapes, so small systems alone would not reach
    all of them."""
    monkeypatch.setenv(var, val)
    for name in ("knn", "aniso_cold"):
        test_setup_hierarchy_matches_oracle(P, oracle_mod, name)


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_apply_pieces_fp64(P, oracle_mod, name):
    s = SYSTEMS[name]()
    n = s.n_cells
    o = oracle_mod.Oracle.from_system(s).setup()
    r = np.random.default_rng(7).normal(size=4 * n)
    with P.Solver.from_system(s).setup() as g:
        rd = _dev(r)

        def run(which, inp, nout):
            out = _dev(np.zeros(nout))
            P.cptr_apply(g.h, which, _dev(inp) if isinstance(inp, np.ndarray) else inp, out)
            return _host(out)

        assert _relerr(run(P.APPLY_RESTRICT, r, 2 * n), o.restrict(r)) < 1e-14
        rh = o.restrict(r)
        assert _relerr(run(P.APPLY_VCYCLE, rh, 2 * n), o.vcycle(rh)) < 1e-10
        y1 = o.first_stage(r)
        assert _relerr(run(P.APPLY_FIRST, r, 4 * n), y1) < 1e-10
        assert _relerr(run(P.APPLY_CORRECTION, r, 4 * n), o.correction(r, y1)) < 1e-10
        assert _relerr(run(P.APPLY_ILU, r, 4 * n), o.ilu_apply(r)) < 1e-10
        assert _relerr(run(P.APPLY_PRECOND, rd, 4 * n), o.precond(r)) < 1e-10


# strip schedule geometries (CPTR_STRIP_P strips, CPTR_STRIP_RC ring rows,
# CPTR_STRIP_RING staging bytes): the default one strip per SM (a few rows each
# here, so nearly every dependency crosses strips), three strips with an
# 8-row solution ring (own rows leave the ring and are read back from global
# memory) and a 4 KiB staging ring (many sub-steps, the ring wraps around)
STRIP_GEOMS = {"default": {}, "evict_wrap": {"CPTR_STRIP_P": "3", "CPTR_STRIP_RC": "8",
                                             "CPTR_STRIP_RING": "4096"}}


@pytest.mark.parametrize("R", [0, 1, 2, 128, 1024, "2:evict_wrap"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_triangular_solve_paths(P, oracle_mod, monkeypatch, R, prec):
    """Each triangular-solve schedule (level-padded kernels R=0, one cluster
    walking the levels R=1, strips R=2, chunked with R rows per thread block)
    gives the oracle's ILU(0) application."""
    if isinstance(R, str):
        R, geom = R.split(":")
        for k, v in STRIP_GEOMS[geom].items():
            monkeypatch.setenv(k, v)
        R = int(R)
    monkeypatch.setenv("CPTR_TRI_R", str(R))
    s = SYSTEMS["knn"]()
    o = oracle_mod.Oracle.from_system(s).setup()
    r = np.random.default_rng(5).normal(size=4 * s.n_cells)
    tol = 1e-10 if prec == "fp64" else 1e-4
    with P.Solver.from_system(s, precision=P.MIXED if prec == "mixed" else P.FP64).setup() as g:
        if R in (0, 1, 2, 128):  # these always fit; 1024 rows in FP64 fall back to R=0
            assert P.cptr_get_info(g.h)["tri_schedule"] == R
        out = _dev(np.zeros(4 * s.n_cells))
        P.cptr_apply(g.h, P.APPLY_ILU, _dev(r), out)
        assert _relerr(_host(out), o.ilu_apply(r)) < tol
        out2 = _dev(np.zeros(4 * s.n_cells))
        P.cptr_apply(g.h, P.APPLY_PRECOND, _dev(r), out2)
        assert _relerr(_host(out2), o.precond(r)) < tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_triangular_solve_paths_bit_identical(P, monkeypatch, prec):
    """Every schedule evaluates each row with the same rounding sequence, so the
    tuner's choice never changes a result (serving relies on this)."""
    s = SYSTEMS["knn"]()
    r = np.random.default_rng(6).normal(size=4 * s.n_cells)
    outs = []
    for R in (0, 1, 2, 128, 256, 1024, "2:evict_wrap"):
        for geom in STRIP_GEOMS.values():
            for k in geom:
                monkeypatch.delenv(k, raising=False)
        if isinstance(R, str):
            R, g_ = R.split(":")
            for k, v in STRIP_GEOMS[g_].items():
                monkeypatch.setenv(k, v)
        monkeypatch.setenv("CPTR_TRI_R", str(R))
        with P.Solver.from_system(s, precision=P.MIXED if prec == "mixed" else P.FP64).setup() as g:
            o1 = _dev(np.zeros(4 * s.n_cells))
            P.cptr_apply(g.h, P.APPLY_ILU, _dev(r), o1)
            o2 = _dev(np.zeros(4 * s.n_cells))
            P.cptr_apply(g.h, P.APPLY_PRECOND, _dev(r), o2)
            outs.append((_host(o1), _host(o2)))
    for a, b in outs[1:]:
        np.testing.assert_array_equal(a, outs[0][0])
        np.testing.assert_array_equal(b, outs[0][1])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_chain_schedule(P, oracle_mod, monkeypatch, prec):
    """The chain schedule (R=3: one quad walks each chain of rows linked to
    their dependency of highest level) is built on a natural-order grid, gives
    the oracle's ILU(0) application and is bit-identical to the level kernels;
    on a kNN pattern, where some dependency points to a later chain, it is
    refused and the level kernels run instead."""
    s = SYSTEMS["aniso_cold"]()
    o = oracle_mod.Oracle.from_system(s).setup()
    r = np.random.default_rng(8).normal(size=4 * s.n_cells)
    tol = 1e-10 if prec == "fp64" else 1e-4
    pr = P.MIXED if prec == "mixed" else P.FP64
    outs = []
    for R in (3, 0):
        monkeypatch.setenv("CPTR_TRI_R", str(R))
        with P.Solver.from_system(s, precision=pr).setup() as g:
            assert P.cptr_get_info(g.h)["tri_schedule"] == R
            out = _dev(np.zeros(4 * s.n_cells))
            P.cptr_apply(g.h, P.APPLY_ILU, _dev(r), out)
            out2 = _dev(np.zeros(4 * s.n_cells))
            P.cptr_apply(g.h, P.APPLY_PRECOND, _dev(r), out2)
            outs.append((_host(out), _host(out2)))
    assert _relerr(outs[0][0], o.ilu_apply(r)) < tol
    assert _relerr(outs[0][1], o.precond(r)) < tol
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    monkeypatch.setenv("CPTR_TRI_R", "3")
    with P.Solver.from_system(SYSTEMS["knn"](), precision=pr).setup() as g:
        assert P.cptr_get_info(g.h)["tri_schedule"] == 0


def test_apply_twice_is_identical(P):
    """Sync-free solves and reductions are deterministic run to run."""
    s = SYSTEMS["knn"]()
    r = _dev(np.random.default_rng(3).normal(size=4 * s.n_cells))
    with P.Solver.from_system(s).setup() as g:
        a = _dev(np.zeros(4 * s.n_cells)); b = _dev(np.zeros(4 * s.n_cells))
        P.cptr_apply(g.h, P.APPLY_PRECOND, r, a)
        P.cptr_apply(g.h, P.APPLY_PRECOND, r, b)
        np.testing.assert_array_equal(_host(a), _host(b))


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_solve_fp64_matches_oracle(P, oracle_mod, name):
    s = SYSTEMS[name]()
    o = oracle_mod.Oracle.from_system(s).setup()
    xo, io = o.solve(s.rhs)
    with P.Solver.from_system(s).setup() as g:
        xg, ig = g.solve(s.rhs)
    assert ig["status"] == 0 and io["status"] == 0
    assert abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
    r = s.rhs - o.spmv(xg)
    assert np.linalg.norm(r) / np.linalg.norm(s.rhs) <= 1e-6


@pytest.mark.parametrize("prec", ["NONE", "ILU", "FIRST"])
def test_solve_other_preconditioners(P, oracle_mod, prec):
    """The first stage alone never corrects the hyperbolic unknowns, so GMRES
    stagnates with it (and nearly so without a preconditioner); those two are
    compared after 10 iterations, before stagnation can amplify rounding."""
    s = config_system("c1")
    pc = {"NONE": (P.PREC_NONE, oracle_mod.PREC_NONE), "ILU": (P.PREC_ILU, oracle_mod.PREC_ILU),
          "FIRST": (P.PREC_FIRST, oracle_mod.PREC_FIRST)}[prec]
    maxit = 400 if prec == "ILU" else 10
    o = oracle_mod.Oracle.from_system(s, precond=pc[1], maxit=maxit).setup()
    xo, io = o.solve(s.rhs)
    with P.Solver.from_system(s, precond=pc[0], maxit=maxit).setup() as g:
        xg, ig = g.solve(s.rhs)
    assert ig["status"] == io["status"]
    assert abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8


def test_solve_chain_one_iteration(P):
    """Eq. 3 with an exact ILU(0) (1D chain of cells): one iteration."""
    s = cartesian(40, 1, 1, pe=1.0, seed=9)
    with P.Solver.from_system(s, tol=1e-10).setup() as g:
        x, info = g.solve(s.rhs)
    assert info["iters"] == 1 and info["status"] == 0


def test_solve_maxit_and_zero_rhs(P, oracle_mod):
    s = config_system("c1")
    o = oracle_mod.Oracle.from_system(s, maxit=3).setup()
    xo, io = o.solve(s.rhs)
    with P.Solver.from_system(s, maxit=3).setup() as g:
        xg, ig = g.solve(s.rhs)
        assert ig["status"] == P._lib.ERR_MAXIT and ig["iters"] == 3
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
        x0, iz = g.solve(np.zeros(4 * s.n_cells), x=np.ones(4 * s.n_cells))
        assert iz["iters"] == 0 and np.all(x0 == 0)


def test_solve_device_buffers_and_restart(P, oracle_mod):
    s = SYSTEMS["random_ragged"]()
    o = oracle_mod.Oracle.from_system(s, restart=4).setup()
    xo, io = o.solve(s.rhs)
    with P.Solver.from_system(s, restart=4).setup() as g:
        b = _dev(s.rhs)
        x = b.new_zeros(b.shape)
        _, ig = g.solve(b, x)
        xg = _host(x)
    assert abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8


@pytest.mark.parametrize("pe", [0.01, 1.0, 100.0])
def test_solve_c2_peclet_sweep_fp64_and_mixed(P, oracle_mod, pe):
    """The 64x64x32 workload at each Peclet number: FP64 parity with the oracle
    and the mixed-precision form within 10% of its iterations."""
    s = config_system("c2", pe=pe)
    o = oracle_mod.Oracle.from_system(s).setup()
    xo, io = o.solve(s.rhs)
    with P.Solver.from_system(s).setup() as g:
        xg, ig = g.solve(s.rhs)
    assert abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
    with P.Solver.from_system(s, precision=P.MIXED).setup() as g:
        xm, im = g.solve(s.rhs)
    assert im["status"] == 0
    assert abs(im["iters"] - io["iters"]) <= max(1, int(0.1 * io["iters"]))
    r = s.rhs - o.spmv(xm)
    assert np.linalg.norm(r) / np.linalg.norm(s.rhs) <= 1e-6


@pytest.mark.parametrize("name", ["c1", "knn"])
def test_solve_mixed_precision(P, oracle_mod, name):
    s = SYSTEMS[name]()
    o = oracle_mod.Oracle.from_system(s).setup()
    xo, io = o.solve(s.rhs)
    with P.Solver.from_system(s, precision=P.MIXED).setup() as g:
        xm, im = g.solve(s.rhs)
    assert im["status"] == 0
    assert abs(im["iters"] - io["iters"]) <= max(1, int(0.1 * io["iters"]))
    r = s.rhs - o.spmv(xm)
    assert np.linalg.norm(r) / np.linalg.norm(s.rhs) <= 1e-6
    # error against the FP64 oracle at the same tolerance, reported by the test log
    err = np.linalg.norm(xm - xo) / np.linalg.norm(xo)
    assert err < 1e-4, err


def test_mixed_apply_error_bound(P, oracle_mod):
    """FP32 preconditioner pieces stay within a few thousand FP32 ulps of FP64."""
    s = SYSTEMS["c1"]()
    n = s.n_cells
    o = oracle_mod.Oracle.from_system(s).setup()
    r = np.random.default_rng(9).normal(size=4 * n)
    with P.Solver.from_system(s, precision=P.MIXED).setup() as g:
        out = _dev(np.zeros(4 * n))
        P.cptr_apply(g.h, P.APPLY_PRECOND, _dev(r), out)
        assert _relerr(_host(out), o.precond(r)) < 1e-3


# ---------------------------------------------------------------- CPR (Section 3.1)
CPR = dict(e0=0, e1=-1)


@pytest.mark.parametrize("name", ["c1", "knn"])
def test_cpr_setup_and_pieces_match_oracle(P, oracle_mod, name):
    """CPR: pressure-only Quasi-IMPES decoupling (1x3 W, 3x3 inverse), scalar
    AMG on the pressure system, and every preconditioner piece."""
    s = SYSTEMS[name]()
    n = s.n_cells
    o = oracle_mod.Oracle.from_system(s, **CPR).setup()
    oa = o.amg()
    with P.Solver.from_system(s, **CPR).setup() as g:
        W = g.copy(0, P.COPY_W, np.float64, 4 * n).reshape(n, 4)[:, :3].reshape(n, 1, 3)
        assert _relerr(W, o.W()) <= 1e-15
        orp, oci, ov = o.ahat()
        info, rp, ci, v = _hier(g, P, 0)
        np.testing.assert_array_equal(rp, orp)
        np.testing.assert_array_equal(ci, oci)
        assert _relerr(v, ov) <= 1e-15
        assert P.cptr_amg_levels(g.h) == oa.nlevels
        for l in range(oa.nlevels - 1):
            np.testing.assert_array_equal(g.copy(l, P.COPY_CF, np.int32, _hier(g, P, l)[0]["n"]),
                                          oa.level_cf(l))
        r = np.random.default_rng(7).normal(size=4 * n)

        def run(which, inp, nout):
            out = _dev(np.zeros(nout))
            P.cptr_apply(g.h, which, _dev(inp), out)
            return _host(out)

        assert _relerr(run(P.APPLY_RESTRICT, r, n), o.restrict(r)) < 1e-14
        rh = o.restrict(r)
        assert _relerr(run(P.APPLY_VCYCLE, rh, n), o.vcycle(rh)) < 1e-10
        y1 = o.first_stage(r)
        assert _relerr(run(P.APPLY_FIRST, r, 4 * n), y1) < 1e-10
        assert _relerr(run(P.APPLY_CORRECTION, r, 4 * n), o.correction(r, y1)) < 1e-10
        assert _relerr(run(P.APPLY_PRECOND, r, 4 * n), o.precond(r)) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cpr_solve_matches_oracle(P, oracle_mod, prec):
    s = SYSTEMS["aniso_cold"]()
    o = oracle_mod.Oracle.from_system(s, **CPR).setup()
    xo, io = o.solve(s.rhs)
    with P.Solver.from_system(s, precision=P.FP64 if prec == "fp64" else P.MIXED,
                              **CPR).setup() as g:
        xg, ig = g.solve(s.rhs)
    assert ig["status"] == 0 and io["status"] == 0
    if prec == "fp64":
        assert abs(ig["iters"] - io["iters"]) <= 1
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
    else:
        assert abs(ig["iters"] - io["iters"]) <= max(1, int(0.1 * io["iters"]))
    r = s.rhs - o.spmv(xg)
    assert np.linalg.norm(r) / np.linalg.norm(s.rhs) <= 1e-6


def test_cpr_vs_cptr_peclet_on_gpu(P):
    """Section 5.3's comparison on the GPU (mixed precision): CPR needs more
    iterations when conduction matters, CPTR stays nearly flat."""
    its = {}
    for pe in (0.01, 100.0):
        s = cartesian(16, 16, 8, pe=pe, seed=1002)
        for name, kw in (("cptr", {}), ("cpr", CPR)):
            with P.Solver.from_system(s, precision=P.MIXED, **kw).setup() as g:
                x, info = g.solve(s.rhs)
            assert info["status"] == 0
            its[name, pe] = info["iters"]
    assert its["cpr", 0.01] > its["cpr", 100.0]
    assert its["cptr", 0.01] < its["cpr", 0.01]


def test_ilu_block_inverses_pivot(P, oracle_mod):
    """Diagonal blocks with zero leading entries: the GPU's 4x4 Gauss-Jordan
    exchanges rows like the oracle, and ILU(0) on the block-tridiagonal chain
    is the exact inverse."""
    from conftest import bsr_from_dense
    from amg_cases import pivoting_chain
    A = pivoting_chain(6)
    rp, ci, v = bsr_from_dense(A)
    o = oracle_mod.Oracle(rp, ci, v, precond=oracle_mod.PREC_ILU).setup()
    r = np.random.default_rng(1).normal(size=A.shape[0])
    with P.Solver(6, rp, ci, v, precond=P.PREC_ILU).setup() as g:
        out = _dev(np.zeros(A.shape[0]))
        P.cptr_apply(g.h, P.APPLY_ILU, _dev(r), out)
        y = _host(out)
    assert _relerr(y, o.ilu_apply(r)) < 1e-12
    assert _relerr(y, np.linalg.solve(A, r)) < 1e-11


def test_gmres_happy_breakdown(P):
    """M = I and three distinct eigenvalues in b: the GPU's FGMRES stops at the
    exact solution after three iterations (h_{4,3} = 0) without dividing by it."""
    from conftest import bsr_from_dense
    from amg_cases import happy_breakdown_case
    A, b = happy_breakdown_case()
    rp, ci, v = bsr_from_dense(A)
    with P.Solver(A.shape[0] // 4, rp, ci, v, precond=P.PREC_NONE, tol=1e-14).setup() as g:
        x, info = g.solve(b)
    assert info["status"] == 0 and info["iters"] == 3
    assert np.isfinite(x).all()
    np.testing.assert_allclose(x, b / np.diag(A), rtol=1e-12)


@pytest.mark.parametrize("restart", [40, 63])
def test_long_restart_cycles_match_oracle(P, oracle_mod, restart):
    """Arnoldi cycles longer than 32 steps (restart at most 63): the second
    CGS pass forms the first 32 dots with the update and the others in an
    offset pass.  ILU(0) alone at tol 1e-12 on a 16x16x8 grid needs 43-44
    steps in one cycle; FP64 to 1e-8 and iterations within one."""
    s = cartesian(16, 16, 8, pe=1.0, seed=5)
    o = oracle_mod.Oracle.from_system(s, precond=oracle_mod.PREC_ILU, restart=restart).setup()
    xo, io = o.solve(s.rhs, tol=1e-12)
    assert io["status"] == 0 and io["iters"] > 32
    with P.Solver.from_system(s, precond=P.PREC_ILU, restart=restart).setup() as g:
        xg, ig = g.solve(s.rhs, tol=1e-12)
    assert ig["status"] == 0 and abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
