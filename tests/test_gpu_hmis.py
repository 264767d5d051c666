"""HMIS coarsening (Section 3.1; on one domain, the classical Ruge-Stueben
first pass) on the GPU path against the oracle.

The library runs the sequential first pass on the host over the strength
graph its setup builds on the GPU, and the oracle runs its own; both must pick
the same C/F splitting on every level (an integer decision: exact), and the
hierarchy built on it (P and the coarse operators to 1e-12), the FP64 solve
(1e-8, iterations within one) and the mixed-precision solve (within 10% of the
oracle's iterations) must follow.
"""
import numpy as np
import pytest

from synth import cartesian, config_system, knn

pytestmark = pytest.mark.gpu

SYSTEMS = {
    "c1": lambda: config_system("c1"),
    "knn": lambda: knn(12, 10, 5, pe=10.0, seed=31),
    "aniso": lambda: cartesian(13, 11, 9, pe=1.0, seed=41, sigma=2.0, layered=True,
                               kv_ratio=0.1),
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
@pytest.mark.parametrize("e1", [3, -1])
def test_hmis_hierarchy_matches_oracle(P, oracle_mod, name, e1):
    s = SYSTEMS[name]()
    o = oracle_mod.Oracle.from_system(s, e1=e1, coarsen=oracle_mod.COARSEN_HMIS).setup()
    oa = o.amg()
    with P.Solver.from_system(s, e1=e1, coarsen=P.COARSEN_HMIS).setup() as g:
        assert P.cptr_amg_levels(g.h) == oa.nlevels
        for l in range(oa.nlevels):
            oi = oa.level_info(l)
            info = P.cptr_level_info(g.h, l)
            assert (info["n"], info["nnz"], info["nc"], info["nnzP"]) == \
                (oi["n"], oi["nnz"], oi["nc"], oi["nnzP"])
            v = g.copy(l, P.COPY_A_VAL, np.float64, info["nnz"])
            assert _relerr(v, oa.level_A(l)[2]) <= 1e-12
            if l < oa.nlevels - 1:
                np.testing.assert_array_equal(g.copy(l, P.COPY_CF, np.int32, info["n"]),
                                              oa.level_cf(l))
                pv = g.copy(l, P.COPY_P_VAL, np.float64, info["nnzP"])
                np.testing.assert_array_equal(
                    g.copy(l, P.COPY_P_COL, np.int32, info["nnzP"]), oa.level_P(l)[1])
                assert _relerr(pv, oa.level_P(l)[2]) <= 1e-12
    # HMIS keeps more C points than PMIS on the first level
    op = oracle_mod.Oracle.from_system(s, e1=e1).setup().amg()
    assert oa.level_info(0)["nc"] >= op.level_info(0)["nc"]


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_hmis_solves_match_oracle(P, oracle_mod, name):
    s = SYSTEMS[name]()
    o = oracle_mod.Oracle.from_system(s, coarsen=oracle_mod.COARSEN_HMIS).setup()
    xo, io = o.solve(s.rhs)
    with P.Solver.from_system(s, coarsen=P.COARSEN_HMIS).setup() as g:
        xg, ig = g.solve(s.rhs)
    assert io["status"] == 0 and ig["status"] == 0
    assert abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
    with P.Solver.from_system(s, coarsen=P.COARSEN_HMIS, precision=P.MIXED).setup() as g:
        xm, im = g.solve(s.rhs)
    assert im["status"] == 0 and abs(im["iters"] - io["iters"]) <= max(1, 0.1 * io["iters"])
    assert np.linalg.norm(s.rhs - o.spmv(xm)) / np.linalg.norm(s.rhs) <= 1e-6


def test_hmis_with_one_aggregate_level(P, oracle_mod):
    """Both coarsenings of the aggregate level use the first pass too."""
    s = SYSTEMS["aniso"]()
    o = oracle_mod.Oracle.from_system(s, coarsen=oracle_mod.COARSEN_HMIS, agg=1).setup()
    oa = o.amg()
    with P.Solver.from_system(s, coarsen=P.COARSEN_HMIS, agg=1).setup() as g:
        assert P.cptr_amg_levels(g.h) == oa.nlevels
        for l in range(oa.nlevels - 1):
            info = P.cptr_level_info(g.h, l)
            np.testing.assert_array_equal(g.copy(l, P.COPY_CF, np.int32, info["n"]),
                                          oa.level_cf(l))


def test_bad_coarsen_refused(P):
    s = SYSTEMS["c1"]()
    with pytest.raises(P.CPTRError):
        P.Solver.from_system(s, coarsen=7)
