"""Newton-loop use of one context: new Jacobian values with the same pattern
(cptr_update_values), a new setup and a new solve.  The result must be
bit-identical to a fresh context's on the same values, and switching back to
the first values must reproduce the first solution exactly: every piece of
setup state (the AMG hierarchy, the ILU(0) factors built on the second
stream, the solve schedule, the captured Arnoldi graph) is rebuilt."""
import numpy as np
import pytest

from synth import config_system

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


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_update_values_matches_fresh_context(P, oracle_mod, prec):
    p = P.MIXED if prec == "mixed" else P.FP64
    s1 = config_system("c1", pe=1.0)
    s2 = config_system("c1", pe=100.0)  # same grid and pattern, other values
    np.testing.assert_array_equal(s1.rowptr, s2.rowptr)
    np.testing.assert_array_equal(s1.col, s2.col)
    with P.Solver.from_system(s2, precision=p).setup() as g:
        x2_fresh, i2_fresh = g.solve(s2.rhs)
    with P.Solver.from_system(s1, precision=p).setup() as g:
        x1, i1 = g.solve(s1.rhs)
        P.cptr_update_values(g.h, np.ascontiguousarray(s2.vals))
        g.setup()
        x2, i2 = g.solve(s2.rhs)
        P.cptr_update_values(g.h, np.ascontiguousarray(s1.vals))
        g.setup()
        x1_again, i1_again = g.solve(s1.rhs)
    assert i2["status"] == P._lib.OK and i2["iters"] == i2_fresh["iters"]
    np.testing.assert_array_equal(x2, x2_fresh)
    assert i1_again["iters"] == i1["iters"]
    np.testing.assert_array_equal(x1_again, x1)
    o = oracle_mod.Oracle.from_system(s2)
    assert np.linalg.norm(s2.rhs - o.spmv(x2)) <= 1e-6 * np.linalg.norm(s2.rhs)
