"""Failure detection on the GPU, without faulting, trapping or hanging it.

Errors are status codes: a non-finite right-hand side ends the solve with
CPTR_ERR_BREAKDOWN (non-finite residual); a singular diagonal block ends the
setup with CPTR_ERR_BREAKDOWN (zero pivot of the decoupling's 2x2 inverse or of
the ILU(0) pivot block); a triangular-solve dependency wait that runs out of
polls (the limit set small with cptr_set_spin_limit, so that a wait on a row
not yet computed gives up at once) makes the solve return CPTR_ERR_TIMEOUT
after every kernel has finished on its own, and the same context then solves
correctly with the default limit.
"""
import numpy as np
import pytest

from synth import cartesian, config_system

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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nan_rhs_is_a_breakdown(P, prec):
    s = config_system("c1")
    b = s.rhs.copy()
    b[17] = np.nan
    with P.Solver.from_system(s, precision=P.FP64 if prec == "fp64" else P.MIXED).setup() as g:
        with pytest.raises(P.CPTRError) as e:
            g.solve(b)
        assert e.value.status == P._lib.ERR_BREAKDOWN
        # the context is still usable
        x, info = g.solve(s.rhs)
        assert info["status"] == P._lib.OK


def _with_block(s, cell, block):
    vals = s.vals.copy()
    t = next(t for t in range(s.rowptr[cell], s.rowptr[cell + 1]) if s.col[t] == cell)
    vals[t] = block.reshape(16)
    return vals


@pytest.mark.parametrize("kind", ["zero", "rank3"])
def test_singular_diagonal_block_is_a_breakdown(P, oracle_mod, kind):
    s = config_system("c1")
    if kind == "zero":
        blk = np.zeros((4, 4))  # the decoupling's D[h,h] is singular
    else:
        # D[h,h] invertible, the 4x4 block of rank 3 (row 3 repeats row 0): the
        # first cell has no lower neighbours, so its ILU(0) pivot block is this one
        blk = s.vals[next(t for t in range(s.rowptr[0], s.rowptr[1]) if s.col[t] == 0)]
        blk = blk.reshape(4, 4).copy()
        blk[3] = blk[0]
    vals = _with_block(s, 0 if kind == "rank3" else 7, blk)
    with pytest.raises(RuntimeError):  # the oracle refuses the same matrix
        oracle_mod.Oracle(s.rowptr, s.col, vals).setup()
    g = P.Solver(s.n_cells, s.rowptr, s.col, vals)
    try:
        with pytest.raises(P.CPTRError) as e:
            g.setup()
        assert e.value.status == P._lib.ERR_BREAKDOWN
    finally:
        g.close()


@pytest.mark.parametrize("R", [0, 1, 2, 3, 128])
def test_dependency_wait_timeout_then_recovery(P, monkeypatch, R):
    """Every triangular-solve schedule (level kernels, cluster, strips, chains,
    chunks) turns a dependency wait that runs out into CPTR_ERR_TIMEOUT."""
    monkeypatch.setenv("CPTR_TRI_R", str(R))
    s = cartesian(32, 32, 16, pe=1.0, seed=77)
    with P.Solver.from_system(s, precision=P.FP64).setup() as g:
        assert P.cptr_get_info(g.h)["tri_schedule"] == R
        x_ref, i_ref = g.solve(s.rhs)
        P.cptr_set_spin_limit(g.h, 1)
        with pytest.raises(P.CPTRError) as e:
            g.solve(s.rhs)
        assert e.value.status == P._lib.ERR_TIMEOUT
        P.cptr_set_spin_limit(g.h, 0)
        x, info = g.solve(s.rhs)
        assert info["status"] == P._lib.OK and info["iters"] == i_ref["iters"]
        np.testing.assert_array_equal(x, x_ref)
