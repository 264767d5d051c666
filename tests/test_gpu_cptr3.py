"""CPTR3 (Section 3.3) on the GPU against the oracle.

The three-stage preconditioner (pressure stage, temperature stage on the
residual the pressure stage leaves, ILU(0) on the residual of both) applied
once matches the oracle's to 1e-10 in FP64 (the stage hierarchies are built
with the same arithmetic as CPTR's, so a 1e-10 agreement needs identical
splits on both stages); FP64 solves match to 1e-8 with iterations within one;
mixed precision reaches the tolerance within 10% of the oracle's iterations.
"""
import numpy as np
import pytest

from synth import cartesian, config_system, knn, with_volume_constraint

pytestmark = pytest.mark.gpu

SYSTEMS = {
    "c1": lambda: config_system("c1"),
    "knn": lambda: knn(12, 10, 5, pe=10.0, seed=31),
    "aniso_cold": lambda: cartesian(13, 11, 9, pe=1.0, seed=41, sigma=2.0, layered=True,
                                    kv_ratio=0.1, cold_dT=40.0),
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
def test_cptr3_apply_matches_oracle(P, oracle_mod, name):
    import torch
    s = SYSTEMS[name]()
    o = oracle_mod.Oracle.from_system(s, precond=oracle_mod.PREC_CPTR3).setup()
    r = np.random.default_rng(4).normal(size=4 * s.n_cells)
    with P.Solver.from_system(s, precond=P.PREC_CPTR3).setup() as g:
        out = torch.zeros(4 * s.n_cells, dtype=torch.float64, device="cuda")
        P.cptr_apply(g.h, P.APPLY_PRECOND, torch.from_numpy(r).cuda(), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # the pressure stage alone, through the single-piece call
        out1 = torch.zeros_like(out)
        P.cptr_apply(g.h, P.APPLY_FIRST, torch.from_numpy(r).cuda(), out1)
        torch.cuda.synchronize()
    assert _relerr(got, o.precond(r)) < 1e-10
    op = oracle_mod.Oracle.from_system(s, e1=-1, precond=oracle_mod.PREC_FIRST).setup()
    assert _relerr(out1.cpu().numpy(), op.first_stage(r)) < 1e-10


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_cptr3_solve_matches_oracle(P, oracle_mod, name):
    s = SYSTEMS[name]()
    o = oracle_mod.Oracle.from_system(s, precond=oracle_mod.PREC_CPTR3).setup()
    xo, io = o.solve(s.rhs)
    with P.Solver.from_system(s, precond=P.PREC_CPTR3).setup() as g:
        xg, ig = g.solve(s.rhs)
    assert ig["status"] == 0 and io["status"] == 0
    assert abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
    with P.Solver.from_system(s, precond=P.PREC_CPTR3, precision=P.MIXED).setup() as g:
        xm, im = g.solve(s.rhs)
    assert im["status"] == 0 and abs(im["iters"] - io["iters"]) <= max(1, 0.1 * io["iters"])
    rel = np.linalg.norm(s.rhs - o.spmv(xm)) / np.linalg.norm(s.rhs)
    assert rel <= 1e-6
    print(f"{name}: CPTR3 iterations oracle {io['iters']} fp64 {ig['iters']} mixed {im['iters']}; "
          f"|x_mixed - x_oracle| / |x_oracle| {np.linalg.norm(xm - xo) / np.linalg.norm(xo):.2e}")


def test_cptr3_with_the_mgr_reduction(P, oracle_mod):
    """CPTR3 after the first MGR reduction (Section 3.4), as the paper's
    framework would chain them: same bars as above."""
    s = with_volume_constraint(config_system("c1"), seed=3)
    o = oracle_mod.Oracle.from_system(s, precond=oracle_mod.PREC_CPTR3, mgr=1).setup()
    xo, io = o.solve(s.rhs)
    with P.Solver.from_system(s, precond=P.PREC_CPTR3, mgr=1).setup() as g:
        xg, ig = g.solve(s.rhs)
    assert ig["status"] == 0 and abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8


def test_cptr3_needs_two_elliptic_unknowns(P):
    s = config_system("c1")
    with pytest.raises(P.CPTRError):
        P.Solver.from_system(s, precond=P.PREC_CPTR3, e1=-1)
