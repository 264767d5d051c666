"""V(nu_pre, nu_post) cycles and the hybrid l1-Gauss-Seidel smoother on the GPU
against the oracle: the V-cycle applied once to 1e-10 (FP64), the whole
preconditioner to 1e-10, FP64 solves to 1e-8 with iterations within one, mixed
precision within 10% of the oracle's iterations."""
import numpy as np
import pytest

from synth import cartesian, config_system, knn

pytestmark = pytest.mark.gpu

SYSTEMS = {
    "c1": lambda: config_system("c1"),
    "knn": lambda: knn(12, 10, 5, pe=10.0, seed=31),
    "aniso_cold": lambda: cartesian(13, 11, 9, pe=1.0, seed=41, sigma=2.0, layered=True,
                                    kv_ratio=0.1, cold_dT=40.0),
}
CYCLES = [(2, 1, 0), (0, 2, 0), (0, 0, 0), (1, 1, 1), (2, 3, 1), (0, 1, 1)]


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


@pytest.mark.parametrize("cyc", CYCLES)
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_vcycle_and_precond(P, oracle_mod, name, cyc):
    import torch
    nu1, nu2, sm = cyc
    kw = dict(nu_pre=nu1, nu_post=nu2, smoother=sm)
    s = SYSTEMS[name]()
    o = oracle_mod.Oracle.from_system(s, **kw).setup()
    rng = np.random.default_rng(12)
    bh = rng.normal(size=2 * s.n_cells)
    r = rng.normal(size=4 * s.n_cells)
    with P.Solver.from_system(s, **kw).setup() as g:
        out = torch.zeros(2 * s.n_cells, dtype=torch.float64, device="cuda")
        P.cptr_apply(g.h, P.APPLY_VCYCLE, torch.from_numpy(bh).cuda(), out)
        out2 = torch.zeros(4 * s.n_cells, dtype=torch.float64, device="cuda")
        P.cptr_apply(g.h, P.APPLY_PRECOND, torch.from_numpy(r).cuda(), out2)
        torch.cuda.synchronize()
        assert _relerr(out.cpu().numpy(), o.vcycle(bh)) < 1e-10
        assert _relerr(out2.cpu().numpy(), o.precond(r)) < 1e-10


@pytest.mark.parametrize("cyc", [(1, 1, 1), (2, 2, 0)])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_solve_matches_oracle(P, oracle_mod, name, cyc):
    nu1, nu2, sm = cyc
    kw = dict(nu_pre=nu1, nu_post=nu2, smoother=sm)
    s = SYSTEMS[name]()
    o = oracle_mod.Oracle.from_system(s, **kw).setup()
    xo, io = o.solve(s.rhs)
    with P.Solver.from_system(s, **kw).setup() as g:
        xg, ig = g.solve(s.rhs)
    assert ig["status"] == 0 and abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
    with P.Solver.from_system(s, precision=P.MIXED, **kw).setup() as g:
        xm, im = g.solve(s.rhs)
    assert im["status"] == 0 and abs(im["iters"] - io["iters"]) <= max(1, 0.1 * io["iters"])
    assert np.linalg.norm(s.rhs - o.spmv(xm)) <= 1e-6 * np.linalg.norm(s.rhs)


def test_smoother_parameters_are_checked(P):
    s = config_system("c1")
    for bad in (dict(nu_pre=-1), dict(nu_post=9), dict(smoother=2)):
        with pytest.raises(P.CPTRError):
            P.Solver.from_system(s, **bad)
