"""Batched solves (one thread block per system, the whole FGMRES loop on the
device) against the per-system path and the oracle.

A system's batched result does not depend on the batch: solved alone and
among others it is bit-identical.  FP64 batched solves match the oracle to
1e-8 with iterations within one; mixed-precision ones reach the tolerance
within 10% of the oracle's iterations.  Configurations the batched kernel
does not run are refused with CPTR_ERR_INVALID and leave the contexts usable.
"""
import numpy as np
import pytest

from synth import cartesian, knn, with_volume_constraint

pytestmark = pytest.mark.gpu


def _systems():
    return [
        cartesian(9, 8, 5, pe=1.0, seed=51),
        cartesian(12, 10, 6, pe=10.0, seed=52, sigma=2.0, layered=True, kv_ratio=0.1),
        knn(10, 9, 4, pe=10.0, seed=53),
        cartesian(7, 6, 4, pe=100.0, seed=54, cold_dT=40.0),
        with_volume_constraint(cartesian(8, 7, 4, pe=1.0, seed=55), seed=5),
    ]


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_11892_gb300 import build
    build.build()
    import paper_2308_11892_gb300 as P
    return P


def _open(P, systems, **kw):
    return [P.Solver.from_system(s, **kw).setup() for s in systems]


def _batch(P, solvers, systems, **kw):
    xs = [np.zeros(4 * s.n_cells) for s in systems]
    st, infos = P.cptr_solve_batch([g.h for g in solvers], [s.rhs for s in systems], xs, **kw)
    return st, xs, infos


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_result_does_not_depend_on_the_batch(P, precision):
    systems = _systems()
    kw = {} if precision == "fp64" else {"precision": P.MIXED}
    solvers = _open(P, systems, **kw)
    try:
        st, xb, ib = _batch(P, solvers, systems)
        assert st == 0
        for k in (0, 3):
            st1, x1, i1 = _batch(P, [solvers[k]], [systems[k]])
            assert st1 == 0 and i1[0]["iters"] == ib[k]["iters"]
            assert np.array_equal(x1[0], xb[k])
        # reversed order, and each system twice in separate batches
        order = list(reversed(range(len(systems))))
        st2, x2, i2 = _batch(P, [solvers[k] for k in order], [systems[k] for k in order])
        for q, k in enumerate(order):
            assert np.array_equal(x2[q], xb[k]) and i2[q]["iters"] == ib[k]["iters"]
    finally:
        for g in solvers:
            g.close()


def test_batch_fp64_matches_oracle(P, oracle_mod):
    systems = _systems()
    solvers = _open(P, systems)
    try:
        st, xb, ib = _batch(P, solvers, systems)
        assert st == 0
        for s, g, x, info in zip(systems, solvers, xb, ib):
            o = oracle_mod.Oracle.from_system(s).setup()
            xo, io = o.solve(s.rhs)
            assert io["status"] == 0 and info["status"] == 0
            assert abs(info["iters"] - io["iters"]) <= 1
            assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-8
            # and the per-system path
            xg, ig = g.solve(s.rhs)
            assert abs(ig["iters"] - info["iters"]) <= 1
            assert np.linalg.norm(x - xg) / np.linalg.norm(xg) <= 1e-8
    finally:
        for g in solvers:
            g.close()


@pytest.mark.parametrize("variant", ["cptr", "cpr", "ilu"])
def test_batch_mixed_reaches_tolerance(P, oracle_mod, variant):
    systems = _systems()[:3]
    kw = {"cpr": {"e1": -1}, "ilu": {"precond": P.PREC_ILU}}.get(variant, {})
    okw = {"cpr": {"e1": -1}, "ilu": {"precond": oracle_mod.PREC_ILU}}.get(variant, {})
    solvers = _open(P, systems, precision=P.MIXED, **kw)
    try:
        st, xb, ib = _batch(P, solvers, systems)
        assert st == 0
        for s, x, info in zip(systems, xb, ib):
            o = oracle_mod.Oracle.from_system(s, **okw).setup()
            _, io = o.solve(s.rhs)
            assert info["status"] == 0
            assert abs(info["iters"] - io["iters"]) <= max(1, 0.1 * io["iters"])
            rel = np.linalg.norm(s.rhs - o.spmv(x)) / np.linalg.norm(s.rhs)
            assert rel <= 1e-6
            assert abs(info["rel_resid"] - rel) <= 1e-9
    finally:
        for g in solvers:
            g.close()


def test_batch_device_buffers_and_initial_guess(P):
    import torch
    systems = _systems()[:2]
    solvers = _open(P, systems)
    try:
        rhs = [torch.from_numpy(s.rhs).cuda() for s in systems]
        xs = [torch.zeros(4 * s.n_cells, dtype=torch.float64, device="cuda") for s in systems]
        st, infos = P.cptr_solve_batch([g.h for g in solvers], rhs, xs)
        assert st == 0
        # restarting from the solution converges at once
        st, again = P.cptr_solve_batch([g.h for g in solvers], rhs, xs)
        assert st == 0 and all(i["iters"] == 0 for i in again)
        # a tighter tolerance through the call's own argument, and maxit
        xs2 = [torch.zeros_like(x) for x in xs]
        st, capped = P.cptr_solve_batch([g.h for g in solvers], rhs, xs2, tol=1e-12, maxit=2)
        assert st == P.ERR_MAXIT and all(i["iters"] == 2 for i in capped)
    finally:
        for g in solvers:
            g.close()


def test_batch_refuses_what_it_does_not_run(P):
    s = _systems()[0]
    s_vc = _systems()[4]  # MGR's first reduction needs the local volume constraint
    good = P.Solver.from_system(s).setup()
    cases = {
        "mgr": dict(mgr=1),
        "hybrid": dict(smoother=P.SMOOTH_HYBRID_GS),
        "restart": dict(restart=40),
        "cptr3": dict(precond=P.PREC_CPTR3),
    }
    try:
        for name, kw in cases.items():
            sk = s_vc if name == "mgr" else s
            with P.Solver.from_system(sk, **kw).setup() as g:
                with pytest.raises(P.CPTRError) as e:
                    _batch(P, [good, g], [s, sk])
                assert e.value.status == P.ERR_INVALID, name
        with P.Solver.from_system(s, precision=P.MIXED).setup() as g:
            with pytest.raises(P.CPTRError):
                _batch(P, [good, g], [s, s])
        with P.Solver.from_system(s) as g:  # not set up
            with pytest.raises(P.CPTRError):
                _batch(P, [good, g], [s, s])
        with pytest.raises(P.CPTRError):
            _batch(P, [good, good], [s, s])
        # the context still solves, alone and batched
        st, x, info = _batch(P, [good], [s])
        assert st == 0 and info[0]["status"] == 0
    finally:
        good.close()
