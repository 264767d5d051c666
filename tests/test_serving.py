"""Serving: continuous batching of independent solves (cptr_server_*).

The GPU test submits a mix of systems of different sizes, kinds and Peclet
numbers to a server with several slots, so that their kernels overlap on the
device, and checks that every result is the same as the same system solved
alone.  Every reduction in the library has a fixed order and every
triangular-solve path evaluates each row's sum in the same order, so "the
same" is bit-for-bit (tolerance 0).
"""
import ctypes
import time

import numpy as np
import pytest

from synth.jacobian import build_request, serving_mix


def _lib():
    from paper_2308_11892_gb300 import build
    build.build()
    import paper_2308_11892_gb300 as P
    return P


def test_server_argument_checks():
    """Host-side validation (no device work)."""
    P = _lib()
    lib = P._lib.load()
    h = ctypes.c_void_p()
    assert lib.cptr_server_create(ctypes.byref(h), 1 << 30, 0, None) == P._lib.ERR_INVALID
    assert lib.cptr_server_create(ctypes.byref(h), 0, 2, None) == P._lib.ERR_INVALID
    assert lib.cptr_server_create(None, 1 << 30, 2, None) == P._lib.ERR_INVALID
    rid = ctypes.c_uint64()
    assert lib.cptr_submit(None, 10, None, None, None, None, 0.0, 0, ctypes.byref(rid)) == \
        P._lib.ERR_INVALID
    assert lib.cptr_poll(None, 1, None, None) == P._lib.ERR_INVALID
    lib.cptr_server_destroy(None)


def _bsr_mv(s, x):
    rows = np.repeat(np.arange(s.n_cells), np.diff(s.rowptr))
    prod = np.einsum("bij,bj->bi", s.vals.reshape(-1, 4, 4), x.reshape(-1, 4)[s.col])
    y = np.zeros((s.n_cells, 4))
    np.add.at(y, rows, prod)
    return y.ravel()


def _mix():
    reqs = serving_mix(n_requests=6, seed=1005, min_cells=1500, max_cells=12000)
    return [(r, build_request(r)) for r in reqs]


def _wait(P, srv, ids, systems, timeout=300.0):
    out = {}
    t0 = time.time()
    while len(out) < len(ids):
        for rid, s in zip(ids, systems):
            if rid in out:
                continue
            x = np.zeros(4 * s.n_cells)
            st, info = P.cptr_poll(srv, rid, x)
            if st != P._lib.PENDING:
                out[rid] = (st, x, info)
        assert time.time() - t0 < timeout, "serving requests did not finish"
        time.sleep(0.002)
    return [out[r] for r in ids]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_results_identical_alone_and_in_the_mix(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = _lib()
    prec = P.FP64 if precision == "fp64" else P.MIXED
    mix = _mix()
    systems = [s for _, s in mix]
    # all requests in flight together on three slots
    srv = P.cptr_server_create(8 << 30, 3, P.params(precision=prec))
    try:
        ids = [P.cptr_submit(srv, s.n_cells, s.rowptr, s.col, s.vals, s.rhs) for s in systems]
        together = _wait(P, srv, ids, systems)
    finally:
        P.cptr_server_destroy(srv)
    # each request alone: one slot, submitted only after the previous one finished
    srv = P.cptr_server_create(8 << 30, 1, P.params(precision=prec))
    try:
        alone = []
        for s in systems:
            rid = P.cptr_submit(srv, s.n_cells, s.rowptr, s.col, s.vals, s.rhs)
            alone += _wait(P, srv, [rid], [s])
    finally:
        P.cptr_server_destroy(srv)
    for (req, s), (st_m, x_m, i_m), (st_a, x_a, i_a) in zip(mix, together, alone):
        assert st_m == P._lib.OK and st_a == P._lib.OK, (req, st_m, st_a)
        assert i_m["iters"] == i_a["iters"]
        np.testing.assert_array_equal(x_m, x_a)
        rel = np.linalg.norm(s.rhs - _bsr_mv(s, x_m)) / np.linalg.norm(s.rhs)
        assert rel <= 1e-6
    # and the same as a direct solve through cptr_solve
    req, s = mix[0]
    with P.Solver.from_system(s, precision=prec).setup() as g:
        x, info = g.solve(s.rhs, np.zeros(4 * s.n_cells))
    np.testing.assert_array_equal(x, together[0][1])


def test_server_limits_argument_checks():
    P = _lib()
    lib = P._lib.load()
    assert lib.cptr_server_set_limits(None, 16, 0) == P._lib.ERR_INVALID


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_small_requests_identical_alone_and_in_the_mix(precision):
    """Requests of at most 6000 cells go through the batched launch, larger
    ones through their slot's own solve: each result is bit-identical alone
    and in the mix, and equal to cptr_solve_batch (small) or cptr_solve
    (large) on the system by itself."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = _lib()
    prec = P.FP64 if precision == "fp64" else P.MIXED
    mix = _mix()
    systems = [s for _, s in mix]
    limit = 6000
    assert any(s.n_cells <= limit for s in systems) and any(s.n_cells > limit for s in systems)
    srv = P.cptr_server_create(8 << 30, 3, P.params(precision=prec))
    try:
        P.cptr_server_set_limits(srv, 4096, limit)
        ids = [P.cptr_submit(srv, s.n_cells, s.rowptr, s.col, s.vals, s.rhs) for s in systems]
        together = _wait(P, srv, ids, systems)
    finally:
        P.cptr_server_destroy(srv)
    srv = P.cptr_server_create(8 << 30, 1, P.params(precision=prec))
    try:
        P.cptr_server_set_limits(srv, 4096, limit)
        alone = []
        for s in systems:
            rid = P.cptr_submit(srv, s.n_cells, s.rowptr, s.col, s.vals, s.rhs)
            alone += _wait(P, srv, [rid], [s])
    finally:
        P.cptr_server_destroy(srv)
    for s, (st_m, x_m, i_m), (st_a, x_a, i_a) in zip(systems, together, alone):
        assert st_m == P._lib.OK and st_a == P._lib.OK
        assert i_m["iters"] == i_a["iters"]
        np.testing.assert_array_equal(x_m, x_a)
        assert np.linalg.norm(s.rhs - _bsr_mv(s, x_m)) / np.linalg.norm(s.rhs) <= 1e-6
        with P.Solver.from_system(s, precision=prec, tri_tune=0).setup() as g:
            if s.n_cells <= limit:
                x = np.zeros(4 * s.n_cells)
                P.cptr_solve_batch([g.h], [s.rhs], [x])
            else:
                x, _ = g.solve(s.rhs, np.zeros(4 * s.n_cells))
        np.testing.assert_array_equal(x, x_m)


@pytest.mark.gpu
def test_full_queue_answers_again():
    """A one-byte budget admits one request at a time; with two requests
    already waiting, the next submission is refused with CPTR_ERR_AGAIN and
    accepted again once the queue has drained."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = _lib()
    big = build_request(serving_mix(n_requests=1, seed=7, min_cells=60000, max_cells=60001)[0])
    s = _mix()[0][1]
    srv = P.cptr_server_create(1, 1, P.params())
    try:
        P.cptr_server_set_limits(srv, 2, 0)
        ids = [P.cptr_submit(srv, big.n_cells, big.rowptr, big.col, big.vals, big.rhs)]
        time.sleep(0.005)  # admitted: the queue is empty again
        ids += [P.cptr_submit(srv, s.n_cells, s.rowptr, s.col, s.vals, s.rhs) for _ in range(2)]
        with pytest.raises(P.CPTRError) as e:
            P.cptr_submit(srv, s.n_cells, s.rowptr, s.col, s.vals, s.rhs)
        assert e.value.status == P._lib.ERR_AGAIN
        done = _wait(P, srv, ids, [big, s, s])
        assert all(st == P._lib.OK for st, _, _ in done)
        rid = P.cptr_submit(srv, s.n_cells, s.rowptr, s.col, s.vals, s.rhs)
        assert _wait(P, srv, [rid], [s])[0][0] == P._lib.OK
    finally:
        P.cptr_server_destroy(srv)


@pytest.mark.gpu
def test_limits_refuse_batching_for_params_it_does_not_run():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = _lib()
    srv = P.cptr_server_create(8 << 30, 1, P.params(smoother=P.SMOOTH_HYBRID_GS))
    try:
        with pytest.raises(P.CPTRError):
            P.cptr_server_set_limits(srv, 16, 5000)
        P.cptr_server_set_limits(srv, 16, 0)
    finally:
        P.cptr_server_destroy(srv)
