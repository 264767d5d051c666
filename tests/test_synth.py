"""Seeded generators: determinism and structure (CPU)."""
import numpy as np
import pytest

from synth import cartesian, config_system, knn, random_bsr, serving_mix


def _check_bsr(s):
    n = s.n_cells
    assert s.rowptr.dtype == np.int32 and s.col.dtype == np.int32
    assert s.rowptr[0] == 0 and s.rowptr[-1] == s.nnzb
    assert s.vals.shape == (s.nnzb, 16) and s.rhs.shape == (4 * n,)
    for i in range(n):
        c = s.col[s.rowptr[i]:s.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c
        assert c.min() >= 0 and c.max() < n


def test_cartesian_shape_and_determinism():
    a = config_system("c1")
    b = config_system("c1")
    _check_bsr(a)
    assert a.n_cells == 500
    nx, ny, nz = 10, 10, 5
    faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    assert a.nnzb == 500 + 2 * faces == 3100
    assert np.array_equal(a.vals, b.vals) and np.array_equal(a.rhs, b.rhs)
    c = cartesian(10, 10, 5, seed=1002)
    assert not np.array_equal(a.vals, c.vals)


def test_peclet_scales_conduction_only():
    lo = cartesian(6, 5, 4, pe=0.01, seed=3)
    hi = cartesian(6, 5, 4, pe=100.0, seed=3)
    assert np.isclose(lo.meta["kappa"] / hi.meta["kappa"], 1e4)
    d = (lo.vals - hi.vals).reshape(-1, 4, 4)
    d[:, 3, 3] = 0.0
    assert np.abs(d).max() == 0.0


def test_knn_structure():
    s = knn(8, 8, 4, pe=10.0, seed=3)
    _check_bsr(s)
    # symmetric block pattern
    pat = set()
    for i in range(s.n_cells):
        for t in range(s.rowptr[i], s.rowptr[i + 1]):
            pat.add((i, int(s.col[t])))
    assert all((j, i) in pat for (i, j) in pat)
    deg = np.diff(s.rowptr) - 1
    assert deg.min() >= 6


def test_random_bsr_and_single_cell():
    _check_bsr(random_bsr(25, seed=1))
    one = cartesian(1, 1, 1, seed=1)
    _check_bsr(one)
    assert one.nnzb == 1


def test_serving_mix_deterministic():
    a = serving_mix(16)
    b = serving_mix(16)
    assert a == b
    assert all(8000 / 4 <= r["dims"][0] ** 2 * r["dims"][2] * 4 for r in a)


@pytest.mark.parametrize("name", ["negated_mixed", "threshold_chain", "sign_flipped_2d"])
def test_pressure_embedding_is_exact(oracle_mod, name):
    """The CPR pressure system of the embedding is the scalar matrix bit for bit
    (zero decoupling weights), and each case has the feature it is named for."""
    from amg_cases import CASES
    from synth import pressure_embedding
    rp, ci, v = CASES[name]()
    s = pressure_embedding(rp, ci, v, seed=3)
    _check_bsr(s)
    o = oracle_mod.Oracle.from_system(s, e0=0, e1=-1).setup()
    np.testing.assert_array_equal(o.W(), 0.0)
    for got, want in zip(o.ahat(), (rp, ci, v)):
        np.testing.assert_array_equal(got, want)
    row = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    diag, off = v[ci == row], v[ci != row]
    if name == "negated_mixed":
        assert (diag < 0).all() and (off < 0).any()
    elif name == "threshold_chain":
        assert (off == -0.25).sum() > 0 and (off == -1.0).sum() > 0
    else:
        assert (diag > 0).all() and (off > 0).mean() > 0.2
