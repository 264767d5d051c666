"""Scalar operators with features that the synthetic Jacobians rarely contain,
for the AMG setup: negative diagonals, positive off-diagonal couplings, and
couplings exactly at the strength threshold.  Each is embedded as the pressure
system of a 4x4-block system (synth.pressure_embedding), so the CUDA setup
builds its hierarchy on it through the CPR first stage.  `pivoting_chain`
is a dense block-tridiagonal matrix whose diagonal blocks need row exchanges
to be inverted (for the block ILU(0) checks); `happy_breakdown_case` a
block-diagonal system whose right-hand side spans a 3-dimensional Krylov
space (for GMRES's exact breakdown)."""
import numpy as np
import scipy.sparse as sp

from synth import poisson1d_csr, poisson3d_csr


def _csr(M):
    M = sp.csr_matrix(M)
    M.sort_indices()
    return M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64)


def negated_mixed(m=16, seed=0):
    """-(7-point Laplacian + a nonsymmetric perturbation of its couplings): every
    diagonal is negative and about a fifth of the couplings have the diagonal's
    sign."""
    rng = np.random.default_rng(seed)
    rp, ci, v = poisson3d_csr(m)
    v = v.copy()
    off = ci != np.repeat(np.arange(rp.size - 1), np.diff(rp))
    v[off] *= rng.uniform(0.5, 1.5, off.sum())
    flip = off & (rng.random(v.size) < 0.2)
    v[flip] = -0.3 * v[flip]
    return rp, ci, -v


def threshold_chain(n=5000):
    """Chain with couplings -1 at distance 1 and exactly -1/4 = -theta at
    distance 2 (strong only under an inclusive threshold), diagonal 3."""
    rows, cols, vals = [], [], []
    for d, a in ((0, 3.0), (1, -1.0), (2, -0.25)):
        i = np.arange(n - d)
        rows += [i, i + d] if d else [i]
        cols += [i + d, i] if d else [i]
        vals += [np.full(i.size, a)] * (2 if d else 1)
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return _csr(M)


def sign_flipped_2d(m=80, seed=1):
    """5-point Laplacian on an m x m grid with a quarter of the couplings made
    positive (+0.2 to +0.6) and the diagonal raised by their size."""
    rng = np.random.default_rng(seed)
    n = m * m
    idx = np.arange(n).reshape(m, m)
    rows, cols = [np.arange(n)], [np.arange(n)]
    for a, b in ((idx[:, :-1], idx[:, 1:]), (idx[:-1, :], idx[1:, :])):
        rows += [a.ravel(), b.ravel()]
        cols += [b.ravel(), a.ravel()]
    rows = np.concatenate(rows); cols = np.concatenate(cols)
    vals = np.where(rows == cols, 4.0, -1.0)
    off = rows != cols
    pos = off & (rng.random(rows.size) < 0.25)
    vals[pos] = rng.uniform(0.2, 0.6, pos.sum())
    extra = np.bincount(rows[pos], weights=vals[pos], minlength=n)
    vals[~off] += extra[rows[~off]]
    M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return _csr(M)


def pivoting_chain(n, seed=3):
    """Block-tridiagonal chain whose diagonal blocks have zero (0,0) and (1,1)
    entries (nonsingular: the first two unknowns are coupled crosswise), so
    inverting them needs row exchanges."""
    rng = np.random.default_rng(seed)
    A = np.zeros((4 * n, 4 * n))
    for i in range(n):
        D = np.array([[0.0, 5.0, 0.1, 0.2], [5.0, 0.0, 0.3, 0.1],
                      [0.1, 0.2, 5.0, 0.0], [0.2, 0.1, 0.0, 5.0]])
        D += np.diag([0.0, 0.0, 1.0, 1.0]) * rng.uniform(0, 1, 4)
        A[4 * i:4 * i + 4, 4 * i:4 * i + 4] = D
        for j in (i - 1, i + 1):
            if 0 <= j < n:
                A[4 * i:4 * i + 4, 4 * j:4 * j + 4] = rng.uniform(-0.2, 0.2, (4, 4))
    return A


def happy_breakdown_case():
    """Block-diagonal A with diagonal blocks c_k I (c_k in {2, 3, 5}) and a
    right-hand side on 12 cells: the Krylov space of b has dimension 3."""
    n = 12
    diag = np.repeat(np.array([2.0, 3.0, 5.0] * 4), 4)
    A = np.diag(diag)
    b = np.random.default_rng(4).normal(size=4 * n)
    return A, b


CASES = {"negated_mixed": negated_mixed, "threshold_chain": threshold_chain,
         "sign_flipped_2d": sign_flipped_2d}
