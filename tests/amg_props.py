"""Properties of the CPTR setup that hold at any size, checked directly from
their definitions (no oracle code): unknown-based strength, PMIS C/F
splitting, ext+i interpolation support and truncation, Galerkin coarse
operators, ILU(0) level sets and the ILU(0) pattern identity (LU)_ij = A_ij.
Used to pin the oracle on generator matrices and to check the GPU setup at
sizes the oracle cannot finish quickly."""
import numpy as np
import scipy.sparse as sp


def strength(rp, ci, v, func, theta=0.25):
    """Strong couplings (i, j): j != i, func[j] == func[i] and
    -s a_ij >= theta max_k(-s a_ik) over same-function off-diagonal k, with
    s = sign(a_ii); a row whose maximum is <= 0 has none."""
    n = rp.size - 1
    row = np.repeat(np.arange(n), np.diff(rp))
    diag = np.zeros(n)
    isd = ci == row
    diag[row[isd]] = v[isd]
    s = np.where(diag < 0, -1.0, 1.0)
    same = (func[ci] == func[row]) & ~isd
    m = np.where(same, -s[row] * v, -np.inf)
    mx = np.full(n, -np.inf)
    nonempty = np.diff(rp) > 0
    if m.size:
        mx[nonempty] = np.maximum.reduceat(m, rp[:-1][nonempty])
    strong = same & (mx[row] > 0) & (-s[row] * v >= theta * mx[row])
    return row[strong], ci[strong]


def check_pmis(cf, si, sj):
    """Every point decided; a C point influences at least one point (lambda >= 1);
    an F point influences nobody or depends strongly on a C point."""
    n = cf.size
    assert np.isin(cf, (-1, 1)).all()
    isC = cf == 1
    infl = np.bincount(sj, minlength=n)
    hasC = np.zeros(n, bool)
    hasC[si[isC[sj]]] = True
    ok = (isC & (infl >= 1)) | (~isC & ((infl == 0) | hasC))
    assert ok.all(), np.nonzero(~ok)[0][:10]
    return isC


def check_interp(isC, si, sj, prp, pci, pv, pmax, rng, samples=2000):
    """C rows of P are unit rows at the point's coarse index; F rows hold at most
    pmax entries whose columns are C points within distance two in the strength
    graph (strong C neighbours, or strong C neighbours of strong F neighbours)."""
    n = isC.size
    cidx = np.cumsum(isC) - 1
    plen = np.diff(prp)
    assert (plen[isC] == 1).all()
    np.testing.assert_array_equal(pci[prp[:-1][isC]], cidx[isC])
    np.testing.assert_array_equal(pv[prp[:-1][isC]], 1.0)
    assert (plen[~isC] <= pmax).all()
    S = sp.csr_matrix((np.ones(si.size), (si, sj)), shape=(n, n))
    fr = np.nonzero(~isC)[0]
    cpts = np.nonzero(isC)[0]
    for i in rng.choice(fr, size=min(samples, fr.size), replace=False):
        si_i = S.indices[S.indptr[i]:S.indptr[i + 1]]
        reach = set(si_i.tolist())
        for k in si_i[~isC[si_i]]:
            reach.update(S.indices[S.indptr[k]:S.indptr[k + 1]].tolist())
        cols = cpts[pci[prp[i]:prp[i + 1]]]
        assert set(cols.tolist()) <= reach, i


def check_galerkin(A, Pm, Ac, rng, samples=500, tol=1e-12):
    """Ac = P^T A P on sampled coarse rows, relative to |P|^T |A| |P|."""
    nc = Pm.shape[1]
    rows = rng.choice(nc, size=min(samples, nc), replace=False)
    Rs = Pm.T.tocsr()[rows]
    ref = (Rs @ A @ Pm).tocsr()
    got = Ac.tocsr()[rows]
    scale = (abs(Rs) @ abs(A) @ abs(Pm)).max(axis=1).toarray().ravel()
    diff = (got - ref).tocoo()
    assert (np.abs(diff.data) <= tol * scale[diff.row] + 1e-300).all()


def check_ilu_levels(rowptr, col, lev):
    """level(i) = 1 + max level of the lower neighbours of row i (0 if none)."""
    row = np.repeat(np.arange(rowptr.size - 1), np.diff(rowptr))
    lower = np.where(col < row, lev[col], -1)
    lmax = np.maximum.reduceat(lower, rowptr[:-1])  # every row holds its diagonal
    np.testing.assert_array_equal(lev, lmax + 1)


def check_ilu_rows(rowptr, col, vals, F, rows, tol=1e-11):
    """(LU)_ij = A_ij on the block pattern of the sampled rows.  F holds the unit
    lower blocks L_ij (j < i), the upper blocks U_ij (j > i) and inv(U_ii)."""
    def blocks(i):
        return {int(col[t]): t for t in range(rowptr[i], rowptr[i + 1])}

    for i in rows:
        bi = blocks(i)
        scale = np.abs(vals[rowptr[i]:rowptr[i + 1]]).max()
        for j, t in bi.items():
            acc = np.zeros((4, 4))
            for k, tk in bi.items():
                if k >= i or k > j:
                    continue
                bk = blocks(k)
                if j in bk:
                    acc += F[tk] @ (np.linalg.inv(F[bk[j]]) if k == j else F[bk[j]])
            if i <= j:
                acc += np.linalg.inv(F[t]) if i == j else F[t]
            assert np.abs(acc - vals[t]).max() <= tol * scale, (i, j)
