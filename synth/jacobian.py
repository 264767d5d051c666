"""Synthetic thermal-compositional Jacobians with 4 unknowns per cell.

The paper (Section 2, Eqs. 1-2) solves two-component, two-phase mass balances
plus an energy balance with four primary unknowns per cell, stored interleaved
(Section 3.1: "interleaved variables").  The default systems here have four
balance-like rows and no volume-constraint row, so CPTR works on all four
unknowns; ``with_volume_constraint`` builds the form with a cell-local
constraint row that the first MGR reduction of Section 3.4 eliminates.  The paper's reservoir
models (Section 4, Table 1) are not available, so these generators build
seeded stand-ins with the same block structure and the same qualitative
operators:

* unknown order inside a 4x4 block: (p, rho_CO2, rho_H2O, T) = 0..3;
* pressure column: TPFA Darcy fluxes with log-normal permeability, weighted
  per equation row by an upwind "mobility" vector;
* rows 1..3 (rho_CO2, rho_H2O, T): first-order upwind convection on the
  row's own unknown, driven by a seeded potential field;
* energy row, T column: thermal conduction on the same stencil, scaled so the
  face-averaged ratio of advective to conductive strength equals the thermal
  Peclet number of Eq. 4;
* a small random diagonally dominant accumulation block per cell, one
  injector-like well cell and a Gaussian right-hand side.

All randomness comes from ``numpy.random.default_rng(seed)`` in a fixed draw
order, so the same call returns bit-identical arrays on every machine.

Output format (block CSR, 4x4 blocks, row-major inside a block):
``rowptr`` int32[N+1], ``col`` int32[nnzb] (sorted per row, diagonal
present), ``vals`` float64[nnzb, 16], ``rhs`` float64[4N].
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Tuple

import numpy as np

BS = 4  # unknowns per cell


@dataclasses.dataclass
class BSRSystem:
    n_cells: int
    rowptr: np.ndarray      # int32 [N+1]
    col: np.ndarray         # int32 [nnzb]
    vals: np.ndarray        # float64 [nnzb, 16]
    rhs: np.ndarray         # float64 [4N]
    meta: Dict

    @property
    def nnzb(self) -> int:
        return int(self.col.shape[0])

    @property
    def n_dof(self) -> int:
        return BS * self.n_cells

    def to_dense(self) -> np.ndarray:
        """Dense (4N x 4N) copy, for tiny systems in tests only."""
        n = self.n_cells
        A = np.zeros((BS * n, BS * n))
        for i in range(n):
            for t in range(self.rowptr[i], self.rowptr[i + 1]):
                j = self.col[t]
                A[BS * i:BS * i + BS, BS * j:BS * j + BS] = self.vals[t].reshape(BS, BS)
        return A


# --------------------------------------------------------------------------
# geometry helpers
# --------------------------------------------------------------------------
def _cartesian_faces(nx: int, ny: int, nz: int):
    """Faces (i<j) of a lexicographic nx*ny*nz grid (x fastest) and their axis."""
    idx = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    fi, fj, ax = [], [], []
    if nx > 1:
        fi.append(idx[:, :, :-1].ravel()); fj.append(idx[:, :, 1:].ravel())
        ax.append(np.zeros(fi[-1].size, np.int8))
    if ny > 1:
        fi.append(idx[:, :-1, :].ravel()); fj.append(idx[:, 1:, :].ravel())
        ax.append(np.ones(fi[-1].size, np.int8))
    if nz > 1:
        fi.append(idx[:-1, :, :].ravel()); fj.append(idx[1:, :, :].ravel())
        ax.append(np.full(fi[-1].size, 2, np.int8))
    if not fi:
        return (np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.int8))
    return np.concatenate(fi), np.concatenate(fj), np.concatenate(ax)


def _morton3(ix: np.ndarray, iy: np.ndarray, iz: np.ndarray) -> np.ndarray:
    def spread(v):
        v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
        v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
        v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
        v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
        v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
        return v
    return spread(ix) | (spread(iy) << np.uint64(1)) | (spread(iz) << np.uint64(2))


# --------------------------------------------------------------------------
# block assembly shared by both geometries
# --------------------------------------------------------------------------
def _assemble(n: int, fi: np.ndarray, fj: np.ndarray, T: np.ndarray, G: np.ndarray,
              phi: np.ndarray, lam: np.ndarray, pe: float, acc_d: np.ndarray,
              acc_o: np.ndarray, inj: int, rhs: np.ndarray, meta: Dict) -> BSRSystem:
    nf = fi.shape[0]
    F = T * (phi[fi] - phi[fj])                 # flux i->j, antisymmetric by construction
    up = np.where(F > 0, fi, fj)
    aF = np.abs(F)
    lam_f = lam[up] * T[:, None]               # (nf, 4): Darcy weight per equation row
    if nf > 0 and np.mean(G) > 0:
        kappa = float(np.mean(aF)) / (pe * float(np.mean(G)))
    else:
        kappa = 0.0
    cond = kappa * G

    Bij = np.zeros((nf, 4, 4))   # block (row fi, col fj)
    Bji = np.zeros((nf, 4, 4))   # block (row fj, col fi)
    Bij[:, :, 0] = -lam_f
    Bji[:, :, 0] = -lam_f
    i_up = up == fi
    for r in (1, 2, 3):
        # outflow from the upwind cell u, inflow into the downwind cell d: A_du[r,r] -= |F|
        Bji[i_up, r, r] -= aF[i_up]
        Bij[~i_up, r, r] -= aF[~i_up]
    Bij[:, 3, 3] -= cond
    Bji[:, 3, 3] -= cond

    D = np.zeros((n, 16))
    for r in range(4):
        D[:, 4 * r] += np.bincount(fi, weights=lam_f[:, r], minlength=n)
        D[:, 4 * r] += np.bincount(fj, weights=lam_f[:, r], minlength=n)
    for r in (1, 2, 3):
        D[:, 5 * r] += np.bincount(up, weights=aF, minlength=n)
    D[:, 15] += np.bincount(fi, weights=cond, minlength=n)
    D[:, 15] += np.bincount(fj, weights=cond, minlength=n)

    sumT = np.bincount(fi, weights=T, minlength=n) + np.bincount(fj, weights=T, minlength=n)
    msum = float(np.mean(sumT)) if n > 0 else 0.0
    alpha = 1e-2 * msum if msum > 0 else 1.0
    acc = 0.1 * acc_o
    acc[:, [0, 5, 10, 15]] += 1.0 + acc_d
    D += alpha * acc
    WI = 10.0 * float(np.max(sumT)) if nf > 0 else 0.0
    D[inj, 0] += WI
    D[inj, 15] += WI

    rows = np.concatenate([np.arange(n, dtype=np.int64), fi, fj])
    cols = np.concatenate([np.arange(n, dtype=np.int64), fj, fi])
    key = rows * n + cols
    perm = np.argsort(key, kind="stable")
    vals = np.concatenate([D, Bij.reshape(nf, 16), Bji.reshape(nf, 16)])[perm]
    col = cols[perm].astype(np.int32)
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnzb exceeds int32 indexing")
    meta = dict(meta)
    meta.update(kappa=kappa, alpha=alpha, WI=WI, injector=int(inj), n_faces=int(nf))
    return BSRSystem(n, rowptr.astype(np.int32), col, np.ascontiguousarray(vals), rhs, meta)


def cartesian(nx: int, ny: int, nz: int, pe: float = 1.0, seed: int = 1001,
              sigma: float = 1.0, layered: bool = False, kv_ratio: float = 1.0,
              cold_dT: float = 0.0) -> BSRSystem:
    """Cartesian nx*ny*nz grid, cells in lexicographic order (x fastest).

    ``layered``: ln k = a(z) + b(cell) with var(a)=0.75 sigma^2, var(b)=0.25 sigma^2.
    ``kv_ratio``: vertical faces use k*kv_ratio (0.1 = 10x vertical anisotropy).
    ``cold_dT``: temperature contrast (K) of a cold plume around the well column,
    Gaussian with a radius of 5 cells; it scales the mobilities by exp(0.02 dT).
    """
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    if layered:
        a = rng.normal(0.0, math.sqrt(0.75) * sigma, nz)
        b = rng.normal(0.0, math.sqrt(0.25) * sigma, n)
        lnk = np.repeat(a, nx * ny) + b
    else:
        lnk = rng.normal(0.0, sigma, n)
    noise = rng.normal(0.0, 0.01, n)
    u = rng.uniform(0.5, 1.5, (n, 3))
    acc_d = rng.uniform(0.0, 1.0, (n, 4))
    acc_o = rng.uniform(-1.0, 1.0, (n, 16))
    rhs = rng.normal(0.0, 1.0, 4 * n)

    k = np.exp(lnk)
    fi, fj, ax = _cartesian_faces(nx, ny, nz)
    ki, kj = k[fi], k[fj]
    vert = ax == 2
    ki = np.where(vert, ki * kv_ratio, ki)
    kj = np.where(vert, kj * kv_ratio, kj)
    G = np.ones(fi.shape[0])
    T = G * 2.0 * ki * kj / (ki + kj)

    zc, yc, xc = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                             indexing="ij")
    xc, yc, zc = xc.ravel(), yc.ravel(), zc.ravel()
    phi = xc + 0.3 * np.sin(2 * np.pi * yc / ny) * np.cos(2 * np.pi * zc / nz) + noise

    lam = np.stack([np.ones(n), 0.5 * u[:, 0], 0.5 * u[:, 1], 0.2 * u[:, 2]], axis=1)
    cx, cy = nx // 2, ny // 2
    if cold_dT != 0.0:
        r2 = (xc - (cx + 0.5)) ** 2 + (yc - (cy + 0.5)) ** 2
        dT = -abs(cold_dT) * np.exp(-r2 / 25.0)
        lam = lam * np.exp(0.02 * dT)[:, None]
    inj = cx + nx * cy  # centre column, bottom layer (z = 0)
    rhs[4 * inj + 0] += 100.0
    rhs[4 * inj + 3] -= 100.0
    meta = dict(kind="cartesian", dims=(nx, ny, nz), pe=pe, seed=seed, sigma=sigma,
                layered=layered, kv_ratio=kv_ratio, cold_dT=cold_dT)
    return _assemble(n, fi, fj, T, G, phi, lam, pe, acc_d, acc_o, inj, rhs, meta)


def knn(gx: int, gy: int, gz: int, box=(10.0, 10.0, 2.0), pe: float = 10.0,
        seed: int = 1003, sigma: float = 1.0, kmin: int = 6, kmax: int = 12) -> BSRSystem:
    """Unstructured cloud: a gx*gy*gz lattice over ``box`` jittered by U(-1/4,1/4) of
    the spacing, Morton-sorted, connected to k_i ~ U{kmin..kmax} nearest
    neighbours (symmetrised by union); geometric factor 1/distance."""
    from scipy.spatial import cKDTree

    n = gx * gy * gz
    rng = np.random.default_rng(seed)
    h = np.array([box[0] / gx, box[1] / gy, box[2] / gz])
    jit = rng.uniform(-0.25, 0.25, (n, 3))
    kk = rng.integers(kmin, kmax + 1, n)
    lnk = rng.normal(0.0, sigma, n)
    noise = rng.normal(0.0, 0.01, n)
    u = rng.uniform(0.5, 1.5, (n, 3))
    acc_d = rng.uniform(0.0, 1.0, (n, 4))
    acc_o = rng.uniform(-1.0, 1.0, (n, 16))
    rhs = rng.normal(0.0, 1.0, 4 * n)

    iz, iy, ix = np.meshgrid(np.arange(gz), np.arange(gy), np.arange(gx), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    pos = (np.stack([ix, iy, iz], axis=1) + 0.5 + jit) * h
    order = np.argsort(_morton3(ix, iy, iz), kind="stable")
    pos = pos[order]
    # per-point draws follow the point to its Morton slot
    kk, lnk, noise, u = kk[order], lnk[order], noise[order], u[order]
    acc_d, acc_o = acc_d[order], acc_o[order]

    kq = min(kmax + 1, n)
    tree = cKDTree(pos)
    dist, nbr = tree.query(pos, k=kq)
    if kq == 1:
        nbr = nbr[:, None]
    src = np.repeat(np.arange(n), kq - 1)
    dst = nbr[:, 1:].ravel()
    keep = (np.tile(np.arange(1, kq), n) <= np.repeat(kk, kq - 1)) & (dst != src) & (dst < n)
    src, dst = src[keep], dst[keep]
    a, b = np.minimum(src, dst), np.maximum(src, dst)
    e = np.unique(a.astype(np.int64) * n + b)
    fi, fj = e // n, e % n
    d = np.linalg.norm(pos[fi] - pos[fj], axis=1)
    G = 1.0 / d
    k = np.exp(lnk)
    T = G * 2.0 * k[fi] * k[fj] / (k[fi] + k[fj])
    phi = (pos[:, 0] + 0.3 * np.sin(2 * np.pi * pos[:, 1] / box[1])
           * np.cos(2 * np.pi * pos[:, 2] / box[2]) + noise)
    lam = np.stack([np.ones(n), 0.5 * u[:, 0], 0.5 * u[:, 1], 0.2 * u[:, 2]], axis=1)
    inj = int(np.argmin(np.linalg.norm(pos - np.array([box[0] / 2, box[1] / 2, 0.0]), axis=1)))
    rhs = rhs.reshape(n, 4)[order].ravel()
    rhs[4 * inj + 0] += 100.0
    rhs[4 * inj + 3] -= 100.0
    meta = dict(kind="knn", dims=(gx, gy, gz), pe=pe, seed=seed, sigma=sigma)
    return _assemble(n, fi, fj, T, G, phi, lam, pe, acc_d, acc_o, inj, rhs, meta)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
CONFIG_NAMES = ("c1", "c2", "c3", "c4")


def config_system(name: str, pe: Optional[float] = None) -> BSRSystem:
    """The four fixed workloads: c1 10x10x5 (Pe 1), c2 64x64x32 (Pe sweep
    {0.01,1,100}, default 1), c3 1M-point kNN (Pe 10), c4 200x200x100 layered
    sigma=2, 10x vertical anisotropy, 40 K cold plume (Pe 1)."""
    if name == "c1":
        return cartesian(10, 10, 5, pe=1.0 if pe is None else pe, seed=1001)
    if name == "c2":
        return cartesian(64, 64, 32, pe=1.0 if pe is None else pe, seed=1002)
    if name == "c3":
        return knn(200, 200, 25, pe=10.0 if pe is None else pe, seed=1003)
    if name == "c4":
        return cartesian(200, 200, 100, pe=1.0 if pe is None else pe, seed=1004, sigma=2.0,
                         layered=True, kv_ratio=0.1, cold_dT=40.0)
    raise KeyError(name)


def config_slab(name: str, nz: int) -> BSRSystem:
    """The generator of workload ``name`` (c2, c3 or c4) on a thinner domain:
    the same horizontal extent and parameters with ``nz`` layers instead of the
    full count (a bounded sample of the workload for slow solvers)."""
    if name == "c2":
        return cartesian(64, 64, nz, pe=1.0, seed=1002)
    if name == "c3":
        return knn(200, 200, nz, box=(10.0, 10.0, 2.0 * nz / 25.0), pe=10.0, seed=1003)
    if name == "c4":
        return cartesian(200, 200, nz, pe=1.0, seed=1004, sigma=2.0, layered=True,
                         kv_ratio=0.1, cold_dT=40.0)
    raise KeyError(name)


def serving_mix(n_requests: int = 512, seed: int = 1005, min_cells: int = 8000,
                max_cells: int = 500000, rate: float = 1.0) -> List[Dict]:
    """Request descriptors for the serving workload: Poisson arrivals (rate per
    second), log-uniform sizes, 50/50 Cartesian (nx = ny = 2 nz) / kNN, log-uniform
    Peclet in [0.01, 100].  Systems are built lazily by :func:`build_request`."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.exp(rng.uniform(math.log(min_cells), math.log(max_cells), n_requests))
    kinds = rng.integers(0, 2, n_requests)
    pes = np.exp(rng.uniform(math.log(0.01), math.log(100.0), n_requests))
    seeds = rng.integers(0, 2**31 - 1, n_requests)
    out = []
    for r in range(n_requests):
        nz = max(1, int(round((sizes[r] / 4.0) ** (1.0 / 3.0))))
        nxy = 2 * nz
        out.append(dict(id=r, t=float(arrivals[r]), kind="cartesian" if kinds[r] == 0 else "knn",
                        dims=(nxy, nxy, nz), pe=float(pes[r]), seed=int(seeds[r])))
    return out


def build_request(req: Dict) -> BSRSystem:
    gx, gy, gz = req["dims"]
    if req["kind"] == "cartesian":
        return cartesian(gx, gy, gz, pe=req["pe"], seed=req["seed"])
    return knn(gx, gy, gz, box=(float(gx) * 0.05, float(gy) * 0.05, float(gz) * 0.08),
               pe=req["pe"], seed=req["seed"])


# --------------------------------------------------------------------------
# generic test matrices (no physics)
# --------------------------------------------------------------------------
def random_bsr(n: int, avg_offdiag: float = 4.0, seed: int = 7, dominance: float = 2.0,
               empty_rows: float = 0.1, lower_only: bool = False) -> BSRSystem:
    """Random 4x4 BSR with an uneven row-length mix, some rows holding only the
    diagonal block, and block-diagonally dominant diagonal blocks."""
    rng = np.random.default_rng(seed)
    blocks = []
    for i in range(n):
        if rng.uniform() < empty_rows or n == 1:
            cnt = 0
        else:
            cnt = int(min(n - 1, rng.poisson(avg_offdiag)))
        cand = np.setdiff1d(np.arange(n), [i])
        if lower_only:
            cand = cand[cand < i]
            cnt = min(cnt, cand.size)
        cols = np.sort(rng.choice(cand, cnt, replace=False)) if cnt > 0 else np.zeros(0, int)
        blocks.append(cols)
    rows, cols = [], []
    for i in range(n):
        c = np.union1d(blocks[i], [i])
        rows.append(np.full(c.size, i)); cols.append(c)
    rows = np.concatenate(rows); cols = np.concatenate(cols)
    vals = rng.uniform(-1.0, 1.0, (rows.size, 16))
    rowsum = np.zeros(n)
    np.add.at(rowsum, rows, np.abs(vals).reshape(-1, 4, 4).sum(axis=2).max(axis=1))
    diag = rows == cols
    vals[diag] += (dominance * rowsum[rows[diag]])[:, None] * np.eye(4).ravel()[None, :]
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    rhs = rng.normal(0.0, 1.0, 4 * n)
    return BSRSystem(n, rowptr.astype(np.int32), cols.astype(np.int32),
                     np.ascontiguousarray(vals), rhs, dict(kind="random", seed=seed))


def block_tridiag_chain(n: int, seed: int = 11) -> BSRSystem:
    """1D chain of n cells with full random 4x4 couplings to both neighbours.

    Its block-lower and block-upper parts have no fill under elimination in
    natural order, so ILU(0) on it equals exact block LU."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                rows.append(i); cols.append(j)
    rows = np.array(rows); cols = np.array(cols)
    vals = rng.uniform(-1.0, 1.0, (rows.size, 16))
    diag = rows == cols
    vals[diag] += 6.0 * np.eye(4).ravel()[None, :]
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    rhs = rng.normal(0.0, 1.0, 4 * n)
    return BSRSystem(n, rowptr.astype(np.int32), cols.astype(np.int32),
                     np.ascontiguousarray(vals), rhs, dict(kind="chain", seed=seed))


def poisson1d_csr(n: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Tridiagonal [-1, 2, -1] of order n as scalar CSR (rowptr, col, val)."""
    rows, cols, vals = [], [], []
    for i in range(n):
        for j, v in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                rows.append(i); cols.append(j); vals.append(v)
    rowptr = np.zeros(n + 1, np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return rowptr, np.array(cols, np.int32), np.array(vals)


def poisson3d_csr(m: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """7-point Laplacian on an m^3 grid with Dirichlet boundaries, scalar CSR."""
    n = m ** 3
    idx = np.arange(n).reshape(m, m, m)
    rows = [np.arange(n)]; cols = [np.arange(n)]; vals = [np.full(n, 6.0)]
    for axis in range(3):
        a = np.take(idx, np.arange(m - 1), axis=axis).ravel()
        b = np.take(idx, np.arange(1, m), axis=axis).ravel()
        rows += [a, b]; cols += [b, a]; vals += [np.full(a.size, -1.0), np.full(a.size, -1.0)]
    rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
    perm = np.argsort(rows.astype(np.int64) * n + cols, kind="stable")
    rowptr = np.zeros(n + 1, np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return rowptr, cols[perm].astype(np.int32), vals[perm]


def pressure_embedding(rowptr: np.ndarray, col: np.ndarray, val: np.ndarray,
                       seed: int = 0) -> BSRSystem:
    """A 4x4-block system whose pressure-only (CPR, e = {p}) Quasi-IMPES system is
    the given scalar CSR matrix exactly.

    Block (i, j) holds val_ij in its (p, p) entry; the (h, p) entries are zero in
    every block and the diagonal blocks have D[p, h] = 0 with D[h, h] diagonally
    dominant, so the decoupling weights are zero and the pressure system is the
    matrix itself.  The remaining (p, h) and (h, h) couplings are seeded small
    random values, which only the full system (ILU, SpMV) sees."""
    rng = np.random.default_rng(seed)
    n = rowptr.size - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    nnzb = col.size
    vals = np.zeros((nnzb, 4, 4))
    vals[:, 0, 0] = val
    off = rows != col
    vals[:, 0, 1:] = rng.uniform(-0.1, 0.1, (nnzb, 3)) * off[:, None]
    vals[:, 1:, 1:] = rng.uniform(-0.1, 0.1, (nnzb, 3, 3))
    diag = ~off
    vals[diag, 1:, 1:] += 4.0 * np.eye(3)
    rhs = rng.normal(0.0, 1.0, 4 * n)
    return BSRSystem(n, np.asarray(rowptr, np.int32), np.asarray(col, np.int32),
                     np.ascontiguousarray(vals.reshape(nnzb, 16)), rhs,
                     dict(kind="pressure_embedding", seed=seed))


def with_volume_constraint(s: BSRSystem, seed: int = 0) -> BSRSystem:
    """The system of Section 3.4 before its first reduction: equation row 2
    becomes a cell-local volume constraint, so the last density (unknown 2,
    rho_H2O) can be eliminated exactly per cell.

    Built from a generator system by reassigning its rows: row 0 (total mass)
    takes over the rho_H2O convection that row 2 carried, in every block, so the
    eliminated unknown still couples neighbouring cells; row 2 of every
    off-diagonal block becomes zero and row 2 of each diagonal block holds seeded
    coefficients of a linearised volume constraint (both densities positive and
    rho_H2O dominant, small negative pressure and temperature sensitivities),
    scaled like the block's density diagonal.  The right-hand side of the
    constraint rows is a small seeded residual."""
    rng = np.random.default_rng(seed)
    n = s.n_cells
    v = s.vals.reshape(-1, 4, 4).copy()
    rows = np.repeat(np.arange(n), np.diff(s.rowptr))
    diag = rows == s.col
    v[:, 0, 2] += v[:, 2, 2]
    v[~diag, 2, :] = 0.0
    scale = np.abs(v[diag, 1, 1])
    coef = np.column_stack([-rng.uniform(0.01, 0.05, n), rng.uniform(0.3, 0.6, n),
                            rng.uniform(0.8, 1.2, n), -rng.uniform(0.01, 0.05, n)])
    v[diag, 2, :] = coef * scale[:, None]
    rhs = s.rhs.copy()
    rhs[2::4] = rng.normal(0.0, 0.01, n) * scale
    meta = dict(s.meta)
    meta.update(volume_constraint_seed=seed)
    return BSRSystem(n, s.rowptr.copy(), s.col.copy(), np.ascontiguousarray(v.reshape(-1, 16)),
                     rhs, meta)
