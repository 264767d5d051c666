import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def bsr_from_dense(A: np.ndarray):
    """Full 4x4-block BSR of a dense matrix (all blocks stored)."""
    n = A.shape[0] // 4
    rowptr = np.arange(0, n * n + 1, n, dtype=np.int32)
    col = np.tile(np.arange(n, dtype=np.int32), n)
    vals = A.reshape(n, 4, n, 4).transpose(0, 2, 1, 3).reshape(n * n, 16).copy()
    return rowptr, col, vals


def bsr_to_dense(rowptr, col, vals, n):
    A = np.zeros((4 * n, 4 * n))
    for i in range(n):
        for t in range(rowptr[i], rowptr[i + 1]):
            j = col[t]
            A[4 * i:4 * i + 4, 4 * j:4 * j + 4] = vals[t].reshape(4, 4)
    return A


def csr_to_dense(rp, ci, v, n, m=None):
    m = n if m is None else m
    A = np.zeros((n, m))
    for i in range(n):
        for t in range(rp[i], rp[i + 1]):
            A[i, ci[t]] += v[t]
    return A
