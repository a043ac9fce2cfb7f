"""Seeded synthetic inputs for RGDBEK, shared by the tests, the smoke check and
the benchmark.  This module holds only input generation (numpy
``default_rng``), none of the method's arithmetic, and imports neither the
oracle nor the CUDA library.

A matrix is returned as ``(row_ptr int64[m+1], col_idx int32[nnz],
vals float64[nnz])`` in CSR form with sorted, distinct column indices per row.

Workloads (the recipe of each is restated in the design notes):
  dense_gaussian      dense i.i.d. N(0,1) m x n matrix stored as CSR, x* ~ N(0,1),
                      b = A x*  (consistent; 1000 x 200 is the small dense case)
  sparse_ls           m x n with k distinct uniform columns per row, N(0,1)
                      values, b = A x* + e with e ~ N(0, sigma^2) (inconsistent
                      least squares; 200000 x 50000, k = 20, sigma = 1e-2 is the
                      large benchmark case)
  sprandn_like        every entry nonzero independently with probability
                      `density`, N(0,1) values, b = A x*  (the random matrices
                      of Tables 1 and 2: 99% sparse)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class System:
    name: str
    m: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    vals: np.ndarray
    b: np.ndarray
    x_true: np.ndarray
    consistent: bool

    @property
    def A(self):
        return (self.row_ptr, self.col_idx, self.vals)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        D = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        D[rows, self.col_idx] = self.vals
        return D


def csr_from_dense(D: np.ndarray):
    m, n = D.shape
    mask = D != 0
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    rows, cols = np.nonzero(mask)
    return row_ptr, cols.astype(np.int32), D[rows, cols].astype(np.float64)


def _csr_matvec(row_ptr, col_idx, vals, x):
    # b = A x for building right-hand sides (input data, not the method)
    m = len(row_ptr) - 1
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    return np.bincount(rows, weights=vals * x[col_idx], minlength=m)


def dense_gaussian(m: int = 1000, n: int = 200, seed: int = 0) -> System:
    rng = np.random.default_rng(seed)
    D = rng.standard_normal((m, n))
    x = rng.standard_normal(n)
    b = D @ x
    rp, ci, av = csr_from_dense(D)
    return System(f"dense_gaussian_{m}x{n}", m, n, rp, ci, av, b, x, True)


def random_rows_csr(rng, m: int, n: int, k: int):
    """k distinct uniformly random columns per row (sorted), N(0,1) values."""
    k = min(k, n)
    cols = rng.integers(0, n, size=(m, k), dtype=np.int64)
    cols.sort(axis=1)
    while True:
        dup = np.any(cols[:, 1:] == cols[:, :-1], axis=1) if k > 1 else np.zeros(m, bool)
        bad = np.nonzero(dup)[0]
        if len(bad) == 0:
            break
        redraw = rng.integers(0, n, size=(len(bad), k), dtype=np.int64)
        redraw.sort(axis=1)
        cols[bad] = redraw
    row_ptr = np.arange(0, m * k + 1, k, dtype=np.int64)
    vals = rng.standard_normal(m * k)
    return row_ptr, cols.reshape(-1).astype(np.int32), vals


def sparse_ls(m: int = 200000, n: int = 50000, k: int = 20, sigma: float = 1e-2,
              seed: int = 1) -> System:
    rng = np.random.default_rng(seed)
    rp, ci, av = random_rows_csr(rng, m, n, k)
    x = rng.standard_normal(n)
    e = sigma * rng.standard_normal(m)
    b = _csr_matvec(rp, ci, av, x) + e
    return System(f"sparse_ls_{m}x{n}_k{k}", m, n, rp, ci, av, b, x, sigma == 0.0)


def sprandn_like(m: int, n: int, density: float = 0.01, seed: int = 0) -> System:
    rng = np.random.default_rng(seed)
    # Bernoulli(density) pattern row by row, N(0,1) values
    counts = rng.binomial(n, density, size=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    cols = np.empty(int(row_ptr[-1]), dtype=np.int32)
    for i in range(m):
        c = rng.choice(n, size=int(counts[i]), replace=False)
        c.sort()
        cols[row_ptr[i]:row_ptr[i + 1]] = c
    vals = rng.standard_normal(len(cols))
    x = rng.standard_normal(n)
    b = _csr_matvec(row_ptr, cols, vals, x)
    return System(f"sprandn_{m}x{n}_d{density}", m, n, row_ptr, cols, vals, b, x, True)


def from_dense(D: np.ndarray, b: np.ndarray, name: str = "dense", x_true=None,
               consistent: bool = False) -> System:
    rp, ci, av = csr_from_dense(D)
    m, n = D.shape
    return System(name, m, n, rp, ci, av, np.asarray(b, np.float64),
                  np.zeros(n) if x_true is None else x_true, consistent)
