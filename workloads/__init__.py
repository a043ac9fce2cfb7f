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
  blur_image          the s^2 x s^2 separable Gaussian blur T (x) T (9 taps,
                      sigma 1.5, taps summing to 1, zero boundary; up to 81
                      nonzeros per row), a blocky test image (uniform [0,1]
                      background under 8-32 random rectangles of U[0,1]
                      values) and b = A x + 1% Gaussian noise
  deblur_regularised  [A; lam I] and [b; 0] for that blur (lam = 0.05): the
                      full-column-rank system of the adjoint workload
  poisson_p1          -Laplace(u) = f on the unit square, P1 elements on a
                      uniform right-triangle grid, Dirichlet rows as identity
                      rows; K x* = b with x* = sin(pi x) sin(pi y) + noise
                      (the mixed-precision workload)
  blur_batch          many blur_image systems of uneven sizes (the batched
                      workload)
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


def gaussian_taps(sigma: float = 1.5, taps: int = 9) -> np.ndarray:
    h = taps // 2
    w = np.exp(-0.5 * (np.arange(-h, h + 1) / sigma) ** 2)
    return w / w.sum()


def blur_csr(side: int, sigma: float = 1.5, taps: int = 9):
    """CSR of T (x) T, T the side x side banded 1-D blur with zero boundary.

    Row p*side + q holds T[p, p'] T[q, q'] at column p'*side + q' (sorted)."""
    w = gaussian_taps(sigma, taps)
    h = taps // 2
    s = side
    off = np.arange(-h, h + 1)
    col1 = np.arange(s)[:, None] + off[None, :]                  # (s, taps)
    ok1 = (col1 >= 0) & (col1 < s)
    val1 = np.where(ok1, w[None, :], 0.0)
    # rows (p, q), entries (a, c): column col1[p, a] * s + col1[q, c]
    cols = col1[:, None, :, None] * s + col1[None, :, None, :]   # (s, s, taps, taps)
    vals = val1[:, None, :, None] * val1[None, :, None, :]
    ok = ok1[:, None, :, None] & ok1[None, :, None, :]
    cols = cols.reshape(s * s, taps * taps)
    vals = vals.reshape(s * s, taps * taps)
    ok = ok.reshape(s * s, taps * taps)
    counts = ok.sum(axis=1)
    row_ptr = np.zeros(s * s + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols[ok].astype(np.int32), vals[ok].astype(np.float64)


def blocky_image(rng, side: int) -> np.ndarray:
    img = rng.random((side, side))
    for _ in range(int(rng.integers(8, 33))):
        r0, r1 = np.sort(rng.integers(0, side + 1, size=2))
        c0, c1 = np.sort(rng.integers(0, side + 1, size=2))
        img[r0:max(r1, r0 + 1), c0:max(c1, c0 + 1)] = rng.random()
    return img.reshape(-1)


def blur_image(side: int = 256, seed: int = 4) -> System:
    rng = np.random.default_rng(seed)
    rp, ci, av = blur_csr(side)
    x = blocky_image(rng, side)
    clean = _csr_matvec(rp, ci, av, x)
    rms = float(np.sqrt(np.mean(clean ** 2)))
    b = clean + 0.01 * rms * rng.standard_normal(side * side)
    return System(f"blur_{side}x{side}", side * side, side * side, rp, ci, av, b, x, False)


def deblur_regularised(side: int = 256, lam: float = 0.05, seed: int = 4) -> System:
    """[A; lam I] x ~ [b; 0] for the blur of `blur_image` (Tikhonov form)."""
    B = blur_image(side, seed)
    N = side * side
    row_ptr = np.concatenate([B.row_ptr, B.row_ptr[-1] + 1 + np.arange(N, dtype=np.int64)])
    col_idx = np.concatenate([B.col_idx, np.arange(N, dtype=np.int32)])
    vals = np.concatenate([B.vals, np.full(N, lam)])
    b = np.concatenate([B.b, np.zeros(N)])
    return System(f"deblur_{side}x{side}_lam{lam}", 2 * N, N, row_ptr, col_idx, vals, b,
                  B.x_true, False)


def poisson_p1_matrix(nx: int, keep_zeros: bool = False):
    """Stiffness matrix of -Laplace(u) = f on [0,1]^2 with u = 0 on the boundary:
    linear (P1) elements on the nx x nx uniform grid, each cell split into two
    right triangles by its (lower-left, upper-right) diagonal.  Element
    matrices are assembled from the gradients of the barycentric basis;
    Dirichlet rows become identity rows and their columns are eliminated from
    the other rows.  Entries that assemble to exactly zero (the couplings
    across the cell diagonals) are dropped unless keep_zeros.

    Returns (row_ptr, col_idx, vals, coords) with coords (N, 2), N = nx^2,
    node (i, j) -> index j * nx + i at (i h, j h), h = 1 / (nx - 1)."""
    h = 1.0 / (nx - 1)
    ii, jj = np.meshgrid(np.arange(nx - 1), np.arange(nx - 1), indexing="xy")
    ii, jj = ii.reshape(-1), jj.reshape(-1)
    n00 = jj * nx + ii
    n10 = n00 + 1
    n01 = n00 + nx
    n11 = n01 + 1
    tris = np.concatenate([np.stack([n00, n10, n11], 1), np.stack([n00, n11, n01], 1)])
    coords = np.stack([np.tile(np.arange(nx) * h, nx), np.repeat(np.arange(nx) * h, nx)], 1)
    P = coords[tris]                                      # (T, 3, 2)
    # gradients of the barycentric functions: grad phi_a = rot(P_b - P_c) / (2 area)
    e = np.stack([P[:, 2] - P[:, 1], P[:, 0] - P[:, 2], P[:, 1] - P[:, 0]], 1)  # opposite edges
    area2 = e[:, 1, 0] * e[:, 2, 1] - e[:, 1, 1] * e[:, 2, 0]
    # K_ab = (e_a . e_b) / (2 area2)  (area2 = twice the area)
    K = np.einsum("tad,tbd->tab", e, e) / (2.0 * area2[:, None, None])
    rows = np.repeat(tris, 3, axis=1).reshape(-1)
    cols = np.tile(tris, (1, 3)).reshape(-1)
    N = nx * nx
    key = rows.astype(np.int64) * N + cols
    uk, inv = np.unique(key, return_inverse=True)
    val = np.zeros(len(uk))
    np.add.at(val, inv, K.reshape(-1))
    r, c = uk // N, uk % N
    bnd = np.zeros(N, bool)
    on = (coords[:, 0] == 0) | (coords[:, 1] == 0) | (np.arange(N) % nx == nx - 1) | \
         (np.arange(N) // nx == nx - 1)
    bnd[on] = True
    keep = ~bnd[r] & ~bnd[c]
    if not keep_zeros:
        keep &= val != 0.0
    r, c, val = r[keep], c[keep], val[keep]
    b_idx = np.nonzero(bnd)[0]
    r = np.concatenate([r, b_idx])
    c = np.concatenate([c, b_idx])
    val = np.concatenate([val, np.ones(len(b_idx))])
    order = np.lexsort((c, r))
    r, c, val = r[order], c[order], val[order]
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=N), out=row_ptr[1:])
    return row_ptr, c.astype(np.int32), val, coords


def poisson_p1(nx: int = 1024, sigma: float = 1e-3, seed: int = 2,
               keep_zeros: bool = False) -> System:
    """K x* = b with x* = sin(pi x) sin(pi y) at the nodes plus N(0, sigma^2)
    noise (consistent, square)."""
    rng = np.random.default_rng(seed)
    rp, ci, av, xy = poisson_p1_matrix(nx, keep_zeros)
    x = np.sin(np.pi * xy[:, 0]) * np.sin(np.pi * xy[:, 1]) + sigma * rng.standard_normal(nx * nx)
    b = _csr_matvec(rp, ci, av, x)
    N = nx * nx
    return System(f"poisson_p1_{nx}x{nx}", N, N, rp, ci, av, b, x, True)


def blur_batch(count: int = 256, side_lo: int = 64, side_hi: int = 512, seed: int = 3) -> list:
    """`count` independent deblurring systems of uneven sizes: side lengths
    uniform in [side_lo, side_hi], each the blur_image recipe with its own
    seed (seed * 100003 + i)."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=count)
    return [blur_image(int(s), seed=seed * 100003 + i) for i, s in enumerate(sides)]
