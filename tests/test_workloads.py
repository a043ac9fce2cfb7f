"""Pins of the input generators to values the paper prints.

The P1 Poisson stiffness matrix generator (the mixed-precision workload) is
pinned to Table 8: at 25 x 25 nodes the paper reports 1152 elements, 99.32 %
sparsity, condition number 2.327776e2 and Frobenius norm 1.028786e2.  These
fix the element assembly, the treatment of the Dirichlet rows (identity rows,
columns eliminated) and the dropping of the couplings that assemble to zero.
"""
import os

import numpy as np

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table8_poisson_fem_matrix.txt")


def _golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_poisson_matrix_matches_table8():
    g = _golden()
    nx = 25
    rp, ci, av, xy = workloads.poisson_p1_matrix(nx)
    N = nx * nx
    assert 2 * (nx - 1) ** 2 == g["elements"]
    D = np.zeros((N, N))
    D[np.repeat(np.arange(N), np.diff(rp)), ci] = av
    assert round(100.0 * (1.0 - len(av) / N ** 2), 2) == g["sparsity_percent"]
    assert float(f"{np.linalg.cond(D):.6e}") == g["condition_number"]
    assert float(f"{np.linalg.norm(D):.6e}") == g["frobenius_norm"]
    # symmetric, Dirichlet rows are identity rows, interior rows sum to zero
    # away from the boundary (a constant is in the kernel of -Laplace)
    assert np.array_equal(D, D.T)
    bnd = (xy[:, 0] == 0) | (xy[:, 1] == 0) | (xy[:, 0] == 1) | (xy[:, 1] == 1)
    assert np.array_equal(D[bnd][:, bnd], np.eye(int(bnd.sum())))
    assert np.all(D[bnd][:, ~bnd] == 0)
    far = np.nonzero(~bnd & (xy[:, 0] > 0.1) & (xy[:, 0] < 0.9) & (xy[:, 1] > 0.1)
                     & (xy[:, 1] < 0.9))[0]
    assert np.allclose(D[far].sum(axis=1), 0.0)


def test_poisson_keep_zeros_gives_seven_point_rows():
    rp, ci, av, _ = workloads.poisson_p1_matrix(9, keep_zeros=True)
    assert np.diff(rp).max() == 7
    rp0, _, _, _ = workloads.poisson_p1_matrix(9)
    assert np.diff(rp0).max() == 5


def test_blur_operator_rows_are_normalised_taps():
    rp, ci, av = workloads.blur_csr(32)
    w = workloads.gaussian_taps()
    assert abs(w.sum() - 1.0) < 1e-15 and len(w) == 9
    # an interior row holds the full 9 x 9 outer product of the taps
    i = 16 * 32 + 16
    row = av[rp[i]:rp[i + 1]]
    assert len(row) == 81 and np.allclose(row, np.outer(w, w).reshape(-1))
    # a corner row is truncated by the zero boundary
    assert rp[1] - rp[0] == 25
