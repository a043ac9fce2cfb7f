"""Randomised parity sweep: many small systems of every kind, with random
options, each solved on the GPU and by the FP64 oracle to a tight tolerance.

Cases (seeded): tall, fat and square; sparse and dense; consistent and
inconsistent; full rank and rank deficient (duplicated or zero rows and
columns); random eta, selection rule, stopping rule, inner precision,
adaptive inner tolerance and launch shape (threads per CTA).  The bar is the FP64 one, 1e-8 relative to
the oracle's solution and to pinv(A) b, except for FP32 inner products on
systems with a null space (their stated bound, 1e-6).
"""
import numpy as np
import pytest

import gpu_util as G
import oracle
import workloads

pytestmark = pytest.mark.gpu

N_CASES = 24


def _case(rng):
    kind = rng.choice(["tall", "fat", "square"])
    if kind == "tall":
        m, n = int(rng.integers(60, 400)), int(rng.integers(10, 60))
    elif kind == "fat":
        m, n = int(rng.integers(10, 60)), int(rng.integers(60, 400))
    else:
        m = n = int(rng.integers(20, 120))
    dense = rng.random() < 0.3
    if dense:
        D = rng.standard_normal((m, n))
    else:
        D = rng.standard_normal((m, n)) * (rng.random((m, n)) < rng.uniform(0.05, 0.3))
    defect = rng.choice(["none", "dup_rows", "zero_cols", "low_rank"])
    if defect == "dup_rows" and m >= 4:
        D[1::2] = D[0:m - m % 2:2][: D[1::2].shape[0]]
    elif defect == "zero_cols":
        D[:, rng.choice(n, size=max(1, n // 10), replace=False)] = 0.0
    elif defect == "low_rank":
        r = int(rng.integers(2, max(3, min(m, n) // 2)))
        D = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    for i in range(m):                    # no empty matrix
        if not D[i].any() and rng.random() < 0.5:
            D[i, rng.integers(n)] = 1.0
    consistent = rng.random() < 0.5
    b = D @ rng.standard_normal(n) if consistent else rng.standard_normal(m)
    opts = dict(eta=float(rng.choice([0.1, 0.3, 0.5, 1.0])),
                selection=int(rng.random() < 0.2),
                stop_rule=2,
                precision=int(rng.random() < 0.3),
                threads=int(rng.choice([0, 256, 512, 1024])),
                seed=int(rng.integers(1 << 30)),
                inner_adapt=float(rng.choice([0.0, 0.0, 0.01, 1.0])))
    return kind, defect, D, b, opts


@pytest.mark.parametrize("case", range(N_CASES))
def test_random_case_matches_oracle_and_pinv(case):
    rg = G.rg()
    rng = np.random.default_rng(1000 + case)
    kind, defect, D, b, o = _case(rng)
    S = workloads.from_dense(D, b)
    if S.nnz == 0:
        pytest.skip("empty matrix")
    s = rg.Solver(S.m, S.n, S.row_ptr, S.col_idx, S.vals, eta_col=o["eta"], eta_row=o["eta"],
                  selection=o["selection"], stop_rule=o["stop_rule"], inner_tol=1e-13,
                  precision=o["precision"], threads_per_block=o["threads"],
                  inner_adapt=o["inner_adapt"])
    res = s.solve(G.dev(S.b), tol=1e-12, max_iter=200000, seed=o["seed"])
    x = G.host(res.x).copy()
    s.close()
    ref = oracle.solve(S.A, S.b, oracle.Options(eta_col=o["eta"], eta_row=o["eta"],
                                                selection=o["selection"], stop_rule=2,
                                                tol=1e-12, inner_tol=1e-13, max_iter=200000,
                                                seed=o["seed"], inner_adapt=o["inner_adapt"]),
                       n=S.n)
    xs = np.linalg.pinv(D, rcond=1e-10) @ b
    label = f"{kind}/{defect}/{o}"
    assert res.stats.status == rg.OK, label
    assert ref.status == 0, label
    null_space = np.linalg.matrix_rank(D, tol=1e-10 * np.linalg.norm(D, 2)) < S.n
    bar = 1e-6 if (o["precision"] and null_space) else 1e-8
    scale = max(np.linalg.norm(xs), 1e-300)
    assert np.linalg.norm(x - xs) <= bar * scale, (label, np.linalg.norm(x - xs) / scale)
    assert np.linalg.norm(x - ref.x) <= bar * scale, label
