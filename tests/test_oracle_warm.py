"""Warm start (x_0 given, z_0 = b): pins of the oracle.

Every update of x lies in range(A^T), so from x_0 the iteration converges to
A^+ b + (I - A^+ A) x_0: the minimum-norm solution plus x_0's null-space part,
checked against numpy's pseudo-inverse on a fat system; and started at the
solution itself it stops before the first iteration.
"""
import numpy as np

import oracle
import workloads


def test_warm_start_limit_keeps_the_null_space_part_of_x0():
    rng = np.random.default_rng(0)
    D = rng.standard_normal((20, 50))
    b = rng.standard_normal(20)
    x0 = rng.standard_normal(50)
    S = workloads.from_dense(D, b)
    r = oracle.solve(S.A, b, oracle.Options(tol=1e-13, inner_tol=1e-14, max_iter=10000), n=50,
                     x0=x0)
    Ap = np.linalg.pinv(D)
    want = Ap @ b + (np.eye(50) - Ap @ D) @ x0
    assert r.status == 0
    assert np.linalg.norm(r.x - want) <= 1e-10 * np.linalg.norm(want)


def test_warm_start_at_the_solution_takes_no_iteration():
    rng = np.random.default_rng(1)
    D = rng.standard_normal((60, 15))
    b = rng.standard_normal(60)
    S = workloads.from_dense(D, b)
    xs = np.linalg.lstsq(D, b, rcond=None)[0]
    r = oracle.solve(S.A, b, oracle.Options(tol=1e-10, max_iter=100), n=15, x0=xs)
    assert r.status == 0 and r.iters == 0
    assert np.array_equal(r.x, xs)
