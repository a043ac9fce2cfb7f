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


def test_resumed_solve_is_bit_identical_to_one_solve():
    """A solve cut into pieces at iterations 7 and 19, each piece resumed from
    the previous piece's (x_k, z_k, k), computes exactly what one uninterrupted
    solve computes: the draws depend only on (seed, k), and every other step
    is a function of (x_k, z_k).  The benchmark's CPU reference arm times the
    oracle this way, one piece per step."""
    import oracle
    import workloads
    S = workloads.sparse_ls(3000, 700, 20, sigma=1e-2, seed=41)
    o = oracle.Options(eta_col=0.1, eta_row=0.1, stop_rule=2, tol=1e-10, max_iter=100000,
                       seed=3)
    full = oracle.solve(S.A, S.b, o, n=S.n)
    assert full.status == 0 and full.iters > 25
    x, z, k = np.zeros(S.n), S.b.copy(), 0
    for stop in (7, 19, 100000):
        oo = oracle.Options(**{**o.__dict__, "max_iter": stop})
        part = oracle.solve(S.A, S.b, oo, n=S.n, resume=(x, z, k))
        x, z, k = part.x, part.z, part.iters
        if part.status == 0:
            break
    assert part.status == 0 and k == full.iters
    assert np.array_equal(x, full.x)
