"""Adaptive inner tolerance (inner_adapt > 0): pins of the oracle.

The block solves of iteration k stop at max(inner_tol, min(0.1, c r_k)), r_k
the stopping rule's measure of x_k.  The outer iteration and its test are
unchanged, so the solve still reaches the least-squares solution (numpy
lstsq) and the consistent solution (x*), with fewer inner LSQR steps.
"""
import numpy as np

import oracle
import workloads


def test_adaptive_inner_tolerance_reaches_the_same_solutions_with_fewer_steps():
    S = workloads.sparse_ls(4000, 1000, 15, sigma=1e-2, seed=3)
    xs = np.linalg.lstsq(S.dense(), S.b, rcond=None)[0]
    fixed = oracle.solve(S.A, S.b, oracle.Options(eta_col=0.2, eta_row=0.2, stop_rule=2,
                                                  tol=1e-12, inner_tol=1e-12), n=S.n)
    adapt = oracle.solve(S.A, S.b, oracle.Options(eta_col=0.2, eta_row=0.2, stop_rule=2,
                                                  tol=1e-12, inner_tol=1e-12, inner_adapt=0.01),
                         n=S.n)
    assert fixed.status == 0 and adapt.status == 0
    assert np.linalg.norm(adapt.x - xs) <= 1e-9 * np.linalg.norm(xs)
    assert adapt.inner_u + adapt.inner_j < 0.8 * (fixed.inner_u + fixed.inner_j)
    C = workloads.dense_gaussian(300, 60, seed=4)
    r = oracle.solve(C.A, C.b, oracle.Options(stop_rule=1, tol=1e-12, inner_tol=1e-12,
                                              inner_adapt=1.0), n=C.n)
    assert r.status == 0
    assert np.linalg.norm(r.x - C.x_true) <= 1e-9 * np.linalg.norm(C.x_true)


def test_adaptive_inner_tolerance_under_each_stopping_rule():
    # consistent sparse system: every rule's measure (relative residual, its
    # square for RSE, normal-equation residual) drives the inner tolerance,
    # and each run reaches x* with fewer LSQR steps than the fixed tolerance
    S = workloads.sprandn_like(1500, 400, 0.02, seed=9)
    for rule, tol in ((1, 1e-11), (2, 1e-11), (3, 1e-22)):
        base = oracle.Options(eta_col=0.3, eta_row=0.3, stop_rule=rule, tol=tol, inner_tol=1e-13)
        fixed = oracle.solve(S.A, S.b, base, n=S.n)
        adapt = oracle.solve(S.A, S.b, oracle.Options(eta_col=0.3, eta_row=0.3, stop_rule=rule,
                                                      tol=tol, inner_tol=1e-13, inner_adapt=0.1),
                             n=S.n)
        assert fixed.status == 0 and adapt.status == 0, rule
        assert np.linalg.norm(adapt.x - S.x_true) <= 1e-8 * np.linalg.norm(S.x_true), rule
        assert adapt.inner_u + adapt.inner_j < fixed.inner_u + fixed.inner_j, rule
