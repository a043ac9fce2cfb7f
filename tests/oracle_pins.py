"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each ``pin_*`` function raises AssertionError when the oracle disagrees with
the fact it checks.  ``test_oracle_pins.py`` runs them against the oracle as
built; ``test_oracle_mutations.py`` runs them against copies of the oracle
with a plausible mistake planted, to show that each mistake is caught.

What the facts are:
  * Philox known answers from numpy.random.Philox, an independent
    implementation of Philox4x64-10.
  * Dense numpy products and norms for the sparse kernels.
  * Hand-computed residual weights (Section 2).
  * Block sampling: draws with probability proportional to the weights
    (chi-square), zero weights never drawn, the block is a sorted set of
    distinct indices, degenerate single-weight and all-zero cases.
  * LSQR (Remark 3.1) against numpy lstsq / pinv, including the minimum-norm
    solution of rank-deficient and underdetermined systems.
  * Algorithm 1 converging to the minimum-norm least-squares solution
    x* = A^+ b (Theorem 2.3), and, for m x 1 and 1 x n matrices, reaching it in
    exactly one iteration (a closed form that needs the row residual to use
    z_{k+1}, as Algorithm 1 states).
  * The Pythagoras identity ||z_{k+1} - r||^2 = ||z_k - r||^2 -
    ||P_U (z_k - r)||^2 of Eq. (5) at every iteration, with P_U computed by
    numpy pinv, and P_U r = 0.
  * Each block update of Eq. (4) with the blocks fixed, against numpy pinv:
    unit-scaled columns and rows, a singular row block (duplicated rows), tall
    and rank-deficient blocks.
  * The linear rate of Theorem 2.3(a): the mean of ||z_k - r||^2/||z_0 - r||^2
    over seeds stays below gamma^k, gamma = 1 - sigma_min^2/||A||_2^2.
  * The mean iteration counts of Tables 1 and 2 (random 99%-sparse matrices,
    eta = 0.5, RSE <= 1e-6) within 20%.
"""
from __future__ import annotations

import os

import numpy as np

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _csr(D):
    return workloads.csr_from_dense(np.asarray(D, dtype=np.float64))


# --------------------------------------------------------------------------
# Philox4x64-10
# --------------------------------------------------------------------------
def pin_philox():
    cases = [((0, 0), (0, 0, 0, 0)), ((5, 7), (0, 0, 0, 0)),
             ((0xDEADBEEF, 0x12345678), (41, 3, 9, 0)),
             ((2**64 - 1, 2**63 + 5), (2**64 - 2, 2**64 - 1, 17, 2**40))]
    for key, ctr in cases:
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                              counter=np.array(ctr, dtype=np.uint64))
        expect = bg.random_raw(8)
        # numpy increments the 256-bit counter (with carry) before each block
        c = list(ctr)
        for blk in range(2):
            i = 0
            while True:
                c[i] = (c[i] + 1) % 2**64
                if c[i] != 0 or i == 3:
                    break
                i += 1
            got = oracle.philox(key, c)
            assert np.array_equal(got, expect[4 * blk:4 * blk + 4]), (key, ctr, blk)


# --------------------------------------------------------------------------
# Sparse products and norms
# --------------------------------------------------------------------------
def pin_spmv():
    rng = np.random.default_rng(11)
    D = rng.standard_normal((37, 23)) * (rng.random((37, 23)) < 0.3)
    D[5, :] = 0.0
    D[:, 7] = 0.0
    A = _csr(D)
    x = rng.standard_normal(23)
    z = rng.standard_normal(37)
    assert np.allclose(oracle.spmv(A, x), D @ x, rtol=1e-13, atol=1e-13)
    assert np.allclose(oracle.spmv_t(A, z, 23), D.T @ z, rtol=1e-13, atol=1e-13)
    assert np.allclose(oracle.row_norms2(A), (D * D).sum(axis=1), rtol=1e-13, atol=0)
    assert np.allclose(oracle.col_norms2(A, 23), (D * D).sum(axis=0), rtol=1e-13, atol=0)


def pin_weights():
    # eps_j = v_j^2 / ||A_j||^2, 0 for a zero-norm column (Section 2)
    v = np.array([3.0, 0.0, -2.0, 5.0, 1.0])
    nrm2 = np.array([9.0, 4.0, 0.0, 5.0, 4.0])
    eps, emax, bad = oracle.weights(v, nrm2)
    assert np.array_equal(eps, [1.0, 0.0, 0.0, 5.0, 0.25])
    assert emax == 5.0 and not bad
    _, _, bad = oracle.weights(np.array([1.0, np.nan]), np.array([1.0, 1.0]))
    assert bad
    _, _, bad = oracle.weights(np.array([1.0, np.inf]), np.array([1.0, 1.0]))
    assert bad


# --------------------------------------------------------------------------
# Block sampling
# --------------------------------------------------------------------------
def pin_sample_law():
    # Draw frequencies follow P(j) = eps_j / sum eps (Section 2).  One draw per
    # call (s = 1) over many counters k gives i.i.d. samples of the law.
    eps = np.array([4.0, 2.0, 1.0, 0.0, 1.0, 8.0, 0.5])
    p = eps / eps.sum()
    counts = np.zeros(len(eps))
    trials = 6000
    for k in range(trials):
        idx = oracle.sample(eps, 1, seed=3, sysid=0, k=k, phase=0)
        assert len(idx) == 1
        counts[idx[0]] += 1
    assert counts[3] == 0, "a zero weight was drawn"
    nz = p > 0
    expected = trials * p[nz]
    chi2 = float(((counts[nz] - expected) ** 2 / expected).sum())
    # 5 degrees of freedom: P(chi2 > 25) < 2e-4
    assert chi2 < 25.0, (chi2, counts, expected)


def pin_sample_sets():
    rng = np.random.default_rng(5)
    eps = rng.random(1000) ** 4
    eps[rng.random(1000) < 0.2] = 0.0
    for k in range(20):
        s = oracle.num_draws(0.3, len(eps))
        assert s == 300
        idx = oracle.sample(eps, s, seed=9, sysid=1, k=k, phase=1)
        assert len(idx) >= 1 and len(idx) <= s
        assert np.all(np.diff(idx) > 0), "block must be sorted and distinct"
        assert np.all(eps[idx] > 0), "zero weights must never be selected"
    # one positive weight: the block is exactly that index
    e1 = np.zeros(50)
    e1[17] = 3.0
    assert list(oracle.sample(e1, 10, 1, 0, 0, 0)) == [17]
    e1[:] = 0.0
    e1[49] = 1e-300
    assert list(oracle.sample(e1, 10, 1, 0, 0, 0)) == [49]
    # all weights zero: empty block
    assert len(oracle.sample(np.zeros(50), 10, 1, 0, 0, 0)) == 0
    # a single index
    assert list(oracle.sample(np.array([2.0]), 1, 1, 0, 0, 0)) == [0]
    # ceil(eta * len) draws, at least one
    assert oracle.num_draws(0.5, 7) == 4 and oracle.num_draws(1e-9, 7) == 1
    assert oracle.num_draws(0.1, 200000) == 20000 and oracle.num_draws(0.1, 50000) == 5000


def pin_greedy():
    # GDBEK threshold set {j : eps_j >= eta max eps} (Section 2)
    eps = np.array([1.0, 5.0, 2.5, 2.4, 0.0, 5.0])
    assert list(oracle.select_greedy(eps, 0.5)) == [1, 2, 5]
    assert list(oracle.select_greedy(eps, 1.0)) == [1, 5]
    assert len(oracle.select_greedy(np.zeros(4), 0.5)) == 0


# --------------------------------------------------------------------------
# LSQR
# --------------------------------------------------------------------------
def pin_lsqr():
    rng = np.random.default_rng(2)
    # tall, full column rank, inconsistent: the least-squares solution
    D = rng.standard_normal((60, 15))
    c = rng.standard_normal(60)
    y, steps = oracle.lsqr(_csr(D), c, 15, tol=1e-14, maxit=500)
    ref = np.linalg.lstsq(D, c, rcond=None)[0]
    assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)
    assert 1 <= steps <= 500
    # fat, full row rank: the minimum-norm solution of a consistent system
    D = rng.standard_normal((10, 40))
    c = rng.standard_normal(10)
    y, _ = oracle.lsqr(_csr(D), c, 40, tol=1e-14, maxit=500)
    ref = np.linalg.pinv(D) @ c
    assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)
    # rank deficient: the minimum-norm least-squares solution
    L = rng.standard_normal((30, 4))
    R = rng.standard_normal((4, 12))
    D = L @ R
    c = rng.standard_normal(30)
    y, _ = oracle.lsqr(_csr(D), c, 12, tol=1e-14, maxit=500)
    ref = np.linalg.pinv(D) @ c
    assert np.linalg.norm(y - ref) <= 1e-9 * np.linalg.norm(ref)
    # zero right-hand side
    y, steps = oracle.lsqr(_csr(D), np.zeros(30), 12)
    assert np.all(y == 0.0) and steps == 0


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------
def _solve_dense(D, b, **kw):
    A = _csr(D)
    o = oracle.Options(**{"tol": 1e-12, "inner_tol": 1e-14, "max_iter": 5000, **kw})
    return oracle.solve(A, b, o, n=D.shape[1])


def pin_solve_min_norm():
    rng = np.random.default_rng(7)
    cases = []
    D = rng.standard_normal((50, 12))
    cases.append((D, D @ rng.standard_normal(12), 1))          # consistent
    cases.append((D, rng.standard_normal(50), 2))              # inconsistent
    L = rng.standard_normal((40, 3))
    cases.append((L @ rng.standard_normal((3, 10)), rng.standard_normal(40), 2))  # rank 3
    F = rng.standard_normal((8, 30))
    cases.append((F, rng.standard_normal(8), 1))               # fat: min-norm
    Z = rng.standard_normal((30, 9))
    Z[4, :] = 0.0
    Z[:, 2] = 0.0
    cases.append((Z, rng.standard_normal(30), 2))              # zero row and column
    for D, b, rule in cases:
        res = _solve_dense(D, b, stop_rule=rule, eta_col=0.5, eta_row=0.5)
        ref = np.linalg.pinv(D) @ b
        err = np.linalg.norm(res.x - ref) / np.linalg.norm(ref)
        assert res.status == 0, res
        assert err <= 1e-8, (D.shape, err)


def pin_one_iteration_closed_forms():
    # m x 1: U = {0}, so z_1 = (I - a a^T/||a||^2) b is the optimal residual,
    # the row residual b - z_1 - A x_0 equals a x*, and any row block with a
    # nonzero entry recovers x* exactly: x_1 = x* = a^T b / ||a||^2.
    rng = np.random.default_rng(4)
    a = rng.standard_normal((25, 1))
    b = rng.standard_normal(25)
    res = _solve_dense(a, b, stop_rule=2, eta_col=0.5, eta_row=0.3, max_iter=1)
    xstar = float(a[:, 0] @ b / (a[:, 0] @ a[:, 0]))
    assert abs(res.x[0] - xstar) <= 1e-12 * abs(xstar)
    assert res.normal_res <= 1e-12
    # 1 x n: z_1 = 0 after any nonempty column block, r = b, and the single
    # row gives x_1 = a b / ||a||^2, the minimum-norm solution.
    a = rng.standard_normal((1, 20))
    b = np.array([1.7])
    res = _solve_dense(a, b, stop_rule=1, eta_col=0.2, eta_row=0.5, max_iter=1)
    xstar = a[0] * b[0] / (a[0] @ a[0])
    assert np.linalg.norm(res.x - xstar) <= 1e-12 * np.linalg.norm(xstar)


def pin_degenerate():
    rng = np.random.default_rng(8)
    D = rng.standard_normal((20, 6))
    # b = 0: x_0 = 0 is the answer, no iteration is run
    res = _solve_dense(D, np.zeros(20), stop_rule=1)
    assert res.iters == 0 and res.status == 0 and np.all(res.x == 0)
    # b orthogonal to range(A) (b lives on zero rows of A): A^T b = 0, A^+ b = 0
    D0 = D.copy()
    D0[[2, 9], :] = 0.0
    b = np.zeros(20)
    b[2], b[9] = 1.5, -0.5
    res = _solve_dense(D0, b, stop_rule=2)
    assert res.status == 0 and res.iters == 0 and np.all(res.x == 0)
    # a NaN in b is reported
    bb = rng.standard_normal(20)
    bb[3] = np.nan
    res = _solve_dense(D, bb, stop_rule=1, max_iter=5)
    assert res.status == -2
    # iteration cap
    res = _solve_dense(D, rng.standard_normal(20), stop_rule=2, max_iter=2, tol=0.0)
    assert res.iters == 2 and res.status == 1


def pin_pythagoras_eq5():
    rng = np.random.default_rng(12)
    D = rng.standard_normal((40, 10))
    D[:, 3] = D[:, 1] + D[:, 2]          # rank deficient
    b = rng.standard_normal(40)
    A = _csr(D)
    o = oracle.Options(eta_col=0.3, eta_row=0.3, tol=1e-13, inner_tol=1e-14, stop_rule=2,
                       max_iter=30)
    res = oracle.solve(A, b, o, n=10, trace=True, keep_iterates=True)
    Dp = np.linalg.pinv(D)
    r_opt = b - D @ (Dp @ b)                 # (I - A A^+) b
    Pn = np.eye(10) - Dp @ D                 # projector onto null(A)
    assert res.iters >= 3
    for k in range(res.iters):
        U = res.lists[k][0]
        e_k = res.zs[k] - r_opt
        e_k1 = res.zs[k + 1] - r_opt
        if len(U):
            AU = D[:, U]
            PU = AU @ np.linalg.pinv(AU)
            assert np.linalg.norm(PU @ r_opt) <= 1e-10 * np.linalg.norm(b)   # P_U r = 0
            lhs = e_k1 @ e_k1
            rhs = e_k @ e_k - (PU @ e_k) @ (PU @ e_k)
            assert abs(lhs - rhs) <= 1e-9 * (e_k @ e_k) + 1e-24, (k, lhs, rhs)
        assert e_k1 @ e_k1 <= e_k @ e_k * (1 + 1e-12) + 1e-26
        # x_k stays in range(A^T): no component in null(A)
        assert np.linalg.norm(Pn @ res.xs[k + 1]) <= 1e-10 * max(np.linalg.norm(res.xs[k + 1]), 1)


def pin_rate_theorem():
    # Theorem 2.3(a) with mu = 1: E||z_k - r||^2 <= gamma^k ||z_0 - r||^2
    rng = np.random.default_rng(21)
    D = rng.standard_normal((60, 15))
    b = rng.standard_normal(60)
    s = np.linalg.svd(D, compute_uv=False)
    gamma = 1.0 - s[-1] ** 2 / s[0] ** 2
    r_opt = b - D @ (np.linalg.pinv(D) @ b)
    K = 8
    ratios = np.zeros(K + 1)
    seeds = 20
    for seed in range(seeds):
        o = oracle.Options(eta_col=0.1, eta_row=0.1, tol=0.0, inner_tol=1e-14, stop_rule=2,
                           max_iter=K, seed=seed)
        res = oracle.solve(_csr(D), b, o, n=15, keep_iterates=True)
        e0 = np.sum((res.zs[0] - r_opt) ** 2)
        ratios += np.array([np.sum((res.zs[k] - r_opt) ** 2) / e0 for k in range(K + 1)])
    ratios /= seeds
    for k in range(K + 1):
        assert ratios[k] <= gamma ** k * (1 + 1e-9), (k, ratios[k], gamma ** k)
    assert ratios[K] < ratios[0]


def read_table_golden():
    rows = []
    with open(os.path.join(GOLDEN, "table1_table2_iterations.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            m, n, method, it = line.split()
            rows.append((int(m), int(n), method, float(it)))
    return rows


def pin_tables_1_2(sizes=((8000, 500), (500, 8000), (8000, 1000)), seeds=10,
                   methods=("RGDBEK", "GDBEK")):
    golden = {(m, n, meth): it for m, n, meth, it in read_table_golden()}
    for (m, n) in sizes:
        for meth in methods:
            its = []
            for seed in range(seeds):
                S = workloads.sprandn_like(m, n, 0.01, seed)
                o = oracle.Options(eta_col=0.5, eta_row=0.5, stop_rule=3, tol=1e-6,
                                   inner_tol=1e-13, max_iter=2000, seed=seed,
                                   selection=0 if meth == "RGDBEK" else 1)
                res = oracle.solve(S.A, S.b, o, n=n)
                assert res.status == 0
                its.append(res.iters)
            paper = golden[(m, n, meth)]
            mean = float(np.mean(its))
            assert abs(mean - paper) <= 0.2 * paper, (m, n, meth, mean, paper)


# --------------------------------------------------------------------------
# The two block updates of Eq. (4), one outer iteration at a time
# --------------------------------------------------------------------------
def _block_steps(D, b, blocks):
    """Run the oracle with the blocks locked and compare every step with the
    closed form z_{k+1} = z_k - A_U pinv(A_U) z_k,
    x_{k+1} = x_k + pinv(A^J)(b_J - z_{k+1,J} - A^J x_k)."""
    m, n = D.shape
    res = oracle.solve(_csr(D), b, oracle.Options(max_iter=len(blocks), stop_rule=2, tol=0.0,
                                                  inner_tol=1e-14, inner_max=2000),
                       n=n, lock=[(np.asarray(u, np.int32), np.asarray(j, np.int32))
                                  for u, j in blocks],
                       trace=True, keep_iterates=True)
    assert res.iters == len(blocks)
    z, x = b.copy(), np.zeros(n)
    for k, (U, J) in enumerate(blocks):
        AU, AJ = D[:, U], D[J, :]
        z_next = z - AU @ (np.linalg.pinv(AU, rcond=1e-12) @ z)
        x_next = x + np.linalg.pinv(AJ, rcond=1e-12) @ (b[J] - z_next[J] - AJ @ x)
        assert np.linalg.norm(res.zs[k + 1] - z_next) <= 1e-10 * max(np.linalg.norm(z_next), 1.0)
        assert np.linalg.norm(res.xs[k + 1] - x_next) <= 1e-10 * max(np.linalg.norm(x_next), 1.0)
        z, x = res.zs[k + 1], res.xs[k + 1]


def pin_block_updates():
    rng = np.random.default_rng(0)
    # uneven column and row norms: the unit scalings of the inner solves matter
    D = rng.standard_normal((40, 25)) * np.exp(rng.uniform(-2, 2, (1, 25)))
    D *= np.exp(rng.uniform(-2, 2, (40, 1)))
    b = rng.standard_normal(40)
    _block_steps(D, b, [(sorted(rng.choice(25, 6, replace=False)),
                         sorted(rng.choice(40, 10, replace=False))) for _ in range(4)])
    # a singular row block: J holds both copies of duplicated rows (the copies
    # scaled by 3, so unit scaling makes them identical rows); b is not in
    # range(A), yet the block system is consistent, since r_k = (b - z_{k+1}) -
    # A x_k lies in range(A)
    B = rng.standard_normal((15, 30))
    D = np.repeat(B, 2, axis=0)
    D[1::2] *= 3.0
    b = rng.standard_normal(30)
    J = list(range(10))
    _block_steps(D, b, [(sorted(rng.choice(30, 8, replace=False)), J),
                        (sorted(rng.choice(30, 8, replace=False)),
                         sorted(rng.choice(30, 12, replace=False)))])
    # tall row blocks (|J| > n), full rank and rank 6
    for (m, n), rank in (((30, 12), None), ((50, 30), 6)):
        D = rng.standard_normal((m, n))
        if rank is not None:
            D = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
        b = rng.standard_normal(m)
        _block_steps(D, b, [(sorted(rng.choice(n, max(2, n // 3), replace=False)),
                             sorted(rng.choice(m, min(m, n + 5), replace=False)))
                            for _ in range(3)])


ALL_PINS = [pin_philox, pin_spmv, pin_weights, pin_sample_law, pin_sample_sets, pin_greedy,
            pin_lsqr, pin_solve_min_norm, pin_one_iteration_closed_forms, pin_degenerate,
            pin_pythagoras_eq5, pin_block_updates, pin_rate_theorem]
