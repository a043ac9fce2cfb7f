"""Pins of the oracle's implicit adjoint (oracle.backward, oracle.backward_dense).

The adjoint has no printed example in the paper, so it is pinned to what the
mathematics fixes, independently of the formula it implements:
  * central finite differences of L(x) = g^T x with x = lstsq(A, b) from
    numpy (full column rank: every entry of A and b);
  * for rank-deficient A = B C, finite differences along perturbations that
    keep the rank ((B + hE) C and B (C + hF)), where the pseudo-inverse is
    differentiable; these also show that the rank term is needed;
  * the scaling identities <dL/db, b> = g^T x and <dL/dA, A> = -g^T x, which
    follow from x(A, t b) = t x and x(t A, b) = x / t at any size;
  * the iterative version (inner Algorithm 1 solves) against the dense one.
"""
import numpy as np

import oracle
import workloads

TIGHT = oracle.Options(tol=1e-14, inner_tol=1e-14, max_iter=20000, eta_col=0.5, eta_row=0.5)


def _loss_lstsq(g, D, b):
    return float(g @ np.linalg.lstsq(D, b, rcond=None)[0])


def test_dense_adjoint_matches_central_differences_full_rank():
    rng = np.random.default_rng(0)
    D = rng.standard_normal((40, 12))
    b = rng.standard_normal(40)
    g = rng.standard_normal(12)
    gb, G = oracle.backward_dense(D, b, g, rank_term=False)
    h = 1e-6
    fd = np.zeros_like(D)
    for i in range(D.shape[0]):
        for j in range(D.shape[1]):
            E = np.zeros_like(D)
            E[i, j] = h
            fd[i, j] = (_loss_lstsq(g, D + E, b) - _loss_lstsq(g, D - E, b)) / (2 * h)
    assert np.abs(fd - G).max() <= 1e-7 * np.abs(G).max()
    fdb = np.array([(_loss_lstsq(g, D, b + h * e) - _loss_lstsq(g, D, b - h * e)) / (2 * h)
                    for e in np.eye(40)])
    assert np.abs(fdb - gb).max() <= 1e-8 * np.abs(gb).max()
    # the full-column-rank case does not need the rank term: it is zero
    _, G1 = oracle.backward_dense(D, b, g, rank_term=True)
    assert np.abs(G1 - G).max() <= 1e-12 * np.abs(G).max()


def test_dense_adjoint_rank_term_on_rank_preserving_directions():
    rng = np.random.default_rng(1)
    m, n, k = 30, 16, 6
    B = rng.standard_normal((m, k))
    C = rng.standard_normal((k, n))
    D = B @ C
    b = rng.standard_normal(m)
    g = rng.standard_normal(n)

    def loss(M):
        return float(g @ (np.linalg.pinv(M, rcond=1e-10) @ b))

    _, G = oracle.backward_dense(D, b, g, rank_term=True, rcond=1e-10)
    _, G0 = oracle.backward_dense(D, b, g, rank_term=False, rcond=1e-10)
    h = 1e-6
    worst_without = 0.0
    for _ in range(4):
        E = rng.standard_normal((m, k))
        F = rng.standard_normal((k, n))
        for dA, fd in (
            (E @ C, (loss((B + h * E) @ C) - loss((B - h * E) @ C)) / (2 * h)),
            (B @ F, (loss(B @ (C + h * F)) - loss(B @ (C - h * F))) / (2 * h)),
        ):
            assert abs(np.sum(G * dA) - fd) <= 1e-6 * max(1.0, abs(fd))
            worst_without = max(worst_without, abs(np.sum(G0 * dA) - fd))
    # without the u p^T term the directional derivatives along B (C + hF) are wrong
    assert worst_without > 1e-2


def test_iterative_adjoint_matches_dense_tall_fat_and_rank_deficient():
    rng = np.random.default_rng(2)
    cases = []
    D = rng.standard_normal((50, 20))
    cases.append((D, False))                                   # tall, full column rank
    cases.append((rng.standard_normal((15, 40)), True))        # fat, full row rank
    B = rng.standard_normal((36, 5))
    cases.append((B @ rng.standard_normal((5, 24)), True))     # rank 5
    for D, rank_term in cases:
        m, n = D.shape
        b = rng.standard_normal(m)
        g = rng.standard_normal(n)
        x = np.linalg.pinv(D, rcond=1e-10) @ b
        S = workloads.from_dense(D, b)
        adj = oracle.backward(S.A, b, x, g, TIGHT, n=n, rank_term=rank_term)
        assert all(s.status == 0 for s in adj.solves)
        gb, G = oracle.backward_dense(D, b, g, rank_term=rank_term, rcond=1e-10)
        assert np.abs(adj.grad_b - gb).max() <= 1e-9 * np.abs(gb).max()
        rows = np.repeat(np.arange(m), np.diff(S.row_ptr))
        assert np.abs(adj.grad_vals - G[rows, S.col_idx]).max() <= 1e-9 * np.abs(G).max()


def test_iterative_adjoint_on_regularised_deblur_matches_differences():
    # [A; 0.05 I] for the 9-tap blur of a 16 x 16 image: 512 x 256, full column rank
    S = workloads.deblur_regularised(16)
    D = S.dense()
    rng = np.random.default_rng(3)
    x = np.linalg.lstsq(D, S.b, rcond=None)[0]
    g = x - S.x_true                         # gradient of 0.5 ||x - x_true||^2
    adj = oracle.backward(S.A, S.b, x, g, oracle.Options(tol=1e-13, inner_tol=1e-14,
                                                         eta_col=0.1, eta_row=0.1,
                                                         max_iter=20000), n=S.n)
    assert all(s.status == 0 for s in adj.solves)
    rows = np.repeat(np.arange(S.m), np.diff(S.row_ptr))
    h = 1e-6
    scale = np.abs(adj.grad_vals).max()
    for e in rng.choice(S.nnz, size=60, replace=False):
        E = np.zeros_like(D)
        E[rows[e], S.col_idx[e]] = h
        fd = (_loss_lstsq(g, D + E, S.b) - _loss_lstsq(g, D - E, S.b)) / (2 * h)
        assert abs(fd - adj.grad_vals[e]) <= 1e-6 * scale
    for i in rng.choice(S.m, size=20, replace=False):
        db = np.zeros(S.m)
        db[i] = h
        fd = (_loss_lstsq(g, D, S.b + db) - _loss_lstsq(g, D, S.b - db)) / (2 * h)
        assert abs(fd - adj.grad_b[i]) <= 1e-7 * np.abs(adj.grad_b).max()
    # scaling identities
    gx = float(g @ x)
    assert abs(float(adj.grad_b @ S.b) - gx) <= 1e-9 * abs(gx)
    assert abs(float(adj.grad_vals @ S.vals) + gx) <= 1e-9 * abs(gx)


def test_transpose_is_the_dense_transpose():
    S = workloads.sprandn_like(23, 17, density=0.2, seed=5)
    tp, ti, tv = oracle.transpose(S.A, S.n)
    T = workloads.System("t", S.n, S.m, tp, ti, tv, np.zeros(S.n), np.zeros(S.m), False)
    assert np.array_equal(T.dense(), S.dense().T)
    for j in range(S.n):
        assert np.all(np.diff(ti[tp[j]:tp[j + 1]]) > 0)
