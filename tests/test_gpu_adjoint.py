"""rgdbek_backward (implicit adjoint of the solve) against the oracle.

Both sides compute w = A^+T g and v = A^+ w by Algorithm 1 solves (w on A^T)
and the entry gradients r_i v_j - w_i x_j (+ u_i p_j with the rank term); the
GPU's come through the C ABI.  Inner solves on both sides stop at a
normal-equation residual of 1e-12, so the two agree to about kappa * 1e-12;
the bar is 1e-8 relative to the largest entry.  The dense pseudo-inverse
gives a second, closed-form reference on the small cases.

Workloads: the Tikhonov-regularised deblur [A; 0.05 I] (A the 9-tap Gaussian
blur T (x) T of an s x s image), at s = 16 and 32 against the oracle and at
s = 256 (131072 x 65536, 5.3e6 nonzeros) on properties that hold at any size;
a sparse least-squares system; fat and rank-deficient dense matrices with the
rank term.
"""
import ctypes

import numpy as np
import pytest

import gpu_util as G
import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-12
ETA = 0.1


@pytest.fixture(scope="module")
def rg():
    return G.rg()


def _gpu_backward(rg, S, x, g, tol=TOL, eta=ETA, rank_term=False, seed=0):
    s = rg.Solver(S.m, S.n, S.row_ptr, S.col_idx, S.vals, eta_col=eta, eta_row=eta,
                  stop_rule=rg.STOP_NORMAL)
    gb, gv, status, st = s.backward(G.dev(S.b), G.dev(x), G.dev(g), tol=tol, max_iter=200000,
                                    seed=seed, rank_term=rank_term, nnz=S.nnz)
    out = G.host(gb).copy(), G.host(gv).copy(), status, st
    s.close()
    return out


def _oracle_backward(S, x, g, tol=TOL, eta=ETA, rank_term=False, seed=0):
    o = oracle.Options(eta_col=eta, eta_row=eta, stop_rule=2, tol=tol, inner_tol=1e-10,
                       max_iter=200000, seed=seed)
    return oracle.backward(S.A, S.b, x, g, o, n=S.n, rank_term=rank_term)


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("side", [16, 32])
def test_backward_deblur_matches_oracle(rg, side):
    S = workloads.deblur_regularised(side)
    x = np.linalg.lstsq(S.dense(), S.b, rcond=None)[0]
    g = x - S.x_true                              # 0.5 ||x - x_true||^2
    gb, gv, status, st = _gpu_backward(rg, S, x, g)
    assert status == rg.OK
    assert st[0].iters > 0 and st[1].iters > 0 and st[2].iters == 0 and st[3].iters == 0
    ref = _oracle_backward(S, x, g)
    assert _rel(gb, ref.grad_b) <= 1e-8
    assert _rel(gv, ref.grad_vals) <= 1e-8
    if side == 16:
        gb_d, Gd = oracle.backward_dense(S.dense(), S.b, g, rank_term=False)
        rows = np.repeat(np.arange(S.m), np.diff(S.row_ptr))
        assert _rel(gb, gb_d) <= 1e-8
        assert _rel(gv, Gd[rows, S.col_idx]) <= 1e-8


def test_backward_sparse_least_squares_matches_oracle(rg):
    S = workloads.sparse_ls(3000, 700, 20, sigma=1e-2, seed=11)
    rng = np.random.default_rng(5)
    x = oracle.solve(S.A, S.b, oracle.Options(eta_col=ETA, eta_row=ETA, stop_rule=2, tol=1e-13,
                                              max_iter=100000), n=S.n).x
    g = rng.standard_normal(S.n)
    gb, gv, status, _ = _gpu_backward(rg, S, x, g)
    assert status == rg.OK
    ref = _oracle_backward(S, x, g)
    assert _rel(gb, ref.grad_b) <= 1e-8
    assert _rel(gv, ref.grad_vals) <= 1e-8
    gx = float(g @ x)
    assert abs(float(gb @ S.b) - gx) <= 1e-8 * abs(gx)
    assert abs(float(gv @ S.vals) + gx) <= 1e-8 * abs(gx)


@pytest.mark.parametrize("shape,rank", [((15, 40), None), ((36, 24), 5)])
def test_backward_rank_term_matches_pseudo_inverse(rg, shape, rank):
    rng = np.random.default_rng(7)
    m, n = shape
    D = rng.standard_normal((m, n))
    if rank is not None:
        D = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
    b = rng.standard_normal(m)
    g = rng.standard_normal(n)
    x = np.linalg.pinv(D, rcond=1e-10) @ b
    S = workloads.from_dense(D, b)
    gb, gv, status, st = _gpu_backward(rg, S, x, g, eta=0.5, rank_term=True)
    assert status == rg.OK and all(s.iters > 0 for s in st)
    gb_d, Gd = oracle.backward_dense(D, b, g, rank_term=True, rcond=1e-10)
    rows = np.repeat(np.arange(m), np.diff(S.row_ptr))
    assert _rel(gb, gb_d) <= 1e-8
    assert _rel(gv, Gd[rows, S.col_idx]) <= 1e-8


def test_backward_grad_b_only_and_argument_errors(rg):
    import torch
    S = workloads.deblur_regularised(16)
    x = np.linalg.lstsq(S.dense(), S.b, rcond=None)[0]
    g = x - S.x_true
    s = rg.Solver(S.m, S.n, S.row_ptr, S.col_idx, S.vals, eta_col=ETA, eta_row=ETA,
                  stop_rule=rg.STOP_NORMAL)
    db, dx, dg = G.dev(S.b), G.dev(x), G.dev(g)
    gb_full, _, _, _ = s.backward(db, dx, dg, tol=TOL, max_iter=200000, seed=3)
    gb_only, gv, status, st = s.backward(db, dx, dg, tol=TOL, max_iter=200000, seed=3,
                                         want_vals=False)
    assert gv is None and status == rg.OK
    assert st[1].iters == 0
    # same seed, same solve: bit-identical
    assert np.array_equal(G.host(gb_only), G.host(gb_full))
    out = torch.empty(S.m, dtype=torch.float64, device="cuda")
    lib, h = rg._lib, s.handle
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    assert lib.rgdbek_backward(h, P(db), P(dx), P(dg), P(out), None, 1e-10, 10, 0, 2,
                               None) == rg.ERR_INVALID_ARG
    assert lib.rgdbek_backward(h, P(db), P(dx), P(dg), P(out), None, -1.0, 10, 0, 0,
                               None) == rg.ERR_INVALID_ARG
    assert lib.rgdbek_backward(h, P(db), P(dx), None, P(out), None, 1e-10, 10, 0, 0,
                               None) == rg.ERR_INVALID_ARG
    bad = G.dev(np.where(np.arange(S.n) == 3, np.nan, g))
    assert lib.rgdbek_backward(h, P(db), P(dx), P(bad), P(out), None, 1e-10, 10, 0, 0,
                               None) == rg.ERR_NONFINITE
    s.close()


def test_backward_full_size_deblur_properties(rg):
    # 256 x 256 image: [A; 0.05 I] is 131072 x 65536 with 5.3e6 nonzeros
    S = workloads.deblur_regularised(256)
    s = rg.Solver(S.m, S.n, S.row_ptr, S.col_idx, S.vals, eta_col=ETA, eta_row=ETA,
                  stop_rule=rg.STOP_NORMAL)
    res = s.solve(G.dev(S.b), tol=1e-11, max_iter=200000, seed=0)
    assert res.stats.status == rg.OK
    x = G.host(res.x).copy()
    g = x - S.x_true
    gb, gv, status, st = s.backward(G.dev(S.b), res.x, G.dev(g), tol=1e-11, max_iter=200000,
                                    seed=1, nnz=S.nnz)
    s.close()
    assert status == rg.OK
    gb, gv = G.host(gb), G.host(gv)
    # A^T w = g (w solves the consistent transposed system)
    assert np.linalg.norm(oracle.spmv_t(S.A, gb, S.n) - g) <= 1e-8 * np.linalg.norm(g)
    # x(A, t b) = t x and x(t A, b) = x / t
    gx = float(g @ x)
    assert abs(float(gb @ S.b) - gx) <= 1e-7 * abs(gx)
    assert abs(float(gv @ S.vals) + gx) <= 1e-7 * abs(gx)
    # sampled entries recomputed on the host as (b_i - (A x)_i) v_j - w_i x_j:
    # w lies in the range of [A; lam I], so w = [A v; lam v] with v = A^+ w,
    # and v is read off the last n entries of w = grad_b
    m0 = S.m - S.n
    lam = 0.05
    rows = np.repeat(np.arange(S.m), np.diff(S.row_ptr))
    r = S.b - oracle.spmv(S.A, x)
    v = gb[m0:] / lam
    rng = np.random.default_rng(9)
    e = rng.choice(S.nnz, size=20000, replace=False)
    expect = r[rows[e]] * v[S.col_idx[e]] - gb[rows[e]] * x[S.col_idx[e]]
    assert _rel(gv[e], expect) <= 1e-6


def test_autograd_function_gradients_wrt_b_lambda_and_values(rg):
    """rgdbek_lstsq under torch.autograd on [A; lam I] x = [b; 0] (16 x 16
    deblur): dL/dlam (through lam's entries of the stacked values) against
    central differences of dense lstsq solutions with h = 1e-6, dL/db and
    dL/dA against the dense pseudo-inverse gradient."""
    import torch
    side, lam0 = 16, 0.05
    S = workloads.deblur_regularised(side, lam=lam0)
    nb = S.m - S.n                                  # blur rows
    nnz_a = int(S.row_ptr[nb])
    dev = "cuda"
    rp = torch.tensor(S.row_ptr, device=dev)
    ci = torch.tensor(S.col_idx, device=dev)
    va = torch.tensor(S.vals[:nnz_a], device=dev, requires_grad=True)
    lam = torch.tensor(lam0, dtype=torch.float64, device=dev, requires_grad=True)
    bb = torch.tensor(S.b[:nb], device=dev, requires_grad=True)
    xt = torch.tensor(S.x_true, device=dev)
    vals = torch.cat([va, lam * torch.ones(S.n, dtype=torch.float64, device=dev)])
    b = torch.cat([bb, torch.zeros(S.n, dtype=torch.float64, device=dev)])
    x = rg.rgdbek_lstsq(rp, ci, vals, b, S.m, S.n, tol=1e-12, eta_col=ETA, eta_row=ETA,
                        stop_rule=rg.STOP_NORMAL)
    loss = ((x - xt) ** 2).sum()
    loss.backward()

    D = S.dense()

    def L(lmb):
        Dl = D.copy()
        Dl[nb:, :] = lmb * np.eye(S.n)
        xs = np.linalg.lstsq(Dl, S.b, rcond=None)[0]
        return float(((xs - S.x_true) ** 2).sum())

    h = 1e-6
    fd = (L(lam0 + h) - L(lam0 - h)) / (2 * h)
    assert abs(float(lam.grad) - fd) <= 1e-6 * abs(fd)
    xs = np.linalg.lstsq(D, S.b, rcond=None)[0]
    gb_d, Gd = oracle.backward_dense(D, S.b, 2 * (xs - S.x_true), rank_term=False)
    rows = np.repeat(np.arange(S.m), np.diff(S.row_ptr))
    assert _rel(G.host(bb.grad), gb_d[:nb]) <= 1e-8
    assert _rel(G.host(va.grad), Gd[rows[:nnz_a], S.col_idx[:nnz_a]]) <= 1e-8


def test_autograd_second_backward_and_handle_release(rg):
    """A second backward through the same graph (retain_graph=True) reuses the
    forward's handle and gives the same gradients; the handle is released with
    the graph (no close inside backward), and a solve that stops at its cap
    warns instead of passing silently."""
    import gc
    import warnings as W

    import torch
    S = workloads.deblur_regularised(16)
    dev = "cuda"
    rp = torch.tensor(S.row_ptr, device=dev)
    ci = torch.tensor(S.col_idx, device=dev)
    vals = torch.tensor(S.vals, device=dev, requires_grad=True)
    b = torch.tensor(S.b, device=dev, requires_grad=True)
    xt = torch.tensor(S.x_true, device=dev)
    x = rg.rgdbek_lstsq(rp, ci, vals, b, S.m, S.n, tol=1e-12, eta_col=ETA, eta_row=ETA,
                        stop_rule=rg.STOP_NORMAL)
    node = x.grad_fn
    solver = node.solver
    assert solver.handle is not None
    loss = ((x - xt) ** 2).sum()
    loss.backward(retain_graph=True)
    g1v, g1b = G.host(vals.grad).copy(), G.host(b.grad).copy()
    assert solver.handle is not None          # still usable after the first backward
    vals.grad = None
    b.grad = None
    loss.backward()
    assert np.array_equal(G.host(vals.grad), g1v)
    assert np.array_equal(G.host(b.grad), g1b)
    # the graph (and with it the handle) goes away with the last reference
    import weakref
    ref = weakref.ref(solver)
    del x, loss, node, solver
    gc.collect()
    assert ref() is None

    # an iteration cap below what the tolerance needs: a warning, not silence
    with W.catch_warnings(record=True) as caught:
        W.simplefilter("always")
        x2 = rg.rgdbek_lstsq(rp, ci, vals, b, S.m, S.n, tol=1e-14, max_iter=3,
                             eta_col=ETA, eta_row=ETA, stop_rule=rg.STOP_NORMAL)
        ((x2 - xt) ** 2).sum().backward()
    msgs = [str(w.message) for w in caught if issubclass(w.category, RuntimeWarning)]
    assert any("forward solve stopped at its cap" in m for m in msgs), msgs
    assert any("adjoint solve" in m for m in msgs), msgs
