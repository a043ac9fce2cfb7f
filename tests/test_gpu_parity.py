"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer and index results (CSC structure, sampled blocks, greedy sets) must
be bit-exact; weights computed from the same inputs must be bit-exact (both
sides divide a correctly rounded square by a norm); floating results of the
solve must agree within ||x - x_oracle|| / ||x_oracle|| <= 1e-8 (FP64 path);
sparse products within 1e-13 relative to the sum of |terms|.
"""
import numpy as np
import pytest

import gpu_util as G
import oracle
import workloads

pytestmark = pytest.mark.gpu

X_TOL = 1e-8


@pytest.fixture(scope="module")
def rg():
    return G.rg()


def random_sparse(m, n, density, seed, empty_rows=(), empty_cols=()):
    rng = np.random.default_rng(seed)
    D = rng.standard_normal((m, n)) * (rng.random((m, n)) < density)
    for i in empty_rows:
        D[i, :] = 0
    for j in empty_cols:
        D[:, j] = 0
    return D


# ---------------------------------------------------------------------------
# Set-up: CSC copy and norms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,density", [((1, 1), 1.0), ((37, 23), 0.3), ((513, 1031), 0.02),
                                           ((2000, 40), 0.9), ((64, 3000), 0.05)])
def test_csc_and_norms(rg, shape, density):
    m, n = shape
    D = random_sparse(m, n, density, seed=m + n, empty_rows=(0,) if m > 2 else (),
                      empty_cols=(n - 1,) if n > 2 else ())
    if not D.any():
        D[0, 0] = 1.5
    rp, ci, av = workloads.csr_from_dense(D)
    s = rg.Solver(m, n, rp, ci, av)
    import torch
    nnz = len(av)
    cp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    ri = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
    cv = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
    rg.rgdbek_get_csc(s.handle, cp, ri, cv)
    # CSC of A is the CSR of A^T: column-major order of the nonzeros
    ccp, cri, ccv = workloads.csr_from_dense(D.T.copy())
    assert np.array_equal(G.host(cp), ccp)
    assert np.array_equal(G.host(ri)[:nnz], cri)
    assert np.array_equal(G.host(cv)[:nnz], ccv)
    rn = torch.empty(m, dtype=torch.float64, device="cuda")
    cn = torch.empty(n, dtype=torch.float64, device="cuda")
    rg.rgdbek_get_norms(s.handle, rn, cn)
    assert np.allclose(G.host(rn), oracle.row_norms2((rp, ci, av)), rtol=1e-14, atol=0)
    assert np.allclose(G.host(cn), oracle.col_norms2((rp, ci, av), n), rtol=1e-14, atol=0)
    s.close()


# ---------------------------------------------------------------------------
# Sparse products (a1 and a5 of every iteration)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["dense_1000x200", "sparse_ragged", "sparse_ls_20000x5000"])
def test_spmv_and_transpose(rg, case):
    import torch
    if case == "dense_1000x200":
        S = workloads.dense_gaussian()
        A, m, n = S.A, S.m, S.n
    elif case == "sparse_ragged":
        D = random_sparse(777, 1234, 0.01, seed=3, empty_rows=(5, 6), empty_cols=(0, 9))
        A, (m, n) = workloads.csr_from_dense(D), D.shape
    else:
        S = workloads.sparse_ls(20000, 5000, 20, seed=4)
        A, m, n = S.A, S.m, S.n
    rng = np.random.default_rng(0)
    x = rng.standard_normal(n)
    z = rng.standard_normal(m)
    s = rg.Solver(m, n, *A)
    y = torch.empty(m, dtype=torch.float64, device="cuda")
    g = torch.empty(n, dtype=torch.float64, device="cuda")
    rg.rgdbek_spmv(s.handle, G.dev(x), y)
    rg.rgdbek_spmv_t(s.handle, G.dev(z), g)
    torch.cuda.synchronize()
    Aabs = (A[0], A[1], np.abs(A[2]))
    scale_y = oracle.spmv(Aabs, np.abs(x)) + 1e-300
    scale_g = oracle.spmv_t(Aabs, np.abs(z), n) + 1e-300
    assert np.all(np.abs(G.host(y) - oracle.spmv(A, x)) <= 1e-13 * scale_y)
    assert np.all(np.abs(G.host(g) - oracle.spmv_t(A, z, n)) <= 1e-13 * scale_g)
    s.close()


@pytest.mark.parametrize("case", ["sparse_ragged", "sparse_ls_20000x5000"])
def test_spmv_f32(rg, case):
    """The FP32 form's products on the float copy of A, against the oracle's
    FP64 products of the same float-rounded values and vectors.  Bound: each
    product a*x rounds once, each lane's Kahan sum adds O(2u), and the tree over
    at most 32 lanes adds 5 roundings, so |error| <= 8 u32 sum|a x|, u32 = 2^-24;
    the test takes 1e-6 (about 17 u32)."""
    import torch
    if case == "sparse_ragged":
        D = random_sparse(777, 1234, 0.01, seed=3, empty_rows=(5, 6), empty_cols=(0, 9))
        A, (m, n) = workloads.csr_from_dense(D), D.shape
    else:
        S = workloads.sparse_ls(20000, 5000, 20, seed=4)
        A, m, n = S.A, S.m, S.n
    rng = np.random.default_rng(1)
    x = rng.standard_normal(n).astype(np.float32)
    z = rng.standard_normal(m).astype(np.float32)
    A32 = (A[0], A[1], A[2].astype(np.float32).astype(np.float64))
    s = rg.Solver(m, n, *A)
    y = torch.empty(m, dtype=torch.float32, device="cuda")
    g = torch.empty(n, dtype=torch.float32, device="cuda")
    rg.rgdbek_spmv_f32(s.handle, 0, torch.from_numpy(x).cuda(), y)
    rg.rgdbek_spmv_f32(s.handle, 1, torch.from_numpy(z).cuda(), g)
    torch.cuda.synchronize()
    Aabs = (A32[0], A32[1], np.abs(A32[2]))
    xd, zd = x.astype(np.float64), z.astype(np.float64)
    scale_y = oracle.spmv(Aabs, np.abs(xd)) + 1e-300
    scale_g = oracle.spmv_t(Aabs, np.abs(zd), n) + 1e-300
    assert np.all(np.abs(y.cpu().numpy() - oracle.spmv(A32, xd)) <= 1e-6 * scale_y)
    assert np.all(np.abs(g.cpu().numpy() - oracle.spmv_t(A32, zd, n)) <= 1e-6 * scale_g)
    # an empty row and an empty column give exact zeros
    if case == "sparse_ragged":
        assert y.cpu().numpy()[5] == 0.0 and g.cpu().numpy()[0] == 0.0
    with pytest.raises(RuntimeError):
        rg.rgdbek_spmv_f32(s.handle, 2, torch.from_numpy(x).cuda(), y)
    s.close()


# ---------------------------------------------------------------------------
# Weights and block selection: bit-exact
# ---------------------------------------------------------------------------
def test_weights_bit_exact(rg):
    import torch
    D = random_sparse(300, 500, 0.05, seed=9, empty_rows=(3,), empty_cols=(7, 8))
    A = workloads.csr_from_dense(D)
    s = rg.Solver(300, 500, *A)
    rn = torch.empty(300, dtype=torch.float64, device="cuda")
    cn = torch.empty(500, dtype=torch.float64, device="cuda")
    rg.rgdbek_get_norms(s.handle, rn, cn)
    rng = np.random.default_rng(1)
    for which, length, norms in ((0, 500, cn), (1, 300, rn)):
        v = rng.standard_normal(length) * np.exp(rng.uniform(-30, 30, length))
        eps = torch.empty(length, dtype=torch.float64, device="cuda")
        emax = rg.rgdbek_weights(s.handle, which, G.dev(v), eps)
        e_ref, emax_ref, bad = oracle.weights(v, G.host(norms))
        assert not bad
        assert np.array_equal(G.host(eps), e_ref)
        assert emax == emax_ref
    v = np.ones(500)
    v[17] = np.nan
    eps = torch.empty(500, dtype=torch.float64, device="cuda")
    with pytest.raises(rg.RGDBEKError) as ei:
        rg.rgdbek_weights(s.handle, 0, G.dev(v), eps)
    assert ei.value.status == rg.ERR_NONFINITE
    s.close()


def _weight_cases():
    rng = np.random.default_rng(17)
    cases = []
    for length in (1, 2, 31, 32, 33, 511, 512, 513, 4097, 50000, 200000):
        e = rng.random(length) ** 3
        e[rng.random(length) < 0.25] = 0.0
        if length > 1:
            e[0] = 0.0
        if not (e > 0).any():
            e[-1] = 1.0
        cases.append((f"len{length}", e))
    e = np.exp(rng.uniform(-700, 0, 3000))
    cases.append(("wide_range", e))
    e = np.zeros(1000)
    e[999] = 2.0
    cases.append(("one_nonzero_last", e))
    cases.append(("all_zero", np.zeros(100)))
    e = np.full(777, 3.25)
    cases.append(("all_equal", e))
    return cases


@pytest.mark.parametrize("name,eps", _weight_cases(), ids=[c[0] for c in _weight_cases()])
def test_sample_bit_exact(rg, name, eps):
    import torch
    L = len(eps)
    m = max(L, 2)
    # any handle whose max(m, n) >= len can sample; a diagonal matrix
    rp = np.arange(m + 1, dtype=np.int64)
    s = rg.Solver(m, 1, rp, np.zeros(m, np.int32), np.ones(m))
    idx = torch.empty(max(L, 1), dtype=torch.int32, device="cuda")
    d_eps = G.dev(eps)
    for (seed, k, phase, frac) in ((0, 0, 0, 0.5), (123456789, 17, 1, 0.1), (2**63 + 7, 3, 0, 1.0)):
        n_draw = oracle.num_draws(frac, L)
        cnt = rg.rgdbek_sample(s.handle, d_eps, n_draw, seed, 5, k, phase, idx)
        ref = oracle.sample(eps, n_draw, seed, 5, k, phase)
        assert cnt == len(ref)
        assert np.array_equal(G.host(idx)[:cnt], ref)
    s.close()


def test_greedy_sets_bit_exact(rg):
    import torch
    rng = np.random.default_rng(2)
    L = 5000
    eps = rng.random(L) ** 2
    eps[::7] = 0.0
    rp = np.arange(L + 1, dtype=np.int64)
    s = rg.Solver(L, 1, rp, np.zeros(L, np.int32), np.ones(L),
                  selection=rg.SELECT_GREEDY, eta_col=0.5, eta_row=0.8)
    idx = torch.empty(L, dtype=torch.int32, device="cuda")
    for phase, eta in ((0, 0.5), (1, 0.8)):
        cnt = rg.rgdbek_sample(s.handle, G.dev(eps), 1, 0, 0, 0, phase, idx)
        ref = oracle.select_greedy(eps, eta)
        assert np.array_equal(G.host(idx)[:cnt], ref)
    s.close()


# ---------------------------------------------------------------------------
# Whole solves against the oracle
# ---------------------------------------------------------------------------
def _solve_both(rg, S, tol, rule, eta, seed, max_iter=5000, inner_tol=1e-13, **kw):
    s = rg.Solver(S.m, S.n, *S.A, eta_col=eta, eta_row=eta, stop_rule=rule,
                  inner_tol=inner_tol, **kw)
    res = s.solve(G.dev(S.b), tol=tol, max_iter=max_iter, seed=seed)
    x = G.host(res.x)
    ref = oracle.solve(S.A, S.b, oracle.Options(eta_col=eta, eta_row=eta, stop_rule=rule, tol=tol,
                                                inner_tol=inner_tol, max_iter=max_iter, seed=seed,
                                                selection=kw.get("selection", 0)), n=S.n)
    s.close()
    return res.stats, x, ref


def test_solve_dense_consistent(rg):
    S = workloads.dense_gaussian(1000, 200, seed=0)
    st, x, ref = _solve_both(rg, S, 1e-12, rg.STOP_REL_RES, 0.5, seed=0)
    assert st.status == rg.OK and ref.status == 0
    assert G.rel(x, ref.x) <= X_TOL
    assert G.rel(x, S.x_true) <= X_TOL
    assert st.rel_res <= 1e-12


def test_solve_sparse_least_squares(rg):
    S = workloads.sparse_ls(4000, 1000, 20, sigma=1e-2, seed=11)
    st, x, ref = _solve_both(rg, S, 1e-11, rg.STOP_NORMAL, 0.1, seed=3)
    assert st.status == rg.OK and ref.status == 0
    assert G.rel(x, ref.x) <= X_TOL
    xs = np.linalg.lstsq(S.dense(), S.b, rcond=None)[0]
    assert G.rel(x, xs) <= X_TOL


@pytest.mark.parametrize("shape", [(40, 12), (12, 40), (333, 77)])
def test_solve_min_norm_rank_deficient(rg, shape):
    rng = np.random.default_rng(sum(shape))
    m, n = shape
    D = rng.standard_normal((m, 4)) @ rng.standard_normal((4, n))
    D[:, 1] = 0.0
    b = rng.standard_normal(m)
    S = workloads.from_dense(D, b)
    st, x, ref = _solve_both(rg, S, 1e-12, rg.STOP_NORMAL, 0.5, seed=1)
    xs = np.linalg.pinv(D) @ b
    assert st.status == rg.OK
    assert G.rel(x, xs) <= X_TOL
    assert G.rel(x, ref.x) <= X_TOL


def test_greedy_mode_solve(rg):
    S = workloads.sparse_ls(3000, 800, 10, sigma=0.0, seed=2)
    st, x, ref = _solve_both(rg, S, 1e-12, rg.STOP_REL_RES, 0.5, seed=0,
                             selection=rg.SELECT_GREEDY)
    assert st.status == rg.OK and ref.status == 0
    assert G.rel(x, ref.x) <= X_TOL
    assert G.rel(x, S.x_true) <= X_TOL


def _gpu_trace(rg, S, eta, seed, iters, rule=2, inner_tol=1e-13, **opts):
    import torch
    s = rg.Solver(S.m, S.n, *S.A, eta_col=eta, eta_row=eta, stop_rule=rule, inner_tol=inner_tol,
                  **opts)
    counts = torch.zeros((iters + 1, 4), dtype=torch.int64, device="cuda")
    lists = torch.zeros(iters * (S.m + S.n) + 1, dtype=torch.int32, device="cuda")
    rg.rgdbek_set_trace(s.handle, counts, lists)
    res = s.solve(G.dev(S.b), tol=0.0, max_iter=iters, seed=seed)
    c = G.host(counts)[:iters]
    li = G.host(lists)
    out, off = [], 0
    for k in range(iters):
        nu, nj = int(c[k, 0]), int(c[k, 1])
        out.append((li[off:off + nu].copy(), li[off + nu:off + nu + nj].copy()))
        off += nu + nj
    x = G.host(res.x)
    s.close()
    return res.stats, c, out, x


def test_lockstep_against_oracle(rg):
    """Same blocks on both sides: the oracle replays the GPU's U_k, J_k."""
    S = workloads.sparse_ls(5000, 1200, 15, sigma=1e-2, seed=21)
    K = 20
    st, counts, lists, x = _gpu_trace(rg, S, 0.2, seed=9, iters=K)
    assert st.status == rg.NOT_CONVERGED and st.iters == K
    ref = oracle.solve(S.A, S.b, oracle.Options(eta_col=0.2, eta_row=0.2, stop_rule=2, tol=0.0,
                                                inner_tol=1e-13, max_iter=K, seed=9),
                       n=S.n, lock=lists, trace=True)
    assert G.rel(x, ref.x) <= 1e-10
    # LSQR step counts agree within one step
    assert np.all(np.abs(ref.counts[:, 2:] - counts[:, 2:]) <= 1)
    # the oracle's own draws in the first iterations coincide with the GPU's
    free = oracle.solve(S.A, S.b, oracle.Options(eta_col=0.2, eta_row=0.2, stop_rule=2, tol=0.0,
                                                 inner_tol=1e-13, max_iter=3, seed=9),
                        n=S.n, trace=True)
    for k in range(3):
        assert np.array_equal(free.lists[k][0], lists[k][0])
        assert np.array_equal(free.lists[k][1], lists[k][1])


def test_deterministic_and_host_api(rg):
    S = workloads.sparse_ls(6000, 1500, 12, sigma=1e-2, seed=8)
    s = rg.Solver(S.m, S.n, *S.A, eta_col=0.2, eta_row=0.2, stop_rule=rg.STOP_NORMAL)
    b = G.dev(S.b)
    r1 = s.solve(b, tol=1e-9, max_iter=2000, seed=4)
    r2 = s.solve(b, tol=1e-9, max_iter=2000, seed=4)
    x1, x2 = G.host(r1.x), G.host(r2.x)
    assert np.array_equal(x1, x2) and r1.stats.iters == r2.stats.iters
    xh = np.zeros(S.n)
    st = rg.rgdbek_solve_host(s.handle, np.ascontiguousarray(S.b), xh, 1e-9, 2000, 4)
    assert np.array_equal(xh, x1) and st.iters == r1.stats.iters
    s.close()


def test_batched_matches_single(rg):
    import torch
    systems = [workloads.sparse_ls(1000 + 300 * i, 300 + 50 * i, 8, sigma=1e-3, seed=30 + i)
               for i in range(3)]
    solvers = [rg.Solver(S.m, S.n, *S.A, eta_col=0.3, eta_row=0.3, stop_rule=rg.STOP_NORMAL)
               for S in systems]
    bs = [G.dev(S.b) for S in systems]
    xs = [torch.empty(S.n, dtype=torch.float64, device="cuda") for S in systems]
    # with the whole grid as the team, each system is solved exactly as
    # rgdbek_solve with one team (col_team = -1) would (system_id = its index)
    solvers[0].set_options(batch_team=solvers[0].info().grid)
    status, stats = rg.rgdbek_solve_batched([s.handle for s in solvers], bs, xs,
                                            [1e-10] * 3, 3000, seed=6)
    assert status == rg.OK
    for i, (S, s) in enumerate(zip(systems, solvers)):
        s.set_options(system_id=i, col_team=-1)
        single = s.solve(bs[i], tol=1e-10, max_iter=3000, seed=6)
        assert np.array_equal(G.host(single.x), G.host(xs[i]))
        assert stats[i].iters == single.stats.iters
        s.close()


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------
def test_edge_cases(rg):
    import torch
    rng = np.random.default_rng(5)
    D = rng.standard_normal((30, 8))
    S = workloads.from_dense(D, rng.standard_normal(30))
    s = rg.Solver(30, 8, *S.A, stop_rule=rg.STOP_NORMAL)
    # b = 0: no iteration, x = 0
    r = s.solve(G.dev(np.zeros(30)), tol=1e-10)
    assert r.stats.status == rg.OK and r.stats.iters == 0 and not G.host(r.x).any()
    # max_iter = 0: x_0 = 0 returned, not converged
    r = s.solve(G.dev(S.b), tol=1e-10, max_iter=0)
    assert r.stats.status == rg.NOT_CONVERGED and r.stats.iters == 0 and not G.host(r.x).any()
    # NaN / Inf in b
    bb = S.b.copy()
    bb[4] = np.nan
    r = s.solve(G.dev(bb), tol=1e-10, raise_on_error=False)
    assert r.stats.status == rg.ERR_NONFINITE
    bb[4] = np.inf
    r = s.solve(G.dev(bb), tol=1e-10, raise_on_error=False)
    assert r.stats.status == rg.ERR_NONFINITE
    # invalid options are rejected
    with pytest.raises(rg.RGDBEKError):
        s.set_options(eta_col=0.0)
    with pytest.raises(rg.RGDBEKError):
        s.set_options(eta_col=0.5, inner_max=0)
    s.set_options(eta_col=0.5, inner_max=200)
    s.close()
    # malformed CSR
    rp = np.array([0, 2, 1, 3], np.int64)
    with pytest.raises(rg.RGDBEKError) as ei:
        rg.Solver(3, 3, rp, np.array([0, 1, 2], np.int32), np.ones(3))
    assert ei.value.status == rg.ERR_BAD_CSR
    rp = np.array([0, 2, 3], np.int64)
    with pytest.raises(rg.RGDBEKError) as ei:
        rg.Solver(2, 3, rp, np.array([1, 1, 2], np.int32), np.ones(3))
    assert ei.value.status == rg.ERR_BAD_CSR
    with pytest.raises(rg.RGDBEKError) as ei:
        rg.Solver(2, 3, rp, np.array([0, 1, 5], np.int32), np.ones(3))
    assert ei.value.status == rg.ERR_BAD_CSR
    with pytest.raises(rg.RGDBEKError) as ei:
        rg.Solver(2, 3, rp, np.array([0, 1, 2], np.int32), np.array([1.0, np.inf, 2.0]))
    assert ei.value.status == rg.ERR_NONFINITE
    # all-zero matrix: both blocks empty at once; x = 0 is A^+ b
    rp = np.zeros(5, np.int64)
    s = rg.Solver(4, 3, rp, np.zeros(0, np.int32), np.zeros(0), stop_rule=rg.STOP_REL_RES)
    r = s.solve(G.dev(np.ones(4)), tol=1e-10)
    assert r.stats.status == rg.OK and not G.host(r.x).any()
    s.close()


def test_one_iteration_closed_forms(rg):
    rng = np.random.default_rng(4)
    a = rng.standard_normal((25, 1))
    b = rng.standard_normal(25)
    S = workloads.from_dense(a, b)
    s = rg.Solver(25, 1, *S.A, eta_col=0.5, eta_row=0.3, stop_rule=rg.STOP_NORMAL,
                  inner_tol=1e-14)
    r = s.solve(G.dev(b), tol=0.0, max_iter=1)
    xstar = a[:, 0] @ b / (a[:, 0] @ a[:, 0])
    assert abs(G.host(r.x)[0] - xstar) <= 1e-12 * abs(xstar)
    s.close()
    a = rng.standard_normal((1, 20))
    S = workloads.from_dense(a, np.array([1.7]))
    s = rg.Solver(1, 20, *S.A, eta_col=0.2, eta_row=0.5, inner_tol=1e-14)
    r = s.solve(G.dev(np.array([1.7])), tol=0.0, max_iter=1)
    xstar = a[0] * 1.7 / (a[0] @ a[0])
    assert G.rel(G.host(r.x), xstar) <= 1e-12
    s.close()


def test_time_budget(rg):
    S = workloads.sparse_ls(20000, 5000, 20, sigma=1e-2, seed=6)
    s = rg.Solver(S.m, S.n, *S.A, eta_col=0.1, eta_row=0.1, stop_rule=rg.STOP_NORMAL,
                  time_budget_s=1e-4)
    r = s.solve(G.dev(S.b), tol=1e-14, max_iter=100000, raise_on_error=False)
    assert r.stats.status == rg.ERR_TIMEOUT
    assert 0 <= r.stats.iters < 100000
    s.close()


def test_inconsistent_row_blocks_take_the_unscaled_solve(rg):
    """Fat least squares with every row duplicated (rank 20 of 40 rows, b not
    in the range): row blocks that hold both copies of a row are singular;
    their systems are consistent in exact arithmetic (the row residual lies in
    range(A)) but only to rounding in floating point, so LSQR may reject the
    row-scaled solve and solve the block again unscaled.  In lockstep the GPU
    makes the same decisions as the oracle (equal LSQR step counts, which
    include both attempts), and both reach pinv(A) b."""
    rng = np.random.default_rng(3)
    B = rng.standard_normal((20, 100))
    D = np.repeat(B, 2, axis=0)
    b = rng.standard_normal(40)
    S = workloads.from_dense(D, b)
    K = 10
    st, counts, lists, x = _gpu_trace(rg, S, 0.5, seed=4, iters=K)
    ref = oracle.solve(S.A, S.b, oracle.Options(eta_col=0.5, eta_row=0.5, stop_rule=2, tol=0.0,
                                                inner_tol=1e-13, max_iter=K, seed=4),
                       n=S.n, lock=lists, trace=True)
    assert G.rel(x, ref.x) <= 1e-10
    assert np.all(np.abs(ref.counts[:, 2:] - counts[:, 2:]) <= 1)
    # some row blocks hold both copies of a row (a singular block)
    assert any(len(set(j // 2 for j in J)) < len(J) for _, J in lists)
    st, x, ref = _solve_both(rg, S, 1e-12, rg.STOP_NORMAL, 0.5, seed=4)
    xs = np.linalg.pinv(D, rcond=1e-10) @ b
    assert st.status == rg.OK
    assert G.rel(x, xs) <= X_TOL
    assert G.rel(x, ref.x) <= X_TOL


def test_warm_start(rg):
    """x read as x_0: the GPU follows the oracle from the same x_0 to
    A^+ b + (I - A^+ A) x_0; from the solution it takes no iteration; the host
    entry point reads x_0 from the host buffer; a non-finite x_0 is reported."""
    import torch
    rng = np.random.default_rng(21)
    D = rng.standard_normal((30, 80))
    b = rng.standard_normal(30)
    x0 = rng.standard_normal(80)
    S = workloads.from_dense(D, b)
    Ap = np.linalg.pinv(D)
    want = Ap @ b + (np.eye(80) - Ap @ D) @ x0
    s = rg.Solver(S.m, S.n, *S.A, eta_col=0.5, eta_row=0.5, stop_rule=rg.STOP_NORMAL,
                  inner_tol=1e-13, warm_start=1)
    xd = G.dev(x0)
    res = s.solve(G.dev(b), tol=1e-12, max_iter=100000, seed=3, x=xd)
    ref = oracle.solve(S.A, b, oracle.Options(eta_col=0.5, eta_row=0.5, stop_rule=2, tol=1e-12,
                                              inner_tol=1e-13, max_iter=100000, seed=3),
                       n=S.n, x0=x0)
    assert res.stats.status == rg.OK
    assert G.rel(G.host(res.x), want) <= 1e-8
    assert G.rel(G.host(res.x), ref.x) <= 1e-8
    # from the solution: no iteration, x unchanged
    xs = G.dev(want)
    res2 = s.solve(G.dev(b), tol=1e-8, max_iter=100, seed=3, x=xs)
    assert res2.stats.iters == 0 and np.array_equal(G.host(xs), want)
    # host buffers
    xh = x0.copy()
    st = rg.rgdbek_solve_host(s.handle, b.copy(), xh, 1e-12, 100000, 3)
    assert st.status == rg.OK and G.rel(xh, want) <= 1e-8
    # non-finite x_0
    bad = x0.copy()
    bad[5] = np.inf
    st = rg.rgdbek_solve(s.handle, G.dev(b), G.dev(bad), 1e-8, 10, 0, raise_on_error=False)
    assert st.status == rg.ERR_NONFINITE
    s.close()


def test_adaptive_inner_tolerance_lockstep_and_solution(rg):
    """inner_adapt > 0: the GPU and the oracle derive the inner tolerance of
    iteration k from the same residual measure, so in lockstep their x and LSQR
    step counts agree; the free-running solve reaches the least-squares
    solution with fewer LSQR steps than at the fixed inner tolerance."""
    S = workloads.sparse_ls(5000, 1200, 15, sigma=1e-2, seed=22)
    K = 12
    st, counts, lists, x = _gpu_trace(rg, S, 0.2, seed=9, iters=K, inner_adapt=0.01)
    ref = oracle.solve(S.A, S.b, oracle.Options(eta_col=0.2, eta_row=0.2, stop_rule=2, tol=0.0,
                                                inner_tol=1e-13, inner_adapt=0.01, max_iter=K,
                                                seed=9),
                       n=S.n, lock=lists, trace=True)
    assert G.rel(x, ref.x) <= 1e-10
    assert np.all(np.abs(ref.counts[:, 2:] - counts[:, 2:]) <= 1)
    xs = np.linalg.lstsq(S.dense(), S.b, rcond=None)[0]
    steps = []
    for adapt in (0.0, 0.01):
        s = rg.Solver(S.m, S.n, *S.A, eta_col=0.2, eta_row=0.2, stop_rule=rg.STOP_NORMAL,
                      inner_tol=1e-13, inner_adapt=adapt)
        res = s.solve(G.dev(S.b), tol=1e-12, max_iter=100000, seed=9)
        s.close()
        assert res.stats.status == rg.OK
        assert G.rel(G.host(res.x), xs) <= X_TOL
        steps.append(res.stats.inner_u + res.stats.inner_j)
    assert steps[1] < 0.8 * steps[0]


def test_eta_tuner(rg):
    """rgdbek_tune_eta scores each candidate by the decrease of the stopping
    measure per second over a short probe and keeps the best: afterwards the
    handle solves exactly as a fresh handle with that eta; bad candidates and
    probe lengths are rejected with the options left as they were."""
    import ctypes
    S = workloads.sparse_ls(5000, 1200, 15, sigma=1e-2, seed=23)
    s = rg.Solver(S.m, S.n, *S.A, eta_col=0.3, eta_row=0.3, stop_rule=rg.STOP_NORMAL)
    b = G.dev(S.b)
    best, scores = s.tune_eta(b, candidates=(0.1, 0.5), probe_iters=10)
    assert best in (0.1, 0.5) and set(scores) == {0.1, 0.5}
    assert all(np.isfinite(v) and v > 0 for v in scores.values())
    assert scores[best] == max(scores.values())
    r1 = s.solve(b, tol=1e-10, max_iter=100000, seed=4)
    f = rg.Solver(S.m, S.n, *S.A, eta_col=best, eta_row=best, stop_rule=rg.STOP_NORMAL)
    r2 = f.solve(b, tol=1e-10, max_iter=100000, seed=4)
    assert r1.stats.iters == r2.stats.iters
    assert np.array_equal(G.host(r1.x), G.host(r2.x))
    f.close()
    best_d, scores_d = s.tune_eta(b, probe_iters=5)
    assert best_d in rg.ETA_CANDIDATES and len(scores_d) == len(rg.ETA_CANDIDATES)
    x = G.dev(np.zeros(S.n))
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    for cands, iters in (((0.0, 0.2), 5), ((1.5,), 5), ((0.2,), 0)):
        C = (ctypes.c_double * len(cands))(*cands)
        assert rg._lib.rgdbek_tune_eta(s.handle, P(b), P(x), C, len(cands), iters, 0, None,
                                       None) == rg.ERR_INVALID_ARG
    # a rejected call changed nothing: the handle still solves with best_d
    r3 = s.solve(b, tol=1e-10, max_iter=100000, seed=4)
    g = rg.Solver(S.m, S.n, *S.A, eta_col=best_d, eta_row=best_d, stop_rule=rg.STOP_NORMAL)
    r4 = g.solve(b, tol=1e-10, max_iter=100000, seed=4)
    assert np.array_equal(G.host(r3.x), G.host(r4.x))
    g.close()
    s.close()


def test_tuners_ignore_the_time_budget(rg):
    """A handle with a tiny time budget still tunes (the probes run their full
    length) and keeps its budget afterwards: the next solve stops on it."""
    S = workloads.sparse_ls(5000, 1200, 15, sigma=1e-2, seed=24)
    s = rg.Solver(S.m, S.n, *S.A, eta_col=0.2, eta_row=0.2, stop_rule=rg.STOP_NORMAL,
                  time_budget_s=1e-5)
    b = G.dev(S.b)
    best, scores = s.tune_eta(b, candidates=(0.1, 0.3), probe_iters=5)
    assert best in (0.1, 0.3) and all(np.isfinite(v) and v > 0 for v in scores.values())
    x = G.dev(np.zeros(S.n))
    block, ms = rg.rgdbek_tune(s.handle, b, x, probe_iters=3)
    assert block in (512, 1024) and all(v > 0 for v in ms.values())
    res = s.solve(b, tol=1e-12, max_iter=100000, seed=1, raise_on_error=False)
    assert res.stats.status == rg.ERR_TIMEOUT
    s.close()


@pytest.mark.parametrize("rule", [1, 3])
def test_adaptive_inner_tolerance_lockstep_other_rules(rg, rule):
    """The inner tolerance follows the relative residual (rule 1) or its square
    (RSE, rule 3) on both sides: over 10 lockstep iterations of a consistent
    system the GPU and the oracle take the same LSQR step counts (the
    decisions tau_k drives) and x agrees.  Under rule 1 the bar is 1e-10
    after 10 iterations.  Under the RSE rule later row solves stop after
    20-40 LSQR steps at a loose tolerance, before LSQR has converged, and
    there the Krylov recurrence amplifies rounding: two CPU builds of the
    oracle that differ only in the order of their dot-product sums drift
    apart by 1.15e-5 after 10 iterations with identical step counts
    (tests/test_oracle_rounding_drift.py).  So under rule 3 x is held to
    1e-10 after 5 iterations and to 1e-4 (ten times that CPU-to-CPU drift)
    after 10."""
    S = workloads.sprandn_like(3000, 800, 0.01, seed=25)

    def both(K):
        st, counts, lists, x = _gpu_trace(rg, S, 0.3, seed=5, iters=K, rule=rule,
                                          inner_adapt=0.1)
        ref = oracle.solve(S.A, S.b, oracle.Options(eta_col=0.3, eta_row=0.3, stop_rule=rule,
                                                    tol=0.0, inner_tol=1e-13, inner_adapt=0.1,
                                                    max_iter=K, seed=5),
                           n=S.n, lock=lists, trace=True)
        return counts, x, ref

    counts, x10, ref = both(10)
    assert np.all(np.abs(ref.counts[:, 2:] - counts[:, 2:]) <= 1)
    d10 = G.rel(x10, ref.x)
    print(f"rule {rule}: |x_gpu - x_oracle| / |x_oracle| after 10 lockstep iterations = {d10:.3e}")
    assert d10 <= (1e-10 if rule == 1 else 1e-4), d10
    _, x5, ref5 = both(5)
    assert G.rel(x5, ref5.x) <= 1e-10


def _replay(rg, blocks, g, r, rn2, cn2, eta_c, eta_r, seed, sysid=0, greedy=False):
    """Replays every iteration's selections on the host (SURVEY's bit-exact
    replay): the oracle's weights on the GPU's own g_k and r_k and the GPU's
    squared norms, then the oracle's sampler (or greedy threshold) with the
    same Philox key and counter; each block must equal the GPU's byte for
    byte."""
    for k, (U, J) in enumerate(blocks):
        ec, emax_c, bad_c = oracle.weights(g[k], cn2)
        er, emax_r, bad_r = oracle.weights(r[k], rn2)
        assert not bad_c and not bad_r
        if greedy:
            Ur = oracle.select_greedy(ec, eta_c, emax_c)
            Jr = oracle.select_greedy(er, eta_r, emax_r)
        else:
            Ur = oracle.sample(ec, oracle.num_draws(eta_c, len(ec)), seed, sysid, k, 0, emax_c)
            Jr = oracle.sample(er, oracle.num_draws(eta_r, len(er)), seed, sysid, k, 1, emax_r)
        assert Ur.dtype == U.dtype and Ur.tobytes() == U.tobytes(), f"U_{k} differs"
        assert Jr.dtype == J.dtype and Jr.tobytes() == J.tobytes(), f"J_{k} differs"


@pytest.mark.parametrize("selection", [0, 1])
def test_selection_replay_over_a_whole_run(rg, selection):
    """Every block of 20 outer iterations (not only the first few) is what the
    oracle's sampler draws when it is replayed on the GPU's own column and row
    residuals g_k = A^T z_k, r_k = b - z_{k+1} - A x_k and the same Philox
    counter (k, phase): the quantised weights, the prefix sums, the draws and
    the compaction are bit-exact on both sides.  Random (Algorithm 1) and
    greedy (GDBEK) selection."""
    S = workloads.sparse_ls(6000, 1500, 20, sigma=1e-2, seed=31)
    eta = 0.1 if selection == 0 else 0.5
    s = rg.Solver(S.m, S.n, *S.A, eta_col=eta, eta_row=eta, stop_rule=rg.STOP_NORMAL,
                  selection=selection)
    rn2, cn2 = G.gpu_norms(rg, s, S)
    st, counts, blocks, g, r, _ = G.traced_solve(rg, s, S, 20, seed=17)
    s.close()
    assert st.iters == 20 and len(blocks) == 20
    assert np.all(np.isfinite(g)) and np.all(np.isfinite(r))
    _replay(rg, blocks, g, r, rn2, cn2, eta, eta, seed=17, greedy=selection == 1)


def test_pass_lane_tuner_and_every_lane_split(rg):
    """rgdbek_tune_spmv times each lane split of the full-matrix passes and
    keeps the fastest; every split (set by hand) gives the products within
    1e-13 of the oracle's (relative to the sum of |terms|), and a solve with
    the tuned split still meets the 1e-8 bar against the oracle."""
    import ctypes
    import torch
    S = workloads.sparse_ls(20000, 5000, 20, sigma=1e-2, seed=4)
    rng = np.random.default_rng(2)
    x, z = rng.standard_normal(S.n), rng.standard_normal(S.m)
    s = rg.Solver(S.m, S.n, *S.A, eta_col=0.2, eta_row=0.2, stop_rule=rg.STOP_NORMAL)
    Aabs = (S.A[0], S.A[1], np.abs(S.A[2]))
    scale_y = oracle.spmv(Aabs, np.abs(x)) + 1e-300
    scale_g = oracle.spmv_t(Aabs, np.abs(z), S.n) + 1e-300
    y = torch.empty(S.m, dtype=torch.float64, device="cuda")
    g = torch.empty(S.n, dtype=torch.float64, device="cuda")
    for L in rg.SPMV_LANE_CANDIDATES:
        rg.rgdbek_set_pass_lanes(s.handle, L, L)
        info = s.info()
        assert (info.lanes_per_row, info.lanes_per_col) == (L, L)
        rg.rgdbek_spmv(s.handle, G.dev(x), y)
        rg.rgdbek_spmv_t(s.handle, G.dev(z), g)
        torch.cuda.synchronize()
        assert np.all(np.abs(G.host(y) - oracle.spmv(S.A, x)) <= 1e-13 * scale_y), L
        assert np.all(np.abs(G.host(g) - oracle.spmv_t(S.A, z, S.n)) <= 1e-13 * scale_g), L
    for bad in (0, 3, 64):
        assert rg._lib.rgdbek_set_pass_lanes(ctypes.c_void_p(s.handle), bad, 1) == rg.ERR_INVALID_ARG
    assert rg._lib.rgdbek_tune_spmv(ctypes.c_void_p(s.handle), 0, None, None, None) \
        == rg.ERR_INVALID_ARG
    lr, lc, us_r, us_c = rg.rgdbek_tune_spmv(s.handle, reps=5)
    assert lr in rg.SPMV_LANE_CANDIDATES and lc in rg.SPMV_LANE_CANDIDATES
    assert us_r[lr] == min(us_r.values()) and us_c[lc] == min(us_c.values())
    assert (s.info().lanes_per_row, s.info().lanes_per_col) == (lr, lc)
    res = s.solve(G.dev(S.b), tol=1e-11, max_iter=100000, seed=3)
    ref = oracle.solve(S.A, S.b, oracle.Options(eta_col=0.2, eta_row=0.2, stop_rule=2,
                                                tol=1e-11, max_iter=100000, seed=3), n=S.n)
    assert res.stats.status == rg.OK
    assert G.rel(G.host(res.x), ref.x) <= X_TOL
    s.close()
