"""The two-team schedule (option col_team).

In Algorithm 1 the column step of iteration k maps z_k to z_{k+1} from z_k
alone, so a team of CTAs can run it one iteration ahead while the other CTAs
run the row step of iteration k.  The schedule computes the iterates of
Algorithm 1 from the same inputs as the one-team schedule; only the partition
of the reductions over CTAs changes (rounding level).  Checked here for every
team size: the solution against the FP64 oracle (1e-8), every block of a run
bit-exact against the oracle's sampler replayed on the GPU's own residuals,
bit-for-bit repeatability, and the exits (tolerance reached at x_0, iteration
cap, warm start, non-finite input, time budget) against the one-team schedule.
"""
import numpy as np
import pytest

import gpu_util as G
import oracle
import workloads
from test_gpu_parity import _replay

pytestmark = pytest.mark.gpu

X_TOL = 1e-8


@pytest.fixture(scope="module")
def rg():
    return G.rg()


@pytest.fixture(scope="module")
def system():
    S = workloads.sparse_ls(6000, 1500, 12, sigma=1e-2, seed=8)
    ref = oracle.solve(S.A, S.b, oracle.Options(eta_col=0.2, eta_row=0.2, stop_rule=2, tol=1e-10,
                                                max_iter=5000, seed=4), n=S.n)
    return S, ref


def _solver(rg, S, col_team, **kw):
    opts = dict(eta_col=0.2, eta_row=0.2, stop_rule=rg.STOP_NORMAL)
    opts.update(kw)
    return rg.Solver(S.m, S.n, *S.A, col_team=col_team, **opts)


@pytest.mark.parametrize("col_team", [1, 2, 7, 19, 0, 1000])
def test_team_sizes_against_the_oracle(rg, system, col_team):
    S, ref = system
    s = _solver(rg, S, col_team)
    grid = s.info().grid
    want = {0: grid // 4, 1000: grid // 2}.get(col_team, col_team)
    assert s.info().col_team == want
    b = G.dev(S.b)
    r1 = s.solve(b, tol=1e-10, max_iter=5000, seed=4)
    assert r1.stats.status == rg.OK and ref.status == 0
    assert r1.stats.normal_res <= 1e-10
    assert G.rel(G.host(r1.x), ref.x) <= X_TOL
    assert abs(int(r1.stats.iters) - int(ref.iters)) <= 2
    # the same team size repeats bit for bit
    r2 = s.solve(b, tol=1e-10, max_iter=5000, seed=4)
    assert np.array_equal(G.host(r1.x), G.host(r2.x))
    assert (r1.stats.iters, r1.stats.inner_u, r1.stats.inner_j, r1.stats.sum_nu,
            r1.stats.sum_nj) == (r2.stats.iters, r2.stats.inner_u, r2.stats.inner_j,
                                 r2.stats.sum_nu, r2.stats.sum_nj)
    s.close()


@pytest.mark.parametrize("m,n,two", [(4000, 1000, True), (6000, 1000, True), (3000, 1000, False),
                                      (2000, 2000, False), (1000, 3000, False)])
def test_automatic_choice_follows_the_shape(rg, m, n, two):
    # two teams (a quarter of the grid on the column steps) only where the row
    # step dominates: at least four rows per column; one team otherwise
    S = workloads.sparse_ls(m, n, 8, sigma=1e-2, seed=3)
    s = rg.Solver(S.m, S.n, *S.A, eta_col=0.2, eta_row=0.2, stop_rule=rg.STOP_NORMAL)
    grid = s.info().grid
    assert s.info().col_team == (grid // 4 if two else 0)
    if m >= 3 * n:
        # tall shapes are well conditioned: either schedule meets the oracle
        # (square and fat random sparse systems converge too slowly to test here)
        ref = oracle.solve(S.A, S.b, oracle.Options(eta_col=0.2, eta_row=0.2, stop_rule=2,
                                                    tol=1e-10, max_iter=5000, seed=6), n=S.n)
        r = s.solve(G.dev(S.b), tol=1e-10, max_iter=5000, seed=6)
        assert r.stats.status == rg.OK and ref.status == 0
        assert G.rel(G.host(r.x), ref.x) <= X_TOL
    s.close()


@pytest.mark.parametrize("col_team", [3, 29])
def test_blocks_replayed_bit_exactly(rg, col_team):
    """Every block of 20 iterations under two teams is the oracle's draw on the
    GPU's own g_k = A^T z_k (formed by the column team) and r_k = b - z_{k+1}
    - A x_k (formed by the row team)."""
    S = workloads.sparse_ls(6000, 1500, 20, sigma=1e-2, seed=31)
    s = _solver(rg, S, col_team, eta_col=0.1, eta_row=0.1)
    assert s.info().col_team == col_team
    rn2, cn2 = G.gpu_norms(rg, s, S)
    st, counts, blocks, g, r, _ = G.traced_solve(rg, s, S, 20, seed=17)
    s.close()
    assert st.iters == 20 and len(blocks) == 20
    assert np.all(np.isfinite(g)) and np.all(np.isfinite(r))
    assert np.all(counts[:, 0] > 0) and np.all(counts[:, 1] > 0)
    _replay(rg, blocks, g, r, rn2, cn2, 0.1, 0.1, seed=17, greedy=False)


def test_counters_match_one_team_in_lockstep(rg):
    """With the oracle's blocks replayed in lockstep, both schedules reach the
    oracle's x_K; their per-iteration block sizes and LSQR step counts agree
    with the oracle's (blocks exactly, steps within one)."""
    S = workloads.sparse_ls(5000, 1200, 15, sigma=1e-2, seed=21)
    K = 12
    for col_team in (-1, 19):
        s = _solver(rg, S, col_team)
        st, counts, blocks, _, _, x = G.traced_solve(rg, s, S, K, seed=9, vectors=False)
        s.close()
        assert st.status == rg.NOT_CONVERGED and st.iters == K
        ref = oracle.solve(S.A, S.b, oracle.Options(eta_col=0.2, eta_row=0.2, stop_rule=2,
                                                    tol=0.0, inner_tol=1e-10, max_iter=K, seed=9),
                           n=S.n, lock=blocks, trace=True)
        assert G.rel(x, ref.x) <= 1e-10
        assert np.array_equal(ref.counts[:, :2], counts[:, :2])
        assert np.all(np.abs(ref.counts[:, 2:] - counts[:, 2:]) <= 1)
        assert st.sum_nu == counts[:, 0].sum() and st.sum_nj == counts[:, 1].sum()
        assert st.inner_u == counts[:, 2].sum() and st.inner_j == counts[:, 3].sum()


@pytest.mark.parametrize("max_iter", [0, 1, 2, 5])
def test_iteration_cap(rg, system, max_iter):
    """At the cap both schedules return x_K with NOT_CONVERGED after exactly K
    iterations, and x_K agrees (the same blocks, rounding-level sums)."""
    S, _ = system
    xs = []
    for col_team in (-1, 19):
        s = _solver(rg, S, col_team)
        res = s.solve(G.dev(S.b), tol=1e-14, max_iter=max_iter, seed=2, raise_on_error=False)
        assert res.stats.status == rg.NOT_CONVERGED and res.stats.iters == max_iter
        xs.append(G.host(res.x))
        s.close()
    if max_iter == 0:
        assert not np.any(xs[0]) and not np.any(xs[1])
    else:
        assert G.rel(xs[1], xs[0]) <= 1e-10


def test_exits_at_x0_warm_start_and_errors(rg, system):
    import torch
    S, ref = system
    s = _solver(rg, S, 19)
    # b = 0: x_0 = 0 already satisfies the rule, no iteration runs
    res = s.solve(G.dev(np.zeros(S.m)), tol=1e-10, max_iter=100, seed=1)
    assert res.stats.status == rg.OK and res.stats.iters == 0 and not np.any(G.host(res.x))
    # warm start at the solution: the test of x_0 holds
    s.set_options(warm_start=1)
    x0 = G.dev(ref.x.copy())
    res = s.solve(G.dev(S.b), tol=1e-6, max_iter=100, seed=1, x=x0)
    assert res.stats.status == rg.OK and res.stats.iters == 0
    assert np.array_equal(G.host(res.x), ref.x)
    # warm start from a perturbed solution converges to the same limit
    x0 = G.dev(ref.x + 1e-3 * np.random.default_rng(0).standard_normal(S.n))
    res = s.solve(G.dev(S.b), tol=1e-10, max_iter=5000, seed=1, x=x0)
    assert res.stats.status == rg.OK and res.stats.normal_res <= 1e-10
    s.set_options(warm_start=0)
    # a non-finite right-hand side
    bad = S.b.copy()
    bad[17] = np.nan
    res = s.solve(G.dev(bad), tol=1e-10, max_iter=100, seed=1, raise_on_error=False)
    assert res.stats.status == rg.ERR_NONFINITE
    # a time budget of 100 us ends the solve between iterations, and the handle
    # solves normally afterwards
    s.set_options(time_budget_s=1e-4)
    res = s.solve(G.dev(S.b), tol=1e-14, max_iter=100000, seed=1, raise_on_error=False)
    assert res.stats.status == rg.ERR_TIMEOUT and res.stats.iters < 100000
    s.set_options(time_budget_s=0.0)
    res = s.solve(G.dev(S.b), tol=1e-10, max_iter=5000, seed=4)
    assert res.stats.status == rg.OK and G.rel(G.host(res.x), ref.x) <= X_TOL
    torch.cuda.synchronize()
    s.close()


def test_fp32_form_and_greedy_under_two_teams(rg, system):
    S, ref = system
    s = _solver(rg, S, 19, precision=rg.PRECISION_FP32_INNER)
    res = s.solve(G.dev(S.b), tol=1e-10, max_iter=5000, seed=4)
    assert res.stats.status == rg.OK and res.stats.normal_res <= 1e-10
    assert G.rel(G.host(res.x), ref.x) <= X_TOL
    s.close()
    T = workloads.sparse_ls(3000, 800, 10, sigma=0.0, seed=2)
    s = _solver(rg, T, 19, eta_col=0.5, eta_row=0.5, selection=rg.SELECT_GREEDY,
                stop_rule=rg.STOP_REL_RES)
    res = s.solve(G.dev(T.b), tol=1e-12, max_iter=5000, seed=0)
    g = oracle.solve(T.A, T.b, oracle.Options(eta_col=0.5, eta_row=0.5, stop_rule=1, tol=1e-12,
                                              max_iter=5000, seed=0, selection=1), n=T.n)
    assert res.stats.status == rg.OK and g.status == 0
    assert G.rel(G.host(res.x), g.x) <= X_TOL
    s.close()


def test_team_tuner(rg, system):
    """rgdbek_tune_teams times one team and column teams of 2/16 .. 5/16 of
    the grid and keeps the fastest; the tuned handle still meets the bar."""
    S, ref = system
    s = _solver(rg, S, 0)
    grid = s.info().grid
    b = G.dev(S.b)
    best, ms = s.tune_teams(b, probe_iters=8)
    cands = [-1] + [min(max(((c + 1) * grid + 8) // 16, 1), grid // 2) for c in range(1, 5)]
    assert len(ms) == rg.COL_TEAM_CANDIDATES and all(v > 0 for v in ms)
    assert best == cands[int(np.argmin(ms))]
    assert s.info().col_team == max(best, 0)
    res = s.solve(b, tol=1e-10, max_iter=5000, seed=4)
    assert res.stats.status == rg.OK and G.rel(G.host(res.x), ref.x) <= X_TOL
    s.close()
