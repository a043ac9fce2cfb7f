"""rgdbek_solve_batched: many independent systems in one persistent launch.

The grid is cut into teams of CTAs; each team solves its systems one after
another, each to its own stopping rule (per-system convergence mask).
Checks, through the C ABI:
  * every system of an uneven batch (sparse least squares of several shapes,
    regularised deblurs, a dense consistent system) reaches the oracle's
    solution within 1e-8, for several team sizes;
  * per-system tolerances and caps are honoured independently;
  * a batch of one with the whole grid as its team is bit-identical to
    rgdbek_solve; repeated batches are bit-identical;
  * the tuner returns one of its candidates and its choice is used;
  * argument errors (a handle listed twice, a team larger than the grid).
"""
import numpy as np
import pytest

import gpu_util as G
import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rg():
    return G.rg()


def _batch_systems():
    out = [workloads.sparse_ls(3000, 700, 20, sigma=1e-2, seed=31),
           workloads.sparse_ls(800, 200, 12, sigma=1e-2, seed=32),
           workloads.sparse_ls(5000, 1200, 15, sigma=0.0, seed=33),
           workloads.sparse_ls(300, 80, 10, sigma=1e-2, seed=34),
           workloads.deblur_regularised(12, seed=35),
           workloads.deblur_regularised(16, seed=36),
           workloads.dense_gaussian(400, 60, seed=37)]
    return out


@pytest.fixture(scope="module")
def systems():
    S = _batch_systems()
    refs = [oracle.solve(s.A, s.b, oracle.Options(eta_col=0.2, eta_row=0.2, stop_rule=2,
                                                  tol=1e-13, max_iter=200000), n=s.n).x
            for s in S]
    return S, refs


def _handles(rg, S, **opts):
    return [rg.Solver(s.m, s.n, s.row_ptr, s.col_idx, s.vals, eta_col=0.2, eta_row=0.2,
                      stop_rule=rg.STOP_NORMAL, **opts) for s in S]


@pytest.mark.parametrize("team", [1, 4, 19])
def test_batched_matches_oracle_for_each_system(rg, systems, team):
    import torch
    S, refs = systems
    hs = _handles(rg, S, batch_team=team)
    bs = [G.dev(s.b) for s in S]
    xs = [torch.empty(s.n, dtype=torch.float64, device="cuda") for s in S]
    status, st = rg.rgdbek_solve_batched([h.handle for h in hs], bs, xs, [1e-12] * len(S),
                                         200000, seed=5)
    assert status == rg.OK
    for i, s in enumerate(S):
        assert st[i].status == rg.OK and st[i].normal_res <= 1e-12
        assert G.rel(G.host(xs[i]), refs[i]) <= 1e-8, i
    for h in hs:
        h.close()


def test_batched_per_system_tolerances_and_caps(rg, systems):
    import torch
    S, _ = systems
    hs = _handles(rg, S, batch_team=8)
    bs = [G.dev(s.b) for s in S]
    xs = [torch.empty(s.n, dtype=torch.float64, device="cuda") for s in S]
    tols = [1e-3, 1e-6, 1e-9, 1e-12, 1e-4, 1e-10, 1e-8]
    status, st = rg.rgdbek_solve_batched([h.handle for h in hs], bs, xs, tols, 200000, seed=1)
    assert status == rg.OK
    for i in range(len(S)):
        assert st[i].normal_res <= tols[i]
    # looser tolerances stop earlier on the same system
    st_loose, st_tight = st[0].iters, None
    status, st2 = rg.rgdbek_solve_batched([h.handle for h in hs], bs, xs,
                                          [1e-12] * len(S), 200000, seed=1)
    st_tight = st2[0].iters
    assert st_loose < st_tight
    # a cap of 3 iterations: every system stops at 3 unless it converged first
    status, st3 = rg.rgdbek_solve_batched([h.handle for h in hs], bs, xs, [0.0] * len(S), 3,
                                          seed=1)
    assert status == rg.NOT_CONVERGED
    assert all(s.iters == 3 and s.status == rg.NOT_CONVERGED for s in st3)
    for h in hs:
        h.close()


def test_batch_of_one_equals_single_solve_and_is_deterministic(rg, systems):
    import torch
    S, _ = systems
    s0 = S[0]
    # the batched kernel runs one team per system: compare with the single
    # solve's one-team schedule
    h = rg.Solver(s0.m, s0.n, s0.row_ptr, s0.col_idx, s0.vals, eta_col=0.2, eta_row=0.2,
                  stop_rule=rg.STOP_NORMAL, col_team=-1)
    grid = h.info().grid
    h.set_options(batch_team=grid)
    b = G.dev(s0.b)
    single = h.solve(b, tol=1e-10, max_iter=100000, seed=7)
    x1 = torch.empty(s0.n, dtype=torch.float64, device="cuda")
    status, st = rg.rgdbek_solve_batched([h.handle], [b], [x1], [1e-10], 100000, seed=7)
    assert status == rg.OK and st[0].iters == single.stats.iters
    assert np.array_equal(G.host(x1), G.host(single.x))
    x2 = torch.empty_like(x1)
    rg.rgdbek_solve_batched([h.handle], [b], [x2], [1e-10], 100000, seed=7)
    assert np.array_equal(G.host(x1), G.host(x2))
    h.close()


def test_tuner_and_argument_errors(rg, systems):
    import torch
    S, refs = systems
    hs = _handles(rg, S)
    H = [h.handle for h in hs]
    bs = [G.dev(s.b) for s in S]
    xs = [torch.empty(s.n, dtype=torch.float64, device="cuda") for s in S]
    team, block, ms, shape_ms = rg.rgdbek_tune_batched(H, bs, xs, [1e-10] * len(S), probe_iters=2)
    assert team in rg.BATCH_TEAM_CANDIDATES and team in ms and len(ms) >= 4
    assert block in (0, 512, 1024) and set(shape_ms) == {512, 1024}
    status, st = rg.rgdbek_solve_batched(H, bs, xs, [1e-12] * len(S), 200000, seed=5)
    assert status == rg.OK
    for i in range(len(S)):
        assert G.rel(G.host(xs[i]), refs[i]) <= 1e-8
    # the same handle twice: two systems cannot share one workspace
    status, _ = rg.rgdbek_solve_batched([H[0], H[0]], bs[:1] * 2, xs[:1] * 2, [1e-8] * 2, 10)
    assert status == rg.ERR_INVALID_ARG
    hs[0].set_options(batch_team=1000)
    status, _ = rg.rgdbek_solve_batched(H[:1], bs[:1], xs[:1], [1e-8], 10)
    assert status == rg.ERR_INVALID_ARG
    for h in hs:
        h.close()


def test_blur_batch_runs_to_its_budget(rg):
    """A small instance of the batched deblurring workload (24 images of sides
    8..24): these systems are ill-conditioned, so they run a fixed budget; each
    reports its iterations and a residual below its starting value."""
    import torch
    S = workloads.blur_batch(24, 8, 24, seed=3)
    hs = [rg.Solver(s.m, s.n, s.row_ptr, s.col_idx, s.vals, eta_col=0.1, eta_row=0.1,
                    stop_rule=rg.STOP_REL_RES) for s in S]
    bs = [G.dev(s.b) for s in S]
    xs = [torch.empty(s.n, dtype=torch.float64, device="cuda") for s in S]
    status, st = rg.rgdbek_solve_batched([h.handle for h in hs], bs, xs, [1e-12] * len(S), 25)
    assert status == rg.NOT_CONVERGED
    for i, s in enumerate(S):
        assert st[i].iters == 25
        r = s.b - oracle.spmv(s.A, G.host(xs[i]))
        assert abs(np.linalg.norm(r) / np.linalg.norm(s.b) - st[i].rel_res) <= 1e-9
        assert st[i].rel_res < 1.0
    for h in hs:
        h.close()


def test_single_solve_shape_tuner(rg, systems):
    """rgdbek_tune times both solve-kernel shapes and keeps the faster; the
    solve after it still reaches the oracle's solution."""
    import torch
    S, refs = systems
    s0 = S[0]
    h = rg.Solver(s0.m, s0.n, s0.row_ptr, s0.col_idx, s0.vals, eta_col=0.2, eta_row=0.2,
                  stop_rule=rg.STOP_NORMAL)
    b = G.dev(s0.b)
    x = torch.empty(s0.n, dtype=torch.float64, device="cuda")
    block, ms = rg.rgdbek_tune(h.handle, b, x, probe_iters=3)
    assert block in (512, 1024) and ms[512] > 0 and ms[1024] > 0
    assert h.info().threads_per_block == block
    res = h.solve(b, tol=1e-12, max_iter=200000, seed=5)
    assert res.stats.status == rg.OK
    assert G.rel(G.host(res.x), refs[0]) <= 1e-8
    h.close()


def test_batched_fp32_inner_matches_oracle(rg, systems):
    """The FP32-inner instantiation of the batched kernel: full-column-rank
    systems of the batch reach the FP64 oracle's solutions within 1e-8."""
    import torch
    S, refs = systems
    pick = [0, 1, 3]                     # sparse least squares, full column rank
    hs = [rg.Solver(S[i].m, S[i].n, S[i].row_ptr, S[i].col_idx, S[i].vals, eta_col=0.2,
                    eta_row=0.2, stop_rule=rg.STOP_NORMAL, precision=rg.PRECISION_FP32_INNER,
                    batch_team=8) for i in pick]
    bs = [G.dev(S[i].b) for i in pick]
    xs = [torch.empty(S[i].n, dtype=torch.float64, device="cuda") for i in pick]
    status, st = rg.rgdbek_solve_batched([h.handle for h in hs], bs, xs, [1e-12] * len(pick),
                                         200000, seed=5)
    assert status == rg.OK
    for k, i in enumerate(pick):
        assert G.rel(G.host(xs[k]), refs[i]) <= 1e-8, i
    for h in hs:
        h.close()


def test_many_right_hand_sides_share_one_matrix(rg, systems):
    """rgdbek_create_like: four right-hand sides of one matrix, each on a
    handle that shares the base's matrix arrays, solved in one batched launch;
    the base can be destroyed first and the others keep working."""
    import torch
    S, refs = systems
    s0 = S[0]
    rng = np.random.default_rng(11)
    base = rg.Solver(s0.m, s0.n, s0.row_ptr, s0.col_idx, s0.vals, eta_col=0.2, eta_row=0.2,
                     stop_rule=rg.STOP_NORMAL)
    derived = [rg.Solver.like(base) for _ in range(3)]
    hs = [base] + derived
    B = [s0.b] + [rng.standard_normal(s0.m) for _ in range(3)]
    bs = [G.dev(b) for b in B]
    xs = [torch.empty(s0.n, dtype=torch.float64, device="cuda") for _ in hs]
    status, st = rg.rgdbek_solve_batched([h.handle for h in hs], bs, xs, [1e-12] * 4, 200000,
                                         seed=2)
    assert status == rg.OK
    o = oracle.Options(eta_col=0.2, eta_row=0.2, stop_rule=2, tol=1e-13, max_iter=200000)
    want = [oracle.solve(s0.A, b, o, n=s0.n).x for b in B]
    for k in range(4):
        assert G.rel(G.host(xs[k]), want[k]) <= 1e-8, k
    base.close()
    res = derived[1].solve(bs[2], tol=1e-12, max_iter=200000, seed=9)
    assert res.stats.status == rg.OK and G.rel(G.host(res.x), want[2]) <= 1e-8
    for h in derived:
        h.close()


def test_batched_per_system_adaptive_inner_tolerance(rg, systems):
    """Each handle brings its own options into the shared launch: every other
    system uses the adaptive inner tolerance (c = 0.1); all reach the oracle's
    solution, and the adaptive ones take no more LSQR steps in total than the
    same systems at the fixed tolerance."""
    import torch
    S, refs = systems
    hs = [rg.Solver(s.m, s.n, s.row_ptr, s.col_idx, s.vals, eta_col=0.2, eta_row=0.2,
                    stop_rule=rg.STOP_NORMAL, batch_team=4, inner_adapt=0.1 if i % 2 else 0.0)
          for i, s in enumerate(S)]
    bs = [G.dev(s.b) for s in S]
    xs = [torch.empty(s.n, dtype=torch.float64, device="cuda") for s in S]
    status, st = rg.rgdbek_solve_batched([h.handle for h in hs], bs, xs, [1e-12] * len(S),
                                         200000, seed=5)
    assert status == rg.OK
    for i in range(len(S)):
        assert st[i].status == rg.OK and st[i].normal_res <= 1e-12
        assert G.rel(G.host(xs[i]), refs[i]) <= 1e-8, i
    for h in hs:
        h.set_options(inner_adapt=0.0)
    status, st0 = rg.rgdbek_solve_batched([h.handle for h in hs], bs, xs, [1e-12] * len(S),
                                          200000, seed=5)
    assert status == rg.OK
    odd = range(1, len(S), 2)
    assert sum(st[i].inner_u + st[i].inner_j for i in odd) \
        <= sum(st0[i].inner_u + st0[i].inner_j for i in odd)
    for h in hs:
        h.close()
