"""The benchmark system at full size (200000 x 50000, 20 nonzeros per row,
b = A x* + e), solved with the launch configuration and options bench.py
times (default grid and block, eta = 0.1, normal-equation stopping rule).

A full oracle solve at this size takes about half a minute, so parity is
checked on what the oracle computes quickly:
  * the first outer iterations: the blocks U_k, J_k drawn by the GPU are
    bit-for-bit the oracle's own draws, and the oracle replaying the GPU's
    blocks reaches the same x_k (relative difference <= 1e-8, the FP64 bound);
  * the converged solution: its normal-equation and relative residuals,
    recomputed on the host with the oracle's sparse products, agree with the
    GPU's reported values and meet the tolerance.
"""
import numpy as np
import pytest

import gpu_util as G
import oracle
import workloads

pytestmark = pytest.mark.gpu

ETA = 0.1
TOL = 1e-8


@pytest.fixture(scope="module")
def system():
    return workloads.sparse_ls(200000, 50000, 20, sigma=1e-2, seed=1)


@pytest.fixture(scope="module")
def rg():
    return G.rg()


def _solver(rg, S):
    return rg.Solver(S.m, S.n, S.row_ptr, S.col_idx, S.vals, eta_col=ETA, eta_row=ETA,
                     stop_rule=rg.STOP_NORMAL)


def test_fullsize_first_iterations_match_oracle(rg, system):
    import torch
    S = system
    K = 2
    s = _solver(rg, S)
    counts = torch.zeros((K + 1, 4), dtype=torch.int64, device="cuda")
    lists = torch.zeros(K * (S.m + S.n) + 1, dtype=torch.int32, device="cuda")
    rg.rgdbek_set_trace(s.handle, counts, lists)
    res = s.solve(G.dev(S.b), tol=0.0, max_iter=K, seed=0)
    assert res.stats.status == rg.NOT_CONVERGED and res.stats.iters == K
    c = G.host(counts)[:K]
    li = G.host(lists)
    gpu_lists, off = [], 0
    for k in range(K):
        nu, nj = int(c[k, 0]), int(c[k, 1])
        gpu_lists.append((li[off:off + nu], li[off + nu:off + nu + nj]))
        off += nu + nj
    x_gpu = G.host(res.x)
    s.close()
    opts = oracle.Options(eta_col=ETA, eta_row=ETA, stop_rule=2, tol=0.0, inner_tol=1e-10,
                          max_iter=K, seed=0)
    free = oracle.solve(S.A, S.b, opts, n=S.n, trace=True)
    for k in range(K):
        assert np.array_equal(free.lists[k][0], gpu_lists[k][0]), f"U_{k} differs"
        assert np.array_equal(free.lists[k][1], gpu_lists[k][1]), f"J_{k} differs"
    assert G.rel(x_gpu, free.x) <= 1e-8


def test_fullsize_converged_solution_properties(rg, system):
    S = system
    s = _solver(rg, S)
    res = s.solve(G.dev(S.b), tol=TOL, max_iter=100000, seed=0)
    st = res.stats
    x = G.host(res.x)
    s.close()
    assert st.status == rg.OK
    t = S.b - oracle.spmv(S.A, x)
    h = oracle.spmv_t(S.A, t, S.n)
    atb = oracle.spmv_t(S.A, S.b, S.n)
    normal = np.linalg.norm(h) / np.linalg.norm(atb)
    rel = np.linalg.norm(t) / np.linalg.norm(S.b)
    assert normal <= TOL * (1 + 1e-6)
    assert abs(normal - st.normal_res) <= 1e-6 * normal
    assert abs(rel - st.rel_res) <= 1e-9 * rel
    # the noise e ~ N(0, 1e-4) bounds the optimal relative residual from below
    assert 1e-4 < rel < 1e-2
