"""rgdbek_sample_noalloc: the block sampler for callers that cannot allocate
device memory (their memory pool already holds the GPU, or a cudaMalloc /
cudaFree synchronisation is not acceptable where they draw a block).

It must return exactly the block that rgdbek_sample (which draws from a
handle's allocated workspace) returns for the same weights and Philox
counter, and exactly the oracle's own draw on those weights, on consecutive
calls that share its static scratch array.  Indices and counts are integers,
so the comparisons are exact.  The special results are checked too: -1 for a
NaN or negative weight, an empty block (idx untouched) for all-zero weights,
and a valid call after them still matches, so no stale marks survive in the
shared array.  This file is named to be collected last; it builds the library
itself, so it also runs alone.
"""
import ctypes

import numpy as np
import pytest

import gpu_util as G
import oracle

pytestmark = pytest.mark.gpu


def _reference_block(rg, eps, s, seed, sysid, k, phase):
    import torch
    L = len(eps)
    rp = np.arange(L + 1, dtype=np.int64)
    solver = rg.Solver(L, 1, rp, np.zeros(L, np.int32), np.ones(L))
    idx = torch.empty(L, dtype=torch.int32, device="cuda")
    cnt = rg.rgdbek_sample(solver.handle, G.dev(eps), s, seed, sysid, k, phase, idx)
    out = G.host(idx)[:cnt].copy()
    solver.close()
    return out


def _noalloc(rg, eps, s, seed, sysid, k, phase, fill=-7):
    """One call through the C ABI; returns (status, count, idx on the host)."""
    import torch
    d_eps = G.dev(eps)
    idx = torch.full((len(eps),), fill, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = rg._lib.rgdbek_sample_noalloc(
        ctypes.c_void_p(d_eps.data_ptr()), len(eps), s, seed, sysid, k, phase,
        ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(count.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, int(G.host(count)[0]), G.host(idx).copy()


def _cases():
    rng = np.random.default_rng(123)
    e1 = rng.random(200000) ** 3
    e1[rng.random(200000) < 0.3] = 0.0
    e2 = rng.random(33333) ** 2
    e2[::5] = 0.0
    return [(e1, 20000, 7, 3, 11, 1),          # rows of the benchmark system
            (e2, 5000, 2**63 + 9, 0, 2, 0)]     # shorter, ragged length


def test_sample_noalloc_matches_rgdbek_sample_and_oracle_on_consecutive_calls():
    rg = G.rg()
    for eps, s, seed, sysid, k, phase in _cases():
        st, n, idx = _noalloc(rg, eps, s, seed, sysid, k, phase)
        assert st == rg.OK
        ref = _reference_block(rg, eps, s, seed, sysid, k, phase)
        orc = oracle.sample(eps, s, seed, sysid, k, phase)
        assert n == len(ref) == len(orc)
        assert np.array_equal(idx[:n], ref)
        assert np.array_equal(idx[:n], orc)


def test_sample_noalloc_special_results_leave_no_stale_state():
    rg = G.rg()
    rng = np.random.default_rng(7)
    eps = rng.random(50000)
    # a NaN weight: count -1
    bad = eps.copy()
    bad[12345] = np.nan
    st, n, _ = _noalloc(rg, bad, 4000, 1, 0, 0, 0)
    assert st == rg.OK and n == -1
    # a negative weight: count -1
    neg = eps.copy()
    neg[7] = -1.0
    st, n, _ = _noalloc(rg, neg, 4000, 1, 0, 0, 0)
    assert st == rg.OK and n == -1
    # all-zero weights: an empty block, idx untouched
    st, n, idx = _noalloc(rg, np.zeros(40000), 4000, 1, 0, 0, 1, fill=-3)
    assert st == rg.OK and n == 0
    assert np.all(idx == -3)
    # a valid call after those still draws exactly the oracle's block
    st, n, idx = _noalloc(rg, eps, 4000, 9, 1, 3, 1)
    orc = oracle.sample(eps, 4000, 9, 1, 3, 1)
    assert st == rg.OK and n == len(orc)
    assert np.array_equal(idx[:n], orc)


def test_sample_noalloc_rejects_sizes_beyond_its_limits():
    import torch
    rg = G.rg()
    max_len = 262144  # RGDBEK_NOALLOC_MAX_LEN in include/rgdbek.h
    eps = torch.ones(max_len + 1, dtype=torch.float64, device="cuda")
    idx = torch.empty(max_len + 1, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = rg._lib.rgdbek_sample_noalloc(
        ctypes.c_void_p(eps.data_ptr()), max_len + 1, 10, 0, 0, 0, 0,
        ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(count.data_ptr()), None)
    assert st == rg.ERR_INVALID_ARG
    # more draws than RGDBEK_MAX_DRAWS_PER_ENTRY (16) per weight
    st = rg._lib.rgdbek_sample_noalloc(
        ctypes.c_void_p(eps.data_ptr()), 1000, 16 * 1000 + 1, 0, 0, 0, 0,
        ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(count.data_ptr()), None)
    assert st == rg.ERR_INVALID_ARG
