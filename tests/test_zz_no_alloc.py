"""rgdbek_sample_noalloc: the block sampler for callers that cannot allocate
device memory (their memory pool already holds the GPU, or a cudaMalloc /
cudaFree synchronisation is not acceptable where they draw a block).

It must return exactly the block that rgdbek_sample (which draws from a
handle's allocated workspace) returns for the same weights and Philox
counter, on consecutive calls that share its static scratch array.  Indices
and counts are integers, so the comparison is exact.  This file is named to
be collected last; it builds the library itself, so it also runs alone.
"""
import ctypes

import numpy as np
import pytest

import gpu_util as G

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


def test_sample_noalloc_matches_rgdbek_sample_on_consecutive_calls():
    import torch
    rg = G.rg()
    rng = np.random.default_rng(123)
    cases = []
    e1 = rng.random(200000) ** 3
    e1[rng.random(200000) < 0.3] = 0.0
    cases.append((e1, 20000, 7, 3, 11, 1))          # rows of the benchmark system
    e2 = rng.random(33333) ** 2
    e2[::5] = 0.0
    cases.append((e2, 5000, 2**63 + 9, 0, 2, 0))     # shorter, ragged length
    for eps, s, seed, sysid, k, phase in cases:
        d_eps = G.dev(eps)
        idx = torch.full((len(eps),), -7, dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        # through the C ABI directly
        st = rg._lib.rgdbek_sample_noalloc(
            ctypes.c_void_p(d_eps.data_ptr()), len(eps), s, seed, sysid, k, phase,
            ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(count.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == rg.OK
        torch.cuda.synchronize()
        n = int(G.host(count)[0])
        ref = _reference_block(rg, eps, s, seed, sysid, k, phase)
        assert n == len(ref)
        assert np.array_equal(G.host(idx)[:n], ref)


def test_sample_noalloc_rejects_lengths_beyond_its_scratch():
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
