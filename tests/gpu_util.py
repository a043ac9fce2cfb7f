"""Helpers for the GPU tests: build/load the CUDA library, move arrays."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def build_library():
    path = os.path.join(ROOT, "paper_2509_19267_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("_rgdbek_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


def rg():
    build_library()
    import paper_2509_19267_gb300 as m
    return m


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def traced_solve(rg, solver, S, iters, seed, tol=0.0, vectors=True):
    """Run `iters` outer iterations (or to tol) on an existing Solver with the
    block trace and, if asked, the per-iteration vectors g_k = A^T z_k and
    r_k recorded.  Returns (stats, counts [K, 4], [(U_k, J_k)], g [K, n],
    r [K, m], x) as host arrays."""
    import torch
    K = iters
    counts = torch.zeros((K + 1, 4), dtype=torch.int64, device="cuda")
    lists = torch.zeros(K * (S.m + S.n) + 1, dtype=torch.int32, device="cuda")
    rg.rgdbek_set_trace(solver.handle, counts, lists)
    g = r = None
    if vectors:
        g = torch.full((K, S.n), float("nan"), dtype=torch.float64, device="cuda")
        r = torch.full((K, S.m), float("nan"), dtype=torch.float64, device="cuda")
        rg.rgdbek_set_trace_vectors(solver.handle, g, r)
    res = solver.solve(dev(S.b), tol=tol, max_iter=K, seed=seed)
    rg.rgdbek_set_trace(solver.handle, None, None)
    rg.rgdbek_set_trace_vectors(solver.handle, None, None)
    n_it = int(res.stats.iters)
    c = host(counts)[:n_it]
    li = host(lists)
    blocks, off = [], 0
    for k in range(n_it):
        nu, nj = int(c[k, 0]), int(c[k, 1])
        blocks.append((li[off:off + nu].copy(), li[off + nu:off + nu + nj].copy()))
        off += nu + nj
    return (res.stats, c, blocks, host(g)[:n_it].copy() if g is not None else None,
            host(r)[:n_it].copy() if r is not None else None, host(res.x).copy())


def gpu_norms(rg, solver, S):
    import torch
    rn = torch.empty(S.m, dtype=torch.float64, device="cuda")
    cn = torch.empty(S.n, dtype=torch.float64, device="cuda")
    rg.rgdbek_get_norms(solver.handle, rn, cn)
    return host(rn).copy(), host(cn).copy()
