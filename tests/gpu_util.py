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
