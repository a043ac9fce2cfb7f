"""GB300 (sm_103a) RGDBEK solver: thin Python binding of the C-ABI library.

RGDBEK (arXiv 2509.19267) solves A x = b, consistent or least squares, with
randomized column and row blocks drawn from residual-derived probabilities
(Algorithm 1).  All arithmetic runs in the CUDA kernels of ``librgdbek.so``;
this module only marshals arguments (torch tensors for device memory and
streams) to the functions declared in ``include/rgdbek.h``, under the same
names.  There is no CPU fallback: importing fails if the library is missing.

Entry points (each a function of the same name as in the header):
  rgdbek_create / rgdbek_destroy / rgdbek_set_options / rgdbek_get_info
  rgdbek_solve, rgdbek_solve_host      one solve (device or host buffers)
  rgdbek_solve_batched                 many systems in one persistent launch
  rgdbek_tune, rgdbek_tune_batched     measured choice of kernel shape / team
  rgdbek_tune_teams                    measured choice of the two-team split
  rgdbek_tune_eta                      measured choice of the block fraction eta
  rgdbek_backward                      implicit adjoint (dL/db, dL/dA)
  rgdbek_spmv, rgdbek_spmv_t, rgdbek_weights, rgdbek_sample,
  rgdbek_sample_noalloc, rgdbek_set_trace, rgdbek_get_norms, rgdbek_get_csc
and two conveniences built on them: ``Solver`` (owns a handle) and
``rgdbek_lstsq`` (the solve as a torch.autograd.Function).

Example:
    s = Solver(m, n, row_ptr, col_idx, vals, eta_col=0.1, eta_row=0.1,
               stop_rule=STOP_NORMAL)
    res = s.solve(b_cuda, tol=1e-8)      # res.x (cuda tensor), res.stats
    gb, gv, status, st = s.backward(b_cuda, res.x, grad_x)
"""
from __future__ import annotations

import ctypes
import os
import warnings
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librgdbek.so")

OK = 0
NOT_CONVERGED = 1
ERR_INVALID_ARG = -1
ERR_NONFINITE = -2
ERR_CUDA = -3
ERR_OOM = -4
ERR_TIMEOUT = -5
ERR_BAD_CSR = -6

SELECT_RANDOM = 0
SELECT_GREEDY = 1
STOP_AUTO = 0
STOP_REL_RES = 1
STOP_NORMAL = 2
STOP_RSE = 3
PHASE_NAMES = ("setup", "col_pass", "col_select", "col_extract", "col_lsqr", "z_update",
               "row_select", "row_extract", "row_lsqr", "residual_pass", "refine")
PRECISION_FP64 = 0
PRECISION_FP32_INNER = 1          # FP32 inner RGDBEK inside FP64 iterative refinement
FP32_INNER_TOL = 1e-6
FP32_REFINE_TOL_MIN = 1e-5

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_int = ctypes.c_int
_dbl = ctypes.c_double
_ptr = ctypes.c_void_p


class rgdbek_options(ctypes.Structure):
    _fields_ = [
        ("eta_col", _dbl), ("eta_row", _dbl), ("selection", _int), ("inner_tol", _dbl),
        ("inner_max", _int), ("stop_rule", _int), ("time_budget_s", _dbl), ("system_id", _u64),
        ("blocks_per_sm", _int), ("threads_per_block", _int), ("precision", _int),
        ("batch_team", _int), ("warm_start", _int), ("inner_adapt", _dbl),
        ("col_team", _int), ("smem_per_cta", _int),
    ]


class rgdbek_stats(ctypes.Structure):
    _fields_ = [
        ("iters", _i64), ("inner_u", _i64), ("inner_j", _i64), ("sum_nu", _i64), ("sum_nj", _i64),
        ("sum_nnz_u", _i64), ("sum_nnz_j", _i64), ("lsqr_nnz_u", _i64), ("lsqr_nnz_j", _i64),
        ("lsqr_n_u", _i64), ("lsqr_n_j", _i64), ("rel_res", _dbl), ("normal_res", _dbl),
        ("rse", _dbl), ("status", _int), ("phase_ms", _dbl * 11), ("refinements", _i64),
    ]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["phase_ms"] = dict(zip(PHASE_NAMES, list(self.phase_ms)))
        return d


class rgdbek_info_t(ctypes.Structure):
    _fields_ = [
        ("m", _i64), ("n", _i64), ("nnz", _i64), ("grid", _int), ("threads_per_block", _int),
        ("lanes_per_row", _int), ("lanes_per_col", _int), ("num_sms", _int),
        ("device_bytes", _i64), ("col_team", _int), ("smem_per_cta", _int),
    ]


# (name, restype, argtypes) of every function declared in include/rgdbek.h
SIGNATURES = [
    ("rgdbek_default_options", None, [ctypes.POINTER(rgdbek_options)]),
    ("rgdbek_create", _int, [ctypes.POINTER(_ptr), _i64, _i64, _i64, _ptr, _ptr, _ptr, _int,
                             ctypes.POINTER(rgdbek_options), _ptr]),
    ("rgdbek_destroy", None, [_ptr]),
    ("rgdbek_create_like", _int, [_ptr, ctypes.POINTER(rgdbek_options), _ptr,
                                  ctypes.POINTER(_ptr)]),
    ("rgdbek_set_options", _int, [_ptr, ctypes.POINTER(rgdbek_options)]),
    ("rgdbek_set_stream", _int, [_ptr, _ptr]),
    ("rgdbek_get_info", _int, [_ptr, ctypes.POINTER(rgdbek_info_t)]),
    ("rgdbek_solve", _int, [_ptr, _ptr, _ptr, _dbl, _i64, _u64, ctypes.POINTER(rgdbek_stats)]),
    ("rgdbek_solve_host", _int, [_ptr, _ptr, _ptr, _dbl, _i64, _u64,
                                 ctypes.POINTER(rgdbek_stats)]),
    ("rgdbek_solve_batched", _int, [_int, _ptr, _ptr, _ptr, _ptr, _i64, _u64,
                                    ctypes.POINTER(rgdbek_stats)]),
    ("rgdbek_tune_batched", _int, [_int, _ptr, _ptr, _ptr, _ptr, _i64, _u64,
                                    ctypes.POINTER(_int), ctypes.POINTER(_int),
                                    ctypes.POINTER(_dbl)]),
    ("rgdbek_tune", _int, [_ptr, _ptr, _ptr, _i64, _u64, ctypes.POINTER(_int),
                           ctypes.POINTER(_dbl)]),
    ("rgdbek_tune_eta", _int, [_ptr, _ptr, _ptr, _ptr, _int, _i64, _u64,
                               ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)]),
    ("rgdbek_tune_teams", _int, [_ptr, _ptr, _ptr, _i64, _u64, ctypes.POINTER(_int), _ptr]),
    ("rgdbek_tune_spmv", _int, [_ptr, _int, ctypes.POINTER(_int), ctypes.POINTER(_int),
                                ctypes.POINTER(_dbl)]),
    ("rgdbek_set_pass_lanes", _int, [_ptr, _int, _int]),
    ("rgdbek_backward", _int, [_ptr, _ptr, _ptr, _ptr, _ptr, _ptr, _dbl, _i64, _u64, _int,
                               ctypes.POINTER(rgdbek_stats)]),
    ("rgdbek_set_trace", _int, [_ptr, _ptr, _i64, _ptr, _i64]),
    ("rgdbek_set_trace_vectors", _int, [_ptr, _ptr, _ptr, _i64]),
    ("rgdbek_spmv", _int, [_ptr, _ptr, _ptr]),
    ("rgdbek_spmv_t", _int, [_ptr, _ptr, _ptr]),
    ("rgdbek_spmv_f32", _int, [_ptr, _int, _ptr, _ptr]),
    ("rgdbek_weights", _int, [_ptr, _int, _ptr, _ptr, ctypes.POINTER(_dbl)]),
    ("rgdbek_sample", _int, [_ptr, _ptr, _i64, _i64, _u64, _u64, _i64, _int, _ptr,
                             ctypes.POINTER(_i64)]),
    ("rgdbek_sample_noalloc", _int, [_ptr, _i64, _i64, _u64, _u64, _i64, _int, _ptr, _ptr, _ptr]),
    ("rgdbek_get_norms", _int, [_ptr, _ptr, _ptr]),
    ("rgdbek_get_csc", _int, [_ptr, _ptr, _ptr, _ptr]),
    ("rgdbek_status_string", ctypes.c_char_p, [_int]),
]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with paper_2509_19267_gb300.build.build() "
            "(nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


class RGDBEKError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


def status_string(status: int) -> str:
    return _lib.rgdbek_status_string(status).decode()


def _check(status: int, where: str, allow=(OK,)) -> int:
    if status not in allow:
        raise RGDBEKError(status, where)
    return status


def _dptr(t) -> int:
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def default_options(**overrides) -> rgdbek_options:
    o = rgdbek_options()
    _lib.rgdbek_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------------------
# Functions named as in the C ABI
# ---------------------------------------------------------------------------
def rgdbek_create(m: int, n: int, row_ptr, col_idx, vals, options: rgdbek_options | None = None,
                  stream=None) -> int:
    """Create a handle from CSR arrays: torch CUDA tensors (int64, int32,
    float64) or host numpy arrays of the same dtypes."""
    h = _ptr()
    nnz = int(vals.shape[0]) if hasattr(vals, "shape") else len(vals)
    is_dev = hasattr(row_ptr, "is_cuda") and row_ptr.is_cuda
    if is_dev:
        ptrs = (_dptr(row_ptr), _dptr(col_idx), _dptr(vals))
    else:
        import numpy as np
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        ptrs = (row_ptr.ctypes.data, col_idx.ctypes.data if nnz else None,
                vals.ctypes.data if nnz else None)
    st = _lib.rgdbek_create(ctypes.byref(h), m, n, nnz, ptrs[0], ptrs[1], ptrs[2], int(is_dev),
                            ctypes.byref(options) if options is not None else None,
                            _stream_ptr(stream))
    _check(st, "rgdbek_create")
    return h.value


def rgdbek_create_like(base: int, options: rgdbek_options | None = None, stream=None) -> int:
    """A handle sharing base's matrix arrays, with its own workspace."""
    h = _ptr()
    _check(_lib.rgdbek_create_like(base, ctypes.byref(options) if options is not None else None,
                                   _stream_ptr(stream), ctypes.byref(h)), "rgdbek_create_like")
    return h.value


def rgdbek_destroy(h: int) -> None:
    _lib.rgdbek_destroy(h)


def rgdbek_set_options(h: int, options: rgdbek_options) -> None:
    _check(_lib.rgdbek_set_options(h, ctypes.byref(options)), "rgdbek_set_options")


def rgdbek_set_stream(h: int, stream=None) -> None:
    _check(_lib.rgdbek_set_stream(h, _stream_ptr(stream)), "rgdbek_set_stream")


def rgdbek_get_info(h: int) -> rgdbek_info_t:
    info = rgdbek_info_t()
    _check(_lib.rgdbek_get_info(h, ctypes.byref(info)), "rgdbek_get_info")
    return info


def rgdbek_solve(h: int, b, x, tol: float, max_iter: int, seed: int = 0,
                 raise_on_error: bool = True) -> rgdbek_stats:
    st = rgdbek_stats()
    status = _lib.rgdbek_solve(h, _dptr(b), _dptr(x), tol, max_iter, seed, ctypes.byref(st))
    st.status = status
    if raise_on_error:
        _check(status, "rgdbek_solve", allow=(OK, NOT_CONVERGED))
    return st


def rgdbek_solve_host(h: int, b, x, tol: float, max_iter: int, seed: int = 0,
                      raise_on_error: bool = True) -> rgdbek_stats:
    """b, x: contiguous float64 host buffers (numpy arrays or pinned CPU tensors)."""
    def hptr(a):
        return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
    st = rgdbek_stats()
    status = _lib.rgdbek_solve_host(h, hptr(b), hptr(x), tol, max_iter, seed, ctypes.byref(st))
    st.status = status
    if raise_on_error:
        _check(status, "rgdbek_solve_host", allow=(OK, NOT_CONVERGED))
    return st


def rgdbek_solve_batched(hs, bs, xs, tols, max_iter: int, seed: int = 0):
    """All systems in one persistent launch; returns (status, [stats])."""
    n = len(hs)
    H = (_ptr * n)(*hs)
    B = (_ptr * n)(*[_dptr(b) for b in bs])
    X = (_ptr * n)(*[_dptr(x) for x in xs])
    T = (_dbl * n)(*tols)
    S = (rgdbek_stats * n)()
    status = _lib.rgdbek_solve_batched(n, H, B, X, T, max_iter, seed, S)
    return status, list(S)


BATCH_TEAM_CANDIDATES = (1, 2, 4, 8, 19, 38, 76, 152)


def rgdbek_tune_batched(hs, bs, xs, tols, probe_iters: int = 3, seed: int = 0):
    """Times the batch with each team size, then each kernel shape at the best
    one; returns (best_team, best_block (0 = automatic), {team: ms},
    {block: ms})."""
    n = len(hs)
    H = (_ptr * n)(*hs)
    B = (_ptr * n)(*[_dptr(b) for b in bs])
    X = (_ptr * n)(*[_dptr(x) for x in xs])
    T = (_dbl * n)(*tols)
    team, block = _int(0), _int(0)
    nc = len(BATCH_TEAM_CANDIDATES)
    ms = (_dbl * (nc + 2))(*([-1.0] * (nc + 2)))
    _check(_lib.rgdbek_tune_batched(n, H, B, X, T, probe_iters, seed, ctypes.byref(team),
                                    ctypes.byref(block), ms), "rgdbek_tune_batched")
    return (team.value, block.value,
            {c: ms[i] for i, c in enumerate(BATCH_TEAM_CANDIDATES) if ms[i] >= 0},
            {blk: ms[nc + i] for i, blk in enumerate((512, 1024)) if ms[nc + i] >= 0})


def rgdbek_tune(h: int, b, x, probe_iters: int = 5, seed: int = 0):
    """Times both solve-kernel shapes; sets the faster. Returns (block, {block: ms})."""
    block = _int(0)
    ms = (_dbl * 2)()
    _check(_lib.rgdbek_tune(h, _dptr(b), _dptr(x), probe_iters, seed, ctypes.byref(block), ms),
           "rgdbek_tune")
    return block.value, {512: ms[0], 1024: ms[1]}


COL_TEAM_CANDIDATES = 5


def rgdbek_tune_teams(h: int, b, x, probe_iters: int = 10, seed: int = 0):
    """Times one team and column teams of 2/16 .. 5/16 of the grid; the handle
    keeps the fastest.  Returns (col_team, [ms per candidate], -1 = skipped)."""
    best = _int(0)
    ms = (_dbl * COL_TEAM_CANDIDATES)()
    _check(_lib.rgdbek_tune_teams(h, _dptr(b), _dptr(x), probe_iters, seed, ctypes.byref(best),
                                  ctypes.cast(ms, ctypes.c_void_p)), "rgdbek_tune_teams")
    return best.value, list(ms)


ETA_CANDIDATES = (0.05, 0.1, 0.2, 0.3, 0.5)


def rgdbek_tune_eta(h: int, b, x, candidates=None, probe_iters: int = 20, seed: int = 0):
    """Scores each candidate eta by -ln(stopping measure) per second over
    probe_iters iterations from x0 = 0; the handle keeps the best.  Returns
    (best_eta, {eta: score})."""
    cands = tuple(ETA_CANDIDATES if candidates is None else candidates)
    C = (_dbl * len(cands))(*cands)
    rate = (_dbl * len(cands))()
    best = _dbl(0.0)
    _check(_lib.rgdbek_tune_eta(h, _dptr(b), _dptr(x), None if candidates is None else C,
                                0 if candidates is None else len(cands), probe_iters, seed,
                                ctypes.byref(best), rate), "rgdbek_tune_eta")
    return best.value, {c: rate[i] for i, c in enumerate(cands)}


SPMV_LANE_CANDIDATES = (1, 2, 4, 8, 16, 32)


def rgdbek_tune_spmv(h: int, reps: int = 10):
    """Times each lane split of the full-matrix passes and keeps the fastest.
    Returns (lanes_row, lanes_col, {lanes: us} for CSR, {lanes: us} for CSC)."""
    lr, lc = _int(0), _int(0)
    nc = len(SPMV_LANE_CANDIDATES)
    us = (_dbl * (2 * nc))()
    _check(_lib.rgdbek_tune_spmv(h, reps, ctypes.byref(lr), ctypes.byref(lc), us),
           "rgdbek_tune_spmv")
    return (lr.value, lc.value, dict(zip(SPMV_LANE_CANDIDATES, list(us)[:nc])),
            dict(zip(SPMV_LANE_CANDIDATES, list(us)[nc:])))


def rgdbek_set_pass_lanes(h: int, lanes_row: int, lanes_col: int) -> None:
    _check(_lib.rgdbek_set_pass_lanes(h, lanes_row, lanes_col), "rgdbek_set_pass_lanes")


ADJ_RANK_TERM = 1


def rgdbek_backward(h: int, b, x, grad_x, grad_b=None, grad_vals=None, tol: float = 1e-10,
                    max_iter: int = 100000, seed: int = 0, flags: int = 0,
                    raise_on_error: bool = True):
    """Implicit adjoint of x = A^+ b: writes dL/db into grad_b and dL/dA (at the
    stored entries, CSR order) into grad_vals.  Returns (status, [4 stats])."""
    S = (rgdbek_stats * 4)()
    status = _lib.rgdbek_backward(h, _dptr(b), _dptr(x), _dptr(grad_x), _dptr(grad_b),
                                  _dptr(grad_vals), tol, max_iter, seed, flags, S)
    if raise_on_error:
        _check(status, "rgdbek_backward", allow=(OK, NOT_CONVERGED))
    return status, list(S)


def rgdbek_set_trace(h: int, counts=None, lists=None) -> None:
    """counts: int64 CUDA tensor of shape (cap, 4); lists: int32 CUDA tensor."""
    if counts is not None and (counts.dim() != 2 or counts.shape[1] != 4):
        raise ValueError("counts must have shape (cap, 4)")
    _check(_lib.rgdbek_set_trace(h, _dptr(counts), counts.shape[0] if counts is not None else 0,
                                 _dptr(lists), lists.shape[0] if lists is not None else 0),
           "rgdbek_set_trace")


def rgdbek_set_trace_vectors(h: int, g=None, r=None) -> None:
    """g: float64 CUDA tensor (cap, n) for A^T z_k; r: float64 CUDA tensor
    (cap, m) for the row residual of iteration k; None, None turns it off."""
    cap = 0
    for t in (g, r):
        if t is not None:
            if t.dim() != 2:
                raise ValueError("trace vectors must be 2-D (iterations, length)")
            cap = t.shape[0] if cap == 0 else min(cap, t.shape[0])
    _check(_lib.rgdbek_set_trace_vectors(h, _dptr(g), _dptr(r), cap),
           "rgdbek_set_trace_vectors")


def rgdbek_spmv(h: int, x, y) -> None:
    _check(_lib.rgdbek_spmv(h, _dptr(x), _dptr(y)), "rgdbek_spmv")


def rgdbek_spmv_f32(h: int, transposed: int, x, y) -> None:
    """FP32 products with the float copy of A: y = A x, or y = A^T x."""
    _check(_lib.rgdbek_spmv_f32(h, int(transposed), _dptr(x), _dptr(y)), "rgdbek_spmv_f32")


def rgdbek_spmv_t(h: int, z, g) -> None:
    _check(_lib.rgdbek_spmv_t(h, _dptr(z), _dptr(g)), "rgdbek_spmv_t")


def rgdbek_weights(h: int, which: int, v, eps) -> float:
    emax = _dbl(0.0)
    _check(_lib.rgdbek_weights(h, which, _dptr(v), _dptr(eps), ctypes.byref(emax)),
           "rgdbek_weights")
    return emax.value


def rgdbek_sample(h: int, eps, s: int, seed: int, sysid: int, k: int, phase: int, idx) -> int:
    cnt = _i64(0)
    _check(_lib.rgdbek_sample(h, _dptr(eps), eps.shape[0], s, seed, sysid, k, phase, _dptr(idx),
                              ctypes.byref(cnt)), "rgdbek_sample")
    return cnt.value


def rgdbek_sample_noalloc(eps, s: int, seed: int, sysid: int, k: int, phase: int, idx, count,
                          stream=None) -> None:
    """Queue the allocation-free sampler; idx (int32) and count (int64, one
    element) are CUDA tensors that receive the block and its size."""
    _check(_lib.rgdbek_sample_noalloc(_dptr(eps), eps.shape[0], s, seed, sysid, k, phase,
                                      _dptr(idx), _dptr(count), _stream_ptr(stream)),
           "rgdbek_sample_noalloc")


def rgdbek_get_norms(h: int, row_norms2=None, col_norms2=None) -> None:
    _check(_lib.rgdbek_get_norms(h, _dptr(row_norms2), _dptr(col_norms2)), "rgdbek_get_norms")


def rgdbek_get_csc(h: int, col_ptr, row_idx, vals) -> None:
    _check(_lib.rgdbek_get_csc(h, _dptr(col_ptr), _dptr(row_idx), _dptr(vals)), "rgdbek_get_csc")


# ---------------------------------------------------------------------------
# Convenience wrapper owning a handle
# ---------------------------------------------------------------------------
@dataclass
class SolveResult:
    x: object
    stats: rgdbek_stats


class Solver:
    """Owns one handle for an m x n CSR matrix on the current CUDA device."""

    def __init__(self, m: int, n: int, row_ptr, col_idx, vals, stream=None, **options):
        self.m, self.n = m, n
        self.options = default_options(**options)
        self.handle = rgdbek_create(m, n, row_ptr, col_idx, vals, self.options, stream)

    @classmethod
    def like(cls, base: "Solver", stream=None, **options) -> "Solver":
        """Another solver for base's matrix (shared on the device, own workspace)."""
        s = cls.__new__(cls)
        s.m, s.n = base.m, base.n
        o = rgdbek_options()
        ctypes.memmove(ctypes.byref(o), ctypes.byref(base.options), ctypes.sizeof(o))
        for k, v in options.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        s.options = o
        s.handle = rgdbek_create_like(base.handle, o, stream)
        return s

    def set_options(self, **options):
        for k, v in options.items():
            setattr(self.options, k, v)
        rgdbek_set_options(self.handle, self.options)

    def info(self) -> rgdbek_info_t:
        return rgdbek_get_info(self.handle)

    def tune_teams(self, b, probe_iters: int = 10, seed: int = 0):
        """Measured choice of the column team (rgdbek_tune_teams); the solver
        keeps it.  Returns (col_team, [ms per candidate])."""
        import torch
        x = torch.empty(self.n, dtype=torch.float64, device=b.device)
        return rgdbek_tune_teams(self.handle, b, x, probe_iters, seed)

    def tune_eta(self, b, candidates=None, probe_iters: int = 20, seed: int = 0):
        """Measured choice of eta (rgdbek_tune_eta); the solver keeps it.
        Returns (best_eta, {eta: score})."""
        import torch
        x = torch.empty(self.n, dtype=torch.float64, device=b.device)
        best, scores = rgdbek_tune_eta(self.handle, b, x, candidates, probe_iters, seed)
        self.options.eta_col = self.options.eta_row = best
        return best, scores

    def solve(self, b, tol: float = 1e-8, max_iter: int = 10000, seed: int = 0, x=None,
              raise_on_error: bool = True) -> SolveResult:
        import torch
        if x is None:  # (with warm_start, x is read as x_0: zeros unless given)
            x = torch.zeros(self.n, dtype=torch.float64, device=b.device)
        st = rgdbek_solve(self.handle, b, x, tol, max_iter, seed, raise_on_error)
        return SolveResult(x, st)

    def backward(self, b, x, grad_x, tol: float = 1e-10, max_iter: int = 100000, seed: int = 0,
                 rank_term: bool = False, want_vals: bool = True, nnz: int | None = None):
        """(grad_b, grad_vals or None, status, stats) for a loss with gradient grad_x."""
        import torch
        grad_b = torch.empty(self.m, dtype=torch.float64, device=b.device)
        grad_vals = None
        if want_vals:
            nnz = self.info().nnz if nnz is None else nnz
            grad_vals = torch.empty(max(nnz, 1), dtype=torch.float64, device=b.device)
        status, st = rgdbek_backward(self.handle, b, x, grad_x, grad_b, grad_vals, tol, max_iter,
                                     seed, ADJ_RANK_TERM if rank_term else 0)
        if grad_vals is not None:
            grad_vals = grad_vals[:nnz]
        return grad_b, grad_vals, status, st

    def close(self):
        if getattr(self, "handle", None):
            rgdbek_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Autograd: the solve as a differentiable function of A's values and b
# ---------------------------------------------------------------------------
def _autograd_function():
    import torch

    class RGDBEKLstsq(torch.autograd.Function):
        """x = A^+ b by rgdbek_solve; backward by rgdbek_backward (the implicit
        adjoint: no iterate is stored or unrolled)."""

        @staticmethod
        def forward(ctx, vals, b, row_ptr, col_idx, m, n, tol, max_iter, seed, adj_tol,
                    rank_term, options):
            solver = Solver(m, n, row_ptr, col_idx, vals.detach().contiguous(), **options)
            res = solver.solve(b.detach().contiguous(), tol=tol, max_iter=max_iter, seed=seed)
            if res.stats.status == NOT_CONVERGED:
                warnings.warn(f"rgdbek_lstsq: the forward solve stopped at its cap of "
                              f"{max_iter} outer iterations before reaching tol={tol:g} "
                              f"(normal-equation residual {res.stats.normal_res:.3e}); the "
                              f"implicit gradient assumes a converged solution",
                              RuntimeWarning, stacklevel=3)
            # the handle lives as long as this graph node: every backward through
            # it (retain_graph=True allows several) reuses it, and it is released
            # with the node when the graph is freed (Solver.__del__)
            ctx.solver = solver
            ctx.nnz = vals.shape[0]
            ctx.adj = (adj_tol, max_iter, seed + 1, rank_term)
            ctx.save_for_backward(b, res.x)
            ctx.stats = res.stats
            return res.x

        @staticmethod
        def backward(ctx, grad_x):
            b, x = ctx.saved_tensors
            adj_tol, max_iter, seed, rank_term = ctx.adj
            if ctx.solver.handle is None:
                raise RuntimeError("rgdbek_lstsq: the solver of this graph node was closed")
            gb, gv, status, st = ctx.solver.backward(b.detach().contiguous(), x,
                                                     grad_x.contiguous(), tol=adj_tol,
                                                     max_iter=max_iter, seed=seed,
                                                     rank_term=rank_term,
                                                     want_vals=ctx.needs_input_grad[0],
                                                     nnz=ctx.nnz)
            if status == NOT_CONVERGED:
                caps = [i for i, s in enumerate(st) if s.status == NOT_CONVERGED]
                warnings.warn(f"rgdbek_lstsq: adjoint solve(s) {caps} stopped at the cap of "
                              f"{max_iter} outer iterations before reaching tol={adj_tol:g}; "
                              f"the gradients are those of the unconverged iterates",
                              RuntimeWarning, stacklevel=2)
            return (gv if ctx.needs_input_grad[0] else None,
                    gb if ctx.needs_input_grad[1] else None,
                    None, None, None, None, None, None, None, None, None, None)

    return RGDBEKLstsq


_LSTSQ = None


def rgdbek_lstsq(row_ptr, col_idx, vals, b, m: int, n: int, tol: float = 1e-10,
                 max_iter: int = 100000, seed: int = 0, adj_tol: float | None = None,
                 rank_term: bool = False, **options):
    """Differentiable minimum-norm least-squares solve x = A^+ b.

    row_ptr (int64, m+1), col_idx (int32, nnz), vals (float64, nnz) and b
    (float64, m) are CUDA tensors; gradients flow to vals (on A's pattern) and
    to b.  Each call creates a handle for the given values; every backward pass
    through the result (several with retain_graph=True) reuses it, and it is
    released with the graph.  A solve or an adjoint solve that stops at
    max_iter before its tolerance issues a RuntimeWarning."""
    global _LSTSQ
    if _LSTSQ is None:
        _LSTSQ = _autograd_function()
    return _LSTSQ.apply(vals, b, row_ptr, col_idx, m, n, tol, max_iter, seed,
                        tol if adj_tol is None else adj_tol, rank_term, options)
