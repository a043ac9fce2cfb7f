"""FP64 CPU oracle for RGDBEK (arXiv 2509.19267) — test infrastructure only.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
in ``paper_2509_19267_gb300``; neither imports the other.

The arithmetic lives in ``rgdbek_oracle.c`` (plain single-threaded C, FP64):
Algorithm 1 of the paper with LSQR as the inner solver (Remark 3.1), the
residual weights and block selection of Section 2, and the greedy threshold
sets of GDBEK.  This module only compiles it with gcc and marshals numpy
arrays through ctypes.

Parity status of each routine (what pins it, in ``tests/test_oracle_*.py``):
  philox        known answers from numpy.random.Philox (independent code)
  spmv/spmv_t   dense numpy products
  norms         dense numpy norms
  weights       hand-computed values
  sample        exact quantised probabilities, chi-square on draw frequencies,
                zero-weight exclusion, single-weight and empty cases
  lsqr          numpy lstsq / pinv (overdetermined, underdetermined, rank
                deficient)
  solve         A^+ b (consistent, inconsistent, rank deficient, fat), the
                one-iteration closed forms for m x 1 and 1 x n systems, the
                Pythagoras identity (Eq. 5) per iteration, the linear-rate
                bound of Theorem 2.3, and the mean iteration counts of
                Tables 1 and 2.
  backward      (implicit adjoint, in this module) central finite
                differences of numpy lstsq / pinv solutions, along
                rank-preserving directions for rank-deficient A, and the
                scaling identities <dL/db, b> = g^T x, <dL/dA, A> = -g^T x
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rgdbek_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_rgdbek.so")

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_dbl = ctypes.c_double
_ptr = ctypes.c_void_p


class _Opts(ctypes.Structure):
    _fields_ = [
        ("eta_col", _dbl), ("eta_row", _dbl), ("selection", ctypes.c_int),
        ("inner_tol", _dbl), ("inner_max", ctypes.c_int), ("stop_rule", ctypes.c_int),
        ("tol", _dbl), ("max_iter", _i64), ("seed", _u64), ("sysid", _u64),
        ("warm", ctypes.c_int), ("inner_adapt", _dbl), ("k0", _i64), ("z_state", _ptr),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [
        ("iters", _i64), ("inner_u", _i64), ("inner_j", _i64),
        ("rel_res", _dbl), ("normal_res", _dbl), ("rse", _dbl), ("status", ctypes.c_int),
    ]


class _Trace(ctypes.Structure):
    _fields_ = [
        ("cap_iters", _i64), ("counts", _ptr), ("list_cap", _i64), ("lists", _ptr),
        ("list_len", _i64), ("n_iters", _i64), ("zs", _ptr), ("xs", _ptr),
        ("lock_counts", _ptr), ("lock_lists", _ptr), ("lock_iters", _i64),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) and return the .so path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _configure(lib):
    lib.orc_philox4x64_10.argtypes = [_ptr, _ptr, _ptr]
    lib.orc_spmv.argtypes = [_i64, _ptr, _ptr, _ptr, _ptr, _ptr]
    lib.orc_spmv_t.argtypes = [_i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr]
    lib.orc_row_norms2.argtypes = [_i64, _ptr, _ptr, _ptr]
    lib.orc_col_norms2.argtypes = [_i64, _i64, _ptr, _ptr, _ptr, _ptr]
    lib.orc_weights.argtypes = [_i64, _ptr, _ptr, _ptr, ctypes.POINTER(ctypes.c_int)]
    lib.orc_weights.restype = _dbl
    lib.orc_num_draws.argtypes = [_dbl, _i64]
    lib.orc_num_draws.restype = _i64
    lib.orc_sample.argtypes = [_i64, _ptr, _dbl, _i64, _u64, _u64, _u64, _u64, _ptr]
    lib.orc_sample.restype = _i64
    lib.orc_select_greedy.argtypes = [_i64, _ptr, _dbl, _dbl, _ptr]
    lib.orc_select_greedy.restype = _i64
    lib.orc_lsqr.argtypes = [_i64, _i64, _ptr, _ptr, _ptr, _ptr, _dbl, _dbl, ctypes.c_int, _ptr]
    lib.orc_lsqr.restype = ctypes.c_int
    lib.orc_solve.argtypes = [_i64, _i64, _ptr, _ptr, _ptr, _ptr, ctypes.POINTER(_Opts), _ptr,
                              ctypes.POINTER(_Stats), ctypes.POINTER(_Trace)]
    lib.orc_solve.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Temporarily route every oracle call through another build of the oracle
    source (used by the tests that plant a mistake in the oracle and check
    that a pin catches it)."""
    global _lib
    saved = _lib
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def build_variant(source_text: str, out_path: str) -> str:
    """Compile a modified copy of the oracle source to out_path."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", out_path,
                           src, "-lm"])
    return out_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _csr(A):
    rp, ci, av = A[0], A[1], A[2]
    return (np.ascontiguousarray(rp, dtype=np.int64), np.ascontiguousarray(ci, dtype=np.int32),
            np.ascontiguousarray(av, dtype=np.float64))


# ---------------------------------------------------------------------------
# Component routines
# ---------------------------------------------------------------------------
def philox(key, ctr) -> np.ndarray:
    """Philox4x64-10 block for a 2-word key and 4-word counter."""
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64).reshape(2))
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64).reshape(4))
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_philox4x64_10(_p(k), _p(c), _p(out))
    return out


def spmv(A, x):
    """y = A x for A = (row_ptr, col_idx, vals, m, n)."""
    rp, ci, av = _csr(A)
    m = len(rp) - 1
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(m)
    _load().orc_spmv(m, _p(rp), _p(ci), _p(av), _p(x), _p(y))
    return y


def spmv_t(A, z, n):
    """g = A^T z."""
    rp, ci, av = _csr(A)
    m = len(rp) - 1
    z = np.ascontiguousarray(z, dtype=np.float64)
    g = np.zeros(n)
    _load().orc_spmv_t(m, n, _p(rp), _p(ci), _p(av), _p(z), _p(g))
    return g


def row_norms2(A):
    rp, ci, av = _csr(A)
    m = len(rp) - 1
    out = np.zeros(m)
    _load().orc_row_norms2(m, _p(rp), _p(av), _p(out))
    return out


def col_norms2(A, n):
    rp, ci, av = _csr(A)
    m = len(rp) - 1
    out = np.zeros(n)
    _load().orc_col_norms2(m, n, _p(rp), _p(ci), _p(av), _p(out))
    return out


def weights(v, norm2):
    """(eps, eps_max, has_nonfinite) with eps_j = v_j^2/norm2_j (0 where norm2_j = 0)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    norm2 = np.ascontiguousarray(norm2, dtype=np.float64)
    eps = np.zeros(len(v))
    nan = ctypes.c_int(0)
    emax = _load().orc_weights(len(v), _p(v), _p(norm2), _p(eps), ctypes.byref(nan))
    return eps, emax, bool(nan.value)


def num_draws(eta: float, length: int) -> int:
    return int(_load().orc_num_draws(eta, length))


def sample(eps, s: int, seed: int, sysid: int, k: int, phase: int, emax=None) -> np.ndarray:
    """Sorted distinct indices from s draws with probabilities proportional to eps."""
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    if emax is None:
        emax = float(eps.max()) if len(eps) else 0.0
    out = np.zeros(max(len(eps), 1), dtype=np.int32)
    cnt = _load().orc_sample(len(eps), _p(eps), emax, s, seed, sysid, k, phase, _p(out))
    return out[:cnt].copy()


def select_greedy(eps, eta: float, emax=None) -> np.ndarray:
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    if emax is None:
        emax = float(eps.max()) if len(eps) else 0.0
    out = np.zeros(max(len(eps), 1), dtype=np.int32)
    cnt = _load().orc_select_greedy(len(eps), _p(eps), emax, eta, _p(out))
    return out[:cnt].copy()


def lsqr(B, c, nb: int, tol: float = 1e-13, maxit: int = 200, fro=None):
    """LSQR from 0 for min ||B y - c||; returns (y, steps)."""
    rp, ci, av = _csr(B)
    mb = len(rp) - 1
    c = np.ascontiguousarray(c, dtype=np.float64)
    if fro is None:
        fro = float(np.sqrt(np.dot(av, av)))
    y = np.zeros(max(nb, 1))
    steps = _load().orc_lsqr(mb, nb, _p(rp), _p(ci), _p(av), _p(c), tol, fro, maxit, _p(y))
    return y[:nb].copy(), int(steps)


# ---------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------
@dataclass
class Options:
    eta_col: float = 0.5
    eta_row: float = 0.5
    selection: int = 0          # 0 randomized (Algorithm 1), 1 greedy threshold (GDBEK)
    inner_tol: float = 1e-10
    inner_max: int = 200
    stop_rule: int = 0          # 0/2 normal equations, 1 relative residual, 3 RSE
    tol: float = 1e-8
    max_iter: int = 10000
    seed: int = 0
    sysid: int = 0
    inner_adapt: float = 0.0    # > 0: inner tolerance tied to the outer residual


@dataclass
class Result:
    x: np.ndarray
    iters: int
    inner_u: int
    inner_j: int
    rel_res: float
    normal_res: float
    rse: float
    status: int
    counts: np.ndarray | None = None   # [iters, 4]: |U_k|, |J_k|, LSQR steps (U), (J)
    lists: list | None = None          # [(U_k, J_k)]
    zs: np.ndarray | None = None
    xs: np.ndarray | None = None
    z: np.ndarray | None = None        # z at the end of a resumed solve


def solve(A, b, opts: Options | None = None, n: int | None = None, trace: bool = False,
          keep_iterates: bool = False, lock: list | None = None, x0=None,
          resume: tuple | None = None) -> Result:
    """Run Algorithm 1 on A = (row_ptr, col_idx, vals) with right-hand side b.

    trace          record |U_k|, |J_k|, LSQR step counts and the index sets
    keep_iterates  also record z_k and x_k (small problems only)
    lock           list of (U_k, J_k) index arrays to use instead of sampling
                   (lockstep replay); iterations past the list sample again
    x0             initial x (a warm start; default 0)
    resume         (x_k, z_k, k) of an earlier piece of the same solve: the solve
                   continues from iteration k (max_iter is then the number of the
                   last iteration, not a count) and Result.z holds z at its end, so
                   that a solve cut into pieces computes exactly what one
                   uninterrupted solve does
    """
    opts = opts or Options()
    rp, ci, av = _csr(A)
    m = len(rp) - 1
    if n is None:
        n = int(ci.max()) + 1 if len(ci) else 0
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(max(n, 1))
    if x0 is not None:
        x[:n] = np.asarray(x0, dtype=np.float64)
    k0 = 0
    zst = None
    if resume is not None:
        xr, zr, k0 = resume
        x[:n] = np.asarray(xr, dtype=np.float64)
        zst = np.ascontiguousarray(np.array(zr, dtype=np.float64))
        if zst.shape != (m,):
            raise ValueError("resume: z must have length m")
    o = _Opts(opts.eta_col, opts.eta_row, opts.selection, opts.inner_tol, opts.inner_max,
              opts.stop_rule, opts.tol, opts.max_iter, opts.seed, opts.sysid,
              1 if (x0 is not None or resume is not None) else 0, opts.inner_adapt,
              int(k0), _p(zst) if zst is not None else None)
    st = _Stats()
    tr = None
    keep = {}
    if trace or keep_iterates or lock is not None:
        cap = int(min(opts.max_iter, 100000))
        counts = np.zeros((max(cap, 1), 4), dtype=np.int64)
        list_cap = int(min(cap * (m + n), 50_000_000))
        lists = np.zeros(max(list_cap, 1), dtype=np.int32)
        tr = _Trace()
        tr.cap_iters = cap
        tr.counts = _p(counts)
        tr.list_cap = list_cap
        tr.lists = _p(lists)
        keep.update(counts=counts, lists=lists)
        if keep_iterates:
            zs = np.zeros((cap + 1, m))
            xs = np.zeros((cap + 1, max(n, 1)))
            tr.zs = _p(zs)
            tr.xs = _p(xs)
            keep.update(zs=zs, xs=xs)
        if lock is not None:
            lc = np.array([[len(u), len(j)] for (u, j) in lock], dtype=np.int64).reshape(-1, 2)
            ll = np.concatenate([np.concatenate([np.asarray(u, np.int32), np.asarray(j, np.int32)])
                                 for (u, j) in lock] + [np.zeros(0, np.int32)]).astype(np.int32)
            ll = np.ascontiguousarray(ll if len(ll) else np.zeros(1, np.int32))
            lc = np.ascontiguousarray(lc if len(lc) else np.zeros((1, 2), np.int64))
            tr.lock_counts = _p(lc)
            tr.lock_lists = _p(ll)
            tr.lock_iters = len(lock)
            keep.update(lc=lc, ll=ll)
    _load().orc_solve(m, n, _p(rp), _p(ci), _p(av), _p(b), ctypes.byref(o), _p(x),
                      ctypes.byref(st), ctypes.byref(tr) if tr is not None else None)
    res = Result(x=x[:n].copy(), iters=int(st.iters), inner_u=int(st.inner_u),
                 inner_j=int(st.inner_j), rel_res=float(st.rel_res),
                 normal_res=float(st.normal_res), rse=float(st.rse), status=int(st.status),
                 z=zst.copy() if zst is not None else None)
    if tr is not None:
        nrec = int(tr.n_iters)
        counts = keep["counts"][:nrec].copy()
        res.counts = counts
        if lock is None and tr.list_len <= tr.list_cap:
            lists, off = [], 0
            for k in range(nrec):
                nu, nj = int(counts[k, 0]), int(counts[k, 1])
                lists.append((keep["lists"][off:off + nu].copy(),
                              keep["lists"][off + nu:off + nu + nj].copy()))
                off += nu + nj
            res.lists = lists
        if keep_iterates:
            res.zs = keep["zs"][:res.iters + 1].copy()
            res.xs = keep["xs"][:res.iters + 1, :n].copy()
    return res


# ---------------------------------------------------------------------------
# Implicit adjoint of the solve
#
# The method converges to x = A^+ b, the minimum-norm least-squares solution
# (the convergence theorem of Section 2).  For a loss L(x) with gradient
# g = dL/dx, the derivative of the pseudo-inverse (Golub and Pereyra, "The
# differentiation of pseudo-inverses and nonlinear least squares problems",
# SIAM J. Numer. Anal. 10, 1973, Theorem 4.3), taken along perturbations that
# keep rank(A), gives
#   dL/db = w,                          w = A^+T g
#   dL/dA = r v^T - w x^T + u p^T,      r = b - A x,  v = A^+ w,
#                                       u = A^+T x,   p = (I - A^+ A) g
# The last term vanishes when A has full column rank (p = 0).  Only the
# entries on A's sparsity pattern are returned.
# ---------------------------------------------------------------------------
def transpose(A, n: int):
    """CSR of A^T (n rows), column indices ascending within each row."""
    rp, ci, av = _csr(A)
    m = len(rp) - 1
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rp))
    order = np.lexsort((rows, ci))          # by column of A, then by row
    counts = np.bincount(ci, minlength=n)
    tp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=tp[1:])
    return tp, rows[order].astype(np.int32), av[order].copy()


@dataclass
class Adjoint:
    grad_b: np.ndarray
    grad_vals: np.ndarray
    w: np.ndarray
    v: np.ndarray
    u: np.ndarray | None
    p: np.ndarray | None
    solves: list          # Result of each inner solve: w, v[, u, q]


def backward(A, b, x, g, opts: Options | None = None, n: int | None = None,
             rank_term: bool = False) -> Adjoint:
    """Gradients of L(x), x = A^+ b, from inner Algorithm 1 solves.

    w solves A^T w = g (minimum norm: w = A^+T g), v solves A v = w, and with
    rank_term u solves A^T u = x and q solves A q = A g (p = g - q).  Solve i
    (0, 1, 2, 3 in that order) uses seed opts.seed + i."""
    import dataclasses
    opts = opts or Options()
    rp, ci, av = _csr(A)
    m = len(rp) - 1
    if n is None:
        n = int(ci.max()) + 1 if len(ci) else 0
    At = transpose(A, n)
    b = np.asarray(b, np.float64)
    x = np.asarray(x, np.float64)
    g = np.asarray(g, np.float64)
    o = [dataclasses.replace(opts, seed=opts.seed + i) for i in range(4)]
    sw = solve(At, g, o[0], n=m)
    sv = solve((rp, ci, av), sw.x, o[1], n=n)
    w, v = sw.x, sv.x
    r = b - spmv((rp, ci, av), x)
    rows = np.repeat(np.arange(m), np.diff(rp))
    gv = r[rows] * v[ci] - w[rows] * x[ci]
    solves = [sw, sv]
    u = p = None
    if rank_term:
        su = solve(At, x, o[2], n=m)
        sq = solve((rp, ci, av), spmv((rp, ci, av), g), o[3], n=n)
        u, p = su.x, g - sq.x
        gv = gv + u[rows] * p[ci]
        solves += [su, sq]
    return Adjoint(grad_b=w.copy(), grad_vals=gv, w=w, v=v, u=u, p=p, solves=solves)


def backward_dense(D, b, g, rank_term: bool = True, rcond: float = 1e-12):
    """The same gradients from the dense pseudo-inverse (small cases): the
    definition written out, for pinning the iterative version.  Returns
    (grad_b, dense dL/dA)."""
    D = np.asarray(D, np.float64)
    Ap = np.linalg.pinv(D, rcond=rcond)
    x = Ap @ b
    w = Ap.T @ g
    v = Ap @ w
    r = b - D @ x
    G = np.outer(r, v) - np.outer(w, x)
    if rank_term:
        u = Ap.T @ x
        p = g - Ap @ (D @ g)
        G = G + np.outer(u, p)
    return w, G
