"""FP64 CPU oracle (test infrastructure only).

A ctypes binding over `glasso_oracle.c`, the plain, slow, obviously correct C
implementation of the multilevel proximal-Newton solver for
    min_{A > 0} -log det A + tr(S A) + lambda * sum_ij |A_ij|
(Treister, Turek, Yavneh, Section 5 eq. MLE_l1_prior; Algorithm 1; Section 7).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA library and the CUDA
library never calls it.  `build()` compiles the C file with gcc; nothing here
depends on the GPU or on torch.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glasso_oracle.c")
_LIB = os.path.join(_HERE, "_glasso_oracle.so")
_lib = None

OK, EINVAL, ENOTPD, ELINESEARCH, EMAXITER = 0, 1, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (plain -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("cycles", C.c_int), ("relaxations", C.c_int),
                ("ls_trials", C.c_int), ("objective", C.c_double), ("rel_kkt", C.c_double),
                ("max_kkt", C.c_double), ("logdet", C.c_double), ("nnz", C.c_int64),
                ("ntrace", C.c_int64), ("max_nnz", C.c_int64)]


_d = C.POINTER(C.c_double)
_i32 = C.POINTER(C.c_int32)
_u8 = C.POINTER(C.c_uint8)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.orc_form_S.argtypes = [_d, C.c_int64, C.c_int64, C.c_int, _d]
        L.orc_cholesky.argtypes = [_d, C.c_int64, _d]
        L.orc_cholesky.restype = C.c_int
        L.orc_logdet_from_chol.argtypes = [_d, C.c_int64]
        L.orc_logdet_from_chol.restype = C.c_double
        L.orc_inverse_from_chol.argtypes = [_d, C.c_int64, _d]
        L.orc_objective.argtypes = [_d, _d, C.c_int64, C.c_double, _d]
        L.orc_objective.restype = C.c_int
        L.orc_free_set.argtypes = [_d, _d, _d, C.c_int64, C.c_double, _i32, _i32, C.c_int64,
                                   _i32, _i32]
        L.orc_free_set.restype = C.c_int64
        L.orc_rel_kkt.argtypes = [_d, _d, _d, C.c_int64, C.c_double, _d]
        L.orc_rel_kkt.restype = C.c_double
        L.orc_hierarchy.argtypes = [_d, _u8, C.c_int64, _u8, C.POINTER(C.c_int)]
        L.orc_hierarchy.restype = C.c_int
        L.orc_cd_sweeps.argtypes = [_d, _d, _d, C.c_int64, C.c_double, _i32, _i32, C.c_int64,
                                    C.c_int, _d, _d]
        L.orc_line_search.argtypes = [_d, _d, _d, C.c_int64, C.c_double, _i32, _i32, C.c_int64,
                                      _d, C.c_double, C.c_double, C.c_int, _d, _d,
                                      C.POINTER(C.c_int)]
        L.orc_line_search.restype = C.c_int
        L.orc_solve.argtypes = [_d, C.c_int64, C.c_double, C.c_double, C.c_int, _d, _d, _d,
                                C.POINTER(Info), _d, C.c_int64, C.c_int, C.c_int, C.c_int]
        L.orc_solve.restype = C.c_int
        L.orc_continuation_lambdas.argtypes = [_d, C.c_int64, C.c_double, _d]
        L.orc_components.argtypes = [_d, C.c_int64, C.c_double, C.POINTER(C.c_int32)]
        L.orc_pcd_direction.argtypes = [_d, _d, _d, C.c_int64, C.c_double, _i32, _i32, C.c_int64,
                                        _d, _d, _d, _d]
        L.orc_pcd_direction.restype = None
        L.orc_pcd.argtypes = [_d, _d, _d, C.c_int64, C.c_double, _i32, _i32, C.c_int64, C.c_int,
                              C.c_int, C.c_double, _d, _d]
        L.orc_pcd.restype = C.c_int
        L.orc_components.restype = C.c_int64
        L.orc_continuation_lambdas.restype = C.c_int
        L.orc_bcd_logdet.argtypes = [_d, C.c_int64, _i32, _i32, C.c_int64, _d, _u8, C.c_double, _d]
        L.orc_bcd_logdet.restype = C.c_int
        L.orc_bcd_iteration.argtypes = [_d, _d, C.c_int64, C.c_double, C.c_int64, _i32, _i32, C.c_int64,
                                        C.c_int, C.c_int, C.c_int, _d, C.POINTER(C.c_int),
                                        C.POINTER(C.c_int)]
        L.orc_bcd_iteration.restype = C.c_int
        L.orc_solve_bcd.argtypes = [_d, C.c_int64, C.c_double, C.c_double, C.c_int, _d, _d,
                                    C.POINTER(Info), C.c_int64, C.c_int, C.c_int, C.c_int]
        L.orc_solve_bcd.restype = C.c_int
        L.orc_bcd_w11.argtypes = [_d, C.c_int64, _u8, _u8, _d, _d]
        L.orc_bcd_w11.restype = C.c_int
        _lib = L
    return _lib


def _p(a, t=_d):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def form_S(X, center: bool = False) -> np.ndarray:
    """a1: S = X^T X / m (optionally centred), eq. cov_estimate."""
    X = _f64(X)
    m, n = X.shape
    S = np.empty((n, n))
    lib().orc_form_S(_p(X), m, n, int(center), _p(S))
    return S


def cholesky(A):
    """a2: (info, L) with A = L L^T; info = k+1 at the first non-positive pivot."""
    A = _f64(A)
    n = A.shape[0]
    L = np.empty((n, n))
    info = lib().orc_cholesky(_p(A), n, _p(L))
    return info, L


def logdet_from_chol(L) -> float:
    L = _f64(L)
    return lib().orc_logdet_from_chol(_p(L), L.shape[0])


def inverse_from_chol(L) -> np.ndarray:
    """a3: W = A^{-1} from the Cholesky factor."""
    L = _f64(L)
    n = L.shape[0]
    W = np.empty((n, n))
    lib().orc_inverse_from_chol(_p(L), n, _p(W))
    return W


def objective(S, A, lam):
    """F(A) (eq. MLE_l1_prior); returns (info, F)."""
    S, A = _f64(S), _f64(A)
    F = C.c_double(0.0)
    info = lib().orc_objective(_p(S), _p(A), A.shape[0], lam, C.byref(F))
    return info, F.value


def free_set(S, W, A, lam, cand=None):
    """a4: free set (eq. active_set) restricted to candidate pairs; returns (i, j) arrays."""
    S, W, A = _f64(S), _f64(W), _f64(A)
    n = A.shape[0]
    if cand is None:
        cap = n * (n + 1) // 2
        ci = cj = None
        nc = 0
    else:
        ci = np.ascontiguousarray(cand[0], dtype=np.int32)
        cj = np.ascontiguousarray(cand[1], dtype=np.int32)
        nc = len(ci)
        cap = max(nc, 1)
    oi = np.empty(cap, dtype=np.int32)
    oj = np.empty(cap, dtype=np.int32)
    cnt = lib().orc_free_set(_p(S), _p(W), _p(A), n, lam,
                             None if ci is None else _p(ci, _i32),
                             None if cj is None else _p(cj, _i32), nc,
                             _p(oi, _i32), _p(oj, _i32))
    return oi[:cnt].copy(), oj[:cnt].copy()


def rel_kkt(S, W, A, lam):
    """Relative KKT residual and max-norm min-norm subgradient."""
    S, W, A = _f64(S), _f64(W), _f64(A)
    mx = C.c_double(0.0)
    r = lib().orc_rel_kkt(_p(S), _p(W), _p(A), A.shape[0], lam, C.byref(mx))
    return r, mx.value


def hierarchy(absg, insupp):
    """a5: per-pair level tags and the number of levels L."""
    absg = _f64(absg)
    insupp = np.ascontiguousarray(insupp, dtype=np.uint8)
    nf = len(absg)
    tag = np.empty(max(nf, 1), dtype=np.uint8)
    L = C.c_int(0)
    lib().orc_hierarchy(_p(absg), _p(insupp, _u8), nf, _p(tag, _u8), C.byref(L))
    return tag[:nf].copy(), L.value


def cd_sweeps(S, W, A, lam, pi, pj, nsweeps, D=None, U=None):
    """a6: CD sweeps on the Newton LASSO; returns (Delta on pairs, U = Delta W)."""
    S, W, A = _f64(S), _f64(W), _f64(A)
    n = A.shape[0]
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    D = np.zeros(len(pi)) if D is None else _f64(D).copy()
    U = np.zeros((n, n)) if U is None else _f64(U).copy()
    lib().orc_cd_sweeps(_p(S), _p(W), _p(A), n, lam, _p(pi, _i32), _p(pj, _i32), len(pi),
                        nsweeps, _p(D), _p(U))
    return D, U


def pcd_direction(S, W, A, lam, pi, pj, D=None, U=None):
    """The PCD direction d (every coordinate's 1-D minimiser at once) and
    b = G + W Delta W on the pairs, at Delta = D (U = Delta W)."""
    S, W, A = _f64(S), _f64(W), _f64(A)
    n = A.shape[0]
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    D = np.zeros(len(pi)) if D is None else _f64(D)
    U = np.zeros((n, n)) if U is None else _f64(U)
    d = np.zeros(len(pi))
    b = np.zeros(len(pi))
    lib().orc_pcd_direction(_p(S), _p(W), _p(A), n, lam, _p(pi, _i32), _p(pj, _i32), len(pi),
                            _p(D), _p(U), _p(d), _p(b))
    return d, b


def pcd(S, W, A, lam, pi, pj, iters, cg=True, D=None, U=None, rtol=0.0):
    """PCD (cg=False) or PCD-CG iterations with exact steps on the Newton
    LASSO (rtol > 0: stop once the direction fell by that factor); returns
    (Delta on pairs, U = Delta W, iterations taken)."""
    S, W, A = _f64(S), _f64(W), _f64(A)
    n = A.shape[0]
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    D = np.zeros(len(pi)) if D is None else _f64(D).copy()
    U = np.zeros((n, n)) if U is None else _f64(U).copy()
    k = lib().orc_pcd(_p(S), _p(W), _p(A), n, lam, _p(pi, _i32), _p(pj, _i32), len(pi), iters,
                      1 if cg else 0, rtol, _p(D), _p(U))
    return D, U, k


def line_search(S, W, A, lam, pi, pj, D, F0, sigma=1e-4, beta=0.5, max_trials=30):
    """a7: Armijo backtracking; returns (status, A_new, F_new, alpha, trials)."""
    S, W = _f64(S), _f64(W)
    A = _f64(A).copy()
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    D = _f64(D)
    F = C.c_double(F0)
    alpha = C.c_double(0.0)
    trials = C.c_int(0)
    rc = lib().orc_line_search(_p(S), _p(W), _p(A), A.shape[0], lam, _p(pi, _i32), _p(pj, _i32),
                               len(pi), _p(D), sigma, beta, max_trials, C.byref(F),
                               C.byref(alpha), C.byref(trials))
    return rc, A, F.value, alpha.value, trials.value


def continuation_lambdas(S, lam):
    """The continuation's stage values lambda_4 > lambda_3 > lambda_2
    (Section 8; lambda_4 = (max_{i != j} |S_ij| + lambda) / 2), empty when the
    solution at lambda is diagonal."""
    S = _f64(S)
    out = np.zeros(3)
    k = lib().orc_continuation_lambdas(_p(S), S.shape[0], lam, _p(out))
    return out[:k].copy()


def components(S, lam):
    """Screening: labels of the connected components of {|S_ij| > lam, i != j}
    (each vertex's component's smallest vertex) and their number."""
    S = _f64(S)
    comp = np.empty(S.shape[0], dtype=np.int32)
    k = lib().orc_components(_p(S), S.shape[0], lam, comp.ctypes.data_as(C.POINTER(C.c_int32)))
    return comp, int(k)


def solve(S, lam, tol=1e-8, max_cycles=200, A0=None, trace_cap=0, one_level=False,
          continuation=False, inner="cd"):
    """a8: the full ML-cycle solve (one_level: the paper's one-level
    comparison, the full free set every cycle; continuation: one relaxation
    at each continuation_lambdas value first).  Returns (A, W, info dict,
    trace array); info["max_nnz"] is the largest nnz(A) at the fine-level
    scans and at return.  inner: "cd" (CD sweeps) or "pcd_cg" (PCD-CG to the
    relative precision 1e-4) for the Newton direction."""
    if inner not in ("cd", "pcd_cg"):
        raise ValueError("inner must be 'cd' or 'pcd_cg'")
    S = _f64(S)
    n = S.shape[0]
    A = np.empty((n, n))
    W = np.empty((n, n))
    info = Info()
    tr = np.zeros((max(trace_cap, 1), 2))
    a0 = None if A0 is None else _f64(A0)
    lib().orc_solve(_p(S), n, lam, tol, max_cycles, None if a0 is None else _p(a0),
                    _p(A), _p(W), C.byref(info), _p(tr), trace_cap, 1 if one_level else 0,
                    1 if continuation else 0, 1 if inner == "pcd_cg" else 0)
    d = {k: getattr(info, k) for k, _ in Info._fields_}
    return A, W, d, tr[: info.ntrace].copy()


# ---- NEXT-4: BCD-IC (Section 6, Algorithm 2) ----------------------------------

_RULES = {"armijo": 0, "paper": 1}


def bcd_logdet(A, pi, pj, D, inI, alpha):
    """log det(A + alpha Delta) by the Schur complement on the index set I
    (eq. logdet_blocks); Delta on the pairs (pi <= pj) must vanish outside
    the rows/columns of I.  Returns (code, log det): code 0, 1 (A_22 not
    positive definite), 2 (the small matrix not), -1 (Delta on the 22 block)."""
    A = _f64(A)
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    D = _f64(D)
    m = np.ascontiguousarray(inI, dtype=np.uint8)
    ld = C.c_double(0.0)
    rc = lib().orc_bcd_logdet(_p(A), A.shape[0], _p(pi, _i32), _p(pj, _i32), len(pi), _p(D),
                              _p(m, _u8), alpha, C.byref(ld))
    return rc, ld.value


def bcd_iteration(S, A, lam, block, cand=None, inner="pcd_cg", nsweeps=1, rule="paper"):
    """One BCD-IC iteration (Algorithm 2) over the column blocks of `block`
    columns; cand = (ci, cj) restricts the block free sets to candidates.
    Returns (status, A_new, F(A_new), line-search evaluations, blocks moved)."""
    S = _f64(S)
    A = _f64(A).copy()
    n = A.shape[0]
    if cand is None:
        ci = cj = None
        nc = 0
    else:
        ci = np.ascontiguousarray(cand[0], dtype=np.int32)
        cj = np.ascontiguousarray(cand[1], dtype=np.int32)
        nc = len(ci)
    F = C.c_double(0.0)
    tr, mv = C.c_int(0), C.c_int(0)
    rc = lib().orc_bcd_iteration(_p(S), _p(A), n, lam, int(block),
                                 None if ci is None else _p(ci, _i32), None if cj is None else _p(cj, _i32),
                                 nc, 1 if inner == "pcd_cg" else 0, nsweeps, _RULES[rule], C.byref(F),
                                 C.byref(tr), C.byref(mv))
    return rc, A, F.value, tr.value, mv.value


def solve_bcd(S, lam, tol=1e-8, block=None, max_cycles=200, A0=None, inner="pcd_cg", rule="paper",
              one_level=False):
    """ML-BCD: the ML-cycle with one BCD-IC iteration (blocks of `block`
    columns, default all n) as the relaxation on each level; one_level: BCD-IC
    alone.  Returns (A, info dict)."""
    S = _f64(S)
    n = S.shape[0]
    A = np.empty((n, n))
    info = Info()
    a0 = None if A0 is None else _f64(A0)
    lib().orc_solve_bcd(_p(S), n, lam, tol, max_cycles, None if a0 is None else _p(a0), _p(A),
                        C.byref(info), int(block or n), 1 if inner == "pcd_cg" else 0, _RULES[rule],
                        1 if one_level else 0)
    return A, {k: getattr(info, k) for k, _ in Info._fields_}


def bcd_w11(A, inI, inN, WN):
    """W_11 = (A^{-1})_{II} from the columns of A^{-1} in the neighbourhood N
    only (the appendix's reduced inversion): W_11 = A_11^{-1} (I - A_12 W_21).
    Returns (code, W_11): 0, 1 (A_11 not positive definite), -1 (A_12 nonzero
    outside N)."""
    A, WN = _f64(A), _f64(WN)
    mI = np.ascontiguousarray(inI, dtype=np.uint8)
    mN = np.ascontiguousarray(inN, dtype=np.uint8)
    m1 = int(mI.sum())
    W11 = np.zeros((max(m1, 1), max(m1, 1)))
    rc = lib().orc_bcd_w11(_p(A), A.shape[0], _p(mI, _u8), _p(mN, _u8), _p(WN), _p(W11))
    return rc, W11[:m1, :m1]
