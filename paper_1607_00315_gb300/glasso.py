"""Thin ctypes binding over libglasso.so (include/glasso.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
Host arrays are numpy float64 (row-major); device arrays are torch CUDA
tensors, passed by pointer.  There is no fallback: `load()` raises when the
library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libglasso.so")

OK, EINVAL, ENOMEM, ENOTPD, ELINESEARCH, EMAXITER, EAGAIN, ETIMEOUT, ECUDA = range(9)
FP64, MIXED = 0, 1
INPUT_S, INPUT_X = 0, 1
F64, F32 = 0, 1
HOST, DEVICE = 0, 1
PROF_CLASSES = 6
PROF_NAMES = ("cholesky", "inverse", "scan", "cd_sweeps", "ls_cholesky", "ns_refine")

_lib = None
INNER = {"cd": 0, "pcd_cg": 1, "auto": 2}


def _inner_code(inner):
    if inner not in INNER:
        raise ValueError(f"inner must be one of {sorted(INNER)}")
    return INNER[inner]


class GlassoError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"glasso status {status}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("device", C.c_int), ("mem_budget_bytes", C.c_size_t), ("precision", C.c_int)]


class Problem(C.Structure):
    _fields_ = [("input", C.c_int), ("dtype", C.c_int), ("location", C.c_int),
                ("data", C.c_void_p), ("n", C.c_int64), ("m", C.c_int64), ("center", C.c_int),
                ("lambda_", C.c_double), ("tol", C.c_double), ("max_cycles", C.c_int),
                ("A0", C.c_void_p), ("one_level", C.c_int), ("continuation", C.c_int),
                ("screen", C.c_int), ("inner", C.c_int)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("cycles", C.c_int), ("relaxations", C.c_int),
                ("ls_trials", C.c_int), ("objective", C.c_double), ("rel_kkt", C.c_double),
                ("max_kkt", C.c_double), ("logdet", C.c_double), ("seconds", C.c_double),
                ("nnz", C.c_int64), ("max_nnz", C.c_int64), ("components", C.c_int64),
                ("max_block", C.c_int64), ("inner_iters", C.c_int64), ("flops", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PATHS = 11
PATH_NAMES = ("cd_lag2", "cd_persist32", "cd_chain64", "ls_series2", "ls_series6", "tc_factor",
              "tc_leaves", "ns_steps", "tc_dag", "tc_tuned", "fused")
FUSED_MAX_N = 512
DEBUG_WAIT_CYCLES, DEBUG_WAIT_UNREACHABLE, DEBUG_LS_REJECT, DEBUG_TC_DAG_TILES = 1, 2, 3, 4


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * PROF_CLASSES), ("launches", C.c_longlong * PROF_CLASSES),
                ("work", C.c_double * PROF_CLASSES), ("kernels", C.c_longlong),
                ("paths", C.c_longlong * PATHS)]


def load():
    """Load libglasso.so; raises when it is missing (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_1607_00315_gb300/build.py "
                           "(the CUDA library is required, there is no CPU path)")
    L = C.CDLL(LIB_PATH)
    vp, i64, d, i32 = C.c_void_p, C.c_int64, C.c_double, C.c_int
    L.glasso_create.argtypes = [C.POINTER(Config), C.POINTER(vp)]
    L.glasso_destroy.argtypes = [vp]
    L.glasso_destroy.restype = None
    L.glasso_set_stream.argtypes = [vp, vp]
    L.glasso_strerror.argtypes = [i32]
    L.glasso_strerror.restype = C.c_char_p
    L.glasso_last_error.argtypes = [vp]
    L.glasso_last_error.restype = C.c_char_p
    L.glasso_solve.argtypes = [vp, C.POINTER(Problem), vp, vp, C.POINTER(Info)]
    L.glasso_solve_batch.argtypes = [vp, C.POINTER(Problem), i32, i32, C.POINTER(vp),
                                     C.POINTER(Info)]
    L.glasso_bcd_logdet.argtypes = [vp, vp, i64, vp, vp, i64, vp, vp, d, C.POINTER(d), C.POINTER(i32)]
    L.glasso_bcd_iteration.argtypes = [vp, vp, vp, i64, d, i64, i32, i32, i32, C.POINTER(d),
                                       C.POINTER(i32), C.POINTER(i32)]
    L.glasso_solve_bcd.argtypes = [vp, vp, i64, d, d, i32, i64, i32, i32, i32, vp, C.POINTER(Info)]
    L.glasso_solve_batch_fused.argtypes = [vp, C.POINTER(Problem), i32, i32, C.POINTER(vp),
                                           C.POINTER(Info)]
    L.glasso_submit.argtypes = [vp, C.POINTER(Problem), vp, C.POINTER(C.c_uint64)]
    L.glasso_poll.argtypes = [vp, C.c_uint64, i64, C.POINTER(Info)]
    L.glasso_set_profiling.argtypes = [vp, i32]
    L.glasso_get_profile.argtypes = [vp, C.POINTER(Profile), i32]
    L.glasso_set_debug.argtypes = [vp, i32, i64]
    L.glasso_pcd.argtypes = [vp, vp, vp, vp, i64, d, vp, vp, i64, i32, i32, d, vp, vp, C.POINTER(i32)]
    L.glasso_form_S.argtypes = [vp, vp, i32, i64, i64, i32, vp]
    L.glasso_potrf.argtypes = [vp, vp, i64, C.POINTER(i32), C.POINTER(d)]
    L.glasso_inverse.argtypes = [vp, vp, i64, vp]
    L.glasso_cholinv_mixed.argtypes = [vp, vp, i64, vp, C.POINTER(i32), C.POINTER(d)]
    L.glasso_free_set.argtypes = [vp, vp, vp, vp, i64, d, vp, vp, i64, vp, vp, vp,
                                  C.POINTER(i64), C.POINTER(d), C.POINTER(d)]
    L.glasso_hierarchy.argtypes = [vp, vp, vp, i64, vp, C.POINTER(i32)]
    L.glasso_cd_sweeps.argtypes = [vp, vp, vp, vp, i64, d, vp, vp, i64, i32, vp, vp]
    L.glasso_line_search.argtypes = [vp, vp, vp, vp, i64, d, vp, vp, i64, vp, d, d, i32,
                                     C.POINTER(d), C.POINTER(d), C.POINTER(i32)]
    L.glasso_objective.argtypes = [vp, vp, vp, i64, d, C.POINTER(d), C.POINTER(i32)]
    L.glasso_components.argtypes = [vp, vp, i64, d, vp, C.POINTER(i64)]
    L.glasso_free_set_noalloc.argtypes = [vp, vp, vp, i64, d, vp, vp, vp, C.POINTER(i64),
                                          C.POINTER(d), C.POINTER(d), vp]
    L.glasso_free_set_noalloc.restype = i32
    for name in ("glasso_create", "glasso_set_stream", "glasso_solve", "glasso_solve_batch",
                 "glasso_submit", "glasso_poll", "glasso_set_profiling", "glasso_get_profile",
                 "glasso_form_S", "glasso_potrf", "glasso_inverse", "glasso_free_set",
                 "glasso_hierarchy", "glasso_cd_sweeps", "glasso_line_search", "glasso_objective",
                 "glasso_components", "glasso_set_debug", "glasso_pcd"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def _ptr(x):
    """Device pointer of a torch tensor, or host pointer of a numpy array."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(type(x))


def strerror(s):
    return load().glasso_strerror(s).decode()


class Context:
    """One solver context on one device (glasso_create / glasso_destroy)."""

    def __init__(self, device=0, precision=FP64, mem_budget_bytes=0):
        L = load()
        h = C.c_void_p()
        cfg = Config(device, mem_budget_bytes, precision)
        s = L.glasso_create(C.byref(cfg), C.byref(h))
        if s != OK:
            raise GlassoError(s, strerror(s))
        self.h = h
        self.L = L

    def close(self):
        if self.h:
            self.L.glasso_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, s, what):
        if s != OK:
            raise GlassoError(s, f"{what}: {strerror(s)} {self.L.glasso_last_error(self.h).decode()}")

    def set_stream(self, stream_handle):
        self._check(self.L.glasso_set_stream(self.h, stream_handle), "set_stream")

    def set_profiling(self, on=True):
        self._check(self.L.glasso_set_profiling(self.h, int(on)), "set_profiling")

    def get_profile(self, reset=False):
        p = Profile()
        self._check(self.L.glasso_get_profile(self.h, C.byref(p), int(reset)), "get_profile")
        d = {PROF_NAMES[c]: dict(ms=p.ms[c], launches=p.launches[c], work=p.work[c])
             for c in range(PROF_CLASSES)}
        d["kernels"] = p.kernels
        d["paths"] = {PATH_NAMES[k]: p.paths[k] for k in range(PATHS)}
        return d

    def set_debug(self, knob, value):
        """Fault injection for tests of the error paths (glasso_set_debug)."""
        self._check(self.L.glasso_set_debug(self.h, int(knob), int(value)), "set_debug")

    # ---------------------------------------------------------------- solver
    @staticmethod
    def problem(data, lam, tol=1e-8, *, samples=False, m=None, n=None, center=False,
                max_cycles=0, A0=None, one_level=False, continuation=False, screen=False,
                inner="cd"):
        """Build a glasso_problem from a numpy array (host) or a torch CUDA tensor."""
        dev = hasattr(data, "data_ptr") and getattr(data, "is_cuda", False)
        if not dev and isinstance(data, np.ndarray) and not data.flags.c_contiguous:
            raise ValueError("host arrays must be C-contiguous")
        if samples:
            mm, nn = data.shape
            dt = F32 if str(data.dtype).endswith("float32") else F64
        else:
            nn = data.shape[0]
            mm = 0
            dt = F64
        p = Problem(INPUT_X if samples else INPUT_S, dt, DEVICE if dev else HOST, _ptr(data),
                    nn if n is None else n, mm if m is None else m, int(center), float(lam),
                    float(tol), int(max_cycles), _ptr(A0), int(bool(one_level)),
                    int(bool(continuation)), int(bool(screen)), _inner_code(inner))
        return p

    def solve(self, data, lam, tol=1e-8, *, samples=False, center=False, max_cycles=0, A0=None,
              A_out=None, W_out=None, want_W=False, check=True, one_level=False,
              continuation=False, screen=False, inner="cd"):
        """glasso_solve (one_level: the paper's one-level comparison method;
        continuation: the paper's continuation stages before the cycles;
        screen: isolated vertices in closed form, the rest as one sub-problem).
        Returns (A, W or None, info dict)."""
        p = self.problem(data, lam, tol, samples=samples, center=center, max_cycles=max_cycles,
                         A0=A0, one_level=one_level, continuation=continuation, screen=screen,
                         inner=inner)
        n = p.n
        if A_out is None:
            if p.location == DEVICE:
                import torch

                A_out = torch.empty((n, n), dtype=torch.float64, device=data.device)
                if want_W and W_out is None:
                    W_out = torch.empty_like(A_out)
            else:
                A_out = np.empty((n, n))
                if want_W and W_out is None:
                    W_out = np.empty((n, n))
        info = Info()
        s = self.L.glasso_solve(self.h, C.byref(p), _ptr(A_out), _ptr(W_out), C.byref(info))
        if check and s not in (OK,):
            raise GlassoError(s, f"solve: {strerror(s)} {self.L.glasso_last_error(self.h).decode()}")
        return A_out, W_out, info.as_dict()

    def solve_batch(self, problems, outs, warm_from_prev=False):
        """glasso_solve_batch over prepared Problem structs; returns info dicts."""
        k = len(problems)
        arr = (Problem * k)(*problems)
        ptrs = (C.c_void_p * k)(*[_ptr(o) for o in outs])
        infos = (Info * k)()
        s = self.L.glasso_solve_batch(self.h, arr, k, int(warm_from_prev), ptrs, infos)
        return s, [infos[i].as_dict() for i in range(k)]

    def solve_batch_fused(self, problems, outs, warm_from_prev=False):
        """glasso_solve_batch_fused (all solves in one persistent launch, n <= 512);
        returns (status, info dicts)."""
        k = len(problems)
        arr = (Problem * k)(*problems)
        ptrs = (C.c_void_p * k)(*[_ptr(o) for o in outs])
        infos = (Info * k)()
        s = self.L.glasso_solve_batch_fused(self.h, arr, k, int(warm_from_prev), ptrs, infos)
        return s, [infos[i].as_dict() for i in range(k)]

    def bcd_logdet(self, A, pi, pj, D, inI, alpha):
        """glasso_bcd_logdet (BCD-IC's Schur-complement log det) on CUDA tensors:
        A (n x n float64), pi/pj (int32) and D (float64) the pairs of Delta,
        inI (uint8) the block mask.  Returns (code, log det)."""
        ld, code = C.c_double(0.0), C.c_int(0)
        self._check(self.L.glasso_bcd_logdet(self.h, _ptr(A), A.shape[0], _ptr(pi), _ptr(pj), len(pi),
                                             _ptr(D), _ptr(inI), float(alpha), C.byref(ld), C.byref(code)),
                    "bcd_logdet")
        return code.value, ld.value

    def bcd_iteration(self, S, A, lam, block, inner="cd", nsweeps=1, rule="paper"):
        """glasso_bcd_iteration on CUDA float64 tensors (A updated in place);
        returns (F, blocks moved, samples evaluated)."""
        F, mv, tr = C.c_double(0.0), C.c_int(0), C.c_int(0)
        self._check(self.L.glasso_bcd_iteration(self.h, _ptr(S), _ptr(A), A.shape[0], float(lam), int(block),
                                                _inner_code(inner), int(nsweeps),
                                                {"armijo": 0, "paper": 1}[rule], C.byref(F), C.byref(mv),
                                                C.byref(tr)), "bcd_iteration")
        return F.value, mv.value, tr.value

    def solve_bcd(self, S, lam, tol=1e-8, block=0, inner="cd", rule="paper", one_level=False, max_cycles=0,
                  A_out=None):
        """glasso_solve_bcd (ML-BCD) on a CUDA float64 S; returns (status, A, info dict)."""
        import torch

        n = S.shape[0]
        A = torch.empty((n, n), dtype=torch.float64, device=S.device) if A_out is None else A_out
        info = Info()
        s = self.L.glasso_solve_bcd(self.h, _ptr(S), n, float(lam), float(tol), int(max_cycles), int(block),
                                    _inner_code(inner), {"armijo": 0, "paper": 1}[rule], int(bool(one_level)),
                                    _ptr(A), C.byref(info))
        return s, A, info.as_dict()

    def submit(self, problem, A_out):
        t = C.c_uint64()
        self._check(self.L.glasso_submit(self.h, C.byref(problem), _ptr(A_out), C.byref(t)),
                    "submit")
        return t.value

    def poll(self, ticket, timeout_us=0):
        info = Info()
        s = self.L.glasso_poll(self.h, ticket, int(timeout_us), C.byref(info))
        return s, info.as_dict()

    # ---------------------------------------------------------- step level
    def form_S(self, X, S, center=False):
        m, n = X.shape
        dt = F32 if str(X.dtype).endswith("float32") else F64
        self._check(self.L.glasso_form_S(self.h, _ptr(X), dt, m, n, int(center), _ptr(S)), "form_S")

    def potrf(self, A):
        info, ld = C.c_int(0), C.c_double(0.0)
        self._check(self.L.glasso_potrf(self.h, _ptr(A), A.shape[0], C.byref(info), C.byref(ld)),
                    "potrf")
        return info.value, ld.value

    def inverse(self, L, W):
        self._check(self.L.glasso_inverse(self.h, _ptr(L), L.shape[0], _ptr(W)), "inverse")

    def cholinv_mixed(self, A, W):
        """FP32 tensor-core factorisation of A and W = A^-1 (unrefined) as FP64;
        returns (info, logdet)."""
        info, ld = C.c_int(0), C.c_double(0.0)
        self._check(self.L.glasso_cholinv_mixed(self.h, _ptr(A), A.shape[0], _ptr(W), C.byref(info),
                                                C.byref(ld)), "cholinv_mixed")
        return info.value, ld.value

    def free_set(self, S, W, A, lam, oi, oj, absg=None, cand=None):
        cnt = C.c_int64(0)
        rk, mk = C.c_double(0.0), C.c_double(0.0)
        ci, cj, nc = (None, None, 0) if cand is None else (_ptr(cand[0]), _ptr(cand[1]), len(cand[0]))
        self._check(self.L.glasso_free_set(self.h, _ptr(S), _ptr(W), _ptr(A), A.shape[0], lam, ci,
                                           cj, nc, _ptr(oi), _ptr(oj), _ptr(absg), C.byref(cnt),
                                           C.byref(rk), C.byref(mk)), "free_set")
        return cnt.value, rk.value, mk.value

    def hierarchy(self, absg, insupp, tag):
        lv = C.c_int(0)
        self._check(self.L.glasso_hierarchy(self.h, _ptr(absg), _ptr(insupp), len(absg), _ptr(tag),
                                            C.byref(lv)), "hierarchy")
        return lv.value

    def cd_sweeps(self, S, W, A, lam, pi, pj, nsweeps, D, U):
        self._check(self.L.glasso_cd_sweeps(self.h, _ptr(S), _ptr(W), _ptr(A), A.shape[0], lam,
                                            _ptr(pi), _ptr(pj), len(pi), nsweeps, _ptr(D), _ptr(U)),
                    "cd_sweeps")

    def pcd(self, S, W, A, lam, pi, pj, iters, D, U, cg=True, rtol=0.0):
        """glasso_pcd: PCD(-CG) iterations on the pair list; D in/out, U = Delta W
        out.  Returns the iterations taken."""
        it = C.c_int(0)
        self._check(self.L.glasso_pcd(self.h, _ptr(S), _ptr(W), _ptr(A), A.shape[0], lam, _ptr(pi),
                                      _ptr(pj), len(pi), int(iters), int(bool(cg)), float(rtol), _ptr(D),
                                      _ptr(U), C.byref(it)), "pcd")
        return it.value

    def line_search(self, S, W, A, lam, pi, pj, D, F_A, sigma=1e-4, max_trials=30):
        Fn, al, tr = C.c_double(0.0), C.c_double(0.0), C.c_int(0)
        s = self.L.glasso_line_search(self.h, _ptr(S), _ptr(W), _ptr(A), A.shape[0], lam, _ptr(pi),
                                      _ptr(pj), len(pi), _ptr(D), F_A, sigma, max_trials,
                                      C.byref(Fn), C.byref(al), C.byref(tr))
        return s, Fn.value, al.value, tr.value

    def components(self, S, lam, comp):
        """glasso_components: comp (device int32, n) receives the smallest
        vertex of each vertex's component of {|S_ij| > lam}; returns the
        number of components."""
        k = C.c_int64(0)
        self._check(self.L.glasso_components(self.h, _ptr(S), S.shape[0], lam, _ptr(comp), C.byref(k)),
                    "components")
        return k.value

    def objective(self, S, A, lam):
        F, info = C.c_double(0.0), C.c_int(0)
        self._check(self.L.glasso_objective(self.h, _ptr(S), _ptr(A), A.shape[0], lam, C.byref(F),
                                            C.byref(info)), "objective")
        return info.value, F.value


NOALLOC_MAX_N = 4096


def free_set_noalloc(S, W, A, lam, oi, oj, absg=None, stream=None):
    """glasso_free_set_noalloc: the level-0 free-set scan without a context and
    without any device allocation (fixed scratch inside the library).
    Returns (status, count, rel_kkt, max_kkt)."""
    L = load()
    cnt = C.c_int64(0)
    rk, mk = C.c_double(0.0), C.c_double(0.0)
    s = L.glasso_free_set_noalloc(_ptr(S), _ptr(W), _ptr(A), A.shape[0], lam, _ptr(oi), _ptr(oj),
                                  _ptr(absg), C.byref(cnt), C.byref(rk), C.byref(mk), stream)
    return s, cnt.value, rk.value, mk.value


EXPORTED = (
    "glasso_create", "glasso_destroy", "glasso_set_stream", "glasso_strerror",
    "glasso_last_error", "glasso_solve", "glasso_solve_batch", "glasso_solve_batch_fused",
    "glasso_submit", "glasso_poll",
    "glasso_set_profiling", "glasso_get_profile", "glasso_form_S", "glasso_potrf",
    "glasso_inverse", "glasso_cholinv_mixed", "glasso_free_set", "glasso_hierarchy", "glasso_cd_sweeps",
    "glasso_line_search", "glasso_objective", "glasso_free_set_noalloc", "glasso_components",
    "glasso_set_debug", "glasso_pcd", "glasso_bcd_logdet", "glasso_bcd_iteration", "glasso_solve_bcd",
)
