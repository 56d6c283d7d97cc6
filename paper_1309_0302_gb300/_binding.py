"""ctypes binding of libgodec (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "godec.h")

BATCH_NO_TUNE = 1
BATCH_POLICIES = 5
PREC_FP32 = 0
PREC_BF16_REFINE = 1
FLAG_NO_REFINE = 2
FLAG_FP64_FACTOR = 4
FLAG_SPARSE_FIRST = 8
FLAG_DENSE_FIRST = 16
MAX_RANK = 64


class GodecParams(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("ldx", C.c_int64), ("r", C.c_int32),
                ("q", C.c_int32), ("k", C.c_int64), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("precision", C.c_int32), ("rank_tol", C.c_double), ("flags", C.c_int32),
                ("reserved", C.c_int32)]


class GodecInfo(C.Structure):
    _fields_ = [("iter", C.c_int32), ("r_eff", C.c_int32), ("rel_err", C.c_double),
                ("obj", C.c_double), ("normX2", C.c_double), ("nnz", C.c_int64),
                ("select_passes", C.c_int32), ("rank_drops", C.c_int32),
                ("launches_per_iter", C.c_int32), ("exact_iters", C.c_int32),
                ("svd_sweeps", C.c_int32), ("chol_shifts", C.c_int32), ("alarms", C.c_int32)]


class GrebsmoParams(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("ldx", C.c_int64), ("lambda", C.c_double),
                ("tau", C.c_double), ("s_cap", C.c_int64), ("dr", C.c_int32), ("K", C.c_int32),
                ("r_max", C.c_int32), ("oversample", C.c_int32), ("q_inc", C.c_int32), ("flags", C.c_int32)]


class GodecError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


_LIB = None
_P = C.c_void_p


def _declare(lib):
    i64p, f32p, f64p, i32p = C.POINTER(C.c_int64), C.POINTER(C.c_float), C.POINTER(C.c_double), C.POINTER(C.c_int32)
    sig = {
        "godec_init": ([C.POINTER(_P), C.POINTER(GodecParams), _P, _P, _P], C.c_int),
        "godec_reset": ([_P], C.c_int),
        "godec_iterate": ([_P, C.c_int32, f64p], C.c_int),
        "godec_solve": ([_P, i32p, f64p], C.c_int),
        "godec_get_L": ([_P, _P, _P, _P, i32p], C.c_int),
        "godec_get_L_dense": ([_P, _P, C.c_int64], C.c_int),
        "godec_get_S": ([_P, _P, _P, C.c_int64, i64p], C.c_int),
        "godec_residual": ([_P, _P, C.c_int64], C.c_int),
        "godec_get_info": ([_P, C.POINTER(GodecInfo)], C.c_int),
        "godec_destroy": ([_P], None),
        "godec_last_error": ([_P], C.c_char_p),
        "godec_status_string": ([C.c_int], C.c_char_p),
        "godec_run_host": ([C.POINTER(GodecParams), _P, _P, C.c_int32, _P, _P, _P, _P, i32p, _P, _P,
                            C.c_int64, i64p, i32p, f64p], C.c_int),
        "godec_profile": ([_P, C.c_int32, f64p, i64p, f64p], C.c_int),
        "godec_profile_trace": ([_P, C.c_int32, i32p, i32p, f32p, f32p, i32p], C.c_int),
        "godec_check_timeout": ([_P, C.c_uint32], C.c_int),
        "godec_hard_threshold": ([_P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, _P, _P, C.c_int64, i64p, _P],
                                 C.c_int),
        "godec_mul_ZB": ([_P, C.c_int64, C.c_int64, C.c_int64, _P, C.c_int32, _P, _P], C.c_int),
        "godec_backward": ([_P, C.c_int64, C.c_int64, C.c_int64, _P, C.c_int32, C.c_int32, C.POINTER(_P), i64p,
                            _P, _P, C.c_int32, _P, C.c_int64, _P, C.c_int64, C.c_int32, _P], C.c_int),
        "godec_mul_ZtC": ([_P, C.c_int64, C.c_int64, C.c_int64, _P, C.c_int32, _P, _P], C.c_int),
        "godec_batch_init": ([C.POINTER(_P), C.c_int32, C.POINTER(GodecParams), C.POINTER(_P), C.POINTER(_P),
                              C.c_int32, _P], C.c_int),
        "godec_batch_iterate": ([_P, C.c_int32], C.c_int),
        "godec_batch_reset": ([_P], C.c_int),
        "godec_batch_problem": ([_P, C.c_int32], _P),
        "godec_batch_tuning": ([_P, i32p, f64p, i32p, i32p], C.c_int),
        "godec_batch_destroy": ([_P], None),
        "godec_batch_last_error": ([_P], C.c_char_p),
        "godec_batch_budgets": ([C.c_int32, i64p, i64p, C.c_int32, C.c_int32, i32p], C.c_int),
        "godec_tc_geometry": ([C.c_int64, C.c_int64, C.c_int32, i64p], C.c_int),
        "godec_grebsmo_init": ([C.POINTER(_P), C.POINTER(GrebsmoParams), _P, _P, _P], C.c_int),
        "godec_naive_init": ([C.POINTER(_P), C.POINTER(GodecParams), _P, _P, _P], C.c_int),
        "godec_lingodec_init": ([C.POINTER(_P), C.POINTER(GodecParams), C.c_double, _P, _P, C.c_int32, _P], C.c_int),
        "godec_lingodec_iterate": ([_P, C.c_int32, f64p], C.c_int),
        "godec_lingodec_get_W": ([_P, _P], C.c_int),
        "godec_mse_train": ([_P, C.c_int64, C.c_int64, C.c_int64, i32p, C.c_int32, i32p, C.c_int64, C.c_int32, _P,
                             C.c_int32, _P, _P, C.c_int64, _P, _P, C.c_int64, i64p, f64p, _P], C.c_int),
        "godec_naive_columns": ([C.c_int64, C.c_int64, C.c_int32], C.c_int),
        "godec_grebsmo_run": ([_P, i32p, f64p, C.c_int32, i32p], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


def library(build_if_missing: bool = True):
    """Load libgodec.so (building it with nvcc first if it is missing or stale)."""
    global _LIB
    if _LIB is None:
        from . import build as _build
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"GoDec CUDA library not found at {path}; run paper_1309_0302_gb300.build")
        _LIB = _declare(C.CDLL(path))
    return _LIB


def header_symbols() -> list[str]:
    """Function names declared in include/godec.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(godec_\w+)\s*\(", txt)))


def _check(status: int, where: str, ctx=None):
    if status != 0:
        lib = library()
        msg = lib.godec_last_error(ctx).decode(errors="replace")
        raise GodecError(status, where, msg)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the GoDec library needs a CUDA device")
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class GoDec:
    """One GoDec-BRP problem on the GPU (Algorithm 1).

    X: CUDA float32 (m, n), row-major (a padded copy is made if its row stride
    is not a multiple of 4 elements).  It is borrowed and must stay unchanged.
    A1: CUDA float32 (n, r) random test matrix.
    """

    def __init__(self, X, A1, r: int, k: int, q: int, tol: float = 1e-7, max_iter: int = 50,
                 rank_tol: float = 0.0, precision: int = PREC_FP32, stream=None, flags: int = 0):
        torch = _torch()
        lib = library()
        if X.dtype != torch.float32 or not X.is_cuda or X.dim() != 2:
            raise ValueError("X must be a 2-D CUDA float32 tensor")
        m, n = X.shape
        if X.stride(1) != 1 or X.stride(0) % 4 or X.stride(0) < n or X.data_ptr() % 16:
            Xp = torch.zeros((m, (n + 3) // 4 * 4), dtype=torch.float32, device=X.device)
            Xp[:, :n] = X
            X = Xp
        self._X = X
        self._A1 = A1.contiguous().to(torch.float32)
        self.m, self.n, self.r, self.k, self.q = m, n, int(r), int(k), int(q)
        self.stream = stream
        p = GodecParams(m=m, n=n, ldx=X.stride(0), r=int(r), q=int(q), k=int(k), tol=float(tol),
                        max_iter=int(max_iter), precision=int(precision), rank_tol=float(rank_tol),
                        flags=int(flags), reserved=0)
        h = C.c_void_p()
        st = lib.godec_init(C.byref(h), C.byref(p), _ptr(X), _ptr(self._A1), _stream_ptr(stream))
        _check(st, "godec_init", None)
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            library().godec_destroy(self._h)
            self._h = None

    __del__ = close

    def reset(self):
        _check(library().godec_reset(self._h), "godec_reset", self._h)

    def iterate(self, n_iter: int = 1) -> float:
        e = C.c_double(0.0)
        _check(library().godec_iterate(self._h, int(n_iter), C.byref(e)), "godec_iterate", self._h)
        return e.value

    def solve(self):
        it, e = C.c_int32(0), C.c_double(0.0)
        _check(library().godec_solve(self._h, C.byref(it), C.byref(e)), "godec_solve", self._h)
        return it.value, e.value

    def check_timeout(self, polls: int = 1000) -> None:
        """Run the timeout self-test (godec_check_timeout): raises GodecError with
        status 5 (GODEC_ERR_TIMEOUT) when the bounded wait gives up, as it must."""
        _check(library().godec_check_timeout(self._h, C.c_uint32(polls)), "godec_check_timeout", self._h)

    def info(self) -> dict:
        inf = GodecInfo()
        _check(library().godec_get_info(self._h, C.byref(inf)), "godec_get_info", self._h)
        return {f: getattr(inf, f) for f, _ in GodecInfo._fields_}

    PROF_CLASSES = ["product", "gram_sum", "chol", "tall_small", "slot_update", "rank_test",
                    "svd_root", "residual", "select_emit", "z_update", "refine", "sparse_proj"]

    def profile(self, n_iter: int):
        """Run n_iter iterations with per-kernel CUDA events; returns per-class totals."""
        nc = len(self.PROF_CLASSES)
        ms = (C.c_double * nc)()
        cnt = (C.c_int64 * nc)()
        bp = C.c_double(0.0)
        _check(library().godec_profile(self._h, int(n_iter), ms, cnt, C.byref(bp)), "godec_profile", self._h)
        return {"ms": {k: ms[i] for i, k in enumerate(self.PROF_CLASSES)},
                "launches": {k: cnt[i] for i, k in enumerate(self.PROF_CLASSES)},
                "bytes_product": bp.value}

    def profile_trace(self):
        """Launches of the last profiled iteration: list of (class, side, t0_ms, t1_ms)."""
        cnt = C.c_int32(0)
        lib = library()
        _check(lib.godec_profile_trace(self._h, 0, None, None, None, None, C.byref(cnt)), "godec_profile_trace", self._h)
        n = cnt.value
        cls, side = (C.c_int32 * max(n, 1))(), (C.c_int32 * max(n, 1))()
        t0, t1 = (C.c_float * max(n, 1))(), (C.c_float * max(n, 1))()
        _check(lib.godec_profile_trace(self._h, n, cls, side, t0, t1, C.byref(cnt)), "godec_profile_trace", self._h)
        return [(self.PROF_CLASSES[cls[i]], side[i], t0[i], t1[i]) for i in range(n)]

    def L(self):
        """(U (m, r_eff), sigma (r_eff,), V (n, r_eff)) as CUDA float32 tensors."""
        torch = _torch()
        dev = self._X.device
        U = torch.empty((self.m, self.r), dtype=torch.float32, device=dev)
        V = torch.empty((self.n, self.r), dtype=torch.float32, device=dev)
        s = torch.empty((self.r,), dtype=torch.float32, device=dev)
        re = C.c_int32(0)
        _check(library().godec_get_L(self._h, _ptr(U), _ptr(s), _ptr(V), C.byref(re)), "godec_get_L", self._h)
        r = re.value
        return U.view(-1)[: self.m * r].view(self.m, r), s[:r], V.view(-1)[: self.n * r].view(self.n, r)

    def L_dense(self):
        """L_t = U diag(sigma) V^T as a dense (m, n) CUDA float32 tensor, written by the library."""
        torch = _torch()
        L = torch.empty((self.m, self.n), dtype=torch.float32, device=self._X.device)
        _check(library().godec_get_L_dense(self._h, _ptr(L), self.n), "godec_get_L_dense", self._h)
        return L

    def S(self):
        """(idx int64 ascending linear indices, val float32) of S as CUDA tensors."""
        torch = _torch()
        nnz = C.c_int64(0)
        lib = library()
        inf = self.info()
        cnt = int(inf["nnz"])
        idx = torch.empty((max(cnt, 1),), dtype=torch.int64, device=self._X.device)
        val = torch.empty((max(cnt, 1),), dtype=torch.float32, device=self._X.device)
        _check(lib.godec_get_S(self._h, _ptr(idx), _ptr(val), cnt, C.byref(nnz)), "godec_get_S", self._h)
        return idx[: nnz.value], val[: nnz.value]

    def residual(self):
        """Dense R = X - L_t (m, n) as a CUDA float32 tensor, from the S-step's kernel."""
        torch = _torch()
        m, n = self._X.shape
        R = torch.empty((m, n), dtype=torch.float32, device=self._X.device)
        _check(library().godec_residual(self._h, _ptr(R), n), "godec_residual", self._h)
        return R


def naive_columns(m: int, n: int, r: int) -> int:
    """Columns p of naive GoDec's subspace iteration (r plus up to 8 oversampling columns)."""
    return int(library().godec_naive_columns(int(m), int(n), int(r)))


class NaiveGoDec(GoDec):
    """Naive GoDec (Sec. 2.1, eq. raw_lss) on the GPU: the L-step is the rank-r truncated SVD of
    X - S by warm-started block subspace iteration (q power steps per iteration), the S-step
    the exact top-k.  omega: CUDA float32 (n, naive_columns(m, n, r)), the first test matrix.
    iterate(), solve(), L(), S() and info() as for GoDec."""

    def __init__(self, X, omega, r: int, k: int, q: int = 2, tol: float = 1e-7, max_iter: int = 50,
                 stream=None, flags: int = 0):
        torch = _torch()
        lib = library()
        if X.dtype != torch.float32 or not X.is_cuda or X.dim() != 2:
            raise ValueError("X must be a 2-D CUDA float32 tensor")
        m, n = X.shape
        if X.stride(1) != 1 or X.stride(0) % 4 or X.stride(0) < n or X.data_ptr() % 16:
            Xp = torch.zeros((m, (n + 3) // 4 * 4), dtype=torch.float32, device=X.device)
            Xp[:, :n] = X
            X = Xp
        p_cols = naive_columns(m, n, r)
        if tuple(omega.shape) != (n, p_cols):
            raise ValueError(f"omega must be ({n}, {p_cols})")
        self._X = X
        self._A1 = omega.contiguous().to(torch.float32)
        self.m, self.n, self.r, self.k, self.q = m, n, int(r), int(k), int(q)
        self.stream = stream
        p = GodecParams(m=m, n=n, ldx=X.stride(0), r=int(r), q=int(q), k=int(k), tol=float(tol),
                        max_iter=int(max_iter), precision=PREC_FP32, rank_tol=0.0, flags=int(flags), reserved=0)
        h = C.c_void_p()
        st = lib.godec_naive_init(C.byref(h), C.byref(p), _ptr(X), _ptr(self._A1), _stream_ptr(stream))
        _check(st, "godec_naive_init", None)
        self._h = h


class LinGoDec(GoDec):
    """LinGoDec (Sec. 4.3) on the GPU: X (users x items) = W F^T + S + G with the item features F
    (n x d) given, rank(W) <= r, S soft-thresholded at lam.  iterate(n) runs n alternations;
    W() returns W (m x d); L(), S() and info() as for GoDec."""

    def __init__(self, X, F, r: int, lam: float, s_cap: int = 0, stream=None, flags: int = 0):
        torch = _torch()
        lib = library()
        if X.dtype != torch.float32 or not X.is_cuda or X.dim() != 2:
            raise ValueError("X must be a 2-D CUDA float32 tensor")
        m, n = X.shape
        if X.stride(1) != 1 or X.stride(0) % 4 or X.stride(0) < n or X.data_ptr() % 16:
            Xp = torch.zeros((m, (n + 3) // 4 * 4), dtype=torch.float32, device=X.device)
            Xp[:, :n] = X
            X = Xp
        if F.dim() != 2 or F.shape[0] != n:
            raise ValueError("F must be (n, d)")
        self._X = X
        self._A1 = F.contiguous().to(torch.float32)
        self.d = int(F.shape[1])
        self.m, self.n, self.r, self.k, self.q = m, n, int(r), int(s_cap), 0
        self.stream = stream
        k = int(s_cap if s_cap > 0 else max(1, m * n // 20))
        p = GodecParams(m=m, n=n, ldx=X.stride(0), r=int(r), q=0, k=k, tol=-1.0, max_iter=1,
                        precision=PREC_FP32, rank_tol=0.0, flags=int(flags), reserved=0)
        h = C.c_void_p()
        st = lib.godec_lingodec_init(C.byref(h), C.byref(p), float(lam), _ptr(X), _ptr(self._A1), self.d,
                                     _stream_ptr(stream))
        _check(st, "godec_lingodec_init", None)
        self._h = h

    def iterate(self, n_iter: int = 1) -> float:
        rel = C.c_double(0.0)
        _check(library().godec_lingodec_iterate(self._h, int(n_iter), C.byref(rel)), "godec_lingodec_iterate",
               self._h)
        return rel.value

    def W(self):
        """W (m, d) as a CUDA float32 tensor."""
        torch = _torch()
        W = torch.empty((self.m, self.d), dtype=torch.float32, device=self._X.device)
        _check(library().godec_lingodec_get_W(self._h, _ptr(W)), "godec_lingodec_get_W", self._h)
        return W


class GreBsmo(GoDec):
    """GreBsmo (Sec. 3.2.1, Algorithm 2) on the GPU: X = U V + S + G with a soft-thresholded S
    and a rank found by greedy increments.

    X: CUDA float32 (m, n), borrowed.  omegas: CUDA float32 (stages, n, dr + oversample), the
    test matrices of the random-projection increments (the first gives the initial V).
    run() returns (rank, errors after each rank stage); then L(), L_dense(), S(), residual()
    and info() read the result as for GoDec.
    """

    def __init__(self, X, omegas, lam: float, dr: int, K: int, tau: float, r_max: int,
                 oversample: int = 6, q_inc: int = 4, s_cap: int = 0, flags: int = 0, stream=None):
        torch = _torch()
        lib = library()
        if X.dtype != torch.float32 or not X.is_cuda or X.dim() != 2:
            raise ValueError("X must be a 2-D CUDA float32 tensor")
        m, n = X.shape
        if X.stride(1) != 1 or X.stride(0) % 4 or X.stride(0) < n or X.data_ptr() % 16:
            Xp = torch.zeros((m, (n + 3) // 4 * 4), dtype=torch.float32, device=X.device)
            Xp[:, :n] = X
            X = Xp
        p_cols = int(dr) + int(oversample)
        if omegas.dim() != 3 or omegas.shape[1] != n or omegas.shape[2] != p_cols:
            raise ValueError("omegas must be (stages, n, dr + oversample)")
        self._X = X
        self._omegas = omegas.contiguous().to(torch.float32)
        self.m, self.n, self.r = m, n, int(r_max)
        self.stream = stream
        self._stages = int(omegas.shape[0])
        p = GrebsmoParams(**{"m": m, "n": n, "ldx": X.stride(0), "lambda": float(lam), "tau": float(tau),
                             "s_cap": int(s_cap if s_cap > 0 else max(1, m * n // 20)), "dr": int(dr),
                             "K": int(K), "r_max": int(r_max), "oversample": int(oversample),
                             "q_inc": int(q_inc), "flags": int(flags)})
        need = 1 + -(-(int(r_max) - int(dr)) // int(dr))
        if self._stages < need:
            raise ValueError(f"omegas needs {need} stages")
        h = C.c_void_p()
        st = lib.godec_grebsmo_init(C.byref(h), C.byref(p), _ptr(X), _ptr(self._omegas), _stream_ptr(stream))
        _check(st, "godec_grebsmo_init", None)
        self._h = h

    def run(self):
        """Run to the stop; returns (rank, list of the relative errors after each stage)."""
        r = C.c_int32(0)
        ns = C.c_int32(0)
        errs = (C.c_double * max(self._stages, 1))()
        _check(library().godec_grebsmo_run(self._h, C.byref(r), errs, self._stages, C.byref(ns)),
               "godec_grebsmo_run", self._h)
        return r.value, [errs[i] for i in range(min(ns.value, self._stages))]

    def iterate(self, n_iter: int = 1):
        raise RuntimeError("GreBsmo runs through run()")


def mse_train(X, labels, ranks, K: int, iters: int, A1s, stream=None):
    """MSE training (Sec. 4.2.1, Algorithm 4) on the GPU.

    X: CUDA float32 (n, p); labels: (n, k) 0/1 array (host); ranks: k ints; A1s: CUDA float32
    (iters, k, p, r_stride), the Gaussian test matrix of each BRP step.  Returns a dict with
    C (k, r_stride, p) orthonormal subspace rows, Lsum (n, p) = sum of the blocks, S_idx,
    S_val (COO) and history (the objective after each outer iteration).
    """
    torch = _torch()
    lib = library()
    if X.dtype != torch.float32 or not X.is_cuda or X.dim() != 2:
        raise ValueError("X must be a 2-D CUDA float32 tensor")
    n, p = X.shape
    if X.stride(1) != 1 or X.stride(0) % 4 or X.stride(0) < p or X.data_ptr() % 16:
        Xp = torch.zeros((n, (p + 3) // 4 * 4), dtype=torch.float32, device=X.device)
        Xp[:, :p] = X
        X = Xp
    lab = np.ascontiguousarray(np.asarray(labels) != 0, dtype=np.int32)
    k = lab.shape[1]
    rk = np.ascontiguousarray(ranks, dtype=np.int32)
    A1s = A1s.contiguous().to(torch.float32)
    r_stride = int(A1s.shape[3])
    C_ = torch.zeros((k, r_stride, p), dtype=torch.float32, device=X.device)
    Ls = torch.empty((n, p), dtype=torch.float32, device=X.device)
    si = torch.empty((max(K, 1),), dtype=torch.int64, device=X.device)
    sv = torch.empty((max(K, 1),), dtype=torch.float32, device=X.device)
    nnz = C.c_int64(0)
    hist = (C.c_double * iters)()
    st = lib.godec_mse_train(_ptr(X), n, p, X.stride(0), lab.ctypes.data_as(C.POINTER(C.c_int32)), k,
                             rk.ctypes.data_as(C.POINTER(C.c_int32)), int(K), int(iters), _ptr(A1s), r_stride,
                             _ptr(C_), _ptr(Ls), p, _ptr(si), _ptr(sv), max(int(K), 1), C.byref(nnz), hist,
                             _stream_ptr(stream))
    _check(st, "godec_mse_train", None)
    return {"C": C_, "Lsum": Ls, "S_idx": si[: nnz.value], "S_val": sv[: nnz.value],
            "history": [hist[i] for i in range(iters)]}


def _mul(name, Z, B, stream=None):
    torch = _torch()
    if Z.dtype != torch.float32 or B.dtype != torch.float32 or not Z.is_cuda:
        raise ValueError("Z and B must be CUDA float32")
    m, n = Z.shape
    if Z.stride(1) != 1 or Z.stride(0) % 4 or Z.data_ptr() % 16:
        Zp = torch.zeros((m, (n + 3) // 4 * 4), dtype=torch.float32, device=Z.device)
        Zp[:, :n] = Z
        Z = Zp
    B = B.contiguous()
    r = B.shape[1]
    out = torch.empty(((n if name == "godec_mul_ZtC" else m), r), dtype=torch.float32, device=Z.device)
    st = getattr(library(), name)(_ptr(Z), m, n, Z.stride(0), _ptr(B), r, _ptr(out), _stream_ptr(stream))
    _check(st, name)
    return out


def hard_threshold(R, k: int, stream=None):
    """Entry-wise hard threshold of a CUDA float32 matrix on the GPU (S-step with L = 0).

    Returns (idx int64 ascending, val float32) CUDA tensors.
    """
    torch = _torch()
    m, n = R.shape
    if R.stride(1) != 1 or R.stride(0) % 4 or R.data_ptr() % 16:
        Rp = torch.zeros((m, (n + 3) // 4 * 4), dtype=torch.float32, device=R.device)
        Rp[:, :n] = R
        R = Rp
    cap = max(1, min(int(k), m * n))
    idx = torch.empty((cap,), dtype=torch.int64, device=R.device)
    val = torch.empty((cap,), dtype=torch.float32, device=R.device)
    nnz = C.c_int64(0)
    st = library().godec_hard_threshold(_ptr(R), m, n, R.stride(0), int(k), _ptr(idx), _ptr(val), cap,
                                        C.byref(nnz), _stream_ptr(stream))
    _check(st, "godec_hard_threshold")
    return idx[: nnz.value], val[: nnz.value]


def mul_ZB(Z, B, stream=None):
    """Y = Z @ B on the GPU (Z m x n, B n x r)."""
    return _mul("godec_mul_ZB", Z, B, stream)


def mul_ZtC(Z, Cm, stream=None):
    """W = Z^T @ C on the GPU (Z m x n, C m x r)."""
    return _mul("godec_mul_ZtC", Z, Cm, stream)


def backward(X, A1, T: int, supports, gU=None, gV=None, gL=None, stream=None, rebuild: bool = False):
    """dLoss/dX of T unrolled q = 0 iterations with frozen supports (godec_backward).

    X (m, n) and A1 (n, r) CUDA float32; ``supports`` the T-1 int64 CUDA tensors of
    linear indices of Omega_1 .. Omega_{T-1}; dLoss/dL_T as gU (m, g) and gV (n, g)
    (meaning gU gV^T) or dense gL (m, n).  ``rebuild``: recompute the iterates in the
    backward sweep instead of keeping them (GODEC_BACKWARD_REBUILD: less memory, slower).
    Returns dX (m, n).
    """
    torch = _torch()
    m, n = X.shape
    r = A1.shape[1]
    for name, t in (("X", X), ("A1", A1), ("gU", gU), ("gV", gV), ("gL", gL)):
        if t is not None and (t.dtype != torch.float32 or not t.is_cuda):
            raise ValueError(f"{name} must be a CUDA float32 tensor")
    if any(s.dtype != torch.int64 or not s.is_cuda for s in supports):
        raise ValueError("supports must be CUDA int64 tensors")
    X = _pad_rows(X)
    A1 = A1.contiguous()
    if len(supports) != T - 1:
        raise ValueError("need T - 1 supports")
    sup = [s.contiguous() for s in supports]
    ptrs = (_P * max(T - 1, 1))(*[_ptr(s) for s in sup]) if T > 1 else None
    nnz = (C.c_int64 * max(T - 1, 1))(*[int(s.numel()) for s in sup]) if T > 1 else None
    dXp = torch.empty((m, (n + 3) // 4 * 4), dtype=torch.float32, device=X.device)
    if gL is not None:
        gL = _pad_rows(gL)
        args = (None, None, 0, _ptr(gL), gL.stride(0))
    else:
        gU, gV = gU.contiguous(), gV.contiguous()
        args = (_ptr(gU), _ptr(gV), gU.shape[1], None, 0)
    st = library().godec_backward(_ptr(X), m, n, X.stride(0), _ptr(A1), r, int(T), ptrs, nnz, *args,
                                  _ptr(dXp), dXp.stride(0), 1 if rebuild else 0, _stream_ptr(stream))
    _check(st, "godec_backward")
    return dXp[:, :n]


def _pad_rows(A):
    """A with unit column stride, a 16-byte multiple row stride and 16-byte alignment."""
    torch = _torch()
    m, n = A.shape
    if A.stride(1) != 1 or A.stride(0) % 4 or A.data_ptr() % 16:
        Ap = torch.zeros((m, (n + 3) // 4 * 4), dtype=torch.float32, device=A.device)
        Ap[:, :n] = A
        return Ap
    return A


def run_host(X: np.ndarray, A1: np.ndarray, r: int, k: int, q: int, n_iter: int, tol: float = 1e-7,
             max_iter: int = 50, rank_tol: float = 0.0, stream=None, out=None) -> dict:
    """Whole run from host arrays through godec_run_host (copies inside the call).

    ``out`` may hold preallocated (ideally pinned) host arrays U, sigma, V, S_idx, S_val.
    """
    lib = library()
    X = np.ascontiguousarray(X, dtype=np.float32)
    A1 = np.ascontiguousarray(A1, dtype=np.float32)
    m, n = X.shape
    out = out or {}
    U = out.get("U", np.empty((m, r), np.float32))
    V = out.get("V", np.empty((n, r), np.float32))
    s = out.get("sigma", np.empty((r,), np.float32))
    Si = out.get("S_idx", np.empty((max(k, 1),), np.int64))
    Sv = out.get("S_val", np.empty((max(k, 1),), np.float32))
    p = GodecParams(m=m, n=n, ldx=(n + 3) // 4 * 4, r=r, q=q, k=k, tol=tol, max_iter=max_iter,
                    precision=0, rank_tol=rank_tol, flags=0, reserved=0)
    re, nnz, it, e = C.c_int32(0), C.c_int64(0), C.c_int32(0), C.c_double(0.0)
    st = lib.godec_run_host(C.byref(p), X.ctypes.data_as(C.c_void_p), A1.ctypes.data_as(C.c_void_p),
                            int(n_iter), _stream_ptr(stream), U.ctypes.data_as(C.c_void_p),
                            s.ctypes.data_as(C.c_void_p), V.ctypes.data_as(C.c_void_p), C.byref(re),
                            Si.ctypes.data_as(C.c_void_p), Sv.ctypes.data_as(C.c_void_p), Si.size,
                            C.byref(nnz), C.byref(it), C.byref(e))
    _check(st, "godec_run_host")
    rr, kk = re.value, nnz.value
    return {"U": U.reshape(-1)[: m * rr].reshape(m, rr), "sigma": s[:rr],
            "V": V.reshape(-1)[: n * rr].reshape(n, rr), "S_idx": Si[:kk], "S_val": Sv[:kk],
            "iters": it.value, "rel_err": e.value, "r_eff": rr}


def _bcheck(status: int, where: str, b=None):
    if status != 0:
        msg = library().godec_batch_last_error(b).decode(errors="replace")
        raise GodecError(status, where, msg)


def _padded(X):
    """X itself, or a copy whose row stride is a multiple of 4 elements (16 bytes)."""
    torch = _torch()
    if X.dtype != torch.float32 or not X.is_cuda or X.dim() != 2:
        raise ValueError("X must be a 2-D CUDA float32 tensor")
    m, n = X.shape
    if X.stride(1) != 1 or X.stride(0) % 4 or X.stride(0) < n or X.data_ptr() % 16:
        Xp = torch.zeros((m, (n + 3) // 4 * 4), dtype=torch.float32, device=X.device)
        Xp[:, :n] = X
        return Xp
    return X


class _Problem(GoDec):
    """Problem i of a GoDecBatch: the GoDec methods on a context the batch owns."""

    def __init__(self, batch, h, X, A1, r, k, q):
        self._batch = batch          # keeps the batch (and its contexts) alive
        self._X, self._A1 = X, A1
        self.m, self.n = X.shape
        self.r, self.k, self.q = int(r), int(k), int(q)
        self.stream = batch.stream
        self._h = h

    def close(self):
        self._h = None               # the batch destroys the context

    __del__ = close


class GoDecBatch:
    """Many GoDec-BRP problems of uneven m, n and r, one CUDA-graph launch per batch
    iteration (godec_batch_* in include/godec.h).

    Xs, A1s: lists of CUDA float32 tensors (m_i, n_i) and (n_i, r_i), borrowed.
    rs, ks, qs: per-problem rank, cardinality and power-step count (ints or lists).
    tune: time the candidate SM-budget policies and keep the fastest (else every
    problem gets all SMs).
    """

    def __init__(self, Xs, A1s, rs, ks, qs, tune: bool = True, rank_tol: float = 0.0, stream=None):
        torch = _torch()
        lib = library()
        cnt = len(Xs)
        if cnt < 1 or len(A1s) != cnt:
            raise ValueError("need as many A1 as X, at least one")
        as_list = lambda v: [int(x) for x in v] if hasattr(v, "__len__") else [int(v)] * cnt
        rs, ks, qs = as_list(rs), as_list(ks), as_list(qs)
        if not (len(rs) == len(ks) == len(qs) == cnt):
            raise ValueError("rs, ks and qs need one entry per problem")
        self._X = [_padded(X) for X in Xs]
        self._A1 = [A.contiguous().to(torch.float32) for A in A1s]
        self.rs, self.ks, self.qs = rs, ks, qs
        self.stream = stream
        params = (GodecParams * cnt)()
        for i, X in enumerate(self._X):
            m, n = Xs[i].shape
            params[i] = GodecParams(m=m, n=n, ldx=X.stride(0), r=rs[i], q=qs[i], k=ks[i], tol=-1.0,
                                    max_iter=1 << 30, precision=PREC_FP32, rank_tol=float(rank_tol), flags=0,
                                    reserved=0)
        xp = (_P * cnt)(*[X.data_ptr() for X in self._X])
        ap = (_P * cnt)(*[A.data_ptr() for A in self._A1])
        h = C.c_void_p()
        st = lib.godec_batch_init(C.byref(h), cnt, params, xp, ap, 0 if tune else BATCH_NO_TUNE,
                                  _stream_ptr(stream))
        _bcheck(st, "godec_batch_init", None)
        self._b = h
        self.count = cnt
        self._shapes = [tuple(X.shape) for X in Xs]

    def close(self):
        if getattr(self, "_b", None):
            library().godec_batch_destroy(self._b)
            self._b = None

    __del__ = close

    def iterate(self, n_iter: int = 1):
        _bcheck(library().godec_batch_iterate(self._b, int(n_iter)), "godec_batch_iterate", self._b)

    def reset(self):
        _bcheck(library().godec_batch_reset(self._b), "godec_batch_reset", self._b)

    def problem(self, i: int) -> GoDec:
        h = library().godec_batch_problem(self._b, int(i))
        if not h:
            raise IndexError(f"problem {i} out of range")
        m, n = self._shapes[i]
        return _Problem(self, C.c_void_p(h), self._X[i][:, :n], self._A1[i], self.rs[i], self.ks[i], self.qs[i])

    def tuning(self) -> dict:
        sm = (C.c_int32 * self.count)()
        ms = (C.c_double * BATCH_POLICIES)()
        pol, rec = C.c_int32(0), C.c_int32(0)
        _bcheck(library().godec_batch_tuning(self._b, sm, ms, C.byref(pol), C.byref(rec)), "godec_batch_tuning",
                self._b)
        return {"sm": list(sm), "policy_ms": list(ms), "policy": pol.value, "recaptures": rec.value}


def batch_budgets(shapes, nsm: int, policy: int):
    """The batched form's SM budgets of one tuner policy (host logic, no device work)."""
    cnt = len(shapes)
    m = (C.c_int64 * cnt)(*[int(a) for a, _ in shapes])
    n = (C.c_int64 * cnt)(*[int(b) for _, b in shapes])
    out = (C.c_int32 * cnt)()
    _check(library().godec_batch_budgets(cnt, m, n, int(nsm), int(policy), out), "godec_batch_budgets")
    return list(out)


def tc_geometry(rows: int, K: int, nsm: int) -> dict:
    """Stream-K geometry of the tensor-core product (host logic, no device work)."""
    out = (C.c_int64 * 6)()
    _check(library().godec_tc_geometry(int(rows), int(K), int(nsm), out), "godec_tc_geometry")
    return dict(zip(("tiles", "ks", "S", "G", "maxseg", "maxpend"), list(out)))
