"""FP64 CPU oracle for the Secant-Avoidance Projection (SAP) algorithm.

TEST INFRASTRUCTURE ONLY.  This package is the correctness bar for the CUDA
library in ``paper_1807_03425_gb300``; the two share no code.  Only the test
suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import it.  The product path never does.

The arithmetic lives in ``sap_oracle.c`` (plain FP64 C, compiled with gcc into
``liboracle_sap.so`` next to this file); this module only marshals arguments.
Conventions: X is N x n row-major FP64 (FP32/BF16 inputs are widened exactly
before the call), U is n x k column-major, i.e. a C-contiguous (k, n) array
whose row c is the basis vector u_c.  Pairs are (i, j) with i < j.

Paper: Kvinge, Farnell, Kirby, Peterson, "A GPU-Oriented Algorithm Design for
Secant-Based Dimensionality Reduction", arXiv:1807.03425 (Sec. IV,
Algorithm 1; Sec. VI-A for dimension estimation; Sec. VII for the
noisy-data threshold).  The soft-min objective is not in the paper; its
definition is stated in ``orc_softmin``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sap_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_sap.so")
_lock = threading.Lock()
_lib = None

MODE_LITERAL = 0
MODE_ANGLE = 1


def build(force: bool = False) -> str:
    """Compile sap_oracle.c into liboracle_sap.so (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        ip = ctypes.POINTER(ctypes.c_int)
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_pair_index.argtypes = [i64, i64, i64]
        lib.orc_pair_index.restype = i64
        lib.orc_ratio.argtypes = [dp, i64, i32, dp, i32, i64, i64, f64]
        lib.orc_ratio.restype = f64
        lib.orc_all_ratios.argtypes = [dp, i64, i32, dp, i32, f64, dp]
        lib.orc_min_secant.argtypes = [dp, i64, i32, dp, i32, f64, i64p, i64p,
                                       dp, dp, i64p]
        lib.orc_min_secant.restype = i32
        lib.orc_update_with_secant.argtypes = [dp, dp, i32, i32, f64, i32, dp, ip]
        lib.orc_update.argtypes = [dp, i64, i32, dp, i32, i64, i64, f64, i32,
                                   dp, ip]
        lib.orc_unit_secant.argtypes = [dp, i32, i64, i64, dp]
        lib.orc_run.argtypes = [dp, i64, i32, dp, i32, f64, i32, f64, i32, dp,
                                dp, i64p]
        lib.orc_run.restype = i32
        lib.orc_estimate_dim.argtypes = [dp, i64, i32, dp, i32, i32, f64, f64,
                                         i32, f64, dp, ip]
        lib.orc_estimate_dim.restype = i32
        lib.orc_softmin.argtypes = [dp, i64, i32, dp, i32, f64, f64, dp, dp]
        lib.orc_softmin.restype = i32
        lib.orc_num_threads.restype = i32
        lib.orc_secant_gram.argtypes = [dp, i64, i32, f64, dp]
        lib.orc_secant_gram.restype = i64
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _x(X):
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    assert X.ndim == 2
    return X


def _u(U):
    """Basis as a C-contiguous (k, n) FP64 array (= n x k column-major)."""
    U = np.ascontiguousarray(np.asarray(U, dtype=np.float64))
    assert U.ndim == 2
    return U


class NoSecantError(RuntimeError):
    """Every pair is excluded (N < 2, duplicates only, or eps too large)."""


def num_threads() -> int:
    return int(_load().orc_num_threads())


def pair_index(i: int, j: int, N: int) -> int:
    return int(_load().orc_pair_index(i, j, N))


def ratio(X, U, i: int, j: int, eps: float = 0.0) -> float:
    """||U^T s_ij|| for one pair; -1 if the pair is excluded (Sec. IV, VII)."""
    X, U = _x(X), _u(U)
    return float(_load().orc_ratio(_dp(X), X.shape[0], X.shape[1], _dp(U),
                                   U.shape[0], i, j, eps))


def all_ratios(X, U, eps: float = 0.0) -> np.ndarray:
    """All N(N-1)/2 ratios in pair-index order; -1 marks excluded pairs."""
    X, U = _x(X), _u(U)
    N = X.shape[0]
    out = np.empty(N * (N - 1) // 2, dtype=np.float64)
    _load().orc_all_ratios(_dp(X), N, X.shape[1], _dp(U), U.shape[0], eps,
                           _dp(out))
    return out


def min_secant(X, U, eps: float = 0.0):
    """Algorithm 1, argmin step.  Returns dict(i, j, r, runner_up, excluded)."""
    X, U = _x(X), _u(U)
    i, j = ctypes.c_int64(), ctypes.c_int64()
    r, r2 = ctypes.c_double(), ctypes.c_double()
    ex = ctypes.c_int64()
    rc = _load().orc_min_secant(_dp(X), X.shape[0], X.shape[1], _dp(U),
                                U.shape[0], eps, ctypes.byref(i),
                                ctypes.byref(j), ctypes.byref(r),
                                ctypes.byref(r2), ctypes.byref(ex))
    if rc != 0:
        raise NoSecantError("every pair is excluded")
    return dict(i=i.value, j=j.value, r=r.value, runner_up=r2.value,
                excluded=ex.value)


def unit_secant(X, i: int, j: int) -> np.ndarray:
    X = _x(X)
    s = np.empty(X.shape[1], dtype=np.float64)
    _load().orc_unit_secant(_dp(X), X.shape[1], i, j, _dp(s))
    return s


def update_with_secant(s, U, alpha: float, mode: int = MODE_LITERAL):
    """Algorithm 1 update (pivot, MGS, rotation, re-orthonormalisation) for a
    given unit secant s.  Returns (U_new as (k, n), pivot t 0-based)."""
    U = _u(U)
    s = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    k, n = U.shape
    out = np.empty_like(U)
    t = ctypes.c_int()
    _load().orc_update_with_secant(_dp(s), _dp(U), n, k, alpha, mode, _dp(out),
                                   ctypes.byref(t))
    return out, t.value


def update(X, U, i: int, j: int, alpha: float, mode: int = MODE_LITERAL):
    """Update toward the unit secant of pair (i, j).  Returns (U_new, t)."""
    X, U = _x(X), _u(U)
    k, n = U.shape
    out = np.empty_like(U)
    t = ctypes.c_int()
    _load().orc_update(_dp(X), X.shape[0], n, _dp(U), k, i, j, alpha, mode,
                       _dp(out), ctypes.byref(t))
    return out, t.value


def step(X, U, alpha: float, eps: float = 0.0, mode: int = MODE_LITERAL):
    """One SAP iteration: evaluate, then update.  Returns (U_new, min_info)."""
    m = min_secant(X, U, eps)
    Un, _ = update(X, U, m["i"], m["j"], alpha, mode)
    return Un, m


def run(X, U0, alpha: float, T: int, eps: float = 0.0,
        mode: int = MODE_LITERAL):
    """T SAP iterations.  Returns (U_T, hist[T+1], argmin[(T+1), 2])."""
    X, U0 = _x(X), _u(U0)
    k, n = U0.shape
    Uo = np.empty_like(U0)
    hist = np.empty(T + 1, dtype=np.float64)
    am = np.empty((T + 1, 2), dtype=np.int64)
    rc = _load().orc_run(_dp(X), X.shape[0], n, _dp(U0), k, alpha, T, eps,
                         mode, _dp(Uo), _dp(hist),
                         am.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc != 0:
        raise NoSecantError("every pair is excluded")
    return Uo, hist, am


def estimate_dim(X, U0full, T: int, alpha: float, threshold: float,
                 eps: float = 0.0, mode: int = MODE_LITERAL):
    """Sec. VI-A sweep over k = 1..kmax (U0full is (kmax, n); basis k uses its
    first k rows).  Returns (k_out or -1, ratios[kmax])."""
    X, U0 = _x(X), _u(U0full)
    kmax, n = U0.shape
    ratios = np.empty(kmax, dtype=np.float64)
    kout = ctypes.c_int()
    rc = _load().orc_estimate_dim(_dp(X), X.shape[0], n, _dp(U0), kmax, T,
                                  alpha, eps, mode, threshold, _dp(ratios),
                                  ctypes.byref(kout))
    if rc != 0:
        raise NoSecantError("every pair is excluded")
    return kout.value, ratios


def softmin(X, U, tau: float, eps: float = 0.0, grad: bool = True):
    """Soft-min objective L(U) = -tau log sum exp(-r_ij/tau) and dL/dU
    (returned as (k, n), like U)."""
    X, U = _x(X), _u(U)
    k, n = U.shape
    L = ctypes.c_double()
    G = np.empty_like(U) if grad else None
    rc = _load().orc_softmin(_dp(X), X.shape[0], n, _dp(U), k, tau, eps,
                             ctypes.byref(L), _dp(G) if grad else None)
    if rc != 0:
        raise NoSecantError("every pair is excluded")
    return (L.value, G) if grad else L.value


def qf(A):
    """Q factor of a thin QR with a non-negative diagonal of R.  A is (k, n)
    (rows are vectors); returns Q in the same (k, n) form."""
    Q, R = np.linalg.qr(np.asarray(A, dtype=np.float64).T)
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return np.ascontiguousarray((Q * sgn).T)


def softmin_ascent_step(X, U, tau: float, eta: float, eps: float = 0.0):
    """One Riemannian gradient-ascent step on the soft-min objective:
    G_R = G - U (U^T G) (tangent projection), U <- qf(U + eta G_R/||G_R||_F).
    Returns (U_new, L, ||G_R||_F).  All arrays are (k, n)."""
    U = _u(U)
    L, G = softmin(X, U, tau, eps)
    # rows are vectors, so the n x k product U (U^T G) is (G U^T) U here
    GR = G - (G @ U.T) @ U
    nr = float(np.linalg.norm(GR))
    if nr == 0.0:
        return U.copy(), L, 0.0
    return qf(U + eta * GR / nr), L, nr


def secant_gram(X, eps: float = 0.0):
    """C = S S^T = sum over kept pairs of s s^T (unit secants s; Sec. IV),
    n x n FP64, and the number of kept pairs."""
    X = _x(X)
    n = X.shape[1]
    C = np.empty((n, n), dtype=np.float64)
    kept = _load().orc_secant_gram(_dp(X), X.shape[0], n, eps, _dp(C))
    if kept < 0:
        raise NoSecantError("every pair is excluded")
    return C, int(kept)


def secant_pca(X, k: int, eps: float = 0.0):
    """The PCA start of Algorithm 1 (Sec. IV): the top k left singular vectors
    of the unit-secant matrix S, i.e. the eigenvectors of S S^T with the k
    largest eigenvalues (numpy's symmetric eigensolver serves as the step),
    each signed so that its entry of largest magnitude is positive.  Returns
    (U as (k, n), the k singular values sqrt(lambda), descending)."""
    C, _ = secant_gram(X, eps)
    lam, V = np.linalg.eigh(C)
    order = np.argsort(lam)[::-1][:k]
    U = V[:, order].T.copy()
    for c in range(k):
        if U[c, np.argmax(np.abs(U[c]))] < 0:
            U[c] = -U[c]
    return np.ascontiguousarray(U), np.sqrt(np.maximum(lam[order], 0.0))
