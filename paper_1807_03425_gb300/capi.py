"""ctypes binding of libsap (include/sap.h).

Module-level functions carry the C names (``sap_create``, ``sap_step`` ...)
and only marshal arguments; ``Sap`` is a small handle wrapper on top.  Arrays
may be NumPy (host) or torch CUDA tensors (device; passed by pointer, no
copy).  A basis is handled as a (k, n) C-contiguous FP64 array, which is the
n x k column-major layout of the C ABI.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SAP_LIBRARY selects another build of the library (e.g. the debug build
# libsap_dbg.so, see build.py)
_LIB_PATH = os.environ.get("SAP_LIBRARY") or os.path.join(_HERE, "libsap.so")
_lib = None

F32, BF16, F64 = 0, 1, 2
PLAIN, RESTRUCTURED = 0, 1
UPDATE_LITERAL, UPDATE_ANGLE = 0, 1
SPLIT_FP16, SPLIT_BF16 = 0, 1
KERNEL_CLASSES = {"gemm_y": 0, "restructured_pass": 1, "plain_pass": 2,
                  "second_tier": 3, "refine": 3, "explicit_recheck": 3, "ydf": 4, "select_update": 5, "update": 5,
                  "softmin_forward": 6, "softmin_backward": 7, "softmin_near": 8,
                  "softmin_other": 9}

STATUS = {0: "SAP_OK", 1: "SAP_E_ARG", 2: "SAP_E_STATE", 3: "SAP_E_NOT_ORTHONORMAL",
          4: "SAP_E_NO_SECANT", 5: "SAP_E_OOM", 6: "SAP_E_CUDA", 7: "SAP_E_TIMEOUT",
          8: "SAP_E_NO_DEVICE", 9: "SAP_E_UNSUPPORTED"}


class SapError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        self.name = STATUS.get(code, "SAP_E_%d" % code)
        super().__init__("%s%s" % (self.name, (": " + msg) if msg else ""))


class Stats(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_dim", ctypes.c_int32),
                ("k", ctypes.c_int32), ("n_pairs", ctypes.c_int64),
                ("n_excluded", ctypes.c_int64), ("n_near", ctypes.c_int64),
                ("last_tier1", ctypes.c_int64), ("last_tier2", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("cert_bound", ctypes.c_double),
                ("y_error_unit", ctypes.c_double), ("ydf_error_unit", ctypes.c_double)]


class Record(ctypes.Structure):
    """One rank's minimum in the multi-GPU split: FP64 squared ratio q and
    the pair (i, j); i = j = -1 when the rank has no candidate."""
    _fields_ = [("q", ctypes.c_double), ("i", ctypes.c_int32), ("j", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("pass_bound", ctypes.c_double), ("pass_stages", ctypes.c_int32),
                ("explicit_blocks_per_sm", ctypes.c_int32), ("update_blocks", ctypes.c_int32),
                ("plain_blocks_per_sm", ctypes.c_int32), ("programmatic_launch", ctypes.c_int32),
                ("refine_tier", ctypes.c_int32), ("us_per_iteration", ctypes.c_double)]


def _tuning_dict(t):
    return {name: getattr(t, name) for name, _ in Tuning._fields_}


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libsap.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError("libsap.so is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    i64p, f64p, i32p = (ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_int32))
    sig = {
        "sap_version": ([], ctypes.c_char_p),
        "sap_status_str": ([i32], ctypes.c_char_p),
        "sap_last_error": ([vp], ctypes.c_char_p),
        "sap_create": ([vp, i64, i32, i32, i32, ctypes.POINTER(vp)], i32),
        "sap_destroy": ([vp], i32),
        "sap_set_stream": ([vp, vp], i32),
        "sap_set_path": ([vp, i32], i32),
        "sap_set_update_mode": ([vp, i32], i32),
        "sap_set_split": ([vp, i32], i32),
        "sap_set_min_secant_length": ([vp, f64], i32),
        "sap_set_basis": ([vp, vp, i32, i32], i32),
        "sap_get_basis": ([vp, vp, i32], i32),
        "sap_min_secant": ([vp, i64p, i64p, f64p], i32),
        "sap_step": ([vp, f64, i64p, i64p, f64p], i32),
        "sap_run": ([vp, f64, i32, vp, vp], i32),
        "sap_get_history": ([vp, vp, vp, i32], i32),
        "sap_estimate_dim": ([vp, vp, i32, i32, f64, f64, i32p, vp], i32),
        "sap_get_sweep_history": ([vp, i32, vp, vp, i32], i32),
        "sap_get_sweep_basis": ([vp, i32, vp, i32], i32),
        "sap_create_batch": ([vp, vp, i32, i32, i32, i32, ctypes.POINTER(vp)], i32),
        "sap_batch_count": ([vp, i32p], i32),
        "sap_set_basis_b": ([vp, i32, vp, i32, i32], i32),
        "sap_get_basis_b": ([vp, i32, vp, i32], i32),
        "sap_min_secant_b": ([vp, i32, i64p, i64p, f64p], i32),
        "sap_run_batch": ([vp, f64, i32, vp, vp], i32),
        "sap_project": ([vp, vp, i32], i32),
        "sap_min_secant_noalloc": ([vp, i64, i32, vp, i32, f64, vp, i64p, i64p, f64p], i32),
        "sap_get_stats": ([vp, ctypes.POINTER(Stats)], i32),
        "sap_set_profiling": ([vp, i32], i32),
        "sap_get_kernel_time": ([vp, i32, f64p, i64p], i32),
        "sap_softmin_forward": ([vp, f64, f64p], i32),
        "sap_softmin_backward": ([vp, f64, f64, vp, i32], i32),
        "sap_softmin_ascent": ([vp, f64, f64, i32, vp], i32),
        "sap_set_pass_bound": ([vp, f64], i32),
        "sap_secant_pca": ([vp, i32, vp, vp], i32),
        "sap_create_subsamples": ([vp, i64, i32, i32, i32, vp, i32, i32, ctypes.POINTER(vp)], i32),
        "sap_estimate_dim_b": ([vp, i32, vp, i32, i32, f64, f64, ctypes.POINTER(i32), vp], i32),
        "sap_project_df": ([vp, vp, vp, i32], i32),
        "sap_autotune": ([vp, f64, i32, ctypes.POINTER(Tuning)], i32),
        "sap_get_tuning": ([vp, ctypes.POINTER(Tuning)], i32),
        "sap_set_tuning": ([vp, ctypes.POINTER(Tuning)], i32),
        "sap_shard_range": ([i64, i32, i32, i64p, i64p, i64p], i32),
        "sap_merge_records": ([ctypes.POINTER(Record), i32, ctypes.POINTER(Record)], i32),
        "sap_create_shard": ([vp, i64, i32, i32, i32, i32, i32, ctypes.POINTER(vp)], i32),
        "sap_shard_min": ([vp, vp, i32], i32),
        "sap_shard_step": ([vp, f64, vp, i32, i32], i32),
        "sap_inject_fault": ([vp, i32], i32),
        "sap_selftest_wait": ([vp, i64], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_names():
    """Names of the C entry points this binding wraps."""
    load_library()
    return sorted(n for n in globals() if n.startswith("sap_") and callable(globals()[n]))


def _ptr(a):
    """(pointer, is_device) of a NumPy array or a torch tensor."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        return ctypes.c_void_p(a.data_ptr()), int(bool(a.is_cuda))
    return a.ctypes.data_as(ctypes.c_void_p), 0


def _check(h, code):
    if code != 0:
        msg = load_library().sap_last_error(h).decode() if h else ""
        raise SapError(code, msg)


# ----------------------------------------------------------- C entry points --

def sap_version():
    return load_library().sap_version().decode()


def sap_status_str(code):
    return load_library().sap_status_str(code).decode()


def sap_last_error(h):
    return load_library().sap_last_error(h).decode()


def sap_create(X, dtype=None):
    """X: (N, n) NumPy array (float32, float64, or uint16 BF16 bits) or a torch
    CUDA tensor (float32, float64, bfloat16).  Returns a handle."""
    lib = load_library()
    if dtype is None:
        dt = str(getattr(X, "dtype", ""))
        if "float64" in dt:
            dtype = F64
        elif "bfloat16" in dt or "uint16" in dt:
            dtype = BF16
        else:
            dtype = F32
    if not hasattr(X, "data_ptr"):
        want = {F32: np.float32, F64: np.float64, BF16: np.uint16}[dtype]
        X = np.ascontiguousarray(X, dtype=want)
    elif not X.is_contiguous():
        raise ValueError("X must be contiguous")
    N, n = X.shape
    p, dev = _ptr(X)
    h = ctypes.c_void_p()
    code = lib.sap_create(p, N, n, dtype, dev, ctypes.byref(h))
    if code != 0:
        raise SapError(code, "sap_create(N=%d, n=%d)" % (N, n))
    return h


def sap_destroy(h):
    _check(None, load_library().sap_destroy(h))


def sap_set_stream(h, stream):
    """stream: torch.cuda.Stream, an integer cudaStream_t, or None."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(h, load_library().sap_set_stream(h, ctypes.c_void_p(stream) if stream else None))


def sap_set_path(h, path):
    _check(h, load_library().sap_set_path(h, path))


def sap_set_update_mode(h, mode):
    _check(h, load_library().sap_set_update_mode(h, mode))


def sap_set_split(h, split):
    _check(h, load_library().sap_set_split(h, split))


def sap_set_min_secant_length(h, eps):
    _check(h, load_library().sap_set_min_secant_length(h, float(eps)))


def sap_secant_pca(h, k, n):
    """PCA start (Sec. IV): sets and returns the basis ((k, n) FP64) and the
    k singular values of the unit-secant matrix."""
    U = np.empty((k, n), dtype=np.float64)
    sv = np.empty(k, dtype=np.float64)
    _check(h, load_library().sap_secant_pca(h, int(k), U.ctypes.data_as(ctypes.c_void_p),
                                            sv.ctypes.data_as(ctypes.c_void_p)))
    return U, sv


def sap_set_pass_bound(h, b_cap):
    _check(h, load_library().sap_set_pass_bound(h, b_cap))


def sap_autotune(h, alpha, iters):
    t = Tuning()
    _check(h, load_library().sap_autotune(h, alpha, iters, ctypes.byref(t)))
    return _tuning_dict(t)


def sap_get_tuning(h):
    t = Tuning()
    _check(h, load_library().sap_get_tuning(h, ctypes.byref(t)))
    return _tuning_dict(t)


def sap_set_tuning(h, **params):
    t = Tuning()
    cur = sap_get_tuning(h) if params.keys() != {n for n, _ in Tuning._fields_} else {}
    cur.update(params)
    for name, _ in Tuning._fields_:
        setattr(t, name, cur.get(name, 0))
    _check(h, load_library().sap_set_tuning(h, ctypes.byref(t)))


def sap_set_basis(h, U):
    """U: (k, n) FP64 (NumPy or torch CUDA tensor), rows = basis vectors."""
    if not hasattr(U, "data_ptr"):
        U = np.ascontiguousarray(U, dtype=np.float64)
    p, dev = _ptr(U)
    _check(h, load_library().sap_set_basis(h, p, U.shape[0], dev))


def sap_get_basis(h, k, n, out=None):
    if out is None:
        out = np.empty((k, n), dtype=np.float64)
    p, dev = _ptr(out)
    _check(h, load_library().sap_get_basis(h, p, dev))
    return out


def sap_min_secant(h):
    i, j, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(h, load_library().sap_min_secant(h, ctypes.byref(i), ctypes.byref(j), ctypes.byref(r)))
    return i.value, j.value, r.value


def sap_step(h, alpha, sync=True):
    lib = load_library()
    if not sync:
        _check(h, lib.sap_step(h, float(alpha), None, None, None))
        return None
    i, j, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(h, lib.sap_step(h, float(alpha), ctypes.byref(i), ctypes.byref(j), ctypes.byref(r)))
    return i.value, j.value, r.value


def sap_run(h, alpha, iters, history=True):
    lib = load_library()
    if not history:
        _check(h, lib.sap_run(h, float(alpha), int(iters), None, None))
        return None
    hist = np.empty(iters + 1, dtype=np.float64)
    am = np.empty((iters + 1, 2), dtype=np.int64)
    _check(h, lib.sap_run(h, float(alpha), int(iters), hist.ctypes.data_as(ctypes.c_void_p),
                          am.ctypes.data_as(ctypes.c_void_p)))
    return hist, am


def sap_get_history(h, count):
    hist = np.empty(count, dtype=np.float64)
    am = np.empty((count, 2), dtype=np.int64)
    _check(h, load_library().sap_get_history(h, hist.ctypes.data_as(ctypes.c_void_p),
                                             am.ctypes.data_as(ctypes.c_void_p), count))
    return hist, am


def sap_estimate_dim(h, U0, iters, alpha, threshold):
    """U0: (k_max, n) FP64; returns (k or -1, ratios[k_max])."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    kmax = U0.shape[0]
    ratios = np.empty(kmax, dtype=np.float64)
    kout = ctypes.c_int32()
    _check(h, load_library().sap_estimate_dim(h, U0.ctypes.data_as(ctypes.c_void_p), kmax,
                                              int(iters), float(alpha), float(threshold),
                                              ctypes.byref(kout),
                                              ratios.ctypes.data_as(ctypes.c_void_p)))
    return kout.value, ratios


def sap_get_sweep_history(h, k, count):
    hist = np.empty(count, dtype=np.float64)
    am = np.empty((count, 2), dtype=np.int64)
    _check(h, load_library().sap_get_sweep_history(h, int(k), hist.ctypes.data_as(ctypes.c_void_p),
                                                   am.ctypes.data_as(ctypes.c_void_p), int(count)))
    return hist, am


def sap_get_sweep_basis(h, k, n, out=None):
    if out is None:
        out = np.empty((k, n), dtype=np.float64)
    p, dev = _ptr(out)
    _check(h, load_library().sap_get_sweep_basis(h, int(k), p, dev))
    return out


def sap_project(h, out):
    """out: (N, k) float32 NumPy array or torch CUDA tensor."""
    p, dev = _ptr(out)
    _check(h, load_library().sap_project(h, p, dev))
    return out


def sap_project_df(h, out_hi, out_lo):
    """Extended-precision projection (hi + lo FP32 pairs, N x k each)."""
    lib = load_library()
    if hasattr(out_hi, "data_ptr"):
        _check(h, lib.sap_project_df(h, ctypes.c_void_p(out_hi.data_ptr()), ctypes.c_void_p(out_lo.data_ptr()), 1))
    else:
        _check(h, lib.sap_project_df(h, out_hi.ctypes.data_as(ctypes.c_void_p),
                                     out_lo.ctypes.data_as(ctypes.c_void_p), 0))
    return out_hi, out_lo


def sap_min_secant_noalloc(X, U, eps=0.0, stream=None):
    """Allocation-free argmin for callers that must not allocate device
    memory: X (N, n) float32 and U (k, n) float64 contiguous torch CUDA
    tensors on one device; returns (i, j, ratio).  Runs on `stream` (a
    torch.cuda.Stream or a raw cudaStream_t), by default torch's current
    stream on X's device, and synchronises it.  Limits N <= 1024, n <= 1024,
    k <= 8; concurrent calls on one device must be serialised (they share a
    fixed scratch array)."""
    import torch
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32
            and X.dim() == 2 and X.is_contiguous()):
        raise TypeError("X must be a contiguous (N, n) float32 CUDA tensor")
    if not (isinstance(U, torch.Tensor) and U.is_cuda and U.dtype == torch.float64
            and U.dim() == 2 and U.is_contiguous()):
        raise TypeError("U must be a contiguous (k, n) float64 CUDA tensor")
    if U.device != X.device or U.shape[1] != X.shape[1]:
        raise ValueError("X and U must share the device and the dimension n")
    if stream is None:
        stream = torch.cuda.current_stream(X.device)
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    i, j, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    code = load_library().sap_min_secant_noalloc(
        ctypes.c_void_p(X.data_ptr()), X.shape[0], X.shape[1], ctypes.c_void_p(U.data_ptr()),
        U.shape[0], float(eps), ctypes.c_void_p(stream) if stream else None,
        ctypes.byref(i), ctypes.byref(j), ctypes.byref(r))
    if code != 0:
        raise SapError(code, "sap_min_secant_noalloc")
    return i.value, j.value, r.value


def sap_shard_range(N, world, rank):
    """(t0, t1, pairs): the tile range [t0, t1) and pair count of `rank` among
    `world` for N points (host only, no device needed)."""
    t0, t1, pairs = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    code = load_library().sap_shard_range(N, world, rank, ctypes.byref(t0), ctypes.byref(t1), ctypes.byref(pairs))
    if code != 0:
        raise SapError(code, "sap_shard_range(N=%d, world=%d, rank=%d)" % (N, world, rank))
    return t0.value, t1.value, pairs.value


def sap_merge_records(recs):
    """The winning record of a sequence of (q, i, j) (host only); None when no
    record holds a pair."""
    arr = (Record * len(recs))(*[Record(float(q), int(i), int(j)) for q, i, j in recs])
    out = Record()
    code = load_library().sap_merge_records(arr, len(recs), ctypes.byref(out))
    if code == 4:
        return None
    if code != 0:
        raise SapError(code, "sap_merge_records")
    return out.q, out.i, out.j


def sap_create_shard(X, world, rank, dtype=None):
    """As sap_create, for rank `rank` of `world` (restructured form)."""
    lib = load_library()
    if dtype is None:
        dtype = BF16 if ("bfloat16" in str(getattr(X, "dtype", "")) or "uint16" in str(getattr(X, "dtype", ""))) else F32
    if not hasattr(X, "data_ptr"):
        X = np.ascontiguousarray(X, dtype={F32: np.float32, BF16: np.uint16}[dtype])
    elif not X.is_contiguous():
        raise ValueError("X must be contiguous")
    N, n = X.shape
    p, dev = _ptr(X)
    h = ctypes.c_void_p()
    code = lib.sap_create_shard(p, N, n, dtype, dev, world, rank, ctypes.byref(h))
    if code != 0:
        raise SapError(code, "sap_create_shard(N=%d, n=%d, world=%d, rank=%d)" % (N, n, world, rank))
    return h


def sap_shard_min(h, out=None):
    """This rank's minimum: into `out` (a 16-byte torch CUDA tensor, no
    synchronisation) or, with out None, returned as (q, i, j)."""
    lib = load_library()
    if out is not None:
        _check(h, lib.sap_shard_min(h, ctypes.c_void_p(out.data_ptr()), 1))
        return out
    r = Record()
    _check(h, lib.sap_shard_min(h, ctypes.byref(r), 0))
    return r.q, r.i, r.j


def sap_shard_step(h, alpha, recs):
    """The update from all ranks' records: a torch CUDA tensor of count x 16
    bytes (no synchronisation) or a sequence of (q, i, j) tuples."""
    lib = load_library()
    if hasattr(recs, "data_ptr"):
        count = recs.numel() * recs.element_size() // 16
        _check(h, lib.sap_shard_step(h, float(alpha), ctypes.c_void_p(recs.data_ptr()), count, 1))
        return
    arr = (Record * len(recs))(*[Record(float(q), int(i), int(j)) for q, i, j in recs])
    _check(h, lib.sap_shard_step(h, float(alpha), ctypes.cast(arr, ctypes.c_void_p), len(recs), 0))


def sap_inject_fault(h, kind):
    """Test hook: the next checked CUDA call of the handle fails (kind 1: an
    allocation failure, 2: a sticky CUDA error).  Returns the status code."""
    return load_library().sap_inject_fault(h, int(kind))


def sap_selftest_wait(budget_cycles, stream=None):
    """Test hook: a kernel whose bounded mbarrier wait runs out after
    budget_cycles SM clocks.  Returns the status code (SAP_E_TIMEOUT)."""
    return load_library().sap_selftest_wait(ctypes.c_void_p(stream) if stream else None, int(budget_cycles))


def sap_get_stats(h):
    s = Stats()
    _check(h, load_library().sap_get_stats(h, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in Stats._fields_}


def sap_set_profiling(h, enable):
    _check(h, load_library().sap_set_profiling(h, int(bool(enable))))


def sap_get_kernel_time(h, kernel_class):
    if isinstance(kernel_class, str):
        kernel_class = KERNEL_CLASSES[kernel_class]
    ms, cnt = ctypes.c_double(), ctypes.c_int64()
    _check(h, load_library().sap_get_kernel_time(h, kernel_class, ctypes.byref(ms),
                                                 ctypes.byref(cnt)))
    return ms.value, cnt.value


def sap_softmin_forward(h, tau):
    L = ctypes.c_double()
    _check(h, load_library().sap_softmin_forward(h, float(tau), ctypes.byref(L)))
    return L.value


def sap_softmin_backward(h, tau, L, k, n, out=None):
    """dL/dU as (k, n) FP64 (NumPy, or the given torch CUDA tensor)."""
    if out is None:
        out = np.empty((k, n), dtype=np.float64)
    p, dev = _ptr(out)
    _check(h, load_library().sap_softmin_backward(h, float(tau), float(L), p, dev))
    return out


def sap_softmin_ascent(h, tau, eta, steps):
    hist = np.empty(int(steps) + 1, dtype=np.float64)
    _check(h, load_library().sap_softmin_ascent(h, float(tau), float(eta), int(steps),
                                                hist.ctypes.data_as(ctypes.c_void_p)))
    return hist


def sap_create_batch(Xs, dtype=None):
    """Xs: list of (N_b, n) NumPy arrays (float32, float64, or uint16 BF16
    bits) of one dtype and n.  Returns a batch handle."""
    lib = load_library()
    if dtype is None:
        dt = str(Xs[0].dtype)
        dtype = F64 if "float64" in dt else (BF16 if "uint16" in dt or "bfloat16" in dt else F32)
    want = {F32: np.float32, F64: np.float64, BF16: np.uint16}[dtype]
    arrs = [np.ascontiguousarray(X, dtype=want) for X in Xs]
    n = arrs[0].shape[1]
    ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data_as(ctypes.c_void_p) for a in arrs])
    Ns = (ctypes.c_int64 * len(arrs))(*[a.shape[0] for a in arrs])
    h = ctypes.c_void_p()
    code = lib.sap_create_batch(ctypes.cast(ptrs, ctypes.c_void_p), ctypes.cast(Ns, ctypes.c_void_p),
                                len(arrs), n, dtype, 0, ctypes.byref(h))
    if code != 0:
        raise SapError(code, "sap_create_batch(B=%d, n=%d)" % (len(arrs), n))
    return h


def sap_create_subsamples(X, idx, dtype=None):
    """X: (N, n) NumPy array (float32, float64 or uint16 BF16 bits); idx:
    (R, m) int64 row indices.  Returns a batch handle of the R subsets."""
    lib = load_library()
    if dtype is None:
        dt = str(X.dtype)
        dtype = F64 if "float64" in dt else (BF16 if "uint16" in dt or "bfloat16" in dt or "int16" in dt else F32)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    R, m = idx.shape
    h = ctypes.c_void_p()
    if hasattr(X, "data_ptr"):  # a contiguous CUDA tensor: rows gathered on the device
        ptr, dev = ctypes.c_void_p(X.contiguous().data_ptr()), 1
    else:
        want = {F32: np.float32, F64: np.float64, BF16: np.uint16}[dtype]
        X = np.ascontiguousarray(X, dtype=want)
        ptr, dev = X.ctypes.data_as(ctypes.c_void_p), 0
    code = lib.sap_create_subsamples(ptr, X.shape[0], X.shape[1], dtype, dev,
                                     idx.ctypes.data_as(ctypes.c_void_p), R, m, ctypes.byref(h))
    if code != 0:
        raise SapError(code, "sap_create_subsamples(N=%d, R=%d, m=%d)" % (X.shape[0], R, m))
    return h


def sap_estimate_dim_b(h, b, U0, iters, alpha, threshold):
    """Dimension sweep of dataset b of a batch; as sap_estimate_dim."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    kmax = U0.shape[0]
    ratios = np.empty(kmax, dtype=np.float64)
    kout = ctypes.c_int32()
    _check(h, load_library().sap_estimate_dim_b(h, int(b), U0.ctypes.data_as(ctypes.c_void_p), kmax, int(iters),
                                                float(alpha), float(threshold), ctypes.byref(kout),
                                                ratios.ctypes.data_as(ctypes.c_void_p)))
    return kout.value, ratios


def sap_batch_count(h):
    b = ctypes.c_int32()
    _check(h, load_library().sap_batch_count(h, ctypes.byref(b)))
    return b.value


def sap_set_basis_b(h, b, U):
    if not hasattr(U, "data_ptr"):
        U = np.ascontiguousarray(U, dtype=np.float64)
    p, dev = _ptr(U)
    _check(h, load_library().sap_set_basis_b(h, int(b), p, U.shape[0], dev))


def sap_get_basis_b(h, b, k, n, out=None):
    if out is None:
        out = np.empty((k, n), dtype=np.float64)
    p, dev = _ptr(out)
    _check(h, load_library().sap_get_basis_b(h, int(b), p, dev))
    return out


def sap_min_secant_b(h, b):
    i, j, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(h, load_library().sap_min_secant_b(h, int(b), ctypes.byref(i), ctypes.byref(j), ctypes.byref(r)))
    return i.value, j.value, r.value


def sap_run_batch(h, alpha, iters, B, history=True):
    lib = load_library()
    if not history:
        _check(h, lib.sap_run_batch(h, float(alpha), int(iters), None, None))
        return None
    hist = np.empty((B, iters + 1), dtype=np.float64)
    am = np.empty((B, iters + 1, 2), dtype=np.int64)
    _check(h, lib.sap_run_batch(h, float(alpha), int(iters), hist.ctypes.data_as(ctypes.c_void_p),
                                am.ctypes.data_as(ctypes.c_void_p)))
    return hist, am


# ------------------------------------------------------------ handle class --

class Sap:
    """One dataset on the GPU.  Methods follow the C entry points."""

    def __init__(self, X, dtype=None):
        self.N, self.n = int(X.shape[0]), int(X.shape[1])
        self.h = sap_create(X, dtype)
        self.k = 0

    def close(self):
        if self.h:
            sap_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        sap_set_stream(self.h, stream)

    def set_path(self, path):
        if isinstance(path, str):
            path = {"plain": PLAIN, "restructured": RESTRUCTURED}[path]
        sap_set_path(self.h, path)

    def set_update_mode(self, mode):
        if isinstance(mode, str):
            mode = {"literal": UPDATE_LITERAL, "angle": UPDATE_ANGLE}[mode]
        sap_set_update_mode(self.h, mode)

    def set_split(self, split):
        if isinstance(split, str):
            split = {"fp16": SPLIT_FP16, "bf16": SPLIT_BF16}[split]
        sap_set_split(self.h, split)

    def set_min_secant_length(self, eps):
        sap_set_min_secant_length(self.h, eps)

    def set_pass_bound(self, b_cap):
        sap_set_pass_bound(self.h, b_cap)

    def secant_pca(self, k):
        U, sv = sap_secant_pca(self.h, k, self.n)
        self.k = int(k)
        return U, sv

    def autotune(self, alpha, iters=16):
        return sap_autotune(self.h, alpha, iters)

    def tuning(self):
        return sap_get_tuning(self.h)

    def set_tuning(self, **params):
        sap_set_tuning(self.h, **params)

    def set_basis(self, U):
        sap_set_basis(self.h, U)
        self.k = int(U.shape[0])

    def get_basis(self, out=None):
        return sap_get_basis(self.h, self.k, self.n, out)

    def min_secant(self):
        return sap_min_secant(self.h)

    def step(self, alpha, sync=True):
        return sap_step(self.h, alpha, sync)

    def run(self, alpha, iters, history=True):
        return sap_run(self.h, alpha, iters, history)

    def get_history(self, count):
        return sap_get_history(self.h, count)

    def estimate_dim(self, U0, iters, alpha, threshold):
        return sap_estimate_dim(self.h, U0, iters, alpha, threshold)

    def sweep_history(self, k, count):
        return sap_get_sweep_history(self.h, k, count)

    def sweep_basis(self, k):
        return sap_get_sweep_basis(self.h, k, self.n)

    def project_df(self):
        hi = np.empty((self.N, self.k), dtype=np.float32)
        lo = np.empty((self.N, self.k), dtype=np.float32)
        return sap_project_df(self.h, hi, lo)

    def project(self, out=None):
        if out is None:
            out = np.empty((self.N, self.k), dtype=np.float32)
        return sap_project(self.h, out)

    def stats(self):
        return sap_get_stats(self.h)

    def set_profiling(self, enable):
        sap_set_profiling(self.h, enable)

    def kernel_time(self, kernel_class):
        return sap_get_kernel_time(self.h, kernel_class)

    def softmin_forward(self, tau):
        return sap_softmin_forward(self.h, tau)

    def softmin_backward(self, tau, L, out=None):
        return sap_softmin_backward(self.h, tau, L, self.k, self.n, out)

    def softmin_ascent(self, tau, eta, steps):
        return sap_softmin_ascent(self.h, tau, eta, steps)


class SapBatch:
    """Several datasets of one dimension run together (uneven sizes)."""

    def __init__(self, Xs, dtype=None, _handle=None):
        self.Ns = [int(X.shape[0]) for X in Xs]
        self.n = int(Xs[0].shape[1])
        self.B = len(Xs)
        self.h = _handle if _handle is not None else sap_create_batch(Xs, dtype)
        self.ks = [0] * self.B

    @classmethod
    def from_subsamples(cls, X, idx, dtype=None):
        """R subsets of the rows of X (idx: (R, m) indices), Sec. VI-C."""
        h = sap_create_subsamples(X, idx, dtype)
        idx = np.asarray(idx)
        return cls([np.empty((idx.shape[1], X.shape[1]))] * idx.shape[0], dtype, _handle=h)

    def estimate_dim(self, b, U0, iters, alpha, threshold):
        return sap_estimate_dim_b(self.h, b, U0, iters, alpha, threshold)

    def close(self):
        if self.h is not None:
            sap_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        sap_set_stream(self.h, stream)

    def set_min_secant_length(self, eps):
        sap_set_min_secant_length(self.h, eps)

    def autotune(self, alpha, iters=4):
        """One launch-parameter set for all datasets, timed on whole batch
        iterations; returns it."""
        return sap_autotune(self.h, alpha, iters)

    def tuning(self):
        """The first dataset's launch parameters (sap_get_tuning)."""
        return sap_get_tuning(self.h)

    def set_tuning(self, **params):
        """Launch parameters of every dataset (sap_set_tuning); unnamed
        parameters keep the first dataset's values."""
        sap_set_tuning(self.h, **params)

    def set_pass_bound(self, b_cap):
        sap_set_pass_bound(self.h, b_cap)

    def set_split(self, split):
        sap_set_split(self.h, {"fp16": SPLIT_FP16, "bf16": SPLIT_BF16}.get(split, split))

    def set_basis(self, b, U):
        sap_set_basis_b(self.h, b, U)
        self.ks[b] = int(U.shape[0])

    def get_basis(self, b):
        return sap_get_basis_b(self.h, b, self.ks[b], self.n)

    def min_secant(self, b):
        return sap_min_secant_b(self.h, b)

    def run(self, alpha, iters, history=True):
        return sap_run_batch(self.h, alpha, iters, self.B, history)

    def stats(self):
        return sap_get_stats(self.h)


class ShardSap:
    """One rank's share of the all-pairs step in the multi-GPU split (one
    process per GPU; see sap_create_shard).  `step` runs one SAP iteration:
    the rank's exact minimum as a 16-byte record, an all-gather of the
    records over `group` (torch.distributed: NCCL between GPUs), and the same
    FP64 update on every rank.  The library runs on torch's current stream,
    so the collective is ordered between the two calls."""

    def __init__(self, X, world, rank, dtype=None):
        import torch
        self.world, self.rank = int(world), int(rank)
        self.N, self.n = int(X.shape[0]), int(X.shape[1])
        self.h = sap_create_shard(X, self.world, self.rank, dtype)
        self.k = 0
        self._rec = torch.empty(16, dtype=torch.uint8, device="cuda")
        self._all = torch.empty(16 * self.world, dtype=torch.uint8, device="cuda")

    def close(self):
        if self.h:
            sap_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        sap_set_stream(self.h, stream)

    def set_basis(self, U):
        sap_set_basis(self.h, U)
        self.k = int(U.shape[0])

    def get_basis(self, out=None):
        return sap_get_basis(self.h, self.k, self.n, out)

    def set_tuning(self, **params):
        sap_set_tuning(self.h, **params)

    def get_history(self, count):
        return sap_get_history(self.h, count)

    def stats(self):
        return sap_get_stats(self.h)

    def min_record(self, out=None):
        return sap_shard_min(self.h, out)

    def step_records(self, alpha, recs):
        sap_shard_step(self.h, alpha, recs)

    def step(self, alpha, group=None):
        import torch.distributed as dist
        sap_shard_min(self.h, self._rec)
        dist.all_gather_into_tensor(self._all, self._rec, group=group)
        sap_shard_step(self.h, alpha, self._all)
