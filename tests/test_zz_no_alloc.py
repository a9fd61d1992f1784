"""The allocation-free argmin entry point (sap_min_secant_noalloc) against the
handle-based one (sap_min_secant, plain form), through the C ABI.

It exists for callers that must not allocate device memory (for instance
while a stream is being captured, or when a framework owns the device memory
pool); its scratch is a fixed file-scope device array shared by all calls,
so the test calls it twice in a row with different inputs and expects each
call to start from a clean state.  Kept in its own file, collected last."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


def _noalloc(lib, Xd, Ud, N, n, k, eps):
    i, j, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    code = lib.sap_min_secant_noalloc(ctypes.c_void_p(Xd.data_ptr()), N, n,
                                      ctypes.c_void_p(Ud.data_ptr()), k, eps, None,
                                      ctypes.byref(i), ctypes.byref(j), ctypes.byref(r))
    return code, i.value, j.value, r.value


def test_noalloc_matches_handle_entry_point():
    torch = pytest.importorskip("torch")
    import paper_1807_03425_gb300 as P
    from paper_1807_03425_gb300 import build
    build.build()
    lib = P.load_library()
    cases = [
        (W.moment_curve(700, 10, 71, np.float32), W.random_basis(20, 4, 72), 0.0),
        (W.moment_curve(1024, 6, 73, np.float32, noise=0.05, noise_seed=74),
         W.random_basis(12, 5, 75), 0.3),
    ]
    for X, U, eps in cases:  # two calls in a row on the shared scratch
        N, n = X.shape
        k = U.shape[0]
        Xd = torch.from_numpy(X).cuda()
        Ud = torch.from_numpy(U).cuda()
        torch.cuda.synchronize()
        code, i, j, r = _noalloc(lib, Xd, Ud, N, n, k, eps)
        assert code == 0, P.capi.sap_status_str(code)
        with P.Sap(X) as s:
            s.set_path("plain")
            if eps > 0:
                s.set_min_secant_length(eps)
            s.set_basis(U)
            i2, j2, r2 = s.min_secant()
        assert (i, j) == (i2, j2)
        assert abs(r - r2) <= REL_TOL * r2


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    import paper_1807_03425_gb300 as P
    lib = P.load_library()
    X = torch.zeros((1025, 4), dtype=torch.float32, device="cuda")
    U = torch.eye(4, dtype=torch.float64, device="cuda")[:2].contiguous()
    code, _, _, _ = _noalloc(lib, X, U, 1025, 4, 2, 0.0)
    assert P.capi.sap_status_str(code) == "SAP_E_ARG"
    code, _, _, _ = _noalloc(lib, X[:10], U, 10, 4, 9, 0.0)
    assert P.capi.sap_status_str(code) == "SAP_E_ARG"
