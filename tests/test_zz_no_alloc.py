"""The allocation-free argmin entry point (sap_min_secant_noalloc) against the
handle-based one (sap_min_secant, plain form), through the C ABI.

It exists for callers that must not allocate device memory (for instance
when a framework owns the device memory pool, or in a loop that cannot
afford an allocation's synchronisation); its scratch is a fixed file-scope
device array shared by all calls, so the tests call it several times in a
row with different inputs and expect each call to start from a clean state.
Kept in its own file, collected last."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


def _noalloc(lib, Xd, Ud, N, n, k, eps, stream=None):
    i, j, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    code = lib.sap_min_secant_noalloc(ctypes.c_void_p(Xd.data_ptr()), N, n,
                                      ctypes.c_void_p(Ud.data_ptr()), k, eps,
                                      ctypes.c_void_p(stream) if stream else None,
                                      ctypes.byref(i), ctypes.byref(j), ctypes.byref(r))
    return code, i.value, j.value, r.value


def _handle_min(P, X, U, eps):
    with P.Sap(X) as s:
        s.set_path("plain")
        if eps > 0:
            s.set_min_secant_length(eps)
        s.set_basis(U)
        return s.min_secant()


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


def test_noalloc_side_stream_smallest_size_and_all_excluded():
    """A call on a torch side stream; the smallest problem (N = 2); and a
    threshold above every pair length, which must return SAP_E_NO_SECANT and
    leave the shared scratch fit for the valid call right after it."""
    torch = pytest.importorskip("torch")
    import paper_1807_03425_gb300 as P
    lib = P.load_library()
    X = W.moment_curve(300, 5, 81, np.float32)
    U = W.random_basis(10, 3, 82)
    Xd = torch.from_numpy(X).cuda()
    Ud = torch.from_numpy(U).cuda()
    torch.cuda.synchronize()
    want = _handle_min(P, X, U, 0.0)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        code, i, j, r = _noalloc(lib, Xd, Ud, 300, 10, 3, 0.0, side.cuda_stream)
    assert code == 0, P.capi.sap_status_str(code)
    assert (i, j) == want[:2] and abs(r - want[2]) <= REL_TOL * want[2]

    # N = 2: one pair, ratio |U^T s| of its unit secant
    X2 = np.array([[1.0, 2.0, 3.0, 0.5], [0.0, -1.0, 2.0, 1.5]], dtype=np.float32)
    U2 = W.random_basis(4, 2, 83)
    code, i, j, r = _noalloc(lib, torch.from_numpy(X2).cuda(), torch.from_numpy(U2).cuda(),
                             2, 4, 2, 0.0)
    assert code == 0, P.capi.sap_status_str(code)
    s = (X2[0].astype(np.float64) - X2[1]) / np.linalg.norm(X2[0].astype(np.float64) - X2[1])
    assert (i, j) == (0, 1) and abs(r - np.linalg.norm(U2 @ s)) <= REL_TOL * r

    # every pair shorter than eps: no secant left
    dmax = max(np.linalg.norm(X[a].astype(np.float64) - X[b]) for a in range(0, 300, 7) for b in range(300))
    code, _, _, _ = _noalloc(lib, Xd, Ud, 300, 10, 3, 10.0 * dmax)
    assert P.capi.sap_status_str(code) == "SAP_E_NO_SECANT"
    code, i, j, r = _noalloc(lib, Xd, Ud, 300, 10, 3, 0.0)
    assert code == 0, P.capi.sap_status_str(code)
    assert (i, j) == want[:2] and abs(r - want[2]) <= REL_TOL * want[2]
