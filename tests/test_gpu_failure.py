"""Failure paths of the C ABI, made to happen without faulting the GPU:
an error injected on the host into the next CUDA call a handle checks
(an allocation failure: SAP_E_OOM, the handle stays usable; a CUDA error:
SAP_E_CUDA, sticky until sap_destroy), and a device-side bounded wait that
runs out (a kernel waiting on an mbarrier nothing arrives on, with the same
bounded wait the library's kernels use): SAP_E_TIMEOUT, after which the
context still works."""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1807_03425_gb300 as P
    from paper_1807_03425_gb300 import build
    build.build()
    return P


def status(P, code):
    return P.capi.sap_status_str(code)


def test_injected_allocation_failure_is_reported_and_not_sticky(P):
    X = W.moment_curve(400, 5, 61, np.float32)
    U3, U4 = W.random_basis(10, 3, 62), W.random_basis(10, 4, 63)
    lib = P.load_library()
    with P.Sap(X) as s:
        s.set_basis(U3)
        assert P.capi.sap_inject_fault(s.h, 1) == 0
        with pytest.raises(P.SapError) as e:
            s.set_basis(U4)            # the first checked CUDA call fails
        assert status(P, e.value.code) == "SAP_E_OOM"
        assert "out of memory" in lib.sap_last_error(s.h).decode()
        # not sticky: the handle works again
        s.set_basis(U4)
        i, j, r = s.min_secant()
        m = O.min_secant(X.astype(np.float64), U4)
        assert (i, j) == (m["i"], m["j"]) and abs(r - m["r"]) <= 1e-5 * m["r"]


def test_injected_cuda_error_is_sticky_until_destroy(P):
    X = W.moment_curve(400, 5, 64, np.float32)
    U = W.random_basis(10, 3, 65)
    lib = P.load_library()
    s = P.Sap(X)
    s.set_basis(U)
    assert P.capi.sap_inject_fault(s.h, 2) == 0
    with pytest.raises(P.SapError) as e:
        s.min_secant()
    assert status(P, e.value.code) == "SAP_E_CUDA"
    # every later call but destroy reports the sticky error
    for call in (lambda: s.min_secant(), lambda: s.set_basis(U), lambda: s.step(0.01), lambda: s.run(0.01, 4)):
        with pytest.raises(P.SapError) as e:
            call()
        assert status(P, e.value.code) == "SAP_E_CUDA"
    assert "sticky" in lib.sap_last_error(s.h).decode()
    assert lib.sap_destroy(s.h) == 0
    s.h = None


def test_device_wait_runs_out_and_context_stays_usable(P):
    torch = pytest.importorskip("torch")
    # ~1 ms of SM clocks: the wait gives up and reports it
    assert status(P, P.capi.sap_selftest_wait(2_000_000)) == "SAP_E_TIMEOUT"
    side = torch.cuda.Stream()
    assert status(P, P.capi.sap_selftest_wait(2_000_000, side.cuda_stream)) == "SAP_E_TIMEOUT"
    # the context is intact: a full SAP step still matches the oracle
    X = W.moment_curve(500, 5, 66, np.float32)
    U = W.random_basis(10, 3, 67)
    with P.Sap(X) as s:
        s.set_basis(U)
        i, j, r = s.step(0.01)
    m = O.min_secant(X.astype(np.float64), U)
    assert (i, j) == (m["i"], m["j"]) and abs(r - m["r"]) <= 1e-5 * m["r"]
    x = torch.arange(10, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == 45.0
