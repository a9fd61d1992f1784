"""GPU parity of the plain form (secants formed on the fly, Sec. IV) through
the C ABI, against the FP64 oracle, in lock-step and free-running."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import check_pair, lockstep, rel_gap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1807_03425_gb300 as P
    from paper_1807_03425_gb300 import build
    build.build()
    return P


def test_c1_fp64_lockstep(P):
    """Moment curve in R^10, N = 200, k = 3, alpha = 0.01, FP64 data."""
    cfg = W.CONFIGS["c1"]
    X = W.moment_curve(cfg["N"], cfg["m"], cfg["data_seed"], np.float64)
    U = W.random_basis(10, cfg["k"], cfg["basis_seed"])
    with P.Sap(X) as s:
        s.set_path("plain")
        for _ in range(25):
            U, _ = lockstep(s, X, U, cfg["alpha"])


@pytest.mark.parametrize("k", [1, 6, 11])
def test_fp64_plain_lockstep_widths(P, k):
    """FP64 data at other basis widths: the pass is compiled per width for
    k <= 8 and generic above (k = 11); N = 150 (ragged 16 x 16 blocks) in
    R^24, lock-step with the oracle."""
    X = W.moment_curve(150, 12, 21 + k, np.float64)
    U = W.random_basis(24, k, 40 + k)
    with P.Sap(X) as s:
        s.set_path("plain")
        for _ in range(6):
            U, _ = lockstep(s, X, U, 0.01)


def test_c1_fp64_free_run_history(P):
    """1000 iterations in captured graphs; the history must follow the
    oracle's exactly up to the first near-tie of the argmin."""
    cfg = W.CONFIGS["c1"]
    X = W.moment_curve(cfg["N"], cfg["m"], cfg["data_seed"], np.float64)
    U0 = W.random_basis(10, cfg["k"], cfg["basis_seed"])
    T = cfg["T"]
    Uo, ho, amo = O.run(X, U0, cfg["alpha"], T)
    with P.Sap(X) as s:
        s.set_path("plain")
        s.set_basis(U0)
        hg, amg = s.run(cfg["alpha"], T)
        Ug = s.get_basis()
    assert hg.shape == (T + 1,) and np.all(np.isfinite(hg))
    # The literal update amplifies rounding differences between the two FP64
    # implementations, so the free-running trajectories agree only until the
    # drift reaches the tolerance or the argmin is nearly tied.
    U = U0
    agree = 0
    for it in range(60):
        m = O.min_secant(X, U)
        if rel_gap(m) <= 1e-6 or abs(hg[it] - ho[it]) > 1e-5 * ho[it]:
            break
        assert tuple(amg[it]) == (m["i"], m["j"]), it
        U, _ = O.update(X, U, m["i"], m["j"], cfg["alpha"])
        agree += 1
    assert agree >= 10
    # the last evaluation is the oracle's minimum of the GPU's final basis
    m = O.min_secant(X, Ug)
    assert abs(hg[-1] - m["r"]) <= 1e-5 * m["r"]
    # graph replays run the same kernels as eager steps: bitwise equal
    with P.Sap(X) as s:
        s.set_path("plain")
        s.set_basis(U0)
        for it in range(40):
            i, j, r = s.step(cfg["alpha"])
            assert (i, j) == tuple(amg[it]) and r == hg[it], it


@pytest.mark.parametrize("N,m,k,seed", [(700, 10, 4, 3), (129, 4, 2, 5), (64, 3, 3, 7)])
def test_fp32_plain_lockstep_ragged(P, N, m, k, seed):
    """FP32 data; N not a multiple of the 64-point block (ragged tail)."""
    X = W.moment_curve(N, m, seed, np.float32)
    X64 = X.astype(np.float64)
    U = W.random_basis(2 * m, k, seed + 1)
    with P.Sap(X) as s:
        s.set_path("plain")
        for _ in range(6):
            U, _ = lockstep(s, X64, U, 0.005)


def test_fp32_plain_angle_mode(P):
    X = W.moment_curve(300, 6, 11, np.float32)
    X64 = X.astype(np.float64)
    U = W.random_basis(12, 3, 12)
    with P.Sap(X) as s:
        s.set_path("plain")
        s.set_update_mode("angle")
        for _ in range(5):
            U, _ = lockstep(s, X64, U, 0.05, mode=O.MODE_ANGLE)


def test_fp32_plain_eps_threshold(P):
    """Sec. VII: noisy moment curve, secants shorter than eps discarded."""
    X = W.moment_curve(400, 5, 21, np.float32, noise=0.1, noise_seed=22)
    X64 = X.astype(np.float64)
    U = W.random_basis(10, 4, 23)
    eps = 2.0
    with P.Sap(X) as s:
        s.set_path("plain")
        s.set_min_secant_length(eps)
        for _ in range(4):
            U, _ = lockstep(s, X64, U, 0.01, eps=eps)
        s.set_min_secant_length(1e9)
        s.set_basis(U)
        with pytest.raises(P.SapError) as e:
            s.min_secant()
        assert e.value.name == "SAP_E_NO_SECANT"


def test_duplicates_and_full_dimension(P):
    X = np.array([[0, 0, 0], [0, 0, 0], [1, 2, 2], [1, 2, 2], [3, 0, 4]], dtype=np.float32)
    with P.Sap(X) as s:
        s.set_path("plain")
        s.set_basis(np.eye(3))
        i, j, r = s.min_secant()
        assert abs(r - 1.0) <= 1e-12           # k = n: every ratio is 1
        assert (i, j) == (0, 2)                 # duplicates (0,1), (2,3) excluded
        s.set_basis(np.eye(3)[:1])
        i, j, r = s.min_secant()
        m = O.min_secant(X.astype(np.float64), np.eye(3)[:1])
        check_pair(X.astype(np.float64), np.eye(3)[:1], m, i, j, r)
    with P.Sap(np.zeros((6, 2), dtype=np.float32)) as s:
        s.set_path("plain")
        s.set_basis(np.eye(2)[:1])
        with pytest.raises(P.SapError) as e:
            s.min_secant()
        assert e.value.name == "SAP_E_NO_SECANT"


def test_rejects_bad_basis(P):
    X = W.moment_curve(50, 3, 1, np.float32)
    with P.Sap(X) as s:
        with pytest.raises(P.SapError) as e:
            s.set_basis(np.ones((2, 6)))
        assert e.value.name == "SAP_E_NOT_ORTHONORMAL"
        with pytest.raises(P.SapError) as e:
            s.step(0.1)
        assert e.value.name == "SAP_E_STATE"


def test_c2_plain_full_size_lockstep(P):
    """Full configuration size (N = 8192, n = 100, k = 5): one lock-step
    evaluation + update of the plain FP32 form against the oracle."""
    cfg = W.CONFIGS["c2"]
    X = W.moment_curve(cfg["N"], cfg["m"], cfg["data_seed"], np.float32)
    U = W.random_basis(100, cfg["k"], cfg["basis_seed"])
    with P.Sap(X) as s:
        s.set_path("plain")
        lockstep(s, X.astype(np.float64), U, cfg["alpha"])


def test_torch_device_buffers_and_stream(P):
    torch = pytest.importorskip("torch")
    X = W.moment_curve(300, 4, 31, np.float32)
    U = W.random_basis(8, 3, 32)
    Xt = torch.from_numpy(X).cuda()
    Ut = torch.from_numpy(U).cuda()
    m = O.min_secant(X.astype(np.float64), U)
    with P.Sap(Xt) as s:
        st = torch.cuda.Stream()
        s.set_stream(st)
        s.set_path("plain")
        s.set_basis(Ut)
        i, j, r = s.min_secant()
        check_pair(X.astype(np.float64), U, m, i, j, r)
        out = torch.empty_like(Ut)
        s.get_basis(out)
        assert torch.equal(out.cpu(), Ut.cpu())
