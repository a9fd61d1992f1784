"""GPU parity of the uneven multi-dataset batch (the noisy-data setting of
Sec. VII on many hyperspectral scenes of different sizes), through the C ABI.

Every dataset of a batch runs its own chain inside one captured graph, so its
trajectory must equal, bit for bit, the same dataset run alone; each dataset
is also checked against the oracle at its first evaluation and at its last
(the oracle's minimum for the GPU's own final basis).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import rel_gap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1807_03425_gb300 as P
    from paper_1807_03425_gb300 import build
    build.build()
    return P


def check_eval(X64, U, i, j, r, eps):
    m = O.min_secant(X64, U, eps)
    if rel_gap(m) > 1e-6:
        assert (i, j) == (m["i"], m["j"])
    else:
        assert O.ratio(X64, U, i, j, eps) <= m["r"] * (1 + 1e-6)
    assert abs(r - m["r"]) <= 1e-5 * m["r"]


def test_uneven_batch_equals_single_runs_and_oracle(P):
    alpha, T, k, eps = 0.01, 12, 4, 0.3
    Xs, Ns = W.hyperspectral_batch(5, 21, n_min=120, n_max=700, n_bands=48)
    Us = [W.random_basis(48, k, 30 + b) for b in range(5)]
    bits = [W.bf16_bits(X) for X in Xs]
    with P.SapBatch(bits, dtype=P.BF16) as sb:
        sb.set_min_secant_length(eps)
        for b in range(5):
            sb.set_basis(b, Us[b])
        hist, am = sb.run(alpha, T)
        Uf = [sb.get_basis(b) for b in range(5)]
        st = sb.stats()
    assert st["n_points"] == sum(Ns) and st["n_excluded"] > 0
    for b in range(5):
        with P.Sap(bits[b], dtype=P.BF16) as s:
            s.set_min_secant_length(eps)
            s.set_basis(Us[b])
            h1, a1 = s.run(alpha, T)
            U1 = s.get_basis()
        assert np.array_equal(hist[b], h1), b
        assert np.array_equal(am[b], a1), b
        assert np.array_equal(Uf[b], U1), b
        X64 = Xs[b].astype(np.float64)
        check_eval(X64, Us[b], int(am[b, 0, 0]), int(am[b, 0, 1]), hist[b, 0], eps)
        check_eval(X64, Uf[b], int(am[b, T, 0]), int(am[b, T, 1]), hist[b, T], eps)


def test_full_size_uneven_batch(P):
    """The full batch workload: 32 hyperspectral scenes, N log-uniform in
    [500, 20000], n = 224 bands, k = 10, eps = 0.05, BF16 data; a few
    iterations.  Each dataset's last evaluation equals the certified minimum
    of its final basis computed alone, and one small dataset is checked
    against the oracle."""
    cfg = W.CONFIGS["c4"]
    Xs, Ns = W.hyperspectral_batch(cfg["B"], cfg["data_seed"])
    Us = [W.random_basis(224, cfg["k"], cfg["basis_seed"] + b) for b in range(cfg["B"])]
    T = 3
    with P.SapBatch([W.bf16_bits(X) for X in Xs], dtype=P.BF16) as sb:
        sb.set_min_secant_length(cfg["eps"])
        for b in range(cfg["B"]):
            sb.set_basis(b, Us[b])
        hist, am = sb.run(cfg["alpha"], T)
        assert np.all(np.isfinite(hist)) and np.all(hist > 0)
        small = int(np.argmin(Ns))
        for b in (small, int(np.argmax(Ns))):
            Ub = sb.get_basis(b)
            with P.Sap(W.bf16_bits(Xs[b]), dtype=P.BF16) as s:
                s.set_min_secant_length(cfg["eps"])
                s.set_basis(Ub)
                i, j, r = s.min_secant()
            assert (i, j) == tuple(am[b, T]) and r == hist[b, T], b
        Us_small = sb.get_basis(small)
    X64 = Xs[small].astype(np.float64)
    check_eval(X64, Us_small, int(am[small, T, 0]), int(am[small, T, 1]), hist[small, T], cfg["eps"])


def test_batch_tuning_applies_to_every_dataset(P):
    """set_tuning on a batch handle reaches every dataset; the second tier in
    its own kernel and inside the pass give the same trajectories, bit for
    bit, for three scenes of different sizes (k = 10: the width-10 pass)."""
    Xs, _ = W.hyperspectral_batch(3, 11, n_min=300, n_max=1500)
    Us = [W.random_basis(224, 10, 40 + b) for b in range(3)]
    runs = []
    for tier in (0, 5):
        with P.SapBatch([W.bf16_bits(X) for X in Xs], dtype=P.BF16) as sb:
            sb.set_min_secant_length(0.05)
            sb.set_tuning(refine_tier=tier, pass_bound=4e-3)
            assert sb.tuning()["refine_tier"] == tier and sb.tuning()["pass_bound"] == 4e-3
            for b in range(3):
                sb.set_basis(b, Us[b])
            runs.append(sb.run(0.01, 6))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


def test_batch_argument_errors(P):
    Xs, _ = W.hyperspectral_batch(2, 3, n_min=50, n_max=80, n_bands=16)
    with P.SapBatch(Xs) as sb:
        with pytest.raises(P.SapError) as e:
            sb.run(0.01, 2)
        assert e.value.code == 2  # no basis yet
        sb.set_basis(0, W.random_basis(16, 2, 1))
        with pytest.raises(P.SapError) as e:
            sb.set_basis(2, W.random_basis(16, 2, 1))
        assert e.value.code == 1
        with pytest.raises(P.SapError) as e:
            P.capi.sap_step(sb.h, 0.01)
        assert e.value.code == 2
        assert P.capi.sap_batch_count(sb.h) == 2
