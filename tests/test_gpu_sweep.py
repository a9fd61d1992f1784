"""GPU parity of the dimension-estimation sweep (Sec. VI-A): every k = 1..k_max
advances together (one tensor-core product for all bases, concurrent
per-basis chains), through the C ABI.

Each basis's trajectory must equal, bit for bit, the single-basis SAP run
from the same start: the FP64 tier decides every argmin exactly and the
update is deterministic, so sharing the product, the stored lengths and the
(k_max) near list may change the candidate lists but not the result.  The
single-basis path itself is pinned to the oracle elsewhere; here the sweep
is also compared with the oracle: the first evaluation (same basis on both
sides), the trajectory walked with the oracle while the two stay within
1e-5, and the last evaluation, which must be the oracle's minimum for the
GPU's own final basis (the update runs in FP32, so free-running
trajectories drift apart; the smallest ratios here are ~1e-9).
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


def images(N, side, seed):
    """Blob images (the sweep's workload) at a reduced side length."""
    s = side / 64.0
    return W.blob_images(N, seed, side=side, sigma=4.0 * s, lo=16.0 * s, hi=48.0 * s)


def follow_oracle(X64, U, hist, argmins, alpha):
    """Walk a GPU trajectory with the oracle: at each iteration the GPU's pair
    must be the oracle's argmin (or, when the oracle's runner-up is within
    1e-6 relative, a pair within 1e-6 of the minimum) and its ratio within
    1e-5; the oracle then updates with the GPU's pair.  Stops when the two
    trajectories' rounding drift exceeds 1e-5.  Returns the iterations
    checked."""
    for it in range(len(hist)):
        m = O.min_secant(X64, U)
        i, j = (int(v) for v in argmins[it])
        if it > 0 and abs(hist[it] - m["r"]) > 1e-5 * m["r"]:
            return it
        if rel_gap(m) > 1e-6:
            assert (i, j) == (m["i"], m["j"]), it
        else:
            assert O.ratio(X64, U, i, j) <= m["r"] * (1 + 1e-6), it
        assert abs(hist[it] - m["r"]) <= 1e-5 * m["r"], it
        if it + 1 < len(hist):
            U, _ = O.update(X64, U, i, j, alpha)
    return len(hist)


def check_final(X64, Ug, hist, argmins):
    """The last evaluation is the oracle's minimum of the GPU's final basis."""
    m = O.min_secant(X64, Ug)
    i, j = (int(v) for v in argmins[-1])
    if rel_gap(m) > 1e-6:
        assert (i, j) == (m["i"], m["j"])
    else:
        assert O.ratio(X64, Ug, i, j) <= m["r"] * (1 + 1e-6)
    assert abs(hist[-1] - m["r"]) <= 1e-5 * m["r"]


def single_runs(P, X, U0, ks, alpha, T):
    out = {}
    with P.Sap(X) as s:
        for k in ks:
            s.set_basis(U0[:k])
            out[k] = s.run(alpha, T)
    return out


@pytest.mark.parametrize("N,side,kmax,T", [(300, 16, 8, 20), (140, 12, 5, 30)])
def test_sweep_equals_single_basis_runs_and_oracle(P, N, side, kmax, T):
    alpha, thr = 0.01, 0.1
    X = images(N, side, 3)
    n = X.shape[1]
    U0 = W.random_basis(n, kmax, 4)
    with P.Sap(X) as s:
        kout, ratios = s.estimate_dim(U0, T, alpha, thr)
        hist = {k: s.sweep_history(k, T + 1) for k in range(1, kmax + 1)}
        Uf = {k: s.sweep_basis(k) for k in (1, 2, kmax)}
    ref = single_runs(P, X, U0, range(1, kmax + 1), alpha, T)
    for k in range(1, kmax + 1):
        hg, amg = hist[k]
        hs, ams = ref[k]
        assert np.array_equal(hg, hs), k
        assert np.array_equal(amg, ams), k
        assert ratios[k - 1] == hg[T]
    assert kout == next((k for k in range(1, kmax + 1) if ratios[k - 1] > thr), -1)
    # against the oracle, following the GPU's pairs (tie-aware lock-step)
    X64 = X.astype(np.float64)
    for k in (1, 2, kmax):
        hg, amg = hist[k]
        assert follow_oracle(X64, U0[:k], hg, amg, alpha) >= 1, k
        check_final(X64, Uf[k], hg, amg)


@pytest.mark.parametrize("tier", [3, 5])
def test_sweep_fused_tiers_equal_single_runs(P, tier):
    """The dimension sweep with the second tier fused into another kernel
    (3: extended precision inside the FP64 recheck, k <= 8; 5: explicit
    FP32 differences inside the all-pairs pass), every basis on its own
    stream, gives the same trajectories, bit for bit, as single-basis runs
    with the default tiers: the tiers only select candidates, the FP64 tier
    decides."""
    alpha, T, kmax = 0.01, 20, 6
    X = images(200, 10, 5)
    n = X.shape[1]
    U0 = W.random_basis(n, kmax, 6)
    with P.Sap(X) as s:
        s.set_tuning(pass_bound=2e-3, pass_stages=0, explicit_blocks_per_sm=1, update_blocks=0,
                     plain_blocks_per_sm=2, programmatic_launch=1, refine_tier=tier)
        s.estimate_dim(U0, T, alpha, 0.1)
        hist = {k: s.sweep_history(k, T + 1) for k in range(1, kmax + 1)}
    ref = single_runs(P, X, U0, range(1, kmax + 1), alpha, T)
    for k in range(1, kmax + 1):
        assert np.array_equal(hist[k][0], ref[k][0]), k
        assert np.array_equal(hist[k][1], ref[k][1]), k


def test_sweep_large_n_split_product(P):
    """64 x 64 images (n = 4096) and k_max = 20: the 256-wide product in K
    slices, the extended-precision explicit tier and n-length updates."""
    alpha, T, kmax = 0.01, 3, 20
    X = images(260, 64, 5)
    U0 = W.random_basis(4096, kmax, 6)
    with P.Sap(X) as s:
        kout, ratios = s.estimate_dim(U0, T, alpha, 0.1)
        hist = {k: s.sweep_history(k, T + 1) for k in (1, 7, 20)}
        Uf = {k: s.sweep_basis(k) for k in (1, 20)}
        st = s.stats()
    assert st["y_error_unit"] < 2e-5  # K slices keep the product's bound small
    ref = single_runs(P, X, U0, (1, 7, 20), alpha, T)
    for k in (1, 7, 20):
        assert np.array_equal(hist[k][0], ref[k][0]), k
        assert np.array_equal(hist[k][1], ref[k][1]), k
    X64 = X.astype(np.float64)
    for k in (1, 20):
        assert follow_oracle(X64, U0[:k], hist[k][0], hist[k][1], alpha) >= 1, k
        check_final(X64, Uf[k], hist[k][0], hist[k][1])


def test_full_size_zero_iterations(P):
    """The full sweep workload (N = 4096 images of 64 x 64, k = 1..20) with no
    iterations: nested initial bases make the min ratios non-decreasing in
    k, each equals the single-basis certified minimum, and each is the
    oracle's ratio of the reported pair."""
    X = W.blob_images(4096, 1)
    U0 = W.random_basis(4096, 20, 2)
    with P.Sap(X) as s:
        kout, ratios = s.estimate_dim(U0, 0, 0.01, 0.1)
        pairs = {k: s.sweep_history(k, 1)[1][0] for k in (1, 10, 20)}
        assert np.all(np.diff(ratios) >= 0)
        for k in (1, 10, 20):
            s.set_basis(U0[:k])
            i, j, r = s.min_secant()
            assert r == ratios[k - 1] and (i, j) == tuple(pairs[k]), k
    X64 = X.astype(np.float64)
    for k in (1, 20):
        i, j = pairs[k]
        assert abs(O.ratio(X64, U0[:k], int(i), int(j)) - ratios[k - 1]) <= 1e-12


def test_sweep_leaves_handle_basis(P):
    X = images(200, 12, 9)
    U = W.random_basis(144, 3, 10)
    U0 = W.random_basis(144, 6, 11)
    with P.Sap(X) as s:
        s.set_basis(U)
        before = s.min_secant()
        s.estimate_dim(U0, 4, 0.01, 0.1)
        assert np.array_equal(s.get_basis(), U)
        assert s.min_secant() == before


def test_sweep_argument_errors(P):
    X = images(100, 12, 1)
    with P.Sap(X) as s:
        with pytest.raises(P.SapError) as e:
            s.estimate_dim(W.random_basis(144, 21, 2), 2, 0.01, 0.1)
        assert e.value.code == 9
        bad = W.random_basis(144, 4, 2)
        bad[1] *= 1.001
        with pytest.raises(P.SapError) as e:
            s.estimate_dim(bad, 2, 0.01, 0.1)
        assert e.value.code == 3
        with pytest.raises(P.SapError) as e:
            s.estimate_dim(W.random_basis(144, 4, 2), 2, 1.5, 0.1)
        assert e.value.code == 1
    with P.Sap(X.astype(np.float64)) as s:
        with pytest.raises(P.SapError) as e:
            s.estimate_dim(W.random_basis(144, 4, 2), 2, 0.01, 0.1)
        assert e.value.code == 9
