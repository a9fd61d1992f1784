"""GPU parity of the restructured form: Y = X U on tensor cores (tcgen05,
split 16-bit operands), the all-pairs pass over stored inverse squared
lengths, the explicit-difference and FP64 rechecks; through the C ABI,
against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import check_pair, lockstep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1807_03425_gb300 as P
    from paper_1807_03425_gb300 import build
    build.build()
    return P


@pytest.mark.parametrize("split", ["fp16", "bf16"])
@pytest.mark.parametrize("N,n,k", [(700, 20, 4), (300, 100, 5), (130, 7, 1), (1000, 64, 12), (257, 40, 20)])
def test_projection_error_within_certified_bound(P, split, N, n, k):
    """The tensor-core product's rows differ from the exact projection by at
    most y_error_unit * ||x_i - mean||: checked on every pair difference
    (translation-free) of a seeded dataset.  Shapes span several 128-row
    tiles, ragged N, n not a multiple of 64, and k across MMA widths."""
    g = np.random.default_rng(N + n + k)
    X = (g.standard_normal((N, n)) + 3.0).astype(np.float32)
    U = W.random_basis(n, k, N)
    X64 = X.astype(np.float64)
    with P.Sap(X) as s:
        s.set_split(split)
        s.set_basis(U)
        Y = np.empty((N, k), dtype=np.float32)
        P.capi.sap_project(s.h, Y)
        st = s.stats()
    eps = st["y_error_unit"]
    assert 0 < eps < (2e-3 if split == "bf16" else 2e-5)
    c32 = X64.mean(axis=0).astype(np.float32).astype(np.float64)
    Yx = (X64 - c32) @ U.T                      # exact projection of the centred data
    nu = np.linalg.norm((X - c32.astype(np.float32)).astype(np.float64), axis=1)
    err = np.abs(Y.astype(np.float64) - Yx)
    assert np.all(err <= eps * nu[:, None] + 1e-30), (err / nu[:, None]).max()
    # the bound is not vacuous: the error is within 3 orders of it
    assert (err / nu[:, None]).max() > eps * 1e-4


@pytest.mark.parametrize("N,n,k", [(700, 20, 4), (300, 100, 5), (130, 7, 1), (257, 300, 12), (200, 1100, 20)])
def test_df_projection_within_certified_bound(P, N, n, k):
    """The double-float projection of the second tier (hi + lo FP32 pairs from
    error-free products of the exact points and the FP64 basis) is within
    ydf_error_unit * ||x_i|| of <x_i, u_c> for every entry: checked against
    an FP64 product on ragged row counts, n across the 256 boundary and
    beyond 1024, and k from 1 to 20."""
    g = np.random.default_rng(7 * N + n + k)
    X = (g.standard_normal((N, n)) + 3.0).astype(np.float32)
    U = W.random_basis(n, k, N + 1)
    with P.Sap(X) as s:
        s.set_basis(U)
        hi, lo = s.project_df()
        eps = s.stats()["ydf_error_unit"]
    assert 0 < eps < 2e-10
    X64 = X.astype(np.float64)
    exact = X64 @ U.T
    got = hi.astype(np.float64) + lo.astype(np.float64)
    xn = np.linalg.norm(X64, axis=1)
    err = np.abs(got - exact)
    assert np.all(err <= eps * xn[:, None]), (err / xn[:, None]).max() / eps
    # far more accurate than one FP32 number, and the comparison is not vacuous
    assert (err / xn[:, None]).max() < 1e-10
    assert np.abs(hi).max() > 0 and np.any(lo != 0)


@pytest.mark.parametrize("N,m,k,seed", [(700, 10, 4, 3), (300, 50, 5, 5), (129, 4, 2, 7), (520, 8, 1, 9)])
def test_restructured_lockstep(P, N, m, k, seed):
    X = W.moment_curve(N, m, seed, np.float32)
    X64 = X.astype(np.float64)
    U = W.random_basis(2 * m, k, seed + 1)
    with P.Sap(X) as s:
        s.set_path("restructured")
        for _ in range(6):
            U, _ = lockstep(s, X64, U, 0.005)
        st = s.stats()
    assert st["n_pairs"] == N * (N - 1) // 2


@pytest.mark.parametrize("k", [9, 13, 20, 27])
def test_restructured_wide_k(P, k):
    """k beyond 8 takes the 2- and 1-column variants of the pass."""
    X = W.moment_curve(400, 16, 41, np.float32)
    X64 = X.astype(np.float64)
    U = W.random_basis(32, k, 42)
    with P.Sap(X) as s:
        s.set_path("restructured")
        for _ in range(3):
            U, _ = lockstep(s, X64, U, 0.01)


def test_restructured_bf16_split_and_eps(P):
    X = W.moment_curve(600, 5, 51, np.float32, noise=0.1, noise_seed=52)
    X64 = X.astype(np.float64)
    U = W.random_basis(10, 4, 53)
    with P.Sap(X) as s:
        s.set_split("bf16")
        s.set_min_secant_length(2.0)
        for _ in range(4):
            U, _ = lockstep(s, X64, U, 0.01, eps=2.0)
        st = s.stats()
        m = O.min_secant(X64, U, 2.0)
        assert st["n_excluded"] == m["excluded"]


def test_restructured_equals_plain_trajectory(P):
    """Both forms hand the FP64 tier a candidate set that contains the FP64
    argmin, and share the update: their trajectories are bitwise equal."""
    X = W.moment_curve(1500, 20, 61, np.float32)
    U0 = W.random_basis(40, 5, 62)
    out = {}
    for path in ("plain", "restructured"):
        with P.Sap(X) as s:
            s.set_path(path)
            s.set_basis(U0)
            out[path] = s.run(0.005, 150) + (s.get_basis(),)
    hp, ap, Up = out["plain"]
    hr, ar, Ur = out["restructured"]
    np.testing.assert_array_equal(ap, ar)
    np.testing.assert_array_equal(hp, hr)
    np.testing.assert_array_equal(Up, Ur)


def test_c2_restructured_full_size(P):
    """Full configuration (N = 8192, n = 100, k = 5, alpha = 0.005): lock-step
    evaluations + updates against the oracle, then a 200-iteration graph run
    whose final evaluation is checked against the oracle's minimum of the
    final basis."""
    cfg = W.CONFIGS["c2"]
    X = W.moment_curve(cfg["N"], cfg["m"], cfg["data_seed"], np.float32)
    X64 = X.astype(np.float64)
    U = W.random_basis(100, cfg["k"], cfg["basis_seed"])
    with P.Sap(X) as s:
        s.set_path("restructured")
        for _ in range(2):
            U, _ = lockstep(s, X64, U, cfg["alpha"])
        s.set_basis(U)
        hist, am = s.run(cfg["alpha"], 200)
        Uf = s.get_basis()
        st = s.stats()
    assert np.abs(Uf @ Uf.T - np.eye(cfg["k"])).max() < 1e-12
    m = O.min_secant(X64, Uf)
    check_pair(X64, Uf, m, int(am[-1, 0]), int(am[-1, 1]), hist[-1])
    assert st["n_near"] > 0 and st["last_tier2"] >= 1


@pytest.mark.parametrize("tier", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("N,n,k", [(600, 300, 3), (450, 40, 1), (700, 100, 5), (800, 60, 12), (650, 48, 10)])
def test_second_tiers_lockstep(P, tier, N, n, k):
    """Every second tier (explicit differences, double-float refine,
    explicit differences fused into the FP64 recheck in FP32 or in extended
    precision, extended precision with a final filter, explicit differences
    inside the all-pairs pass) gives the oracle's argmin, ratio and update in
    lock-step, for n on both sides of the 256 switch (above it the FP32
    fused tiers fall back to the separate one), n = 100 (the one-warp update
    of n <= 128 with a ragged last row group), k = 1 (where ties in the
    ratio are dense) and k = 12 (the padded compute width)."""
    g = np.random.default_rng(N + n)
    t = g.random(N) * 2 * np.pi
    # a curve on a 2-torus linearly embedded in R^n (short secants abound)
    base = np.stack([np.cos(t), np.sin(t), np.cos(3 * t), np.sin(3 * t), np.cos(7 * t) * 0.5], axis=1)
    Q, _ = np.linalg.qr(g.standard_normal((n, 5)))
    X = (base @ Q.T + 0.5).astype(np.float32)
    X64 = X.astype(np.float64)
    U = W.random_basis(n, k, N + 3)
    with P.Sap(X) as s:
        s.set_path("restructured")
        s.set_tuning(pass_bound=2e-3, pass_stages=0, explicit_blocks_per_sm=2, update_blocks=0,
                     plain_blocks_per_sm=2, programmatic_launch=0, refine_tier=tier)
        for _ in range(5):
            U, _ = lockstep(s, X64, U, 0.01)


@pytest.mark.parametrize("k", [3, 9, 10, 12, 16])
def test_tier_forms_agree_bitwise(P, k):
    """The second tier in its own kernel (explicit FP32, double-float) and
    inside the pass (with the FP64 tier, a one-block update over the pass's
    results) select different candidates but take the same FP64 decisions:
    15 iterations give bitwise-identical histories, argmins and bases, for
    the exact and the padded compute widths of the pass (k = 9, 10 use the
    width-10 pass, k = 12 the width-12 one)."""
    X = W.moment_curve(1100, 16, 70 + k, np.float32)
    U0 = W.random_basis(32, k, 71 + k)
    runs = []
    for tier in (0, 1, 5):
        with P.Sap(X) as s:
            s.set_path("restructured")
            s.set_tuning(refine_tier=tier)
            s.set_basis(U0)
            hist, am = s.run(0.01, 15)
            runs.append((hist, am, s.get_basis()))
    for other in runs[1:]:
        for a, b in zip(runs[0], other):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("tier", [0, 5])
def test_bf16_data_tiers_lockstep(P, tier):
    """BF16 data (the hyperspectral workload's input type), n = 224, k = 10:
    the explicit tier in its own kernel and inside the pass (which reads the
    exact FP32 widening of the BF16 points) follow the oracle in lock-step
    on the BF16 values, with ε = 0.05 excluding short secants."""
    Xs, _ = W.hyperspectral_batch(1, 17, n_min=900, n_max=900)
    Xb = W.to_bf16_exact(Xs[0])
    X64 = Xb.astype(np.float64)
    U = W.random_basis(224, 10, 18)
    with P.Sap(W.bf16_bits(Xb), dtype=P.BF16) as s:
        s.set_path("restructured")
        s.set_min_secant_length(0.05)
        s.set_tuning(refine_tier=tier)
        for _ in range(3):
            U, _ = lockstep(s, X64, U, 0.01, eps=0.05)
