"""GPU parity of the soft-min objective, its hand-written backward and the
Riemannian ascent (torch.autograd.Function on top), against the FP64 oracle.

Tolerances are derived from the arithmetic of the kernels, per pair, from
the oracle's own values (ratio r, length d, point norms), so a dropped term,
a wrong weight or a transposed operand fails while rounding does not:

* ratio: r~ = sqrt(q w) with w = 1/d^2 from explicit FP32 differences
  (relative error gamma_{n+3}), q = |y_i - y_j|^2 from hi+lo FP32 Y (the
  difference exact to 2u of its size, plus an absolute a_ij =
  sqrt(k) n 2^-45 (|x_i| + |x_j|) / d_ij from the extended-precision
  product), sqrt.approx (2^-22):
      |r~ - r| <= rho_r r + a_ij,  rho_r = gamma_{n+3}/2 + gamma_{k+2} + 2u + 2^-22;
* weights: exp(x) via ex2.approx (2^-21 relative) of an FP32 argument
  (error u (M + r)/tau), FP32 tile sums then FP64:
      |L~ - L| <= sum p (rho_r r + a) + tau (2^-21 + gamma_40) + 2u sum p (L + r);
* gradient: each pair's term p_ij g_ij has |g_ij|_F = 1;
      |dp| <= p ((|dr| + |dL|)/tau + u (L + r)/tau + 2^-21),
  the coefficient and product add rho_t = gamma_{n+3} + 2^-21 + 4u, the
  per-warp FP32 sums gamma_32, and the Laplacian form (row and column sums
  of c_ij (y_i - y_j), size p/d, in FP32 trees of depth <= 24 within a
  tile and extended precision across tiles, times x - mean) adds, with
  margin, sqrt(k) gamma_34 p (nu_i + nu_j)/d_ij.
Each bound is taken x1.2.  The finite-difference check uses h = 1e-3 with a
tolerance of 2e-2 relative (truncation ~ h^2/tau^2 at tau = 0.01).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

U_ = 2.0 ** -24


def gam(m):
    return m * U_ / (1 - m * U_)


@pytest.fixture(scope="module")
def P():
    import paper_1807_03425_gb300 as P
    from paper_1807_03425_gb300 import build
    build.build()
    return P


def pair_arrays(X64, eps=0.0):
    N = X64.shape[0]
    iu, ju = np.triu_indices(N, 1)
    d = np.linalg.norm(X64[iu] - X64[ju], axis=1)
    keep = (d > 0) & ~(d < eps)
    return iu[keep], ju[keep], d[keep], keep


def bounds(X64, U, tau, L, eps=0.0):
    """Per-call error bounds on L and on dL/dU (Frobenius) from the oracle's
    values, as derived in the module docstring."""
    N, n = X64.shape
    k = U.shape[0]
    r_all = O.all_ratios(X64, U, eps)
    iu, ju, d, keep = pair_arrays(X64, eps)
    r = r_all[keep]
    assert np.all(r >= 0)
    p = np.exp(-(r - L) / tau)
    raw = np.linalg.norm(X64, axis=1)
    c32 = X64.astype(np.float32).mean(axis=0, dtype=np.float64)
    nu = np.linalg.norm(X64 - c32, axis=1)
    rho_r = gam(n + 3) / 2 + gam(k + 2) + 2 * U_ + 2.0 ** -22
    a = np.sqrt(k) * n * 2.0 ** -45 * (raw[iu] + raw[ju]) / d
    dr = rho_r * r + a
    bL = 1.2 * (np.sum(p * dr) + tau * (2.0 ** -21 + gam(40)) + 2 * U_ * np.sum(p * (L + r)))
    rho_t = gam(n + 3) + 2.0 ** -21 + 4 * U_
    dp = (dr + bL) / tau + U_ * (L + r) / tau + 2.0 ** -21
    lap = np.sqrt(k) * gam(34) * (nu[iu] + nu[ju]) / d
    bG = 1.2 * np.sum(p * (dp + rho_t + gam(32) + lap))
    return bL, bG, r.min(), len(r)


def moment_case(N, seed=1, m=50, k=5):
    X = W.moment_curve(N, m, seed, np.float32)
    U = W.random_basis(2 * m, k, seed + 1)
    return X, X.astype(np.float64), U


@pytest.mark.parametrize("N,tau", [(600, 0.01), (300, 0.05), (129, 0.002)])
def test_forward_and_backward_match_oracle(P, N, tau):
    X, X64, U = moment_case(N)
    Lo, Go = O.softmin(X64, U, tau)
    bL, bG, rmin, npairs = bounds(X64, U, tau, Lo)
    with P.Sap(X) as s:
        s.set_basis(U)
        st = s.stats()
        Lg = s.softmin_forward(tau)
        Gg = s.softmin_backward(tau, Lg)
    assert abs(Lg - Lo) <= bL, (Lg, Lo, bL)
    err = np.linalg.norm(Gg - Go)
    assert err <= bG, (err, bG, np.linalg.norm(Go))
    # log-sum-exp bounds of the exact objective hold for the GPU value too
    assert rmin - tau * np.log(npairs) - bL <= Lg <= rmin + bL
    # the case exercises the explicit near-pair path as well as the pass
    if N == 600:
        assert st["n_near"] > 0


def test_results_are_reproducible(P):
    X, X64, U = moment_case(400, seed=3)
    with P.Sap(X) as s:
        s.set_basis(U)
        L1 = s.softmin_forward(0.01)
        G1 = s.softmin_backward(0.01, L1)
        L2 = s.softmin_forward(0.01)
        G2 = s.softmin_backward(0.01, L2)
    assert L1 == L2
    assert np.array_equal(G1, G2)


def test_gradient_is_horizontal_and_matches_finite_differences(P):
    """L depends only on span U, so U^T G is symmetric; along a retraction
    qf(U + hE) the derivative is <G, (I - U U^T) E> (E scaled so that its
    horizontal part has unit norm: h is then the length of the step)."""
    tau, h = 0.01, 1e-3
    X, X64, U = moment_case(500, seed=5)
    Lo = O.softmin(X64, U, tau, grad=False)
    bL, bG, _, _ = bounds(X64, U, tau, Lo)
    g = np.random.default_rng(11)
    with P.Sap(X) as s:
        s.set_basis(U)
        L0 = s.softmin_forward(tau)
        G = s.softmin_backward(tau, L0)
        A = G @ U.T
        assert np.abs(A - A.T).max() <= 2 * bG
        for _ in range(3):
            E = g.standard_normal(U.shape)
            ER = E - (E @ U.T) @ U
            E, ER = E / np.linalg.norm(ER), ER / np.linalg.norm(ER)  # a unit step in span
            s.set_basis(O.qf(U + h * E))
            Lp = s.softmin_forward(tau)
            s.set_basis(O.qf(U - h * E))
            Lm = s.softmin_forward(tau)
            fd = (Lp - Lm) / (2 * h)
            an = float(np.sum(G * ER))
            assert abs(fd - an) <= 2e-2 * abs(an) + 2 * bL / (2 * h) + bG * np.linalg.norm(ER), (fd, an)


def test_eps_and_bf16_data(P):
    """Noisy-data variant: BF16 hyperspectral-like pixels with the
    short-secant threshold (excluded pairs count nowhere)."""
    tau, eps = 0.02, 0.4  # excludes about 4% of the pairs (noise floor ~0.11)
    E = W.endmembers(7, n_bands=60)
    Xb = W.hyperspectral(350, 7, E, 0.01, bf16=True)  # BF16-exact FP32 values
    X64 = Xb.astype(np.float64)
    U = W.random_basis(Xb.shape[1], 4, 8)
    Lo, Go = O.softmin(X64, U, tau, eps)
    bL, bG, _, _ = bounds(X64, U, tau, Lo, eps)
    with P.Sap(W.bf16_bits(Xb), dtype=P.BF16) as s:
        s.set_min_secant_length(eps)
        s.set_basis(U)
        Lg = s.softmin_forward(tau)
        Gg = s.softmin_backward(tau, Lg)
        assert s.stats()["n_excluded"] > 0
    assert abs(Lg - Lo) <= bL
    assert np.linalg.norm(Gg - Go) <= bG


@pytest.mark.parametrize("k", [1, 3, 8])
def test_other_widths(P, k):
    tau = 0.02
    X, X64, U = moment_case(300, seed=k, m=12, k=k)
    Lo, Go = O.softmin(X64, U, tau)
    bL, bG, _, _ = bounds(X64, U, tau, Lo)
    with P.Sap(X) as s:
        s.set_basis(U)
        Lg = s.softmin_forward(tau)
        Gg = s.softmin_backward(tau, Lg)
    assert abs(Lg - Lo) <= bL
    assert np.linalg.norm(Gg - Go) <= bG


def test_ascent_matches_oracle_steps(P):
    """Three Riemannian ascent steps on the device against the oracle's.
    Per step the update moves U by eta G_R/|G_R|, so a gradient error e
    moves it by at most 2 eta e/|G_R| (Frobenius); the bases are compared as
    projectors (sign- and rotation-free), and the recorded L values within
    their own bound plus |G| times the basis drift so far."""
    tau, eta, steps = 0.01, 0.005, 3
    X, X64, U = moment_case(400, seed=9)
    Uo = U.copy()
    ref, drift = [], 0.0
    for _ in range(steps + 1):
        L, Gf = O.softmin(X64, Uo, tau)
        bL, bG, _, _ = bounds(X64, Uo, tau, L)
        ref.append((L, bL + 2 * np.linalg.norm(Gf) * drift))
        if len(ref) > steps:
            break
        GR = Gf - (Gf @ Uo.T) @ Uo
        drift += 2 * eta * bG / np.linalg.norm(GR)
        Uo, _, _ = O.softmin_ascent_step(X64, Uo, tau, eta)
    with P.Sap(X) as s:
        s.set_basis(U)
        hist = s.softmin_ascent(tau, eta, steps)
        Ug = s.get_basis()
        # the handle's SAP state follows the new basis
        i, j, r = s.min_secant()
    for q, (L, tolL) in enumerate(ref):
        assert abs(hist[q] - L) <= tolL, (q, hist[q], L, tolL)
    assert np.abs(Ug @ Ug.T - np.eye(U.shape[0])).max() <= 1e-12
    assert np.abs(Ug.T @ Ug - Uo.T @ Uo).max() <= 2 * drift + 1e-12
    mo = O.min_secant(X64, Ug)
    assert abs(r - mo["r"]) <= 1e-5 * mo["r"]


def test_autograd_function(P):
    import torch
    from paper_1807_03425_gb300.autograd import softmin
    tau = 0.01
    X, X64, U = moment_case(300, seed=13)
    Lo, Go = O.softmin(X64, U, tau)
    bL, bG, _, _ = bounds(X64, U, tau, Lo)
    with P.Sap(X) as s:
        Ut = torch.tensor(U, device="cuda", requires_grad=True)
        L = softmin(Ut, s, tau)
        (3.0 * L).backward()
        g = Ut.grad.cpu().numpy()
        s.set_basis(U)
        Gd = s.softmin_backward(tau, float(L))
    assert abs(float(L) - Lo) <= bL
    assert np.array_equal(g, 3.0 * Gd)
    assert np.linalg.norm(g / 3.0 - Go) <= bG


def test_full_size_properties(P):
    """At the full size (moment curve m = 50, N = 16384, k = 5, tau = 0.01)
    the oracle is too slow pair by pair; properties that hold at any size:
    min r - tau log P <= L <= min r (min r from the certified SAP argmin),
    U^T G symmetric, and the ascent keeps U orthonormal while moving it."""
    tau = 0.01
    X = W.moment_curve(16384, 50, 1, np.float32)
    U = W.random_basis(100, 5, 2)
    with P.Sap(X) as s:
        s.set_path(P.RESTRUCTURED)
        s.set_basis(U)
        _, _, rmin = s.min_secant()
        L = s.softmin_forward(tau)
        G = s.softmin_backward(tau, L)
        P_ = 16384 * 16383 // 2 - s.stats()["n_excluded"]
        hist = s.softmin_ascent(tau, 0.005, 2)
        Ug = s.get_basis()
    assert rmin - tau * np.log(P_) - 1e-6 <= L <= rmin + 1e-6
    A = G @ U.T
    assert np.abs(A - A.T).max() <= 1e-4 * np.abs(A).max() + 1e-9
    assert hist[0] == L
    assert np.all(np.isfinite(hist))
    assert np.abs(Ug @ Ug.T - np.eye(5)).max() <= 1e-12
    assert np.abs(Ug.T @ Ug - U.T @ U).max() > 1e-4  # the basis moved


def test_argument_errors(P):
    X, X64, U = moment_case(200, seed=2)
    with P.Sap(X) as s:
        with pytest.raises(P.SapError) as e:
            s.softmin_forward(0.01)
        assert e.value.code == 2  # no basis
        s.set_basis(U)
        for bad in (0.0, -1.0, float("inf"), float("nan")):
            with pytest.raises(P.SapError) as e:
                s.softmin_forward(bad)
            assert e.value.code == 1
        s.set_basis(W.random_basis(100, 9, 3))
        with pytest.raises(P.SapError) as e:
            s.softmin_forward(0.01)
        assert e.value.code == 9
    with P.Sap(X64) as s:
        s.set_basis(U)
        with pytest.raises(P.SapError) as e:
            s.softmin_forward(0.01)
        assert e.value.code == 9
