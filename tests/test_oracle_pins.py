"""Pins for the FP64 oracle: each test ties it to something other than itself
(hand-derived closed forms, textbook identities, invariances, brute force on
tiny inputs), chosen so that a dropped term, a wrong sign, a transposed
operand or a wrong index fails at least one of them.

Paper: Kvinge et al., arXiv:1807.03425.  Sec. III-C (a projection never
lengthens a secant, so ratios are <= 1); Sec. IV and Algorithm 1 (ratio,
argmin, pivot, MGS, rotation); Sec. VI-A (dimension sweep); Sec. VII (length
threshold).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W


def _ev(e):
    """Evaluate a closed-form string from the golden file."""
    return float(eval(str(e), {"sqrt": math.sqrt, "__builtins__": {}}))


@pytest.fixture(scope="module")
def hand(golden_dir):
    with open(os.path.join(golden_dir, "hand_cases.json")) as f:
        return json.load(f)


# ---------------------------------------------------------------- ratios ----

def test_hand_ratio_cases(hand):
    for case in hand["ratio_cases"]:
        X = np.array(case["X"], dtype=np.float64)
        U = np.array(case["U"], dtype=np.float64)
        r = O.all_ratios(X, U)
        want = np.array([_ev(e) for e in case["ratios"]])
        np.testing.assert_allclose(r, want, rtol=0, atol=1e-15, err_msg=case["name"])
        m = O.min_secant(X, U)
        assert (m["i"], m["j"]) == tuple(case["argmin"]), case["name"]
        assert abs(m["r"] - _ev(case["min"])) <= 1e-15
        assert abs(m["runner_up"] - _ev(case["runner_up"])) <= 1e-15


def test_pair_index_enumerates_upper_triangle():
    N = 7
    seen = [O.pair_index(i, j, N) for i in range(N) for j in range(i + 1, N)]
    assert seen == list(range(N * (N - 1) // 2))


def _brute_ratios(X, U):
    """Brute force through the orthogonal projector P = U^T U (rows are basis
    vectors): r^2 = s^T P s for the unit secant s -- a different formula from
    the oracle's ||U s||, equal for orthonormal rows."""
    P = U.T @ U
    out = []
    for i, j in itertools.combinations(range(X.shape[0]), 2):
        s = (X[i] - X[j]) / np.linalg.norm(X[i] - X[j])
        out.append(math.sqrt(max(0.0, float(s @ P @ s))))
    return np.array(out)


@pytest.mark.parametrize("N,n,k,seed", [(2, 3, 1, 0), (4, 5, 2, 1), (5, 4, 3, 2), (6, 7, 2, 3)])
def test_brute_force_tiny(N, n, k, seed):
    g = np.random.default_rng(seed)
    X = g.standard_normal((N, n))
    U = W.random_basis(n, k, seed + 10)
    r = O.all_ratios(X, U)
    np.testing.assert_allclose(r, _brute_ratios(X, U), rtol=1e-13, atol=1e-15)
    # argmin by sorting (ratio, pair index)
    order = sorted((rv, p) for p, rv in enumerate(r))
    pairs = list(itertools.combinations(range(N), 2))
    m = O.min_secant(X, U)
    assert pairs[order[0][1]] == (m["i"], m["j"])
    assert m["r"] == order[0][0]
    if len(order) > 1:
        assert m["runner_up"] == order[1][0]


def test_full_dimension_gives_unit_ratios():
    """k = n: the projection is the identity on R^n, every ratio is 1."""
    X = W.moment_curve(40, 3, 5, np.float64)
    r = O.all_ratios(X, np.eye(6))
    assert np.abs(r - 1.0).max() <= 1e-14


def test_ratios_bounded_by_one():
    """Sec. III-C: a projection satisfies the upper Lipschitz bound with
    m2 = 1, so 0 <= r <= 1."""
    X = W.moment_curve(60, 5, 3, np.float64)
    U = W.random_basis(10, 3, 4)
    r = O.all_ratios(X, U)
    assert r.min() >= 0.0 and r.max() <= 1.0 + 1e-15


def test_data_in_subspace_is_isometric():
    """Points inside span(U): every secant lies in the span, r = 1."""
    g = np.random.default_rng(7)
    U = W.random_basis(9, 4, 8)
    X = g.standard_normal((25, 4)) @ U
    r = O.all_ratios(X, U)
    assert np.abs(r - 1.0).max() <= 1e-13


def test_naive_projection_of_moment_curve_closed_form():
    """First-three-coordinates projection of the Sec. V curve: as the sample
    gets dense the minimum tends to the tangent limit at sin 2t = 0,
    ||(-sin t, cos t, -2 sin 2t)|| / ||phi'(t)|| = 1/sqrt(1+4+9+16+25)."""
    X = W.moment_curve(2000, 5, 1, np.float64)
    m = O.min_secant(X, np.eye(10)[:3])
    lim = 1.0 / math.sqrt(55.0)
    assert lim <= m["r"] <= lim + 2e-6


def test_permutation_invariance():
    X = W.moment_curve(50, 5, 11, np.float64)
    U = W.random_basis(10, 3, 12)
    m = O.min_secant(X, U)
    perm = np.random.default_rng(13).permutation(50)
    m2 = O.min_secant(X[perm], U)
    assert m2["r"] == pytest.approx(m["r"], rel=1e-13)
    # point a of X[perm] is original point perm[a]
    assert sorted((perm[m2["i"]], perm[m2["j"]])) == [m["i"], m["j"]]


def test_joint_rotation_invariance_and_update_equivariance():
    """x -> R x, u -> R u leaves every ratio unchanged; the update commutes
    with R."""
    X = W.moment_curve(40, 4, 21, np.float64)
    U = W.random_basis(8, 3, 22)
    R = W.random_basis(8, 8, 23)  # orthogonal 8 x 8
    Xr, Ur = X @ R.T, U @ R.T
    np.testing.assert_allclose(O.all_ratios(Xr, Ur), O.all_ratios(X, U), rtol=1e-12)
    m = O.min_secant(X, U)
    Un, _ = O.update(X, U, m["i"], m["j"], 0.05)
    Unr, _ = O.update(Xr, Ur, m["i"], m["j"], 0.05)
    np.testing.assert_allclose(Unr, Un @ R.T, atol=1e-13)


# ---------------------------------------------------------------- update ----

def test_hand_update_cases(hand):
    for case in hand["update_cases"]:
        U = np.array(case["U"], dtype=np.float64)
        s = np.array([_ev(e) for e in case["s"]])
        mode = O.MODE_ANGLE if case["mode"] == "angle" else O.MODE_LITERAL
        Un, t = O.update_with_secant(s, U, _ev(case["alpha"]), mode)
        want = np.array([[_ev(e) for e in row] for row in case["U_new"]])
        assert t == case["pivot"], case["name"]
        np.testing.assert_allclose(Un, want, atol=1e-15, err_msg=case["name"])


def _chosen_secant_closed_form(r, a, mode):
    """Ratio of the chosen secant after one update (derived from Sec. IV):
    s = v + e with |v| = r, |e| = sqrt(1-r^2), v in span U, e orthogonal to it;
    the other new columns are orthogonal to both, so only u1' sees s."""
    if mode == O.MODE_LITERAL:
        return ((1 - a) * r * r + a * (1 - r * r)) / math.sqrt(
            (1 - a) ** 2 * r * r + a * a * (1 - r * r))
    return ((1 - a) * r + a * math.sqrt(1 - r * r)) / math.sqrt((1 - a) ** 2 + a * a)


@pytest.mark.parametrize("mode", [O.MODE_LITERAL, O.MODE_ANGLE])
@pytest.mark.parametrize("alpha", [0.0, 0.005, 0.01, 0.3])
def test_update_closed_form_orthonormality_and_span(mode, alpha):
    X = W.moment_curve(60, 5, 31, np.float64)
    U = W.random_basis(10, 3, 32)
    m = O.min_secant(X, U)
    s = O.unit_secant(X, m["i"], m["j"])
    Un, _ = O.update(X, U, m["i"], m["j"], alpha, mode)
    # orthonormal columns after the step
    assert np.abs(Un @ Un.T - np.eye(3)).max() <= 1e-14
    # closed form for the chosen secant
    want = _chosen_secant_closed_form(m["r"], alpha, mode)
    assert np.linalg.norm(Un @ s) == pytest.approx(want, rel=1e-12)
    # span pin: q1 = normalised P P^T s leaves, u1' enters, the other new
    # columns stay inside the old span, so for every secant s'
    #   r'^2 = r^2 - (q1.s')^2 + (u1'.s')^2
    v = U.T @ (U @ s)
    q1 = v / np.linalg.norm(v)
    for i, j in [(0, 1), (3, 17), (m["i"], m["j"]), (5, 59), (20, 21)]:
        sp = O.unit_secant(X, i, j)
        lhs = np.linalg.norm(Un @ sp) ** 2
        rhs = np.linalg.norm(U @ sp) ** 2 - (q1 @ sp) ** 2 + (Un[0] @ sp) ** 2
        assert lhs == pytest.approx(rhs, abs=1e-13)
    if alpha == 0.0:
        # alpha = 0 keeps the span: same projector
        np.testing.assert_allclose(Un.T @ Un, U.T @ U, atol=1e-14)


def test_update_keeps_span_when_secant_in_span():
    U = W.random_basis(7, 3, 41)
    s = U.T @ np.array([0.3, -0.5, 0.2])
    s /= np.linalg.norm(s)
    Un, _ = O.update_with_secant(s, U, 0.2)
    np.testing.assert_allclose(Un.T @ Un, U.T @ U, atol=1e-14)


def test_run_history_matches_stepwise():
    X = W.moment_curve(80, 5, 51, np.float64)
    U0 = W.random_basis(10, 3, 52)
    UT, hist, am = O.run(X, U0, 0.01, 5)
    U = U0
    for it in range(6):
        m = O.min_secant(X, U)
        assert hist[it] == m["r"] and tuple(am[it]) == (m["i"], m["j"])
        if it < 5:
            U, _ = O.update(X, U, m["i"], m["j"], 0.01)
    np.testing.assert_array_equal(UT, U)


def test_sap_raises_min_ratio_on_moment_curve():
    """Sec. V: SAP improves the shortest projected secant; 100 iterations at
    alpha = 0.01 lift it well above the start."""
    X = W.moment_curve(200, 5, 1, np.float64)
    U0 = W.random_basis(10, 3, 2)
    _, hist, _ = O.run(X, U0, 0.01, 100)
    assert hist[-1] > 5 * hist[0]


# ------------------------------------------------------------- threshold ----

def test_threshold_exclusion_hand_case():
    """Sec. VII: discard secants shorter than l before normalising.  Lengths
    here: |p0p1| = 1, |p0p2| = 2, |p1p2| = sqrt5.  eps = 2 keeps d == 2."""
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 2, 0]], dtype=np.float64)
    U = np.array([[1.0, 0, 0]])
    r = O.all_ratios(X, U, eps=2.0)
    assert r[0] == -1.0 and r[1] == 0.0 and r[2] == pytest.approx(1 / math.sqrt(5))
    m = O.min_secant(X, U, eps=2.0)
    assert (m["i"], m["j"], m["excluded"]) == (0, 2, 1)
    # eps = 0 is the unthresholded algorithm
    np.testing.assert_array_equal(O.all_ratios(X, U, 0.0), O.all_ratios(X, U))
    with pytest.raises(O.NoSecantError):
        O.min_secant(X, U, eps=3.0)


def test_duplicates_are_not_secants():
    X = np.array([[1, 2], [1, 2], [3, 2]], dtype=np.float64)
    m = O.min_secant(X, np.array([[1.0, 0.0]]))
    assert m["excluded"] == 1 and (m["i"], m["j"]) == (0, 2)
    with pytest.raises(O.NoSecantError):
        O.min_secant(X[:2], np.array([[1.0, 0.0]]))


# ------------------------------------------------------------ dimension -----

def test_estimate_dim_coordinate_simplex():
    """Points 0, e1..e4 in R^6 with U0 = e1..e6 and no iterations: for k < 4
    the secant e4 is orthogonal to span(e1..ek) (ratio 0); at k = 4 every
    secant lies in the span (ratio 1).  So the sweep returns 4."""
    X = np.vstack([np.zeros(6), np.eye(6)[:4]])
    U0 = np.eye(6)
    k, ratios = O.estimate_dim(X, U0, T=0, alpha=0.01, threshold=0.1)
    assert k == 4
    np.testing.assert_allclose(ratios, [0, 0, 0, 1, 1, 1], atol=1e-15)


def test_estimate_dim_matches_runs():
    X = W.moment_curve(60, 3, 61, np.float64)
    U0 = W.random_basis(6, 4, 62)
    k, ratios = O.estimate_dim(X, U0, T=7, alpha=0.02, threshold=0.3)
    for kk in range(1, 5):
        _, hist, _ = O.run(X, U0[:kk], 0.02, 7)
        assert ratios[kk - 1] == hist[-1]
    assert k == next((kk + 1 for kk in range(4) if ratios[kk] > 0.3), -1)


# -------------------------------------------------------------- soft-min ----

def test_softmin_single_pair_closed_form():
    """One pair: L = r exactly and dL/dU = s (U s)^T / r (rows: u_c)."""
    X = np.array([[0.0, 0, 0], [1.0, 2.0, 2.0]])
    U = W.random_basis(3, 2, 71)
    L, G = O.softmin(X, U, tau=0.05)
    s = (X[0] - X[1]) / 3.0
    z = U @ s
    r = np.linalg.norm(z)
    assert L == pytest.approx(r, rel=1e-14)
    np.testing.assert_allclose(G, np.outer(z, s) / r, atol=1e-14)


def test_softmin_bounds_symmetry_and_finite_differences():
    X = W.moment_curve(40, 4, 81, np.float64)
    U = W.random_basis(8, 3, 82)
    tau = 0.05
    L, G = O.softmin(X, U, tau)
    r = O.all_ratios(X, U)
    P = r.size
    # log-sum-exp bounds: min r - tau ln P <= L <= min r
    assert r.min() - tau * math.log(P) - 1e-14 <= L <= r.min() + 1e-14
    # L depends on span(U) only, so U^T G is symmetric
    S = U @ G.T
    assert np.abs(S - S.T).max() <= 1e-12 * max(1.0, np.abs(S).max())
    # central finite differences, h = 1e-6 (the FP64 oracle can afford it)
    h = 1e-6
    for (c, l) in [(0, 0), (1, 3), (2, 7), (0, 5)]:
        Up, Um = U.copy(), U.copy()
        Up[c, l] += h
        Um[c, l] -= h
        fd = (O.softmin(X, Up, tau, grad=False) - O.softmin(X, Um, tau, grad=False)) / (2 * h)
        assert fd == pytest.approx(G[c, l], rel=1e-6, abs=1e-8)


def test_softmin_ascent_step_stays_orthonormal():
    X = W.moment_curve(40, 4, 91, np.float64)
    U = W.random_basis(8, 3, 92)
    Un, L, nr = O.softmin_ascent_step(X, U, 0.05, 0.01)
    assert nr > 0
    assert np.abs(Un @ Un.T - np.eye(3)).max() <= 1e-14
    assert O.softmin(X, Un, 0.05, grad=False) > L


def test_softmin_ascent_step_hand_cases(hand):
    """Closed forms of one Grassmann ascent step on a single secant, where
    dL/dU has a non-zero radial part U(U^T G): the result fails if the
    tangent projection is dropped, if the step is normalised by ||G||
    instead of ||G_R||, or if qf returns a negative diagonal of R."""
    for case in hand["ascent_cases"]:
        X = np.array(case["X"], dtype=np.float64)
        U = np.array(case["U"], dtype=np.float64)
        want = np.array([[_ev(e) for e in row] for row in case["U_new"]])
        Un, L, nr = O.softmin_ascent_step(X, U, case["tau"], _ev(case["eta"]))
        np.testing.assert_allclose(Un, want, rtol=0, atol=1e-15, err_msg=case["name"])
        assert abs(L - _ev(case["L"])) <= 1e-15, case["name"]
        assert abs(nr - _ev(case["norm_GR"])) <= 4e-15, case["name"]  # a few ulps


def test_qf_hand_case():
    """qf of the rows (3,4,0), (1,0,2): q1 = (3,4,0)/5; the second row minus
    its projection 3/5 q1 is (16,-12,50)/25, of length 2 sqrt(29)/5, so
    q2 = (8,-6,25)/(5 sqrt(29)); both R diagonal entries positive."""
    Q = O.qf(np.array([[3.0, 4.0, 0.0], [1.0, 0.0, 2.0]]))
    want = np.array([[0.6, 0.8, 0.0], np.array([8.0, -6.0, 25.0]) / (5 * math.sqrt(29))])
    np.testing.assert_allclose(Q, want, rtol=0, atol=1e-15)


# ---------------------------------------------------------------- secant PCA --
# The PCA start of Algorithm 1 (Sec. IV): top-k left singular vectors of the
# unit-secant matrix S.


def test_secant_pca_hand_triangle():
    """Points (0,0), (1,0), (0,1): unit secants (-1,0), (0,-1), (1,-1)/sqrt2,
    so S S^T = [[3/2, -1/2], [-1/2, 3/2]] with eigenvalues 2 and 1; the first
    direction is (1,-1)/sqrt2 (first entry positive), singular value sqrt2."""
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    C, kept = O.secant_gram(X)
    assert kept == 3
    assert np.allclose(C, [[1.5, -0.5], [-0.5, 1.5]], atol=1e-15)
    U, sv = O.secant_pca(X, 1)
    assert np.allclose(U, [[2 ** -0.5, -(2 ** -0.5)]], atol=1e-15)
    assert abs(sv[0] - 2 ** 0.5) < 1e-15


@pytest.mark.parametrize("N,n,k,seed", [(6, 3, 2, 1), (7, 5, 3, 2), (8, 4, 1, 3)])
def test_secant_pca_matches_svd_of_explicit_secants(N, n, k, seed):
    """Against numpy's SVD of the explicitly built n x p secant matrix."""
    X = np.random.default_rng(seed).standard_normal((N, n))
    cols = [(X[i] - X[j]) / np.linalg.norm(X[i] - X[j]) for i in range(N) for j in range(i + 1, N)]
    S = np.array(cols).T
    Us, sv, _ = np.linalg.svd(S, full_matrices=False)
    U, svo = O.secant_pca(X, k)
    assert np.allclose(svo, sv[:k], rtol=1e-12)
    Pu, Ps = U.T @ U, Us[:, :k] @ Us[:, :k].T
    assert np.abs(Pu - Ps).max() < 1e-10
    assert np.abs(U @ U.T - np.eye(k)).max() < 1e-13


def test_secant_gram_trace_counts_kept_pairs():
    """trace(S S^T) = number of kept unit secants: duplicates and pairs
    shorter than eps do not count (Sec. II, Sec. VII)."""
    g = np.random.default_rng(4)
    X = g.standard_normal((30, 6))
    X[7] = X[3]
    X[12] = X[11] + 1e-3
    C, kept = O.secant_gram(X)
    assert kept == 30 * 29 // 2 - 1 and abs(np.trace(C) - kept) < 1e-10
    C2, kept2 = O.secant_gram(X, eps=0.01)
    assert kept2 == kept - 1 and abs(np.trace(C2) - kept2) < 1e-10


def test_secant_pca_of_subspace_data_is_isometric():
    """Points in a k0-dimensional affine subspace: the top k0 secant
    directions span it, every unit secant keeps its length (min ratio 1) and
    the next singular value is zero."""
    g = np.random.default_rng(5)
    A = np.linalg.qr(g.standard_normal((9, 3)))[0].T  # 3 x 9, orthonormal rows
    X = g.standard_normal((40, 3)) @ A + 0.7
    U, sv = O.secant_pca(X, 4)
    assert sv[3] < 1e-6 * sv[0]
    m = O.min_secant(X, U[:3])
    assert abs(m["r"] - 1.0) < 1e-12
    assert np.abs(U[:3].T @ U[:3] - A.T @ A).max() < 1e-10


def test_secant_pca_rotation_equivariance():
    g = np.random.default_rng(6)
    X = g.standard_normal((25, 5)) * np.array([3.0, 2.0, 1.0, 0.5, 0.2])
    Q = np.linalg.qr(g.standard_normal((5, 5)))[0]
    U, sv = O.secant_pca(X, 2)
    V, sv2 = O.secant_pca(X @ Q, 2)
    assert np.allclose(sv, sv2, rtol=1e-12)
    # rows of U are vectors: the rotated data's directions are U Q, up to sign
    dots = np.abs(np.sum((U @ Q) * V, axis=1))
    assert np.allclose(dots, 1.0, atol=1e-10)
