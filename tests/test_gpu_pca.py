"""The PCA start of Algorithm 1 (sap_secant_pca): the top k left singular
vectors of the unit-secant matrix, formed on the device in FP64 as
Xc^T L X and diagonalised by the library's FP64 Jacobi solver, against the FP64 oracle (which sums
s s^T pair by pair and diagonalises with numpy)."""
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


def scaled(N, n, seed, dtype=np.float32):
    """Gaussian points with decaying scales (clear gaps between the secant
    directions) plus an offset."""
    g = np.random.default_rng(seed)
    scales = 3.0 * 0.8 ** np.arange(n)
    return (g.standard_normal((N, n)) * scales + 1.5).astype(dtype)


def compare(Ug, svg, Uo, svo):
    assert np.allclose(svg, svo, rtol=1e-10, atol=0)
    assert np.abs(Ug - Uo).max() < 1e-8, np.abs(Ug - Uo).max()
    assert np.abs(Ug @ Ug.T - np.eye(Ug.shape[0])).max() < 1e-12


@pytest.mark.parametrize("N,n,k", [(300, 7, 1), (517, 40, 3), (700, 100, 5), (65, 12, 12), (130, 1, 1),
                                   (300, 33, 4)])
def test_secant_pca_matches_oracle(P, N, n, k):
    """Ragged point counts around the 64-point blocks, k up to n; odd n (the
    Jacobi round-robin has an unpaired index) and n = 1."""
    X = scaled(N, n, N + n)
    with P.Sap(X) as s:
        Ug, svg = s.secant_pca(k)
        assert np.array_equal(s.get_basis(), Ug)
        i, j, r = s.min_secant()
    Uo, svo = O.secant_pca(X.astype(np.float64), k)
    compare(Ug, svg, Uo, svo)
    m = O.min_secant(X.astype(np.float64), Uo)
    assert abs(r - m["r"]) <= 1e-5 * m["r"] + 1e-13


def test_secant_pca_threshold_and_fp64_data(P):
    """Pairs shorter than eps and duplicates are not secants (Sec. II,
    Sec. VII); FP64 data takes the same path."""
    X = scaled(400, 20, 3, np.float64)
    X[17] = X[5]
    X[30] = X[29] + 1e-3
    for eps in (0.0, 0.05, 1.5):
        with P.Sap(X) as s:
            if eps:
                s.set_min_secant_length(eps)
            Ug, svg = s.secant_pca(4)
        Uo, svo = O.secant_pca(X, 4, eps)
        compare(Ug, svg, Uo, svo)


def test_secant_pca_of_subspace_data_is_isometric(P):
    """Points on a 3-dimensional affine subspace of R^30: the PCA start
    already keeps every secant's length (min ratio 1, Sec. IV)."""
    g = np.random.default_rng(9)
    A = np.linalg.qr(g.standard_normal((30, 3)))[0].T
    X = (g.standard_normal((900, 3)) @ A + 0.5).astype(np.float32)
    with P.Sap(X) as s:
        U, sv = s.secant_pca(3)
        _, _, r = s.min_secant()
    assert abs(r - 1.0) < 1e-6
    assert np.abs(U.T @ U - A.T @ A).max() < 1e-5


def test_secant_pca_errors(P):
    X = scaled(50, 6, 1)
    with P.Sap(X) as s:
        for k in (0, 7):
            with pytest.raises(P.SapError) as e:
                s.secant_pca(k)
            assert e.value.code == 1
