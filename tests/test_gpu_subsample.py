"""Repeated point subsampling (Sec. VI-C): a batch of random subsets of one
point set, each with its own dimension sweep.  Each subset must behave
exactly like a handle created from its gathered rows, and its first
evaluation must be the oracle's minimum."""
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


def pixels(N, bands, seed):
    E = W.endmembers(seed, bands)
    return W.hyperspectral(N, seed + 1, E, noise=0.01, bf16=False)


def test_subsets_equal_standalone_handles_and_oracle(P):
    X = pixels(3000, 24, 5)
    idx = W.subsample_indices(3000, 3, 200, 6)
    U0 = W.random_basis(24, 6, 7)
    with P.SapBatch.from_subsamples(X, idx) as sb:
        assert P.capi.sap_batch_count(sb.h) == 3
        got = [sb.estimate_dim(b, U0, 10, 0.01, 0.1) for b in range(3)]
        first = [sb.estimate_dim(b, U0, 0, 0.01, 0.1) for b in range(3)]
    for b in range(3):
        with P.Sap(X[idx[b]]) as s:
            k_ref, r_ref = s.estimate_dim(U0, 10, 0.01, 0.1)
        assert got[b][0] == k_ref and np.array_equal(got[b][1], r_ref), b
        # zero iterations: the ratio of each k is the oracle's minimum for U0[:k]
        X64 = X[idx[b]].astype(np.float64)
        for k in (1, 3, 6):
            m = O.min_secant(X64, U0[:k])
            assert abs(first[b][1][k - 1] - m["r"]) <= 1e-5 * m["r"] + 1e-13, (b, k)


def test_device_rows_and_duplicates(P):
    import torch
    X = pixels(800, 16, 11)
    idx = W.subsample_indices(800, 2, 120, 12)
    idx[1, 5] = idx[1, 6]  # a duplicated row: its pair is excluded, nothing else changes
    U0 = W.random_basis(16, 4, 13)
    with P.SapBatch.from_subsamples(X, idx) as a, \
            P.SapBatch.from_subsamples(torch.from_numpy(X).cuda(), idx) as b:
        for q in range(2):
            ra = a.estimate_dim(q, U0, 5, 0.01, 0.1)
            rb = b.estimate_dim(q, U0, 5, 0.01, 0.1)
            assert ra[0] == rb[0] and np.array_equal(ra[1], rb[1])
        assert a.stats()["n_excluded"] == 1


def test_subsample_argument_errors(P):
    X = pixels(100, 8, 1)
    for bad in (np.array([[0, 100]]), np.array([[-1, 3]]), np.zeros((1, 1), dtype=np.int64)):
        with pytest.raises(P.SapError) as e:
            P.capi.sap_create_subsamples(X, bad)
        assert e.value.code == 1
    with P.SapBatch.from_subsamples(X, W.subsample_indices(100, 2, 30, 2)) as sb:
        with pytest.raises(P.SapError) as e:
            sb.estimate_dim(2, W.random_basis(8, 3, 1), 2, 0.01, 0.1)
        assert e.value.code == 1
