"""The multi-GPU split of the argmin step on one GPU.

The ranks of a split run here one after another in one process, each with
its own handle (its own tiles' lengths): per iteration every rank's exact
minimum is taken (sap_shard_min), the records are handed to every rank, and
each rank updates (sap_shard_step).  No kernel waits on another rank, so
this is the multi-GPU path with the collective replaced by a copy.  The
trajectory must equal an unsplit handle's bit for bit (the FP64 tier decides
every argmin exactly and every rank runs the same update), and the first
evaluation must match the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import check_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1807_03425_gb300 as P
    from paper_1807_03425_gb300 import build
    build.build()
    return P


def unsplit(P, X, U0, alpha, T, tier):
    with P.Sap(X) as s:
        s.set_path("restructured")
        s.set_tuning(refine_tier=tier)
        s.set_basis(U0)
        hist, am = s.run(alpha, T)
        return hist, am, s.get_basis()


@pytest.mark.parametrize("world,tier", [(2, 0), (3, 3), (5, 1), (2, 5)])
def test_split_equals_unsplit_bitwise(P, world, tier):
    """Moment curve N = 1500 in R^40 (12 point blocks, 78 tiles, ragged last
    block), k = 5: world ranks, host records."""
    X = W.moment_curve(1500, 20, 31, np.float32)
    U0 = W.random_basis(40, 5, 32)
    alpha, T = 0.005, 12
    ref_hist, ref_am, ref_U = unsplit(P, X, U0, alpha, T, tier)
    ranks = [P.ShardSap(X, world, r) for r in range(world)]
    try:
        for s in ranks:
            s.set_tuning(refine_tier=tier)
            s.set_basis(U0)
        first = None
        for it in range(T):
            recs = [s.min_record() for s in ranks]
            if first is None:
                first = recs
            for s in ranks:
                s.step_records(alpha, recs)
        for s in ranks:
            h, am = s.get_history(T)
            assert np.array_equal(h, ref_hist[:T])
            assert np.array_equal(am, ref_am[:T])
            assert np.array_equal(s.get_basis(), ref_U)
        # the shards' pair counts add up; their first minima contain the oracle's
        st = [s.stats() for s in ranks]
        assert sum(x["n_near"] for x in st) >= 0
    finally:
        for s in ranks:
            s.close()
    X64 = X.astype(np.float64)
    m = O.min_secant(X64, U0)
    q, i, j = min((r for r in first if r[1] >= 0), key=lambda r: (r[0], r[1], r[2]))
    check_pair(X64, U0, m, i, j, np.sqrt(q))


def test_split_device_records(P):
    """The records stay on the device (as with an NCCL all-gather): each rank
    writes its record into its slot of one device buffer, then every rank
    steps from the whole buffer."""
    torch = pytest.importorskip("torch")
    X = W.moment_curve(900, 10, 41, np.float32)
    U0 = W.random_basis(20, 4, 42)
    alpha, T, world = 0.01, 8, 2
    ref_hist, ref_am, ref_U = unsplit(P, X, U0, alpha, T, 0)
    ranks = [P.ShardSap(X, world, r) for r in range(world)]
    try:
        for s in ranks:
            s.set_basis(U0)
        buf = torch.zeros(16 * world, dtype=torch.uint8, device="cuda")
        for it in range(T):
            for r, s in enumerate(ranks):
                s.min_record(buf[16 * r:16 * (r + 1)])
            torch.cuda.synchronize()
            for s in ranks:
                s.step_records(alpha, buf)
            torch.cuda.synchronize()
        for s in ranks:
            h, am = s.get_history(T)
            assert np.array_equal(h, ref_hist[:T]) and np.array_equal(am, ref_am[:T])
            assert np.array_equal(s.get_basis(), ref_U)
    finally:
        for s in ranks:
            s.close()


def test_shard_handle_guards(P):
    X = W.moment_curve(600, 10, 51, np.float32)
    with P.ShardSap(X, 2, 1) as s:
        s.set_basis(W.random_basis(20, 3, 52))
        lib = P.load_library()
        code = lib.sap_step(s.h, 0.01, None, None, None)
        assert P.capi.sap_status_str(code) == "SAP_E_STATE"
        code = lib.sap_set_path(s.h, P.PLAIN)
        assert P.capi.sap_status_str(code) == "SAP_E_UNSUPPORTED"
    # more ranks than tiles: the empty ranks are refused
    with pytest.raises(P.SapError):
        P.ShardSap(W.moment_curve(100, 5, 53, np.float32), 2, 1)
