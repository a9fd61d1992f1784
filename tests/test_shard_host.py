"""The multi-GPU split of the argmin step, checked on the CPU.

Algorithm 1's argmin (Sec. IV of Kvinge et al., arXiv:1807.03425) is a
minimum over all pairs, so it splits over disjoint pair sets: each rank owns
a contiguous range of 128 x 128 pair tiles (row-major over the upper
triangle, equal pair counts, from the library's host code) and finds its
exact minimum; the ranks exchange 16-byte records and every rank takes the
winner.  Here the ranks are `gloo` processes that evaluate their shards with
the FP64 oracle, exchange records over the process group and merge them with
the library's host merge; the result must be the oracle's unsplit argmin,
exactly, iteration after iteration."""
import os
import socket

import numpy as np
import pytest

from paper_1807_03425_gb300 import capi

TILE = 128


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1807_03425_gb300 import build
    build.build()
    return capi.load_library()


def tile_order(N):
    nb = (N + TILE - 1) // TILE
    return [(I, J) for I in range(nb) for J in range(I, nb)]


def tile_pairs(N, I, J):
    rI, rJ = min(TILE, N - I * TILE), min(TILE, N - J * TILE)
    return rI * (rI - 1) // 2 if I == J else rI * rJ


@pytest.mark.parametrize("N", [2, 127, 128, 129, 300, 1000, 8192, 92681])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_shard_ranges_cover_every_pair_once_and_balance(N, world):
    tiles = tile_order(N)
    P = N * (N - 1) // 2
    bounds = [capi.sap_shard_range(N, world, r) for r in range(world)]
    assert bounds[0][0] == 0 and bounds[-1][1] == len(tiles)
    for r in range(world - 1):
        assert bounds[r][1] == bounds[r + 1][0]          # contiguous, disjoint
    counts = [sum(tile_pairs(N, *tiles[t]) for t in range(t0, t1)) for t0, t1, _ in bounds]
    assert [b[2] for b in bounds] == counts
    assert sum(counts) == P
    if len(tiles) >= world:
        # every rank is within one tile's pairs of an equal share
        assert max(abs(c - P / world) for c in counts) <= TILE * TILE


def test_shard_range_rejects_bad_arguments():
    for args in [(1, 2, 0), (100, 0, 0), (100, 2, 2), (100, 2, -1), (92682, 2, 0), (100, 4097, 0)]:
        with pytest.raises(capi.SapError):
            capi.sap_shard_range(*args)


def test_merge_records_takes_the_lexicographic_minimum():
    m = capi.sap_merge_records
    assert m([(0.5, 3, 9), (0.25, 7, 8), (0.75, 0, 1)]) == (0.25, 7, 8)
    # equal q: the smallest pair index, i first, then j
    assert m([(0.25, 7, 8), (0.25, 2, 90), (0.25, 2, 40)]) == (0.25, 2, 40)
    # a rank without a candidate contributes i = -1
    assert m([(float("inf"), -1, -1), (0.5, 4, 5)]) == (0.5, 4, 5)
    assert m([(float("inf"), -1, -1), (0.0, -1, -1)]) is None
    assert m([]) is None


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, T, alpha, eps):
    import torch
    import torch.distributed as dist

    import oracle as O
    import workloads as W
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, world_size=world, rank=rank)
    try:
        X = W.moment_curve(300, 5, 7, np.float64)
        X[17] = X[3]                       # a duplicate point: its pair is excluded
        N = X.shape[0]
        U0 = W.random_basis(10, 3, 8)
        U = U0.copy()
        # this rank's pairs, from the library's split
        t0, t1, npairs = capi.sap_shard_range(N, world, rank)
        mask = np.zeros(N * (N - 1) // 2, dtype=bool)
        tiles = tile_order(N)
        iu, ju = np.triu_indices(N, 1)
        blk_i, blk_j = iu // TILE, ju // TILE
        for t in range(t0, t1):
            I, J = tiles[t]
            mask |= (blk_i == I) & (blk_j == J)
        assert int(mask.sum()) == npairs
        hist = []
        for _ in range(T):
            r = O.all_ratios(X, U, eps)    # -1 marks excluded pairs
            ok = mask & (r >= 0)
            if ok.any():
                cand = np.flatnonzero(ok)
                p = cand[np.argmin(r[cand])]  # first minimum: smallest pair index
                rec = torch.tensor([r[p] * r[p], float(iu[p]), float(ju[p])], dtype=torch.float64)
            else:
                rec = torch.tensor([np.inf, -1.0, -1.0], dtype=torch.float64)
            parts = [torch.empty(3, dtype=torch.float64) for _ in range(world)]
            dist.all_gather(parts, rec)
            q, i, j = capi.sap_merge_records([(float(v[0]), int(v[1]), int(v[2])) for v in parts])
            m = O.min_secant(X, U, eps)
            assert (i, j) == (m["i"], m["j"])
            assert q == m["r"] * m["r"]
            hist.append(m["r"])
            U, _ = O.update(X, U, i, j, alpha)
        Uo, ho, _ = O.run(X, U0, alpha, T, eps)
        assert np.array_equal(U, Uo)
        assert np.array_equal(np.array(hist), ho[:T])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,eps", [(2, 0.0), (3, 0.05)])
def test_gloo_ranks_reproduce_the_unsplit_oracle(world, eps):
    """world gloo processes on the CPU: per iteration each evaluates its own
    tiles' pairs in FP64, the 16-byte records are all-gathered and merged,
    and every rank updates with the winner; after T iterations the basis and
    the history equal the unsplit oracle's bit for bit."""
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    mp.spawn(_rank_main, args=(world, _free_port(), 4, 0.01, eps), nprocs=world, join=True)
