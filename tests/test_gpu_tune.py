"""The launch-parameter autotuner (sap_autotune / sap_set_tuning).  Launch
parameters never change a result: every setting evaluates certified
candidate sets and takes the same FP64 decisions, so trajectories must be
bitwise identical whatever the tuner chose.  Also checked against the FP64
oracle at the first and last evaluation, and the on-disk cache across
processes."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import check_pair

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_1807_03425_gb300 as P
    from paper_1807_03425_gb300 import build
    build.build()
    return P


def trajectory(s, U0, alpha, T):
    s.set_basis(U0)
    hist, am = s.run(alpha, T)
    return hist, am, s.get_basis()


EXTREMES = [
    dict(pass_bound=0.05, pass_stages=2, explicit_blocks_per_sm=1, update_blocks=38, plain_blocks_per_sm=1,
         programmatic_launch=1, refine_tier=1),
    dict(pass_bound=1e-4, pass_stages=3, explicit_blocks_per_sm=4, update_blocks=304, plain_blocks_per_sm=4,
         programmatic_launch=0, refine_tier=0),
    dict(pass_bound=2e-3, pass_stages=0, explicit_blocks_per_sm=2, update_blocks=0, plain_blocks_per_sm=2,
         programmatic_launch=1, refine_tier=-1),
    dict(pass_bound=4e-3, pass_stages=0, explicit_blocks_per_sm=1, update_blocks=76, plain_blocks_per_sm=2,
         programmatic_launch=0, refine_tier=1),
    dict(pass_bound=1e-3, pass_stages=2, explicit_blocks_per_sm=2, update_blocks=152, plain_blocks_per_sm=2,
         programmatic_launch=1, refine_tier=2),
    dict(pass_bound=8e-3, pass_stages=0, explicit_blocks_per_sm=1, update_blocks=38, plain_blocks_per_sm=2,
         programmatic_launch=0, refine_tier=2),
    dict(pass_bound=4e-3, pass_stages=0, explicit_blocks_per_sm=1, update_blocks=76, plain_blocks_per_sm=2,
         programmatic_launch=1, refine_tier=3),
    dict(pass_bound=5e-4, pass_stages=3, explicit_blocks_per_sm=4, update_blocks=0, plain_blocks_per_sm=2,
         programmatic_launch=0, refine_tier=3),
    dict(pass_bound=4e-3, pass_stages=0, explicit_blocks_per_sm=2, update_blocks=152, plain_blocks_per_sm=2,
         programmatic_launch=1, refine_tier=4),
    dict(pass_bound=2e-3, pass_stages=0, explicit_blocks_per_sm=1, update_blocks=76, plain_blocks_per_sm=2,
         programmatic_launch=1, refine_tier=5),
    dict(pass_bound=1.6e-2, pass_stages=2, explicit_blocks_per_sm=2, update_blocks=0, plain_blocks_per_sm=2,
         programmatic_launch=0, refine_tier=5),
]


@pytest.mark.parametrize("path", ["restructured", "plain"])
def test_tuning_never_changes_results(P, path):
    """Moment curve N = 1500 in R^40 (12 row tiles, ragged), k = 5, 40
    iterations: the default, the tuned and three hand-set parameter sets
    give bitwise-identical histories, argmins and final bases."""
    X = W.moment_curve(1500, 20, 11, np.float32)
    U0 = W.random_basis(40, 5, 12)
    alpha, T = 0.005, 40
    with P.Sap(X) as s:
        s.set_path(path)
        ref = trajectory(s, U0, alpha, T)
        tuned = s.autotune(alpha, 8)
        assert tuned["us_per_iteration"] > 0
        assert s.tuning() == tuned
        runs = [trajectory(s, U0, alpha, T)]
        for t in EXTREMES:
            s.set_tuning(**t)
            got = s.tuning()
            for key, v in t.items():
                assert got[key] == v
            runs.append(trajectory(s, U0, alpha, T))
            if path == "restructured":
                assert s.stats()["cert_bound"] == t["pass_bound"]
    for h, am, U in runs:
        assert np.array_equal(h, ref[0]) and np.array_equal(am, ref[1]) and np.array_equal(U, ref[2])
    X64 = X.astype(np.float64)
    m = O.min_secant(X64, U0)
    check_pair(X64, U0, m, int(ref[1][0, 0]), int(ref[1][0, 1]), ref[0][0])


def test_pass_bound_trades_near_list_for_filtering(P):
    """A larger cap shortens the near list (pairs above it are evaluated from
    explicit differences); the minimum found is the same."""
    X = W.moment_curve(2000, 30, 3, np.float32)
    U = W.random_basis(60, 4, 4)
    with P.Sap(X) as s:
        s.set_basis(U)
        near, res = [], []
        for b in (2e-4, 2e-3, 2e-2):
            s.set_pass_bound(b)
            res.append(s.min_secant())
            near.append(s.stats()["n_near"])
        with pytest.raises(P.SapError) as e:
            s.set_pass_bound(0.5)
        assert e.value.code == 1
    assert near[0] > near[1] > near[2]
    assert res[0] == res[1] == res[2]


def test_batch_autotune_keeps_results(P):
    Xs, Ns = W.hyperspectral_batch(3, 21, n_min=200, n_max=900, n_bands=24)
    Us = [W.random_basis(24, 3, 30 + b) for b in range(3)]
    out = []
    with P.SapBatch(Xs) as sb:
        for tune in (False, True):
            for b in range(3):
                sb.set_basis(b, Us[b])
            if tune:
                chosen = sb.autotune(0.01, 4)
                # one set for every dataset, timed on whole batch iterations
                assert chosen["us_per_iteration"] > 0 and sb.tuning() == chosen
                for b in range(3):
                    sb.set_basis(b, Us[b])
            out.append(sb.run(0.01, 12))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


CHILD = r"""
import json, sys
sys.path.insert(0, %(root)r)
import numpy as np
import workloads as W
import paper_1807_03425_gb300 as P
X = W.moment_curve(900, 10, 5, np.float32)
U = W.random_basis(20, 3, 6)
with P.Sap(X) as s:
    s.set_basis(U)
    before = s.tuning()
    if sys.argv[1] == "tune":
        s.autotune(0.01, 4)
    print(json.dumps({"before": before, "after": s.tuning()}))
"""


def test_tuning_cache_file_across_processes(P, tmp_path):
    """With SAP_TUNE_CACHE set, a second process starts a handle of the same
    shape with the first process's choice, without timing anything."""
    path = tmp_path / "tune.txt"
    env = dict(os.environ, SAP_TUNE_CACHE=str(path))
    code = CHILD % {"root": ROOT}
    a = json.loads(subprocess.run([sys.executable, "-c", code, "tune"], env=env, check=True,
                                  capture_output=True, text=True).stdout)
    assert path.exists() and path.read_text().startswith("sap-tune 3 900 20 3 ")
    b = json.loads(subprocess.run([sys.executable, "-c", code, "load"], env=env, check=True,
                                  capture_output=True, text=True).stdout)
    launch = ("pass_bound", "pass_stages", "explicit_blocks_per_sm", "update_blocks", "plain_blocks_per_sm",
              "programmatic_launch", "refine_tier")
    assert {k: b["before"][k] for k in launch} == {k: a["after"][k] for k in launch}
    assert b["before"]["us_per_iteration"] > 0
