"""The debug build (compiled with SAP_DEBUG_BOUNDS): every index a kernel
reads from data -- a pair from a candidate or near list, a tile's block
coordinates, a recent argmin pair -- is checked before it addresses memory,
and an index out of range makes the call return SAP_E_BOUNDS instead of
touching memory (no trap): it stands in for a memory checker's
out-of-bounds checks.

The debug library runs every form of the path -- the restructured form with
each second tier (the in-pass tiers included), the plain form in FP32 and
FP64, an uneven batch and a dimension sweep -- without a bounds report, and
its results equal the ordinary library's bit for bit (the checks change no
arithmetic)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, %(root)r)
import numpy as np
import workloads as W
import paper_1807_03425_gb300 as P
out = {}
X = W.moment_curve(1500, 20, 3, np.float32)
U0 = W.random_basis(40, 5, 4)
for tier in (0, 1, 3, 4, 5):
    with P.Sap(X) as s:
        s.set_path("restructured")
        s.set_tuning(refine_tier=tier, programmatic_launch=1)
        s.set_basis(U0)
        h, am = s.run(0.01, 10)
        out["restructured_%%d" %% tier] = [h.tolist(), am.tolist()]
U12 = W.random_basis(40, 12, 5)
with P.Sap(X) as s:
    s.set_path("restructured")
    s.set_basis(U12)
    h, am = s.run(0.01, 6)
    out["restructured_k12"] = [h.tolist(), am.tolist()]
for dt in (np.float32, np.float64):
    Xp = W.moment_curve(400, 10, 6, dt)
    with P.Sap(Xp) as s:
        s.set_path("plain")
        s.set_basis(W.random_basis(20, 3, 7))
        h, am = s.run(0.01, 8)
        out["plain_%%s" %% np.dtype(dt).name] = [h.tolist(), am.tolist()]
Xs, _ = W.hyperspectral_batch(3, 8, n_min=300, n_max=1200, n_bands=24)
with P.SapBatch(Xs) as sb:
    for b in range(3):
        sb.set_basis(b, W.random_basis(24, 3, 10 + b))
    h, am = sb.run(0.01, 6)
    out["batch"] = [np.asarray(h).tolist(), np.asarray(am).tolist()]
with P.Sap(X) as s:
    k, ratios = s.estimate_dim(W.random_basis(40, 6, 11), 6, 0.01, 0.1)
    out["sweep"] = [int(k), ratios.tolist()]
print("RESULT " + json.dumps(out))
"""


def run_child(lib):
    env = dict(os.environ)
    if lib:
        env["SAP_LIBRARY"] = lib
    else:
        env.pop("SAP_LIBRARY", None)
    p = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}], capture_output=True, text=True, env=env,
                       timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    line = [l for l in p.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_debug_bounds_build_runs_clean_and_matches():
    from paper_1807_03425_gb300 import build
    dbg = build.build(debug_bounds=True)
    assert os.path.basename(dbg) == "libsap_dbg.so"
    ref = run_child(None)
    got = run_child(dbg)   # an SAP_E_BOUNDS would raise in the child
    assert set(got) == set(ref)
    for key in ref:
        assert got[key] == ref[key], key
