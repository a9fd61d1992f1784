"""Shared helpers of the GPU parity tests (compare the CUDA library, through
its C ABI, with the FP64 oracle on the same seeded inputs).

Bar (from the method's tolerance statement): the argmin pair must equal the
oracle's whenever the oracle's relative gap to the runner-up exceeds 1e-6;
otherwise the GPU's pair must be within 1e-6 (relative) of the oracle's
minimum.  The min ratio and the updated basis (column-wise up to sign) must
agree within 1e-5 relative.
"""
import numpy as np

import oracle as O

REL_GAP = 1e-6
REL_TOL = 1e-5


def rel_gap(m):
    return (m["runner_up"] - m["r"]) / max(m["r"], 1e-300)


def check_pair(X64, U, m, i, j, r, eps=0.0):
    """The GPU's (i, j, r) against the oracle's min_secant result m."""
    assert 0 <= i < j < X64.shape[0]
    if rel_gap(m) > REL_GAP:
        assert (i, j) == (m["i"], m["j"]), (i, j, m)
    else:
        ro = O.ratio(X64, U, i, j, eps)
        assert ro >= 0 and ro <= m["r"] * (1 + REL_GAP) + 1e-300, (ro, m)
    assert abs(r - m["r"]) <= REL_TOL * m["r"] + 1e-13, (r, m["r"])


def check_basis(Ug, Uo):
    """Column-wise equality up to sign, within 1e-5 (columns are unit)."""
    dots = np.abs((Ug * Uo).sum(axis=1))
    assert np.all(np.abs(dots - 1.0) <= REL_TOL), dots
    sign = np.sign((Ug * Uo).sum(axis=1))[:, None]
    assert np.abs(Ug - sign * Uo).max() <= REL_TOL
    P_g, P_o = Ug.T @ Ug, Uo.T @ Uo
    assert np.abs(P_g - P_o).max() <= REL_TOL


def lockstep(sap, X64, U, alpha, mode=O.MODE_LITERAL, eps=0.0):
    """Give the GPU the oracle's basis, run one step on both, compare.
    Returns the oracle's new basis (to continue in lock-step)."""
    m = O.min_secant(X64, U, eps)
    sap.set_basis(U)
    i, j, r = sap.step(alpha)
    check_pair(X64, U, m, i, j, r, eps)
    Ug = sap.get_basis()
    # the oracle's update for the pair the GPU chose (same pair unless tied)
    Uo, _ = O.update(X64, U, i, j, alpha, mode)
    check_basis(Ug, Uo)
    return Uo, m
