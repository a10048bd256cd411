"""The oracle on the paper's own 2D example (Section 6.2): Newton totals are
independent of p and close to the printed 24.

The paper does not state its Newton tolerance; with an absolute l2 tolerance
of 1e-6 the oracle needs 27 (p=4) and 28 (p=6) Newton steps on the 10x10
mesh.  The pin is the printed value within a window set by that unknown
tolerance, and the p-independence the paper reports.
"""
import os

import numpy as np
import pytest
from scipy.special import j0

from paper_2412_13733_gb300 import workloads as W
from oracle.hpg import ObstacleOracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_newton_counts.txt")


def printed(name):
    for line in open(GOLDEN):
        if line.startswith(name):
            return int(line.split("|")[2].split()[0])
    raise KeyError(name)


@pytest.mark.slow
def test_oscillatory_obstacle_newton_totals():
    phi = lambda X: (1 + j0(20 * X[:, 0])) * (1 + j0(20 * X[:, 1]))
    alphas = W.alpha_list(2.0 ** -7, 2.0 ** -3)
    totals = []
    for p in (4, 6):
        o = ObstacleOracle([W.uniform(0, 1, 10)] * 2, p, W.const_field(100.0), phi, None, beta=0.0)
        r = o.solve(alphas, tol=1e-6)
        assert r["converged"]
        totals.append(sum(r["newton"]))
    ref = printed("oscillatory_obstacle_2d")
    assert abs(totals[0] - totals[1]) <= 1, totals
    assert all(ref <= t <= ref + 6 for t in totals), (totals, ref)


def test_box3d_newton_totals_independent_of_h_and_p():
    """Section 6.5 (3D solver study): the paper prints 16 Newton steps for every
    (p, N) it runs.  The literal alpha rule gives eight subproblems where the
    paper counts six (each extra subproblem at alpha = 2 costs two steps at the
    tolerance used here), so the printed value is pinned within [16, 22], and
    the h- and p-independence within 2."""
    ref = printed("obstacle_3d")
    totals = {}
    for p, m in ((2, 4), (2, 8), (3, 4)):
        w = W.workload(f"box3d_p{p}_m{m}")
        o = ObstacleOracle(w["breakpoints"], w["p"], w["f"], w["phi"], None, beta=w["beta"])
        r = o.solve(w["alphas"], tol=w["tol"])
        assert r["converged"]
        assert len(r["newton"]) == 8
        totals[(p, m)] = sum(r["newton"])
    assert max(totals.values()) - min(totals.values()) <= 2, totals
    assert all(ref <= t <= ref + 6 for t in totals.values()), (totals, ref)
