"""Write stored oracle results for the full-size workloads (calls only ``oracle/``).

Usage: python tests/golden/make_golden.py [radial32] [sine3d] [torsion]
Each run stores u (full, caller sign), psi, Newton counts per proximal step and
metadata in tests/golden/<name>_oracle.npz.

The 3D workload (sine3d, 8^3 hexes, p = 6) solves each Newton system by exact
block elimination of psi (``linear="eliminate_psi"``): the direct sparse LU of
the whole Newton matrix needs more than the host's 62 GB, the eliminated system
about 7 GB; both give the same delta up to rounding (pinned in
tests/test_oracle_newton.py).
"""
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2412_13733_gb300 import workloads as W  # noqa: E402
from oracle.hpg import ObstacleOracle  # noqa: E402
from oracle.gradient import GradientOracle  # noqa: E402


def run(name):
    w = W.workload(name)
    t0 = time.time()
    if w["kind"] == "gradient":
        o = GradientOracle(w["breakpoints"], w["p"], w["f"], w["phi"], beta=w["beta"])
    else:
        linear = "eliminate_psi" if w["dim"] == 3 else "direct"
        o = ObstacleOracle(w["breakpoints"], w["p"], w["f"], w["phi"], w["g"], beta=w["beta"], lower=w["lower"],
                           linear=linear)
    r = o.solve(w["alphas"], tol=w["tol"], log=lambda s: print(name, s, flush=True))
    dt = time.time() - t0
    out = os.path.join(HERE, f"{name}_oracle.npz")
    np.savez_compressed(out, u=r["u"], psi=r["psi"], newton=np.array(r["newton"]), alphas=np.array(w["alphas"]),
                        converged=r["converged"], seconds=dt, host=platform.processor() or platform.machine(),
                        cores=os.cpu_count())
    print(name, "done", dt, "s", r["newton"], r["converged"], out)


if __name__ == "__main__":
    for nm in (sys.argv[1:] or ["radial32"]):
        run(nm)
