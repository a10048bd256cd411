"""Pins of the thermoforming QVI oracle (Section 6.4).

* Constant g: when Phi_0 + xi T - u <= 0 everywhere, g is the constant g_0 and the T
  equation (grad T, grad q) + gamma (T, q) = g_0 (1, q) has the closed-form solution
  T = g_0 / gamma, the constant function (hats g_0 / gamma, bubbles 0).
* Taylor test: where 0 < s < 1, g is affine, so the T residual is affine in T and
  F(T + e h) - F(T) - e J h must vanish to round-off for the assembled Jacobian J (a
  wrong sign, factor or index leaves an O(e) remainder).
* The fixed point on a small mesh converges (successive H^1 differences fall below the
  tolerance) and its T satisfies the T equation to the Newton tolerance.
"""
import numpy as np

from paper_2412_13733_gb300 import workloads as W
from oracle.hpg import alpha_schedule
from oracle.qvi import QVIOracle


def _qvi(Phi0, xi, m=2, p=3, f=100.0):
    return QVIOracle([W.uniform(0, 1, m)] * 2, p, W.const_field(f), Phi0, xi, gamma=1.0, g0=0.2)


def test_constant_g_gives_constant_temperature():
    q = _qvi(lambda X: np.full(X.shape[0], -10.0), lambda X: 0.1 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]))
    u = np.zeros(q.sp.Nu)
    T, it, res = q.T_newton(u, np.zeros(q.sp.Nu))
    want = np.zeros(q.sp.Nu)
    nh = [ms.m + 1 for ms in q.sp.meshes]            # hats first in each 1D numbering
    for j in range(nh[1]):
        for i in range(nh[0]):
            want[i + q.sp.N1[0] * j] = 0.2
    assert res < 1e-11 and it <= 2
    assert np.max(np.abs(T - want)) < 1e-12


def test_temperature_jacobian_taylor():
    q = _qvi(lambda X: 0.5 + 0.0 * X[:, 0], lambda X: 0.1 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]), p=4)
    rng = np.random.default_rng(3)
    u = 0.01 * rng.normal(size=q.sp.Nu)
    T = 0.05 * rng.normal(size=q.sp.Nu)
    h = rng.normal(size=q.sp.Nu)
    F0 = q.T_residual(T, u)
    J = q.T_jacobian(T, u)
    for e in (1e-1, 1e-2, 1e-3):
        r = np.linalg.norm(q.T_residual(T + e * h, u) - F0 - e * (J @ h))
        assert r <= 1e-10 * e * np.linalg.norm(J @ h), (e, r)


def test_fixed_point_converges_on_a_small_mesh():
    Phi0 = lambda X: 1.1 - 2 * np.maximum(np.abs(X[:, 0] - 0.5), np.abs(X[:, 1] - 0.5)) \
        + np.cos(8 * np.pi * X[:, 0]) * np.cos(8 * np.pi * X[:, 1]) / 10
    xi = lambda X: np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])
    q = _qvi(Phi0, xi, m=2, p=3)
    r = q.solve(alpha_schedule(2.0 ** -6, 1.0, growth_log2=2.0), tol=3e-3)
    h = r["history"]
    assert h[-1]["du_h1"] is not None and h[-1]["du_h1"] <= 3e-3
    assert np.linalg.norm(q.T_residual(r["T"], r["u"])) < 1e-10
    d = [x["du_h1"] for x in h[1:]]
    assert all(b < a for a, b in zip(d, d[1:])), d


def test_fixed_point_count_of_table_3():
    """Section 6.4's setup on the 4 x 4 mesh at p = 6: the fixed point stops after 4
    iterations (Table 3), each T solve taking one or two Newton steps (Table 3's average
    1.5 at p = 6)."""
    w = W.workload("thermoforming_p6")
    q = QVIOracle(w["breakpoints"], w["p"], w["f"], w["Phi0"], w["xi"], gamma=w["gamma"], g0=w["g0"],
                  beta=w["beta"])
    r = q.solve(w["alphas"], tol=w["qvi_tol"])
    assert r["iterations"] == 4
    assert all(1 <= h["t_newton"] <= 3 for h in r["history"])
    assert r["history"][-1]["du_h1"] <= 3e-3 < r["history"][-2]["du_h1"]
