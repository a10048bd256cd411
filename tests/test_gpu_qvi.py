"""Thermoforming QVI (Section 6.4) through the C ABI against the oracle's fixed point.

The device runs every step: the obstacle Phi_0 + xi T_i written at the latent Gauss
points, the hpG obstacle solve, the temperature Newton with (A + gamma M)^{-1}-
preconditioned GMRES, and the H^1 stopping test.  The oracle takes the same steps with
direct sparse solves.  Both stop on the same test, so the iteration counts must agree,
and u and T agree to the solvers' tolerances.  At degrees the oracle's fixed point is
too slow for, the checks are properties: the fixed-point count of Table 3 and the T
equation evaluated by the oracle at the device's (u, T)."""
import numpy as np
import pytest

from paper_2412_13733_gb300 import workloads as W
from oracle.qvi import QVIOracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2412_13733_gb300 import hpg
    c = hpg.Context(0)
    yield c
    c.close()


def _setup(ctx, w):
    from paper_2412_13733_gb300 import hpg
    bps = w["breakpoints"]
    d = len(bps)
    P = hpg.Problem(ctx, d, [b[0] for b in bps], [b[-1] for b in bps], [len(b) - 1 for b in bps], w["p"],
                    hpg.HPG_OBSTACLE_UPPER)
    P.set_rhs(w["f_const"])
    P.set_dirichlet(None)
    # Section 6.4's rule: alpha_1 = 2^-6, alpha_{k+1} = 4 alpha_k, stop once alpha_k = 1 (the
    # oracle takes the same four values as a list)
    P.set_alpha_growth(2.0 ** -6, 4.0, 1.0)
    prm = hpg.default_params()
    prm.beta = w["beta"]
    prm.newton_tol = 1e-10
    P.set_params(prm)
    Xl = P.quad_points()
    Xq = P.qvi_points()
    return P, (w["Phi0"](Xl), w["xi"](Xl), w["Phi0"](Xq), w["xi"](Xq))


def _case(name):
    if name == "thermoforming_p6":
        return W.workload(name)
    if name == "thermo_3x5_p4":
        w = W.workload("thermoforming_p4")
        w.update(name=name, breakpoints=[W.uniform(0, 1, 3), W.uniform(0, 1, 5)])
        return w
    if name == "thermo3d_2x2x2_p3":
        w = W.workload("thermoforming_p3")
        w.update(name=name, dim=3, breakpoints=[W.uniform(0, 1, 2)] * 3, f_const=100.0, f=W.const_field(100.0))
        return w
    raise KeyError(name)


@pytest.mark.parametrize("name", ["thermoforming_p6", "thermo_3x5_p4", "thermo3d_2x2x2_p3"])
def test_qvi_matches_oracle(ctx, name):
    w = _case(name)
    P, data = _setup(ctx, w)
    rc, st = P.qvi_solve(*data, gamma=w["gamma"], g0=w["g0"], tol=w["qvi_tol"])
    q = QVIOracle(w["breakpoints"], w["p"], w["f"], w["Phi0"], w["xi"], gamma=w["gamma"], g0=w["g0"],
                  beta=w["beta"])
    r = q.solve(w["alphas"], tol=w["qvi_tol"], newton_tol=1e-10)
    assert rc == 0 and st["converged"] == 1
    assert P.stats()["alpha_steps"] == len(w["alphas"])     # the growth rule gives the oracle's list
    assert st["iterations"] == r["iterations"], (st, [h["du_h1"] for h in r["history"]])
    # per-iteration H^1 differences (the fixed point's contraction), then u and T
    want = [h["du_h1"] for h in r["history"][1:]]
    got = st["du_h1"][1:]
    np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-7)
    u, T = P.u(), P.qvi_T()
    assert np.max(np.abs(u - r["u"])) <= 1e-6 * max(1.0, np.max(np.abs(r["u"]))), name
    assert np.max(np.abs(T - r["T"])) <= 1e-7 * max(1.0, np.max(np.abs(r["T"]))), name
    # the device T solves the oracle's T equation for the device u
    assert np.linalg.norm(q.T_residual(T, u)) <= 1e-9
    # T Newton counts per iteration within one of the oracle's
    tn = [h["t_newton"] for h in r["history"]]
    assert all(abs(a - b) <= 1 for a, b in zip(st["t_newton_per_fp"], tn)), (st["t_newton_per_fp"], tn)
    P.free()


@pytest.mark.parametrize("p", [12, 22])
def test_qvi_fixed_point_count_at_high_degree(ctx, p):
    """Table 3: four fixed-point iterations at every degree on the 4 x 4 mesh, one to three
    temperature Newton steps each; the device (u, T) satisfies the oracle's T equation."""
    w = W.workload(f"thermoforming_p{p}")
    P, data = _setup(ctx, w)
    rc, st = P.qvi_solve(*data, gamma=w["gamma"], g0=w["g0"], tol=w["qvi_tol"])
    assert rc == 0 and st["converged"] == 1
    assert st["iterations"] == 4, st
    assert all(1 <= t <= 3 for t in st["t_newton_per_fp"]), st
    assert st["t_krylov_total"] <= 8 * st["t_newton_total"], st
    q = QVIOracle(w["breakpoints"], w["p"], w["f"], w["Phi0"], w["xi"], gamma=w["gamma"], g0=w["g0"],
                  beta=w["beta"])
    u, T = P.u(), P.qvi_T()
    assert np.linalg.norm(q.T_residual(T, u)) <= 1e-9
    P.free()


def test_qvi_argument_errors(ctx):
    from paper_2412_13733_gb300 import hpg
    w = W.workload("thermoforming_p3")
    P, data = _setup(ctx, w)
    for bad in ((0.0, 4.0, 1.0), (1.0, 0.5, 1.0), (1.0, 2.0, -1.0)):
        with pytest.raises(hpg.HpgError):
            P.set_alpha_growth(*bad)
    with pytest.raises(hpg.HpgError):
        P.set_alpha_growth(1.0, 2.0, 4.0, max_steps=hpg.HPG_MAX_ALPHA + 1)
    P.set_alpha_growth(2.0 ** -6, 4.0, 1.0)
    with pytest.raises(hpg.HpgError):
        P.qvi_T()                                     # no QVI solve yet
    rc, _ = P.qvi_solve(data[0][:-1], data[1], data[2], data[3], check=False)
    assert rc == hpg.STATUS.index("HPG_ERR_ARG")      # short latent array
    rc, _ = P.qvi_solve(*data, gamma=-1.0, check=False)
    assert rc == hpg.STATUS.index("HPG_ERR_ARG")
    rc, _ = P.qvi_solve(*data, max_fp=hpg.HPG_QVI_MAX_FP + 1, check=False)
    assert rc == hpg.STATUS.index("HPG_ERR_ARG")
    # a fixed point cut off after one iteration reports the cap, keeping T
    rc, st = P.qvi_solve(*data, max_fp=1, check=False)
    assert rc == hpg.STATUS.index("HPG_ERR_NEWTON_CAP") and st["iterations"] == 1
    assert np.all(np.isfinite(P.qvi_T()))
    # the problem solves again afterwards (its constraint is the last mould)
    rc, st = P.qvi_solve(*data, check=False)
    assert rc == 0 and st["converged"] == 1
    P.free()
    L = hpg.Problem(ctx, 2, [0, 0], [1, 1], [2, 2], 3, hpg.HPG_OBSTACLE_LOWER)
    L.set_rhs(1.0)
    L.set_alphas([0.5, 1.0])
    Xl, Xq = L.quad_points(), L.qvi_points()
    rc, _ = L.qvi_solve(np.zeros(len(Xl)), np.zeros(len(Xl)), np.zeros(len(Xq)), np.zeros(len(Xq)), check=False)
    assert rc == hpg.STATUS.index("HPG_ERR_ARG")
    L.free()


def test_qvi_mixed_precision_matches_oracle(ctx):
    """The QVI with HPG_MIXED obstacle solves: the same fixed point as the oracle's (count,
    u, T) at the tolerances of the FP64 comparison."""
    from paper_2412_13733_gb300 import hpg
    w = W.workload("thermoforming_p6")
    P, data = _setup(ctx, w)
    prm = hpg.default_params()
    prm.beta = w["beta"]
    prm.newton_tol = 1e-10
    prm.precision = hpg.HPG_MIXED
    P.set_params(prm)
    rc, st = P.qvi_solve(*data, gamma=w["gamma"], g0=w["g0"], tol=w["qvi_tol"])
    q = QVIOracle(w["breakpoints"], w["p"], w["f"], w["Phi0"], w["xi"], gamma=w["gamma"], g0=w["g0"],
                  beta=w["beta"])
    r = q.solve(w["alphas"], tol=w["qvi_tol"], newton_tol=1e-10)
    assert rc == 0 and st["converged"] == 1 and st["iterations"] == r["iterations"], st
    u, T = P.u(), P.qvi_T()
    assert np.max(np.abs(u - r["u"])) <= 1e-6 * max(1.0, np.max(np.abs(r["u"])))
    assert np.max(np.abs(T - r["T"])) <= 1e-7 * max(1.0, np.max(np.abs(r["T"])))
    P.free()


def _mould_problem(ctx, precision, p=22):
    """Obstacle solve with the thermoforming mould Phi_0 (the QVI's first iterate) at degree p
    on the 4 x 4 mesh; beta = 1e-6 makes the S-hat cell blocks badly conditioned."""
    from paper_2412_13733_gb300 import hpg
    w = W.workload(f"thermoforming_p{p}")
    P = hpg.Problem(ctx, 2, [0.0, 0.0], [1.0, 1.0], [4, 4], p, hpg.HPG_OBSTACLE_UPPER)
    P.set_rhs(w["f_const"])
    P.set_alphas(w["alphas"])
    P.set_params(hpg.default_params(beta=w["beta"], precision=precision))
    P.set_constraint_values(w["Phi0"](P.quad_points()))
    return P


def test_mixed_fallback_to_fp64_steps(ctx):
    """At p = 22 a mixed proximal step fails (the FP32 elimination of an S-hat block meets a
    non-positive pivot, the line search ends on a non-finite point): the step is solved again
    from its start in FP64, as is the rest of the solve, and the result is the FP64 one; in
    a lockstep group the member is solved again on its own, bit for bit as alone."""
    from paper_2412_13733_gb300 import hpg
    ref = _mould_problem(ctx, hpg.HPG_FP64)
    ref.solve()
    u_ref = ref.u().copy()
    sr = ref.stats()
    assert sr["fp64_from_step"] == 0 and sr["fp64_newton_steps"] == 0
    A = _mould_problem(ctx, hpg.HPG_MIXED)
    assert A.solve(check=False) == 0
    sa = A.stats()
    assert sa["fp64_from_step"] >= 1 and sa["fp64_newton_steps"] >= 1, sa
    assert sa["newton_total"] >= sum(sa["newton_per_step"])           # discarded mixed steps count
    # both end on FP64 Newton steps at the same residual tolerance; at beta = 1e-6 the psi
    # block of eq. (pG-matrix) is nearly singular on the contact set, so two such solves from
    # slightly different starting points agree to the max-norm bar of the QVI comparisons
    assert sa["final_residual"] <= 1e-10 and sr["final_residual"] <= 1e-10
    assert np.max(np.abs(A.u() - u_ref)) <= 1e-6 * max(1.0, np.max(np.abs(u_ref)))
    assert all(abs(a - b) <= 1 for a, b in zip(sa["newton_per_step"], sr["newton_per_step"]))
    B1, B2 = _mould_problem(ctx, hpg.HPG_MIXED), _mould_problem(ctx, hpg.HPG_MIXED)
    assert ctx.solve_batch([B1, B2], check=False) == 0
    for B in (B1, B2):
        assert np.array_equal(B.u(), A.u())
        sb = B.stats()
        assert sb["newton_per_step"] == sa["newton_per_step"]
        assert sb["fp64_from_step"] == sa["fp64_from_step"]
    for P in (ref, A, B1, B2):
        P.free()
