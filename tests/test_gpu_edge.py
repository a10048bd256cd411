"""Edge and degenerate cases of the CUDA path: argument checks, the trivial fixed
point, a non-finite constraint, and the largest 2D size of the request stream."""
import numpy as np
import pytest

from paper_2412_13733_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2412_13733_gb300 import hpg
    c = hpg.Context(0)
    yield c
    c.close()


def test_invalid_problem_arguments_are_rejected(ctx):
    from paper_2412_13733_gb300 import hpg
    bad = [(1, [0.0], [1.0], [4], 4, hpg.HPG_OBSTACLE_UPPER),       # dimension 1
           (2, [0.0, 0.0], [1.0, 1.0], [0, 4], 4, hpg.HPG_OBSTACLE_UPPER),   # no cells
           (2, [0.0, 0.0], [1.0, -1.0], [4, 4], 4, hpg.HPG_OBSTACLE_UPPER),  # hi < lo
           (2, [0.0, 0.0], [1.0, 1.0], [4, 4], 1, hpg.HPG_OBSTACLE_UPPER),   # p = 1: no bubbles, n = 0
           (2, [0.0, 0.0], [1.0, 1.0], [4, 4], 4, 7)]                        # unknown kind
    for dim, lo, hi, cells, p, kind in bad:
        with pytest.raises(hpg.HpgError) as ei:
            hpg.Problem(ctx, dim, lo, hi, cells, p, kind)
        assert ei.value.code == 1


def _flat(f, phi, m=3, p=4):
    return dict(name="flat", kind="obstacle", lower=False, dim=2, breakpoints=[W.uniform(0, 1, m)] * 2, p=p,
                f=W.const_field(f), f_const=f, phi=W.const_field(phi), g=None,
                alphas=W.alpha_list(2.0 ** -7, 2.0 ** -3), beta=1e-4, tol=1e-10)


@pytest.mark.parametrize("precision", [0, 1])
def test_zero_load_under_unit_obstacle_is_the_trivial_fixed_point(ctx, precision):
    """f = 0, phi = 1, u = 0 on the boundary: (u, psi) = (0, 0) solves every
    subproblem of eq. (pG) (e^{-0} = phi), so no Newton step is taken."""
    from paper_2412_13733_gb300 import hpg
    P = hpg.from_workload(ctx, _flat(0.0, 1.0), hpg.default_params(precision=precision))
    P.solve()
    st = P.stats()
    assert st["status"] == 0
    assert st["newton_total"] == 0
    assert np.abs(P.u()).max() < 1e-14 and np.abs(P.psi()).max() < 1e-14
    P.free()


def test_nonfinite_constraint_is_rejected(ctx):
    from paper_2412_13733_gb300 import hpg
    P = hpg.from_workload(ctx, _flat(10.0, 0.2), hpg.default_params(precision=0))
    vals = np.full(P.n_quad, 0.2)
    vals[len(vals) // 2] = np.nan
    with pytest.raises(hpg.HpgError) as ei:
        P.set_constraint_values(vals)
    assert ei.value.code == 6            # HPG_ERR_NONFINITE
    P.solve()                            # the previous constraint stays in force
    assert P.stats()["status"] == 0
    P.free()


def test_largest_request_size_residual_property(ctx):
    """m = 32, p = 10 (n1 = 319, the largest size of the request stream), mixed
    path with the request stream's Newton cap of 200 per proximal step: the
    oracle's residual of eq. (pG) at the GPU's final state."""
    from paper_2412_13733_gb300 import hpg
    from oracle.hpg import ObstacleOracle
    phi = lambda X: 0.3 + 0.1 * np.sin(2 * np.pi * X[:, 0]) * np.sin(2 * np.pi * X[:, 1])
    w = dict(name="big", kind="obstacle", lower=False, dim=2, breakpoints=[W.uniform(0, 1, 32)] * 2, p=10,
             f=W.const_field(50.0), f_const=50.0, phi=phi, g=None, alphas=W.alpha_list(2.0 ** -7, 2.0 ** -3),
             beta=1e-4, tol=1e-10)
    P = hpg.from_workload(ctx, w, hpg.default_params(precision=1, newton_max=200))
    P.set_alphas(w["alphas"][:-1])
    P.solve()
    psi_prev = P.psi()
    P.set_alphas(w["alphas"])
    P.solve()
    st = P.stats()
    assert st["status"] == 0 and st["final_residual"] <= 1e-10
    o = ObstacleOracle(w["breakpoints"], w["p"], w["f"], w["phi"], None, beta=w["beta"])
    F = o.residual(P.u(), P.psi(), psi_prev, w["alphas"][-1])
    assert np.linalg.norm(F) <= 2e-10, np.linalg.norm(F)
    P.free()


def test_l2_error_is_the_mass_norm(ctx):
    """hpg_l2_error gives ||u_h - u_ref||_L2 through the exact 1D mass matrices: it
    equals the oracle's assembled mass-matrix norm for an arbitrary reference."""
    from paper_2412_13733_gb300 import hpg
    from tests.gpu_helpers import case, oracle_for, mass_norm
    for name in ("radial_3x3_p5", "sine3d_3x2x2"):
        w = case(name)
        o = oracle_for(w)
        P = hpg.from_workload(ctx, w)
        P.solve()
        ref = np.random.default_rng(3).standard_normal(P.n_u_full)
        err, nrm = P.l2_error(ref)
        assert abs(err - mass_norm(o, P.u() - ref)) <= 1e-12 * err
        assert abs(nrm - mass_norm(o, ref)) <= 1e-12 * nrm
        P.free()


def test_fma_peak_probe(ctx):
    """The roofline denominators of the ALU-bound kernels: FP32 and FP64 FMA rates
    measured on this device lie between a quarter of and just above the unit-count
    figures (128 FP32 FMA per SM per clock; FP64 1.25 TFLOP/s nominal)."""
    from paper_2412_13733_gb300 import hpg
    f32, sms = ctx.fma_peak(hpg.HPG_MIXED)
    f64, _ = ctx.fma_peak(hpg.HPG_FP64)
    derived32 = sms * 128 * 2 * 2.07e9 / 1e12
    assert 0.25 * derived32 <= f32 <= 1.1 * derived32, (f32, derived32)
    assert 0.05 <= f64 <= 0.5 * f32, f64
