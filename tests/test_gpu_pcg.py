"""The iterative (inexact) A_alpha^{-1}: conjugate gradients on the stiffness matrix
preconditioned by block Jacobi over the entities of the hierarchical basis (the
vertex functions' Q1 block solved exactly by fast diagonalisation, the bubble blocks
of every edge, face and cell interior by their dense inverses).  Section 6.5 compares
algebraic-multigrid CG with the Cholesky factorisation of A; here the exact inverse is
the fast diagonalisation, so CG is checked against it, and against the oracle inside
the flexible-GMRES strategies that accept an inexact A_alpha^{-1}."""
import numpy as np
import pytest

from tests.gpu_helpers import case, oracle_for, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2412_13733_gb300 import hpg
    c = hpg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("name", ["radial_3x3_p5", "aniso_upper", "sine3d_3x2x2", "box3d_p3_m4", "single_cell"])
def test_pcg_equals_fast_diagonalisation(ctx, name):
    from paper_2412_13733_gb300 import hpg
    w = case(name)
    o = oracle_for(w)
    P = hpg.from_workload(ctx, w)
    u, psi, psi_prev = random_state(o, 3)
    alpha = 0.37
    P.set_state(u, psi, psi_prev, alpha)
    b = np.random.default_rng(4).standard_normal(P.n_u)
    want = P.apply_stiffness_inv(b, hpg.HPG_FP64)
    got, its = P.stiffness_solve_pcg(b, alpha, rtol=1e-13, atol=0.0)
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want), (name, its)
    assert 1 <= its <= 300
    P.free()


def test_pcg_iterations_grow_slowly_with_degree(ctx):
    """The preconditioned system's condition grows like a power of log p, so the CG
    iteration count for A x = 1 (the experiment of Section 6.5, tolerance 1e-6) stays
    within a small multiple of its p = 2 value up to p = 6 on 4^3 hexes."""
    from paper_2412_13733_gb300 import hpg, workloads as W
    its = {}
    for p in (2, 4, 6):
        w = W.workload(f"box3d_p{p}_m4")
        P = hpg.from_workload(ctx, w)
        P.set_state(np.zeros(P.n_u_full), np.zeros(P.n_psi), np.zeros(P.n_psi), 1.0)
        x, its[p] = P.stiffness_solve_pcg(np.ones(P.n_u), 1.0, rtol=1e-6, atol=1e-6)
        assert np.all(np.isfinite(x))
        P.free()
    assert its[6] <= 4 * its[2] + 10, its


@pytest.mark.parametrize("strategy", [1, 2])
@pytest.mark.parametrize("name", ["radial_3x3_p5", "box3d_p2_m4"])
def test_fgmres_with_inexact_inverse_matches_oracle(ctx, name, strategy):
    """FGMRES with P_D or P_L P_D whose A_alpha^{-1} is CG (relative tolerance 1e-12):
    the same fixed points as the oracle (Newton counts +-1 per step, u_h to 1e-9)."""
    from paper_2412_13733_gb300 import hpg
    from tests.gpu_helpers import mass_norm
    w = case(name)
    o = oracle_for(w)
    r = o.solve(w["alphas"], tol=w["tol"])
    P = hpg.from_workload(ctx, w, hpg.default_params(strategy=strategy, ainv_pcg=1, ainv_rtol=1e-12))
    P.solve()
    st = P.stats()
    assert st["status"] == 0
    for a, b in zip(st["newton_per_step"], r["newton"]):
        assert abs(a - b) <= 1
    assert st["ainv_iters"] >= st["ainv_total"] > 0
    err = mass_norm(o, P.u() - r["u"]) / mass_norm(o, r["u"])
    assert err <= 1e-9, err
    P.free()
