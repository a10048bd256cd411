"""The iterative (inexact) A_alpha^{-1}: conjugate gradients on the stiffness matrix with
three two-level additive Schwarz preconditioners sharing the coarse vertex (Q1) space,
solved exactly by fast diagonalisation: (1) block Jacobi over the entities of the
hierarchical basis, (2) overlapping cell patches, (3) overlapping vertex-star patches
whose tensor boxes are solved by fast diagonalisation.  Section 6.5 compares
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


@pytest.mark.parametrize("precond", [1, 2, 3])
@pytest.mark.parametrize("name", ["radial_3x3_p5", "aniso_upper", "sine3d_3x2x2", "box3d_p3_m4", "single_cell"])
def test_pcg_equals_fast_diagonalisation(ctx, name, precond):
    from paper_2412_13733_gb300 import hpg
    w = case(name)
    o = oracle_for(w)
    P = hpg.from_workload(ctx, w)
    u, psi, psi_prev = random_state(o, 3)
    alpha = 0.37
    P.set_state(u, psi, psi_prev, alpha)
    b = np.random.default_rng(4).standard_normal(P.n_u)
    want = P.apply_stiffness_inv(b, hpg.HPG_FP64)
    got, its = P.stiffness_solve_pcg(b, alpha, rtol=1e-13, atol=0.0, precond=precond)
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want), (name, its)
    assert 1 <= its <= 300
    P.free()


def test_pcg_table_of_section_6_5(ctx):
    """The experiment of Section 6.5's CG table on 4^3 hexes: A x = 1 to absolute and
    relative tolerance 1e-6; x is A^{-1} 1 (checked against the fast diagonalisation).
    The vertex-star patches keep the count nearly independent of p (the paper's AMG-CG:
    20, 76, 165 at p = 2, 4, 6); the cell patches and the non-overlapping entity blocks
    do not."""
    from paper_2412_13733_gb300 import hpg, workloads as W
    its = {}
    for p in (2, 4, 6):
        w = W.workload(f"box3d_p{p}_m4")
        P = hpg.from_workload(ctx, w)
        P.set_state(np.zeros(P.n_u_full), np.zeros(P.n_psi), np.zeros(P.n_psi), 1.0)
        ones = np.ones(P.n_u)
        ref = P.apply_stiffness_inv(ones, hpg.HPG_FP64)
        for pc in (1, 2, 3):
            x, its[(pc, p)] = P.stiffness_solve_pcg(ones, 1.0, rtol=1e-6, atol=1e-6, precond=pc)
            assert np.linalg.norm(x - ref) <= 1e-3 * np.linalg.norm(ref)
        P.free()
    assert its[(1, 2)] <= 40 and its[(1, 6)] < 1000, its
    assert its[(2, 6)] < its[(1, 6)], its
    # the vertex-star patches: at most about twice the p = 2 count at p = 6
    assert its[(3, 6)] <= 2 * its[(3, 2)] + 10 and its[(3, 6)] < its[(2, 6)], its


@pytest.mark.parametrize("precond", [1, 3])
@pytest.mark.parametrize("strategy", [1, 2])
@pytest.mark.parametrize("name", ["radial_3x3_p5", "box3d_p2_m4"])
def test_fgmres_with_inexact_inverse_matches_oracle(ctx, name, strategy, precond):
    """FGMRES with P_D or P_L P_D whose A_alpha^{-1} is CG (relative tolerance 1e-12):
    the same fixed points as the oracle (Newton counts +-1 per step, u_h to 1e-9)."""
    from paper_2412_13733_gb300 import hpg
    from tests.gpu_helpers import mass_norm
    w = case(name)
    o = oracle_for(w)
    r = o.solve(w["alphas"], tol=w["tol"])
    P = hpg.from_workload(ctx, w, hpg.default_params(strategy=strategy, ainv_pcg=precond, ainv_rtol=1e-12))
    P.solve()
    st = P.stats()
    assert st["status"] == 0
    for a, b in zip(st["newton_per_step"], r["newton"]):
        assert abs(a - b) <= 1
    assert st["ainv_iters"] >= st["ainv_total"] > 0
    err = mass_norm(o, P.u() - r["u"]) / mass_norm(o, r["u"])
    assert err <= 1e-9, err
    P.free()
