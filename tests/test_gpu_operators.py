"""GPU parity of every operator on the hpG Newton path against the CPU oracle.

Each operator is called through the C ABI on a random state and compared
entry by entry with the oracle's sparse/dense FP64 reference:
  residual of eq. (pG)/(pG:gradient), the Newton matrix G of eq.
  (pG-matrix), A_alpha^{-1}, the S-hat cell blocks of eq.
  (schur-preconditioner), S-hat^{-1}, S of eq. (schur4), and a full Newton
  direction by eq. (schur2) + GMRES.
Tolerances: FP64 kernels 1e-11 relative (round-off of sums of a few hundred
terms); FP32 kernels 1e-4 relative (single precision on operators with
condition numbers up to ~1e3 on these sizes).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from tests.gpu_helpers import case, oracle_for, random_state, rel_entry as rel

pytestmark = pytest.mark.gpu

OBSTACLE_CASES = ["radial_3x3_p5", "aniso_upper", "p2", "single_cell", "sine3d_small", "sine3d_3x2x2"]
ALL_CASES = OBSTACLE_CASES + ["torsion_small", "torsion_3x3_p3", "grad3d_2x3x2_p3"]


@pytest.fixture(scope="module")
def ctx():
    from paper_2412_13733_gb300 import hpg
    c = hpg.Context(0)
    yield c
    c.close()


def _setup(ctx, name, seed=0, alpha=0.05):
    from paper_2412_13733_gb300 import hpg
    w = case(name)
    o = oracle_for(w)
    P = hpg.from_workload(ctx, w)
    u, psi, psi_prev = random_state(o, seed)
    P.set_state(u, psi, psi_prev, alpha)
    return w, o, P, (u, psi, psi_prev, alpha)


@pytest.mark.parametrize("name", ALL_CASES)
def test_sizes_match(ctx, name):
    w, o, P, _ = _setup(ctx, name)
    assert P.n_u_full == o.sp.Nu
    assert P.n_u == len(o.interior)
    assert P.n_psi == o.sp.Npsi


@pytest.mark.parametrize("name", ALL_CASES)
def test_residual(ctx, name):
    w, o, P, (u, psi, psi_prev, alpha) = _setup(ctx, name)
    F, nrm = P.residual()
    Fo = o.residual(u, psi, psi_prev, alpha)
    assert rel(F, Fo) < 1e-11
    assert abs(nrm - np.linalg.norm(Fo)) < 1e-11 * np.linalg.norm(Fo)


@pytest.mark.parametrize("name", ALL_CASES)
def test_newton_apply(ctx, name):
    w, o, P, (u, psi, psi_prev, alpha) = _setup(ctx, name)
    x = np.random.default_rng(3).normal(size=P.n_u + P.n_psi)
    y = P.apply_newton(x)
    G = o.jacobian(psi, alpha)
    assert rel(y, G @ x) < 1e-11


@pytest.mark.parametrize("name", ALL_CASES)
def test_stiffness_inverse(ctx, name):
    from paper_2412_13733_gb300 import hpg
    w, o, P, (u, psi, psi_prev, alpha) = _setup(ctx, name)
    x = np.random.default_rng(4).normal(size=P.n_u)
    ref = spla.spsolve((alpha * o.A00).tocsc(), x)
    assert rel(P.apply_stiffness_inv(x, hpg.HPG_FP64), ref) < 1e-10
    assert rel(P.apply_stiffness_inv(x, hpg.HPG_MIXED), ref) < 1e-4


@pytest.mark.parametrize("name", ALL_CASES)
def test_shat_blocks_and_inverse(ctx, name):
    from paper_2412_13733_gb300 import hpg
    from oracle.schur import SchurOracle
    w, o, P, (u, psi, psi_prev, alpha) = _setup(ctx, name)
    blocks = P.factor_precond(hpg.HPG_FP64, dump=True)
    if w["kind"] == "gradient":
        ref = o.D_blocks(psi) + o.beta * np.array(
            [o.Kpsi[c * blocks.shape[1]:(c + 1) * blocks.shape[1], c * blocks.shape[1]:(c + 1) * blocks.shape[1]]
             .toarray() for c in range(o.sp.Nc)])
    else:
        ref = -SchurOracle(o).shat_blocks(psi, alpha)
    assert rel(blocks.ravel(), ref.ravel()) < 1e-12
    x = np.random.default_rng(5).normal(size=P.n_psi)
    nb = blocks.shape[1]
    want = -np.linalg.solve(ref, x.reshape(-1, nb)[..., None])[..., 0].ravel()
    assert rel(P.apply_precond_inv(x, hpg.HPG_FP64), want) < 1e-10
    P.factor_precond(hpg.HPG_MIXED)
    assert rel(P.apply_precond_inv(x, hpg.HPG_MIXED), want) < 1e-4


@pytest.mark.parametrize("name", ALL_CASES)
def test_schur_apply(ctx, name):
    from paper_2412_13733_gb300 import hpg
    w, o, P, (u, psi, psi_prev, alpha) = _setup(ctx, name)
    x = np.random.default_rng(6).normal(size=P.n_psi)
    # S = -(D + E + B^T A_alpha^{-1} B), from the oracle's Newton matrix blocks
    G = o.jacobian(psi, alpha).tocsr()
    ni = len(o.interior)
    A = G[:ni, :ni]
    B = G[:ni, ni:]
    C = G[ni:, ni:]                  # -D - E
    want = C @ x - B.T @ spla.spsolve(A.tocsc(), B @ x)
    assert rel(P.apply_schur(x, hpg.HPG_FP64), want) < 1e-10
    assert rel(P.apply_schur(x, hpg.HPG_MIXED), want) < 1e-4


@pytest.mark.parametrize("name", ALL_CASES)
def test_newton_direction(ctx, name):
    from paper_2412_13733_gb300 import hpg
    w, o, P, (u, psi, psi_prev, alpha) = _setup(ctx, name)
    F = o.residual(u, psi, psi_prev, alpha)
    want = spla.spsolve(o.jacobian(psi, alpha), F)
    d64, its = P.newton_direction(hpg.HPG_FP64, rtol=1e-12)
    assert its >= 1
    assert rel(d64, want) < 1e-8
    dmx, its2 = P.newton_direction(hpg.HPG_MIXED, rtol=1e-10)
    assert rel(dmx, want) < 1e-7


def _fdm_case(name):
    from paper_2412_13733_gb300 import workloads as W
    if name == "rect_30x20_p5":
        # n1 = (149, 99): two 128-row tensor-core tiles with a ragged second one, ragged N tiles
        return dict(name=name, kind="obstacle", lower=False, dim=2,
                    breakpoints=[W.uniform(0.0, 1.5, 30), W.uniform(0.0, 1.0, 20)], p=5,
                    f=W.const_field(10.0), f_const=10.0, phi=lambda X: 0.3 + 0.0 * X[:, 0], g=None,
                    alphas=W.alpha_list(2.0 ** -7, 2.0 ** -3), beta=1e-4, tol=1e-10)
    return case(name)


@pytest.mark.parametrize("name", ["rect_30x20_p5", "radial_3x3_p5", "p2", "sine3d_3x2x2", "torsion_3x3_p3"])
def test_stiffness_inverse_every_pass_variant(ctx, name):
    """Every fast-diagonalisation pass variant (SIMT tiles and the tcgen05 3xTF32
    kernels) against a sparse direct solve of alpha A."""
    from paper_2412_13733_gb300 import hpg
    w = _fdm_case(name)
    o = oracle_for(w)
    alpha = 0.05
    x = np.random.default_rng(6).normal(size=len(o.interior))
    ref = spla.spsolve((alpha * o.A00).tocsc(), x)
    u, psi, psi_prev = random_state(o, 0)
    for prec, count, tol in ((hpg.HPG_MIXED, hpg.fdm_tile_count(hpg.HPG_MIXED), 1e-4),
                             (hpg.HPG_FP64, hpg.fdm_tile_count(hpg.HPG_FP64), 1e-10)):
        assert count >= 1
        for v in range(count):
            kw = {"fdm_tile_f32": v} if prec == hpg.HPG_MIXED else {"fdm_tile_f64": v}
            P = hpg.from_workload(ctx, w, hpg.default_params(**kw))
            P.set_state(u, psi, psi_prev, alpha)
            st = P.stats()
            assert (st["fdm_tile_f32"] if prec == hpg.HPG_MIXED else st["fdm_tile_f64"]) == v
            err = rel(P.apply_stiffness_inv(x, prec), ref)
            assert err < tol, (prec, v, err)
            P.free()


@pytest.mark.parametrize("strategy", [1, 2, 3])
@pytest.mark.parametrize("name", ["radial_3x3_p5", "sine3d_3x2x2", "torsion_3x3_p3"])
def test_newton_direction_fgmres(ctx, name, strategy):
    """The Newton direction by flexible GMRES on G with each block preconditioner
    equals the sparse direct solve of eq. (pG-matrix)."""
    from paper_2412_13733_gb300 import hpg
    w, o, P, (u, psi, psi_prev, alpha) = _setup(ctx, name)
    P.set_params(hpg.default_params(precision=0, strategy=strategy, beta=w["beta"]))
    F = o.residual(u, psi, psi_prev, alpha)
    want = spla.spsolve(o.jacobian(psi, alpha), F)
    d, its = P.newton_direction(hpg.HPG_FP64, rtol=1e-12)
    assert rel(d, want) < 1e-8
