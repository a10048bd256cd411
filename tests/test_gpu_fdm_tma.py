"""The TMA-fed tcgen05 fast diagonalisation (3xTF32 products, FP32 accumulation).

A_alpha^{-1} is applied as 2d dense passes (Section 4.4's inverse of the stiffness
matrix by the tensor product of the 1D generalised eigenvectors).  Checked here:
* every TMA variant (N tiles of 64, 128, 256, 32) against a sparse direct solve of
  alpha A on small meshes (isotropic, anisotropic 2D and 3D, ragged tiles);
* at the full sizes of the 32 x 32 p = 8 and 8^3 p = 6 workloads, the residual
  ||alpha A y - x|| / ||x|| of the device's y with the oracle's assembled A (the
  FP32 bar of the other variants);
* complete mixed-precision solves with a TMA variant forced against the oracle, and
  lockstep groups with it bitwise equal to solving alone."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from tests.gpu_helpers import case, oracle_for, random_state, rel, mass_norm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2412_13733_gb300 import hpg
    c = hpg.Context(0)
    yield c
    c.close()


def _tma_variants():
    """The TMA-fed variants are the last four (N tiles of 64, 128, 256 and 32 columns)."""
    from paper_2412_13733_gb300 import hpg
    n = hpg.fdm_tile_count(hpg.HPG_MIXED)
    return list(range(n - 4, n))


def _rect():
    from paper_2412_13733_gb300 import workloads as W
    return dict(name="rect_30x20_p5", kind="obstacle", lower=False, dim=2,
                breakpoints=[W.uniform(0.0, 1.5, 30), W.uniform(0.0, 1.0, 20)], p=5,
                f=W.const_field(10.0), f_const=10.0, phi=lambda X: 0.3 + 0.0 * X[:, 0], g=None,
                alphas=W.alpha_list(2.0 ** -7, 2.0 ** -3), beta=1e-4, tol=1e-10)


@pytest.mark.parametrize("name", ["rect_30x20_p5", "radial_3x3_p5", "p2", "sine3d_3x2x2", "torsion_3x3_p3"])
def test_tma_variants_against_direct_solve(ctx, name):
    from paper_2412_13733_gb300 import hpg
    w = _rect() if name == "rect_30x20_p5" else case(name)
    o = oracle_for(w)
    alpha = 0.05
    x = np.random.default_rng(6).normal(size=len(o.interior))
    ref = spla.spsolve((alpha * o.A00).tocsc(), x)
    u, psi, psi_prev = random_state(o, 0)
    for v in _tma_variants():
        P = hpg.from_workload(ctx, w, hpg.default_params(fdm_tile_f32=v))
        P.set_state(u, psi, psi_prev, alpha)
        assert P.stats()["fdm_tile_f32"] == v
        err = rel(P.apply_stiffness_inv(x, hpg.HPG_MIXED), ref)
        assert err < 1e-4, (name, v, err)
        # entry by entry: no tile, slice or row of the padded layouts is lost
        y = P.apply_stiffness_inv(x, hpg.HPG_MIXED)
        assert np.max(np.abs(y - ref)) <= 1e-4 * np.max(np.abs(ref)), (name, v)
        P.free()


@pytest.mark.parametrize("wname", ["radial32", "sine3d"])
def test_tma_full_size_residual(ctx, wname):
    from paper_2412_13733_gb300 import hpg, workloads as W
    w = W.workload(wname)
    o = oracle_for(w)
    alpha = w["alphas"][-1]
    x = np.random.default_rng(11).normal(size=len(o.interior))
    u0 = np.zeros(o.sp.Nu)
    for v in _tma_variants():
        P = hpg.from_workload(ctx, w, hpg.default_params(precision=hpg.HPG_MIXED, fdm_tile_f32=v))
        P.set_state(u0, np.zeros(o.sp.Npsi), np.zeros(o.sp.Npsi), alpha)
        y = P.apply_stiffness_inv(x, hpg.HPG_MIXED)
        r = alpha * (o.A00 @ y) - x
        assert np.linalg.norm(r) <= 2e-4 * np.linalg.norm(x), (wname, v)
        P.free()


@pytest.mark.parametrize("name", ["radial_3x3_p5", "sine3d_3x2x2"])
def test_tma_full_solve_against_oracle(ctx, name):
    from paper_2412_13733_gb300 import hpg
    w = case(name)
    o = oracle_for(w)
    r = o.solve(w["alphas"], tol=w["tol"])
    v = _tma_variants()[1]
    P = hpg.from_workload(ctx, w, hpg.default_params(precision=hpg.HPG_MIXED, fdm_tile_f32=v))
    P.solve()
    st = P.stats()
    assert st["status"] == 0 and st["fdm_tile_f32"] == v
    assert all(abs(a - b) <= 1 for a, b in zip(st["newton_per_step"], r["newton"]))
    e = mass_norm(o, P.u() - r["u"]) / mass_norm(o, r["u"])
    assert e <= 1e-8, e
    P.free()


def test_tma_lockstep_group_equals_alone(ctx):
    from paper_2412_13733_gb300 import hpg, workloads as W
    base = case("radial_3x3_p5")
    ws = []
    for i in range(4):
        w = dict(base)
        c = 0.02 * i
        w["phi"] = (lambda f0, c: (lambda X: f0(X) + c))(base["phi"], c)
        ws.append(w)
    for v in (_tma_variants()[0], _tma_variants()[3]):
        prm = lambda: hpg.default_params(precision=hpg.HPG_MIXED, fdm_tile_f32=v)
        alone = []
        for w in ws:
            P = hpg.from_workload(ctx, w, prm())
            P.solve()
            st = P.stats()
            alone.append((P.u(), st["newton_per_step"], st["krylov_total"]))
            P.free()
        probs = [hpg.from_workload(ctx, w, prm()) for w in ws]
        for rep in range(2):
            ctx.solve_batch(probs)
            for P, (u, newton, kry) in zip(probs, alone):
                st = P.stats()
                assert st["status"] == 0 and st["fdm_tile_f32"] == v
                assert st["newton_per_step"] == newton and st["krylov_total"] == kry
                assert np.array_equal(P.u(), u)
        for P in probs:
            P.free()


def test_tune_batch_group_equals_alone(ctx):
    """hpg_params.fdm_tune_batch tunes the variant for the time per problem in a lockstep
    group; the group then runs that variant, so alone and batched results stay equal bit
    for bit whichever variant wins."""
    from paper_2412_13733_gb300 import hpg
    base = case("radial_3x3_p5")
    ws = []
    for i in range(4):
        w = dict(base)
        w["phi"] = (lambda f0, c: (lambda X: f0(X) + c))(base["phi"], 0.02 * i)
        ws.append(w)
    prm = lambda: hpg.default_params(precision=hpg.HPG_MIXED, fdm_tune_batch=4)
    alone = []
    for w in ws:
        P = hpg.from_workload(ctx, w, prm())
        P.solve()
        alone.append((P.u(), P.stats()["fdm_tile_f32"]))
        P.free()
    probs = [hpg.from_workload(ctx, w, prm()) for w in ws]
    ctx.solve_batch(probs)
    for P, (u, v) in zip(probs, alone):
        st = P.stats()
        assert st["status"] == 0 and st["fdm_tile_f32"] == v, (st["fdm_tile_f32"], v)
        assert np.array_equal(P.u(), u), (v, float(np.max(np.abs(P.u() - u))))
    for P in probs:
        P.free()
