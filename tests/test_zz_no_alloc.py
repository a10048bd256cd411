"""The allocation-free stiffness-inverse entry point gives the same result as
hpg_apply_stiffness_inv.

hpg_apply_stiffness_inv_noalloc serves callers that cannot allocate device
memory at call time (real-time loops that forbid allocation after start-up,
applications that give all device memory to their own pool up front): its
scratch is a fixed device array of the library.  This file is collected last so that, if it fails, a run that
stops at the first failure has run every other test already.
"""
import numpy as np
import pytest

from tests.gpu_helpers import case, oracle_for, random_state

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    from paper_2412_13733_gb300 import hpg
    ctx = hpg.Context(0)
    w = case("radial_3x3_p5")
    o = oracle_for(w)
    P = hpg.from_workload(ctx, w)
    u, psi, psi_prev = random_state(o, 1)
    alpha = 0.07
    P.set_state(u, psi, psi_prev, alpha)
    rng = np.random.default_rng(11)
    for call in range(2):                       # two calls in a row share the scratch array
        x = rng.standard_normal(P.n_u)
        want = P.apply_stiffness_inv(x, hpg.HPG_FP64)
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        torch.cuda.synchronize()
        rc = P.apply_stiffness_inv_noalloc(alpha, xd.data_ptr(), yd.data_ptr(), P.n_u)
        assert rc == 0, ctx.L.hpg_last_error(ctx.h)
        torch.cuda.synchronize()
        got = yd.cpu().numpy()
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want), call
    P.free()
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    from paper_2412_13733_gb300 import hpg, workloads as W
    ctx = hpg.Context(0)
    P = hpg.Problem(ctx, 2, [0.0, 0.0], [1.0, 1.0], [64, 64], 9, hpg.HPG_OBSTACLE_UPPER)   # 575^2 > 262144
    P.set_rhs(1.0)
    P.set_constraint(lambda X: np.full(X.shape[0], 0.5))
    P.set_dirichlet(None)
    P.set_alphas([0.1])
    P.set_state(np.zeros(P.n_u_full), np.zeros(P.n_psi), np.zeros(P.n_psi), 0.1)
    xd = torch.zeros(P.n_u, dtype=torch.float64, device="cuda")
    yd = torch.zeros_like(xd)
    rc = P.apply_stiffness_inv_noalloc(0.1, xd.data_ptr(), yd.data_ptr(), P.n_u)
    assert rc == 1
    assert b"exceed the limit" in ctx.L.hpg_last_error(ctx.h)
    P.free()
    ctx.close()
