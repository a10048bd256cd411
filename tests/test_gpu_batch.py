"""Batched solves (hpg_solve_batch): problems of different kind, dimension, h
and p in flight together give exactly the results of solving each alone."""
import numpy as np
import pytest

from tests.gpu_helpers import case

pytestmark = pytest.mark.gpu

MIX = ["radial4", "aniso_upper", "p2", "single_cell", "sine3d_small", "torsion_small", "radial_3x3_p5"]


@pytest.fixture(scope="module")
def ctx():
    from paper_2412_13733_gb300 import hpg
    c = hpg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("workers", [1, 3, 8])
def test_batch_equals_alone(ctx, precision, workers):
    from paper_2412_13733_gb300 import hpg
    alone = {}
    for name in MIX:
        P = hpg.from_workload(ctx, case(name), hpg.default_params(precision=precision))
        P.solve()
        alone[name] = (P.u(), P.psi(), P.stats()["newton_per_step"])
        P.free()
    ctx.set_concurrency(workers)
    probs = [hpg.from_workload(ctx, case(name), hpg.default_params(precision=precision)) for name in MIX]
    ctx.solve_batch(probs)
    for name, P in zip(MIX, probs):
        u, psi, newton = alone[name]
        assert P.stats()["status"] == 0
        assert P.stats()["newton_per_step"] == newton
        assert np.array_equal(P.u(), u), name
        assert np.array_equal(P.psi(), psi), name
        P.free()
    ctx.set_concurrency(8)


def test_batch_rejects_duplicates(ctx):
    from paper_2412_13733_gb300 import hpg
    P = hpg.from_workload(ctx, case("radial4"))
    with pytest.raises(hpg.HpgError):
        ctx.solve_batch([P, P])
    P.free()


def _variants(name, k):
    """k problems of one shape (same mesh, degree and kind) with different data, so
    that their Newton and Krylov counts differ inside a lockstep group."""
    from paper_2412_13733_gb300 import workloads as W
    out = []
    for i in range(k):
        w = dict(case(name))
        base = w.get("f_const") or 0.0
        w["f_const"] = base + 6.0 * i
        w["f"] = W.const_field(w["f_const"])
        phi0 = w["phi"]
        w["phi"] = (lambda f0, c: (lambda X: f0(X) + c))(phi0, 0.02 * i)
        out.append(w)
    return out


GROUP_SHAPES = ["radial_3x3_p5", "sine3d_3x2x2", "torsion_3x3_p3", "aniso_upper"]


@pytest.mark.parametrize("precision,kf32", [(0, 0), (1, 0), (1, 1)])
def test_lockstep_groups_equal_alone(ctx, precision, kf32):
    """Same-shape problems of a batch run as lockstep groups (one launch per step for
    the whole group).  Every problem gets exactly what it gets alone: the same Newton
    counts per step, Krylov iterations, refinement sweeps and bits of u and psi,
    though the problems of a group need different numbers of iterations."""
    from paper_2412_13733_gb300 import hpg
    ws = [w for name in GROUP_SHAPES for w in _variants(name, 4)]
    prm = lambda: hpg.default_params(precision=precision, krylov_f32=kf32)
    alone = []
    for w in ws:
        P = hpg.from_workload(ctx, w, prm())
        P.solve()
        st = P.stats()
        alone.append((P.u(), P.psi(), st["newton_per_step"], st["krylov_total"], st["refine_total"]))
        P.free()
    counts = {tuple(a[2]) for a in alone}
    assert len(counts) > len(GROUP_SHAPES)          # the groups really hold diverging problems
    ctx.set_concurrency(3)
    probs = [hpg.from_workload(ctx, w, prm()) for w in ws]
    for rep in range(2):                            # the second batch reuses the cached groups
        ctx.solve_batch(probs)
        for w, P, (u, psi, newton, kry, ref) in zip(ws, probs, alone):
            st = P.stats()
            assert st["status"] == 0
            assert st["newton_per_step"] == newton, (w["name"], st["newton_per_step"], newton)
            assert st["krylov_total"] == kry and st["refine_total"] == ref, w["name"]
            assert np.array_equal(P.u(), u), w["name"]
            assert np.array_equal(P.psi(), psi), w["name"]
    for P in probs:
        P.free()
    ctx.set_concurrency(8)


def test_lockstep_group_member_failure_is_its_own(ctx):
    """A problem of a group that hits its Newton cap fails alone: the others of the
    group finish and equal their solves alone."""
    from paper_2412_13733_gb300 import hpg
    ws = _variants("radial_3x3_p5", 3)
    alone = []
    for w in ws:
        P = hpg.from_workload(ctx, w)
        P.solve()
        alone.append(P.u())
        P.free()
    probs = [hpg.from_workload(ctx, w) for w in ws]
    probs[1].set_params(hpg.default_params(newton_max=1))
    rc = ctx.solve_batch(probs, check=False)
    assert rc == 4                                   # HPG_ERR_NEWTON_CAP, the failing member's
    assert probs[1].stats()["status"] == 4
    for i in (0, 2):
        assert probs[i].stats()["status"] == 0
        assert np.array_equal(probs[i].u(), alone[i])
    for P in probs:
        P.free()


def test_lockstep_group_mixed_fallback_equals_alone(ctx):
    """A mixed problem whose proximal step hits the Newton cap is solved again from that
    step's start in FP64 (where, with a cap of two steps, it hits the cap again).  In a
    lockstep group that member leaves the group and is solved on its own afterwards: its
    status, counts and iterate equal its solve alone, and the other members are unaffected."""
    from paper_2412_13733_gb300 import hpg
    ws = _variants("radial_3x3_p5", 3)
    prm = lambda i: hpg.default_params(precision=hpg.HPG_MIXED, newton_max=2 if i == 1 else 50)
    alone = []
    for i, w in enumerate(ws):
        P = hpg.from_workload(ctx, w, prm(i))
        rc = P.solve(check=False)
        alone.append((rc, P.stats(), P.u().copy()))
        P.free()
    rc1, st1, _ = alone[1]
    assert rc1 == 4 and st1["fp64_from_step"] == 1 and st1["fp64_newton_steps"] == 2, st1
    assert st1["newton_total"] == 4                  # two mixed steps discarded, two in FP64
    for i in (0, 2):
        assert alone[i][0] == 0 and alone[i][1]["fp64_from_step"] == 0
    probs = [hpg.from_workload(ctx, w, prm(i)) for i, w in enumerate(ws)]
    assert ctx.solve_batch(probs, check=False) == 4
    for (rc, st, u), P in zip(alone, probs):
        sb = P.stats()
        assert sb["status"] == rc
        for key in ("fp64_from_step", "fp64_newton_steps", "newton_total", "krylov_total"):
            assert sb[key] == st[key], key
        assert sb["newton_per_step"] == st["newton_per_step"]
        assert np.array_equal(P.u(), u)
    for P in probs:
        P.free()
