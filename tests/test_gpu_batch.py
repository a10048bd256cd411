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
