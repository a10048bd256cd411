"""Request loop (continuous batching): requests submitted while others are on
the GPU are admitted as workers and memory free up, overlap on the device, and
each result is exactly the one the same problem gives when solved alone."""
import time

import numpy as np
import pytest

from tests.gpu_helpers import case

pytestmark = pytest.mark.gpu

MIX = ["radial4", "aniso_upper", "p2", "single_cell", "sine3d_small", "torsion_small", "radial_3x3_p5",
       "sine3d_3x2x2", "torsion_3x3_p3"]


@pytest.fixture(scope="module")
def alone():
    from paper_2412_13733_gb300 import hpg
    ctx = hpg.Context(0)
    out = {}
    for name in MIX:
        P = hpg.from_workload(ctx, case(name), hpg.default_params(precision=1))
        P.solve()
        out[name] = (P.u(), P.psi())
        P.free()
    ctx.close()
    return out


def _drain(ctx, tickets, timeout_s=120.0):
    t0 = time.time()
    left = dict(tickets)
    while left and time.time() - t0 < timeout_s:
        for t in list(left):
            done, res = ctx.poll(t)
            if done:
                assert res == 0
                left.pop(t)
        time.sleep(0.002)
    assert not left, "requests did not finish"


def test_staggered_requests_match_alone(alone):
    from paper_2412_13733_gb300 import hpg
    ctx = hpg.Context(0)
    ctx.server_start(workers=4)
    probs = {name: hpg.from_workload(ctx, case(name), hpg.default_params(precision=1)) for name in MIX}
    tickets = {}
    for name in MIX[:3]:
        tickets[ctx.submit(probs[name])] = name
    time.sleep(0.005)
    for name in MIX[3:]:                       # arrive while the first ones run
        tickets[ctx.submit(probs[name])] = name
    _drain(ctx, tickets)
    for t, name in tickets.items():
        P = probs[name]
        u, psi = alone[name]
        assert np.array_equal(P.u(), u), name
        assert np.array_equal(P.psi(), psi), name
        q, run, lat = ctx.ticket_times(t)
        assert lat >= run > 0.0
    for P in probs.values():
        P.free()
    assert ctx.server_memory()[0] == 0
    ctx.server_stop()
    ctx.close()


def test_memory_admission_serialises_when_budget_is_tight(alone):
    from paper_2412_13733_gb300 import hpg
    ctx = hpg.Context(0)
    names = ["radial4", "p2", "radial_3x3_p5"]
    probs = [hpg.from_workload(ctx, case(n), hpg.default_params(precision=1)) for n in names]
    biggest = max(ctx.server_memory(P)[1] for P in probs)
    ctx.server_start(workers=4, budget_bytes=int(biggest * 1.5))     # room for one request at a time
    tickets = [ctx.submit(P) for P in probs]
    for t in tickets:
        assert ctx.wait(t, 60000.0) == 0
    # finished requests hand their device memory back to the budget
    assert ctx.server_memory()[0] == 0
    # submits were back to back, so queued/running times give the run intervals: no overlap
    iv = sorted((q, q + r) for q, r, _ in (ctx.ticket_times(t) for t in tickets))
    for (s0, e0), (s1, e1) in zip(iv, iv[1:]):
        assert s1 >= e0 - 0.5, iv
    for n, P in zip(names, probs):
        assert np.array_equal(P.u(), alone[n][0])
        P.free()
    assert ctx.server_memory()[0] == 0
    ctx.server_stop()
    ctx.close()


def test_bounded_wait_times_out_without_faulting():
    from paper_2412_13733_gb300 import hpg
    ctx = hpg.Context(0)
    ctx.server_start(workers=1)
    w = case("radial_3x3_p5")
    slow = hpg.from_workload(ctx, w)
    slow.set_alphas(w["alphas"] * 6)           # a long request
    t = ctx.submit(slow)
    with pytest.raises(hpg.HpgError) as ei:     # not available to the client while in the loop
        slow.u()
    assert ei.value.code == 11                  # HPG_ERR_BUSY
    with pytest.raises(hpg.HpgError) as ei:
        ctx.wait(t, 0.01)
    assert ei.value.code == 8                   # HPG_ERR_TIMEOUT, the request keeps running
    assert ctx.wait(t, 120000.0) == 0
    slow.free()
    ctx.server_stop()
    ctx.close()


def test_component_calls_refuse_a_problem_in_the_loop():
    """While a request is queued or running, a worker owns the problem's device
    buffers; the component operators and the allocation-free apply must refuse it
    (HPG_ERR_BUSY) instead of launching on buffers the worker may release."""
    from paper_2412_13733_gb300 import hpg
    ctx = hpg.Context(0)
    w = case("radial_3x3_p5")
    slow = hpg.from_workload(ctx, w)
    slow.solve()                                # device state exists before submission
    torch = pytest.importorskip("torch")
    x = np.zeros(slow.n_u)
    xd = torch.zeros(slow.n_u, dtype=torch.float64, device="cuda")
    yd = torch.zeros_like(xd)
    torch.cuda.synchronize()
    slow.set_alphas(w["alphas"] * 12)          # a request that outlives the calls below (120 steps)
    ctx.server_start(workers=1)
    t = ctx.submit(slow)
    calls = [lambda: slow.apply_stiffness_inv(x, hpg.HPG_FP64), lambda: slow.residual(),
             lambda: slow.factor_precond(hpg.HPG_FP64)]
    for call in calls:
        with pytest.raises(hpg.HpgError) as ei:
            call()
        assert ei.value.code == 11, ei.value            # HPG_ERR_BUSY
    assert slow.apply_stiffness_inv_noalloc(0.5, xd.data_ptr(), yd.data_ptr(), slow.n_u) == 11
    assert ctx.wait(t, 120000.0) == 0
    slow.free()
    ctx.server_stop()
    ctx.close()


def test_failed_request_reports_its_message():
    from paper_2412_13733_gb300 import hpg
    ctx = hpg.Context(0)
    ctx.server_start(workers=2)
    P = hpg.from_workload(ctx, case("radial_3x3_p5"), hpg.default_params(newton_max=1))
    ok = hpg.from_workload(ctx, case("p2"))
    t_bad, t_ok = ctx.submit(P), ctx.submit(ok)
    assert ctx.wait(t_bad, 120000.0) == 4               # HPG_ERR_NEWTON_CAP
    assert ctx.wait(t_ok, 120000.0) == 0
    msg = ctx.ticket_error(t_bad)
    assert "Newton cap" in msg and "proximal step" in msg, msg
    assert ctx.ticket_error(t_ok) == ""
    P.free()
    ok.free()
    ctx.server_stop()
    ctx.close()
