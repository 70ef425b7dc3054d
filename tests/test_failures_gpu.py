"""Failure detection without faulting the GPU.

* A tile wait forced to give up at once (the wait bound set to 0 polls): the sweep records the
  error, lets its in-flight copies land and returns; the state reports OT_ETIMEDOUT and the context
  keeps working.
* A time budget ends a solve early with stop reason "time".
* A non-finite coordinate makes the iteration report OT_ENUMERIC; in the server only that request
  fails.
"""
import numpy as np
import pytest

import ot_inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2609_33814_b300")


def test_device_wait_bound_reports_timeout_and_context_survives():
    ctx = P.Context(0)
    prob = I.grid_problem(32, 1)
    P.lib().ot_debug_set_wait_limit(ctx.handle, 0)
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, cert_every=0)
    with pytest.raises(P.OTError) as e:
        S.step(1)
    assert e.value.status == P.OT_ETIMEDOUT
    S.close()
    P.lib().ot_debug_set_wait_limit(ctx.handle, 1 << 26)
    f, g, res = ctx.solve(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega,
                          max_iters=100, cert_every=50)
    assert res["iters"] == 100 and np.isfinite(f).all()
    ctx.close()


def test_time_budget_stops_solve():
    ctx = P.Context(0)
    prob = I.grid_problem(64, 2)
    f, g, res = ctx.solve(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega,
                          max_iters=10 ** 8, cert_every=10, time_budget_s=0.3)
    assert res["stop"] == "time" and 0 < res["iters"] < 10 ** 8
    assert res["elapsed_s"] >= 0.3
    ctx.close()


def test_nan_coordinate_reports_numeric_error():
    ctx = P.Context(0)
    prob = I.grid_problem(16, 3)
    x = prob.x.copy()
    x[17, 1] = np.nan
    S = ctx.state(x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, cert_every=0)
    with pytest.raises(P.OTError) as e:
        S.step(1)
    assert e.value.status == P.OT_ENUMERIC
    S.close()
    # in the server only the bad request fails
    srv = P.Server(ctx, hbm_budget_bytes=1 << 30, max_slots=4)
    bad = srv.submit(x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, max_iters=100,
                     cert_every=50)
    good = srv.submit(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, max_iters=100,
                      cert_every=50)
    with pytest.raises(P.OTError) as e:
        srv.wait(bad, 60.0)
    assert e.value.status == P.OT_ENUMERIC
    f, g, res = srv.wait(good, 60.0)
    assert res["iters"] == 100 and np.isfinite(f).all()
    srv.close()
    ctx.close()
