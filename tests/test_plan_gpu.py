"""Barycentric projection and marginal errors of the implicit output plan (App. G output, Tables 3
and 4) through ot_plan_project, against the oracle's dense form and its sampled-row form.

Tolerances: the GPU forms exponents in float-float and sums in Kahan-compensated FP32, so row and
column sums carry ~1e-7 relative error: sums are compared at 1e-6 relative, projections at 1e-5
absolute (targets lie in [0, 1]), and the marginal-error statistics at 1e-6 of the total mass
(1e-5 for the maxima relative to single masses).
"""
import numpy as np
import pytest

import oracle as O
import ot_inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2609_33814_b300")


@pytest.fixture(scope="module")
def ctx():
    return P.Context(0)


def _oracle_plan(S, plan, eta, lam, b, best_iter):
    """The oracle's (log u, log v, eps) for the GPU state's plan."""
    if plan == P.OT_PLAN_BEST:
        eps = O.eps_schedule(eta, lam, best_iter)
        return S.get(P.OT_F_BEST) / eps, np.log(b) + S.get(P.OT_G_BEST) / eps, eps
    eps = O.eps_schedule(eta, lam, S.k - 1)
    lv = S.get(P.OT_LOG_BETA_HAT) if plan == P.OT_PLAN_LATEST else S.get(P.OT_LOG_BETA_TILDE)
    return S.get(P.OT_LOG_ALPHA_HAT), lv, eps


CASES = [("grid", 16, 1.0), ("grid", 24, 1.5), ("ragged3", 0, 1.0)]


@pytest.mark.parametrize("kind,s,lam", CASES)
@pytest.mark.parametrize("plan", [0, 1, 2])
def test_projection_parity(ctx, kind, s, lam, plan):
    if kind == "grid":
        prob = I.grid_problem(s, 31, "gaussmix", "cauchy")
    else:
        x = I.rgb_cloud(1500, 41)
        y = I.rgb_cloud(1031, 42)
        prob = I.Problem(x, y, I.uniform_weights(1500, 43), I.uniform_weights(1031, 44), 1.0 / 3.0, 1.0, "ragged3")
    a = prob.a / prob.a.sum()
    b = prob.b / prob.b.sum()
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0, lam=lam,
                  cert_every=20, precision="mufu")
    res = S.step(60)
    y_hat, row, col, err = S.project(plan)
    lu, lv, eps = _oracle_plan(S, plan, 1.0, lam, b, res["best_iter"])
    assert err["eps"] == pytest.approx(eps, rel=1e-15)
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    D = O.plan_diagnostics(lu, lv, C, eps, prob.y, a, b)
    assert np.abs(row / D["row_sums"] - 1).max() <= 1e-6
    assert np.abs(col / D["col_sums"] - 1).max() <= 1e-6
    assert np.abs(y_hat - D["y_hat"]).max() <= 1e-5
    for key in ("row_l1", "col_l1", "row_max_abs", "col_max_abs"):
        assert abs(err[key] - D[key]) <= 1e-6, key
    for key in ("row_max_rel", "col_max_rel"):
        assert abs(err[key] - D[key]) <= 1e-5, key
    # the exact marginal of each plan, as the certificate construction makes it
    if plan == P.OT_PLAN_INTERMEDIATE:
        assert err["row_max_rel"] <= 1e-5
    if plan == P.OT_PLAN_BEST:
        assert err["col_max_rel"] <= 1e-5
    S.close()


def test_projection_sampled_rows_rgb(ctx):
    n = 1 << 18
    prob = I.rgb_problem(n, seed=51)
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=1.0, eps0=0.1, lam=1.0,
                  cert_every=10, precision="mufu")
    res = S.step(20)
    b = prob.b / prob.b.sum()
    rows = np.sort(np.random.default_rng(4).choice(n, size=8, replace=False))
    for plan in (P.OT_PLAN_BEST, P.OT_PLAN_INTERMEDIATE):
        y_hat, row, col, err = S.project(plan)
        lu, lv, eps = _oracle_plan(S, plan, 0.1, 1.0, b, res["best_iter"])
        if plan == P.OT_PLAN_BEST:
            assert err["col_max_rel"] <= 1e-5
        else:
            assert err["row_max_rel"] <= 1e-5
        lr, yh = O.projection_sampled(rows, prob.x, prob.y, lu, lv, prob.kappa, eps, chunk=1 << 16)
        assert np.abs(row[rows] / np.exp(lr) - 1).max() <= 1e-6
        assert np.abs(y_hat[rows] - yh).max() <= 1e-5
        assert abs(row.sum() - col.sum()) <= 1e-6
    S.close()


def test_projection_needs_a_certificate_and_an_iteration(ctx):
    prob = I.grid_problem(8, 3)
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, cert_every=0)
    with pytest.raises(P.OTError) as e:
        S.project(P.OT_PLAN_LATEST)
    assert e.value.status == P.OT_EINVAL
    S.step(3)
    with pytest.raises(P.OTError) as e:
        S.project(P.OT_PLAN_BEST)
    assert e.value.status == P.OT_EINVAL
    S.project(P.OT_PLAN_LATEST)
    S.close()


@pytest.mark.parametrize("kind,s,lam", CASES)
@pytest.mark.parametrize("plan", [0, 1, 2])
def test_rounding_cost_parity(ctx, kind, s, lam, plan):
    """Cost of the rounded plan (row scaling, column scaling, rank-one correction) and of the
    unrounded one against the oracle's dense rounding, at 1e-6 relative."""
    if kind == "grid":
        prob = I.grid_problem(s, 33, "gaussmix", "sparse")
    else:
        x = I.rgb_cloud(900, 45)
        y = I.rgb_cloud(700, 46)
        prob = I.Problem(x, y, I.uniform_weights(900, 47), I.uniform_weights(700, 48), 1.0 / 3.0, 1.0, "ragged3")
    a = np.maximum(prob.a, 1e-15); a = a / a.sum()
    b = np.maximum(prob.b, 1e-15); b = b / b.sum()
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, zero_mass_floor=1e-15,
                  eps0=1.0, lam=lam, cert_every=20, precision="mufu")
    res = S.step(40)
    cr, cu = S.round_cost(plan)
    lu, lv, eps = _oracle_plan(S, plan, 1.0, lam, b, res["best_iter"])
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    R = O.round_plan(lu, lv, C, eps, a, b)
    assert abs(cu / R["cost_unrounded"] - 1) <= 1e-6
    assert abs(cr / R["cost"] - 1) <= 1e-6, (cr, R["cost"])
    assert cr >= res["L_best"] - 1e-12  # a feasible plan's cost bounds the dual from above
    S.close()


def test_rounding_bounds_pstar_for_an_old_kernel_method(ctx):
    """Annealed Sinkhorn (no certificate available) still gets a feasible upper bound by rounding:
    on a line it stays above the exact p* and approaches it."""
    x = I.random_cloud(3000, 1, 61)
    y = I.random_cloud(2500, 1, 62)
    a, b = I.uniform_weights(3000, 63), I.uniform_weights(2500, 64)
    pstar = O.pstar_1d(x[:, 0], a, y[:, 0], b, 1.0)
    S = ctx.state(x, y, a, b, cost_scale=1.0, omega=1.0, eps0=1.0, cert_every=0, algorithm="as")
    gaps = []
    for it in (50, 450):
        S.step(it)
        cr, _ = S.round_cost(P.OT_PLAN_LATEST)
        assert cr >= pstar - 1e-12
        gaps.append(cr - pstar)
    assert gaps[1] < gaps[0]
    S.close()
