"""Late-iteration parity at full size: the GPU's next iteration against the oracle started from the
GPU's own state, on sampled rows and columns.

The dense oracle cannot run a whole solve at these sizes, and FP32 trajectories re-inject rounding
every iteration, so each comparison covers exactly one iteration of Algorithm 1: the state after k
iterations is read back, the oracle forms beta-tilde = beta^k + (beta^k - beta^{k-1}) / lambda and
the row update log alpha-hat_i = log r_i - LSE_j(log beta-tilde_j - C_ij / eps) on sampled rows,
then the column update log beta-hat_j = log c_j - LSE_i(log alpha-hat_i - C_ij / eps) on sampled
columns from the GPU's own alpha-hat (``oracle.row_lse_sampled`` with the roles of the clouds
swapped), all in FP64 with the costs formed on the fly.

These states are deep in the schedule (eps down to 2e-5), where the fast sweeps run on their late
paths: shift hints from the previous iteration, 32 to 64 micro-split partials merged per point,
pack offsets of a drifted gauge, and, once the hints are withdrawn (a state written back with
``ot_state_set``), the exact-maximum recompute of tiles whose sum overflows.  ``ot_state_counters``
shows which of those paths ran.

Each error is stated twice:
* in cost units, ||eps delta||_inf / max(||f||_inf, ||g||_inf) <= 1e-5 (the potential tolerance);
* in log units, |delta log alpha-hat| and |delta log beta-hat| against a bound derived from the
  arithmetic.  Plain FP32 sweeps: every partial value of z = h_q - G + <A_p, w_q> (base 2; G the
  pack offset) is at most Z = max|h - G| + sum_k max|A_k| max|w_k| in magnitude and takes at most
  d + 2 roundings of 2^-24 relative, and the log-sum-exp is 1-Lipschitz in its terms; the offset the
  GPU used is up to two iterations older than the one formed here, so Z is doubled:
  bound = ln 2 (2 (d + 2) 2^-24 Z + 2^-16).  Refined sweeps (refine_on = 2^-8, which switches the
  refinement on at these states): the dominant terms are formed in float-float and rounded once at
  their own small size, and the terms left in FP32 carry about refine_tol, so
  bound = 8 refine_tol + 2^-16.
"""
import numpy as np
import pytest

import oracle as O
import ot_inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2609_33814_b300")
torch = pytest.importorskip("torch")

TOL_POT = 1e-5
LOG2E = 1.4426950408889634
REFINE_TOL = 1e-5  # the library's default refine_tol


@pytest.fixture(scope="module")
def ctx():
    return P.Context(0)


def _weights(prob):
    a = np.maximum(prob.a, 1e-15)
    b = np.maximum(prob.b, 1e-15)
    return a / a.sum(), b / b.sum()


def _log_bound(u, w, lv, kappa, eps, d):
    """Derived FP32 bound (natural log units) for the sweep over tile-side points w with scalings lv,
    thread-side points u."""
    u = u.astype(np.float64)
    w = w.astype(np.float64)
    h = (lv - kappa * (w ** 2).sum(1) / eps) * LOG2E - LOG2E * lv[0]
    A = 2.0 * kappa * LOG2E / eps * np.abs(u).max(0)
    Z = np.abs(h).max() + float((A * np.abs(w).max(0)).sum())
    return np.log(2.0) * (2 * (d + 2) * 2.0 ** -24 * Z + 2.0 ** -16)


def _sample(n, rng, count):
    return np.unique(np.concatenate([rng.choice(n, count, replace=False), [0, n - 1]]))


def _next_iteration_parity(S, prob, eta, lam, rng, count=24):
    """One GPU iteration from the state after S.k iterations against the oracle; returns the errors."""
    a, b = _weights(prob)
    k = S.k
    lb, lbp = S.get(P.OT_LOG_BETA), S.get(P.OT_LOG_BETA_PREV)
    lbt = lb + (lb - lbp) / lam
    eps = O.eps_schedule(eta, lam, k)
    S.step(1)
    lah, lbh = S.get(P.OT_LOG_ALPHA_HAT), S.get(P.OT_LOG_BETA_HAT)
    assert np.isfinite(lah).all() and np.isfinite(lbh).all()
    rows = _sample(prob.n, rng, count)
    cols = _sample(prob.m, rng, count)
    ref_r = np.log(a[rows]) - O.row_lse_sampled(rows, prob.x, prob.y, lbt, prob.kappa, eps)
    ref_c = np.log(b[cols]) - O.row_lse_sampled(cols, prob.y, prob.x, lah, prob.kappa, eps)
    scale = max(np.abs(eps * lah).max(), np.abs(eps * (lbh - np.log(b))).max())
    out = {"k": k, "eps": eps,
           "rows_log": float(np.abs(lah[rows] - ref_r).max()), "cols_log": float(np.abs(lbh[cols] - ref_c).max()),
           "rows_bound": _log_bound(prob.x, prob.y, lbt, prob.kappa, eps, prob.d),
           "cols_bound": _log_bound(prob.y, prob.x, lah, prob.kappa, eps, prob.d)}
    out["rows_cost"] = eps * out["rows_log"] / scale
    out["cols_cost"] = eps * out["cols_log"] / scale
    return out


def _assert_parity(e, what, refined=False):
    assert e["rows_cost"] <= TOL_POT and e["cols_cost"] <= TOL_POT, (what, e)
    if refined:
        rb = cb = 8 * REFINE_TOL + 2.0 ** -16
    else:
        rb, cb = e["rows_bound"], e["cols_bound"]
    assert e["rows_log"] <= rb and e["cols_log"] <= cb, (what, e)


def _withdraw_hints(S, lam):
    """Write the state back unchanged: the stored shift hints are withdrawn, so the next iteration
    starts its running shifts from each micro-split's first chunk."""
    k = S.k
    la, lb, lbp = S.get(P.OT_LOG_ALPHA), S.get(P.OT_LOG_BETA), S.get(P.OT_LOG_BETA_PREV)
    S.set(P.OT_LOG_ALPHA, la, k)
    S.set(P.OT_LOG_BETA, lb, k)
    S.set(P.OT_LOG_BETA_PREV, lbp, k)


@pytest.mark.parametrize("refine", [False, True])
@pytest.mark.parametrize("lam,checkpoints", [(1.0, (20000, 50000)), (1.99, (20000,))])
def test_grid128_deep_in_the_schedule(ctx, lam, checkpoints, refine):
    """A 128 x 128 grid (the serving stream's largest requests) at k = 2e4 and 5e4 (eps = 5e-5, 2e-5),
    with the fast sweeps in plain FP32 and refined (their dominant terms in float-float)."""
    prob = I.grid_problem(128, 2609, "gaussmix", "cauchy")
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0, lam=lam,
                  precision="mufu", cert_every=0, zero_mass_floor=1e-15, refine_on=2.0 ** -8 if refine else 0.0)
    rng = np.random.default_rng(7)
    done = 0
    for kc in checkpoints:
        S.step(kc - done)
        c = S.counters()
        e = _next_iteration_parity(S, prob, 1.0, lam, rng)
        c1 = S.counters()
        assert c1["splits_fast"] == (32, 32), c1
        assert (c1["tiles_refined"] > c["tiles_refined"]) == refine, (c, c1)
        _assert_parity(e, ("hinted", kc), refine)
        # the same iteration's successor without hints: the overflow recompute path runs
        _withdraw_hints(S, lam)
        e2 = _next_iteration_parity(S, prob, 1.0, lam, rng)
        _assert_parity(e2, ("no hints", kc), refine)
        assert S.counters()["tile_recomputes"] > c1["tile_recomputes"]
        done = S.k
    S.close()


@pytest.mark.parametrize("s", [256, 512])
def test_large_grids_sixty_four_splits(ctx, s):
    """256^2 and 512^2 O-BDRS instances (the batched configuration's sizes, 64 micro-split partials
    per point) at k = 500, hinted and unhinted."""
    import torch as T
    prob = I.grid_problem(s, 300 + s, "sparse", "gaussmix")
    dev = [T.from_numpy(v).cuda() for v in (prob.x, prob.y, prob.a, prob.b)]
    S = ctx.state(*dev, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0, lam=1.5, precision="mufu", cert_every=0,
                  zero_mass_floor=1e-15)
    S.step(500)
    assert S.counters()["splits_fast"] == (64, 64)
    rng = np.random.default_rng(s)
    _assert_parity(_next_iteration_parity(S, prob, 1.0, 1.5, rng, count=16), ("hinted", s))
    _withdraw_hints(S, 1.5)
    _assert_parity(_next_iteration_parity(S, prob, 1.0, 1.5, rng, count=16), ("no hints", s))
    S.close()


def test_rgb_two_pow_20_at_k200(ctx):
    """Colour-transfer size, n = m = 2^20 RGB points (d = 3), eps0 = 0.1, at k = 200."""
    n = 1 << 20
    prob = I.rgb_problem(n, seed=41)
    dev = [torch.from_numpy(v).cuda() for v in (prob.x, prob.y, prob.a, prob.b)]
    S = ctx.state(*dev, cost_scale=prob.kappa, omega=1.0, eps0=0.1, lam=1.0, precision="mufu", cert_every=0)
    del dev
    S.step(200)
    rng = np.random.default_rng(11)
    _assert_parity(_next_iteration_parity(S, prob, 0.1, 1.0, rng, count=12), "rgb hinted")
    S.close()


def test_server_batch_certificate_potentials_at_k500(ctx):
    """The batched configuration (5 x 256^2 + 3 x 512^2, O-BDRS) in one server lane to 500 iterations:
    the returned certificate potentials satisfy g = eps log(B / c) with B = c / (K^T A), A = exp(f /
    eps), i.e. g_j = -eps LSE_i((f_i - C_ij) / eps), on sampled columns of every instance."""
    sizes = [256, 256, 512, 256, 512, 256, 512, 256]
    classes = ["uniform", "gaussmix", "cauchy", "sparse"]
    probs = [I.grid_problem(s, 100 + i, classes[i % 4], classes[(i + 1) % 4]) for i, s in enumerate(sizes)]
    lams = [1.5 if i % 2 else 1.99 for i in range(8)]
    srv = P.Server(ctx, hbm_budget_bytes=32 << 30, max_slots=8)
    ids = []
    for p, lam in zip(probs, lams):
        dev = [torch.from_numpy(v).cuda() for v in (p.x, p.y, p.a, p.b)]
        ids.append(srv.submit(*dev, cost_scale=p.kappa, omega=p.omega, zero_mass_floor=1e-15, eps0=1.0, lam=lam,
                              max_iters=500, cert_every=100, precision="mufu"))
    rng = np.random.default_rng(2)
    for rid, p, lam in zip(ids, probs, lams):
        f, g, res = srv.wait(rid, 600.0)
        assert res["iters"] == 500 and res["L_best"] <= res["U_best"], p.name
        eps = O.eps_schedule(1.0, lam, res["best_iter"])
        cols = _sample(p.m, rng, 12)
        g_ref = -eps * O.row_lse_sampled(cols, p.y, p.x, f / eps, p.kappa, eps)
        scale = max(np.abs(f).max(), np.abs(g).max())
        assert np.abs(g[cols] - g_ref).max() / scale <= 1e-6, p.name
    srv.close()
