"""Parity at the benchmark configurations' sizes, where the dense oracle cannot run a whole solve.

* 32x32 grid, FP64, eps0 = 1, lambda = 1, 2000 iterations, certificate every 100: the oracle
  re-evaluates the certificate (Prop. 3, Algorithm 2) from the final GPU state, and takes one
  iteration of Algorithm 1 from it, for comparison with the GPU's next iteration.
* A batch of 8 uneven O-BDRS instances (5 x 256^2 and 3 x 512^2 grids) in one server lane:
  sampled rows of the first iteration's potentials against the oracle's on-the-fly LSE.
* The large colour-transfer size (n = m = 10,022,870, d = 3): sampled rows of the first row sweep.
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


def test_grid32_fp64_2000_iterations(ctx):
    prob = I.grid_problem(32, seed=2609)
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0, lam=1.0,
                  precision="fp64", cert_every=100)
    res = S.step(2000)
    assert res["iters"] == 2000 and res["n_certs"] == 20
    assert res["L_best"] <= res["U_best"]
    # the oracle's certificate of the GPU state after iteration 1999 (a certificate iteration)
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    lah, lbh, lbt = S.get(P.OT_LOG_ALPHA_HAT), S.get(P.OT_LOG_BETA_HAT), S.get(P.OT_LOG_BETA_TILDE)
    eps = O.eps_schedule(1.0, 1.0, 1999)
    cert = O.certificate(lah, lbh, lbt, prob.a, prob.b, C, eps, prob.omega)
    assert abs(cert["U"] - res["U"]) <= 1e-6 and abs(cert["L"] - res["L"]) <= 1e-6, (cert["U"], res["U"])
    # one more iteration from that state on both sides
    st = O.DualState(S.get(P.OT_LOG_ALPHA), S.get(P.OT_LOG_BETA), S.get(P.OT_LOG_BETA_PREV), lah, lbh, lbt,
                     2000, eps)
    st1 = O.dual_obdrs_step(st, np.log(prob.a), np.log(prob.b), C, 1.0, 1.0)
    S.step(1)
    f_g = st1.eps * S.get(P.OT_LOG_ALPHA_HAT)
    f_o = st1.eps * st1.log_alpha_hat
    g_g = st1.eps * (S.get(P.OT_LOG_BETA_HAT) - np.log(prob.b))
    g_o = st1.eps * (st1.log_beta_hat - np.log(prob.b))
    scale = max(np.abs(f_o).max(), np.abs(g_o).max())
    assert max(np.abs(f_g - f_o).max(), np.abs(g_g - g_o).max()) / scale <= 1e-9
    S.close()


def test_batch_of_eight_uneven_obdrs_instances(ctx):
    import torch
    sizes = [256, 256, 512, 256, 512, 256, 512, 256]
    classes = ["uniform", "gaussmix", "cauchy", "sparse"]
    probs = [I.grid_problem(s, 100 + i, classes[i % 4], classes[(i + 1) % 4]) for i, s in enumerate(sizes)]
    lams = [1.5 if i % 2 else 1.99 for i in range(8)]
    srv = P.Server(ctx, hbm_budget_bytes=32 << 30, max_slots=8)
    ids = []
    for p, lam in zip(probs, lams):
        dev = [torch.from_numpy(v).cuda() for v in (p.x, p.y, p.a, p.b)]
        ids.append(srv.submit(*dev, cost_scale=p.kappa, omega=p.omega, zero_mass_floor=1e-15, eps0=1.0, lam=lam,
                              max_iters=1, cert_every=1, precision="mufu"))
    rng = np.random.default_rng(1)
    for rid, p, lam in zip(ids, probs, lams):
        f, g, res = srv.wait(rid, 300.0)
        assert res["iters"] == 1 and res["L"] <= res["U"]
        a = np.maximum(p.a, 1e-15)
        a = a / a.sum()
        rows = np.sort(rng.choice(p.n, size=16, replace=False))
        lse = O.row_lse_sampled(rows, p.x, p.y, np.zeros(p.m), p.kappa, 1.0)  # k = 0: eps = eta, beta-tilde = 1
        f_o = 1.0 * (np.log(a[rows]) - lse)
        assert np.abs(f[rows] - f_o).max() / np.abs(f_o).max() <= 1e-6, p.name
    srv.close()


def test_large_colour_transfer_size_sampled_rows(ctx):
    import torch
    n = 4238 * 2365
    prob = I.rgb_problem(n, seed=5)
    eta = 0.01
    dev = [torch.from_numpy(v).cuda() for v in (prob.x, prob.y, prob.a, prob.b)]
    S = ctx.state(*dev, cost_scale=prob.kappa, omega=1.0, eps0=eta, cert_every=0)
    del dev
    S.step(1)
    lah = S.get(P.OT_LOG_ALPHA_HAT)
    rows = np.sort(np.random.default_rng(3).choice(n, size=6, replace=False))
    lse = O.row_lse_sampled(rows, prob.x, prob.y, np.zeros(n), prob.kappa, eta, chunk=1 << 20)
    ref = np.log(prob.a[rows]) - lse
    err = np.abs(eta * (lah[rows] - ref)).max() / np.abs(eta * ref).max()
    assert err <= 1e-5, err
    S.close()


def test_translation_bound_at_colour_transfer_size(ctx):
    """p* between a measure and its translate is kappa ||v||^2 at any size (the optimal plan is the
    translation), so the certificate must bracket it: L_best <= p* <= U_best at 2^20 points, d = 3.
    Colours are quantised to multiples of 2^-10 and v too, so y = x + v is exact in float32."""
    n = 1 << 20
    x = np.round(I.rgb_cloud(n, seed=11).astype(np.float64) * 1024.0) / 1024.0
    v = np.array([52.0, -31.0, 17.0]) / 1024.0
    y = x + v
    a = np.full(n, 1.0 / n)
    kappa = 1.0 / 3.0
    pstar = O.pstar_translation(v, kappa)
    f, g, res = ctx.solve(x.astype(np.float32), y.astype(np.float32), a, a, cost_scale=kappa, omega=0.0,
                          eps0=0.1, lam=1.0, max_iters=20, cert_every=10)
    assert res["n_certs"] == 2
    assert res["L_best"] <= pstar + 1e-12 and pstar <= res["U_best"] + 1e-12, (res["L_best"], pstar, res["U_best"])


def test_one_dimensional_monotone_bound():
    """On a line the monotone coupling is optimal for a convex cost: p* (exact, O(n log n) on the
    host) must lie in [L_best, U_best] at n = m = 2^17 with non-uniform weights, and the gap closes."""
    ctx = P.Context(0)
    n = 1 << 17
    x = I.random_cloud(n, 1, seed=21)
    y = I.random_cloud(n, 1, seed=22)
    a = I.uniform_weights(n, 23)
    b = I.uniform_weights(n, 24)
    pstar = O.pstar_1d(x[:, 0], a, y[:, 0], b, 1.0)
    gaps = []
    for iters in (100, 400):
        f, g, res = ctx.solve(x, y, a, b, cost_scale=1.0, omega=1.0, eps0=1.0, lam=1.0, max_iters=iters,
                              cert_every=50)
        assert res["L_best"] <= pstar + 1e-12 and pstar <= res["U_best"] + 1e-12, (iters, res, pstar)
        gaps.append(res["U_best"] - res["L_best"])
    assert gaps[1] < gaps[0]
    ctx.close()


@pytest.mark.parametrize("cls", ["uniform", "gaussmix", "cauchy", "sparse"])
@pytest.mark.parametrize("lam", [1.0, 1.99])
def test_certificate_and_rounding_bracket_lp_pstar(ctx, cls, lam):
    """The GPU's certified bounds bracket the exact transport LP value (scipy HiGHS) on 12 x 12 grid
    histograms of every class, and the rounded plan's cost is at least p*."""
    from exact_lp import lp_pstar
    prob = I.grid_problem(12, 22, cls, "cauchy")
    a = np.maximum(prob.a, 1e-15); a = a / a.sum()
    b = np.maximum(prob.b, 1e-15); b = b / b.sum()
    pstar = lp_pstar(a, b, O.cost_matrix(prob.x, prob.y, prob.kappa))
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, zero_mass_floor=1e-15,
                  eps0=1.0, lam=lam, cert_every=50, precision="mufu")
    res = S.step(500)
    # 1e-6: the certificate's stated absolute accuracy in the float-float sweeps
    assert res["L_best"] <= pstar + 1e-6 and pstar <= res["U_best"] + 1e-6, (res["L_best"], pstar, res["U_best"])
    assert res["U_best"] - res["L_best"] < 0.05
    f_round, _ = S.round_cost(P.OT_PLAN_BEST)
    assert f_round >= pstar - 1e-6
    S.close()
