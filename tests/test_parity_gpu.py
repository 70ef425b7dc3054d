"""GPU parity: the CUDA sweeps through the C ABI against the FP64 oracle.

Tolerances (stated per result, from the arithmetic of each precision mode):
* potentials f = eps log alpha-hat, g = eps (log beta-hat - log c), compared as
  ||delta||_inf / max(||f||_inf, ||g||_inf):  1e-5 for the FP32 sweeps, 1e-9 for FP64;
* certificate bounds U, L: 1e-6 absolute (certificate iterations use compensated or FP64 sweeps).
"""
import numpy as np
import pytest

import oracle as O
import ot_inputs as I

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2609_33814_b300")

TOL_POT = {"mufu": 1e-5, "poly": 1e-5, "split": 1e-5, "comp": 1e-5, "fp64": 1e-9}
TOL_CERT = 1e-6


@pytest.fixture(scope="module")
def ctx():
    return P.Context(0)


def _problem(kind, seed):
    if kind == "grid16":
        return I.grid_problem(16, seed)
    if kind == "grid32":
        return I.grid_problem(32, seed)
    if kind == "grid16_gauss":
        return I.grid_problem(16, seed, "gaussmix", "cauchy")
    if kind == "grid16_sparse":
        return I.grid_problem(16, seed, "sparse", "uniform")
    if kind == "ragged3":
        x = I.random_cloud(1000, 3, seed)
        y = I.random_cloud(777, 3, seed + 1)
        return I.Problem(x, y, I.uniform_weights(1000, seed + 2), I.uniform_weights(777, seed + 3),
                         1.0 / 3.0, 1.0, "ragged3")
    if kind == "line":
        x = I.random_cloud(300, 1, seed)
        y = I.random_cloud(200, 1, seed + 1)
        return I.Problem(x, y, I.uniform_weights(300, seed + 2), I.uniform_weights(200, seed + 3),
                         1.0, 1.0, "line")
    if kind == "one_row":
        x = I.random_cloud(1, 2, seed)
        y = I.random_cloud(5, 2, seed + 1)
        return I.Problem(x, y, np.ones(1), I.uniform_weights(5, seed + 3), 0.5, 1.0, "one_row")
    if kind == "one_col":
        x = I.random_cloud(5, 2, seed)
        y = I.random_cloud(1, 2, seed + 1)
        return I.Problem(x, y, I.uniform_weights(5, seed + 2), np.ones(1), 0.5, 1.0, "one_col")
    # 2-D packs whose tiles share a coordinate along aligned runs of points take the fast sweeps'
    # run variant; these cases cover the other coordinate, no runs, and runs on one side only
    if kind == "grid16_cm":  # column-major grid: the first coordinate is constant along each run
        p = I.grid_problem(16, seed)
        return I.Problem(np.ascontiguousarray(p.x[:, ::-1]), np.ascontiguousarray(p.y[:, ::-1]), p.a, p.b,
                         p.kappa, p.omega, kind)
    if kind == "grid48":
        return I.grid_problem(48, seed, "gaussmix", "uniform")
    if kind == "grid20_perm":  # a grid in random order: no runs
        p = I.grid_problem(20, seed)
        rng = np.random.default_rng(seed)
        px, py = rng.permutation(400), rng.permutation(400)
        return I.Problem(p.x[px], p.y[py], p.a[px], p.b[py], p.kappa, p.omega, kind)
    if kind == "grid_mixed":  # 24 x 24 sources (runs of 24 straddle the aligned groups), 16 x 17 targets
        x, y = _grid_xy(24, 24), _grid_xy(16, 17)
        kappa = 1.0 / float(((x[:, None, :] - y[None, :, :]) ** 2).sum(-1).max())
        return I.Problem(x, y, I.uniform_weights(576, seed), I.uniform_weights(272, seed + 1), kappa, 1.0, kind)
    raise ValueError(kind)


def _grid_xy(sx, sy):
    """Integer coordinates of an sx-by-sy pixel grid, row-major (the first coordinate varies fastest)."""
    iy, ix = np.meshgrid(np.arange(sy), np.arange(sx), indexing="ij")
    return np.stack([ix.ravel(), iy.ravel()], axis=1).astype(np.float32)


def _potential_err(st_o, lah, lbh, eps, logc):
    f_o = eps * st_o.log_alpha_hat
    g_o = eps * (st_o.log_beta_hat - logc)
    f_g = eps * lah
    g_g = eps * (lbh - logc)
    scale = max(np.abs(f_o).max(), np.abs(g_o).max(), 1e-300)
    return max(np.abs(f_g - f_o).max(), np.abs(g_g - g_o).max()) / scale


def _gpu_state(ctx, prob, eta, lam, precision, cert_every, st_o=None):
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega,
                  eps0=eta, lam=lam, precision=precision, cert_every=cert_every, max_iters=10 ** 6)
    if st_o is not None and st_o.k > 0:
        S.set(P.OT_LOG_ALPHA, st_o.log_alpha, st_o.k)
        S.set(P.OT_LOG_BETA, st_o.log_beta, st_o.k)
        S.set(P.OT_LOG_BETA_PREV, st_o.log_beta_prev, st_o.k)
    return S


CASES = [("grid16", 1.0, 0), ("grid16", 1.0, 7), ("grid32", 1.0, 3), ("grid16_gauss", 1.5, 5),
         ("grid16_sparse", 1.99, 4), ("ragged3", 1.5, 3), ("line", 1.0, 6), ("one_row", 1.2, 2),
         ("one_col", 1.0, 2), ("grid16_cm", 1.0, 5), ("grid48", 1.3, 4), ("grid20_perm", 1.0, 3),
         ("grid_mixed", 1.5, 6)]


@pytest.mark.parametrize("precision", ["mufu", "poly", "split", "comp", "fp64"])
@pytest.mark.parametrize("kind,lam,k0", CASES)
def test_one_step_parity(ctx, kind, lam, k0, precision):
    """The same FP64 state goes into the GPU and the oracle; one iteration of Algorithm 1."""
    prob = _problem(kind, seed=11)
    eta = 1.0 if kind.startswith("grid") else 0.5
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    st0 = O.dual_obdrs(prob.a, prob.b, C, eta, lam, k0)
    st1 = O.dual_obdrs_step(st0, np.log(prob.a), np.log(prob.b), C, eta, lam)
    S = _gpu_state(ctx, prob, eta, lam, precision, cert_every=0, st_o=st0)
    S.step(1)
    assert S.k == k0 + 1
    lah = S.get(P.OT_LOG_ALPHA_HAT)
    lbh = S.get(P.OT_LOG_BETA_HAT)
    err = _potential_err(st1, lah, lbh, st1.eps, np.log(prob.b))
    assert err <= TOL_POT[precision], (kind, precision, err)
    # the rest of the returned tuple of Algorithm 1
    la, lb, lt = S.get(P.OT_LOG_ALPHA), S.get(P.OT_LOG_BETA), S.get(P.OT_LOG_BETA_TILDE)
    np.testing.assert_allclose(lt, st1.log_beta_tilde, rtol=1e-12, atol=1e-9)
    sc = max(np.abs(st1.log_alpha).max(), np.abs(st1.log_beta).max(), 1.0)
    assert np.abs(la - st1.log_alpha).max() / sc <= 2 * TOL_POT[precision] + 1e-12
    assert np.abs(lb - st1.log_beta).max() / sc <= 2 * TOL_POT[precision] + 1e-12
    S.close()


@pytest.mark.parametrize("precision", ["mufu", "fp64"])
@pytest.mark.parametrize("kind,lam,k0", [("grid16", 1.0, 0), ("grid16", 1.0, 9), ("grid16_gauss", 1.5, 20),
                                         ("ragged3", 1.99, 12), ("line", 1.0, 30)])
def test_certificate_parity(ctx, kind, lam, k0, precision):
    """A certificate iteration (compensated / FP64 sweeps) against Prop. 3 + Algorithm 2 in FP64."""
    prob = _problem(kind, seed=5)
    eta = 1.0 if kind.startswith("grid") else 0.5
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    st0 = O.dual_obdrs(prob.a, prob.b, C, eta, lam, k0)
    st1 = O.dual_obdrs_step(st0, np.log(prob.a), np.log(prob.b), C, eta, lam)
    cert_o = O.certificate_of(st1, prob.a, prob.b, C, prob.omega)
    S = _gpu_state(ctx, prob, eta, lam, precision, cert_every=1, st_o=st0)
    res = S.step(1)
    assert res["n_certs"] == 1
    assert abs(res["U"] - cert_o["U"]) <= TOL_CERT, (res["U"], cert_o["U"])
    assert abs(res["L"] - cert_o["L"]) <= TOL_CERT, (res["L"], cert_o["L"])
    # the certificate potentials it reports
    f = S.get(P.OT_F_CERT)
    g = S.get(P.OT_G_CERT)
    scale = max(np.abs(cert_o["f"]).max(), np.abs(cert_o["g"]).max())
    assert np.abs(f - cert_o["f"]).max() / scale <= 1e-6
    assert np.abs(g - cert_o["g"]).max() / scale <= 1e-6
    # the standalone certificate pass agrees with the fused one
    S2 = _gpu_state(ctx, prob, eta, lam, precision, cert_every=0, st_o=st0)
    S2.step(1)
    c2 = S2.certificate()
    assert abs(c2["U"] - res["U"]) <= TOL_CERT and abs(c2["L"] - res["L"]) <= TOL_CERT
    S.close()
    S2.close()


def test_fp64_trajectory_matches_oracle(ctx):
    """Config-1-style run (grid, eps0 = 1, lambda = 1) over many iterations, FP64 sweeps."""
    prob = I.grid_problem(16, seed=3)
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    ro = O.solve(prob.a, prob.b, C, 1.0, 1.0, 400, 100, prob.omega)
    f, g, res = ctx.solve(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega,
                          eps0=1.0, lam=1.0, max_iters=400, cert_every=100, precision="fp64")
    assert res["iters"] == 400 and res["n_certs"] == 4
    assert abs(res["U_best"] - ro["U_best"]) <= TOL_CERT
    assert abs(res["L_best"] - ro["L_best"]) <= TOL_CERT
    scale = max(np.abs(ro["best"]["f"]).max(), np.abs(ro["best"]["g"]).max())
    assert res["best_iter"] + 1 == ro["best"]["k"]
    assert np.abs(f - ro["best"]["f"]).max() / scale <= 1e-9
    assert np.abs(g - ro["best"]["g"]).max() / scale <= 1e-9


@pytest.mark.parametrize("precision", ["mufu", "comp"])
def test_fp32_trajectory_error_is_small(ctx, precision):
    """FP32 sweeps re-inject rounding every iteration; the trajectory error stays well below 1e-4."""
    prob = I.grid_problem(16, seed=4, cls_a="gaussmix", cls_b="gaussmix")
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    ro = O.solve(prob.a, prob.b, C, 1.0, 1.0, 300, 100, prob.omega)
    f, g, res = ctx.solve(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega,
                          eps0=1.0, lam=1.0, max_iters=300, cert_every=100, precision=precision)
    scale = max(np.abs(ro["best"]["f"]).max(), np.abs(ro["best"]["g"]).max())
    err = max(np.abs(f - ro["best"]["f"]).max(), np.abs(g - ro["best"]["g"]).max()) / scale
    assert err <= 1e-4, err
    assert abs(res["U_best"] - ro["U_best"]) <= 1e-5
    assert abs(res["L_best"] - ro["L_best"]) <= 1e-5


@pytest.mark.parametrize("precision", ["mufu", "split"])
@pytest.mark.parametrize("kind,lam,k", [("grid32", 1.0, 1200), ("grid16_gauss", 1.5, 600), ("ragged3", 1.0, 300)])
def test_hinted_sweep_late_iteration(ctx, precision, kind, lam, k):
    """Late iterations (small eps, wide exponent ranges) where the fast sweeps start their running
    shifts from the previous iteration's log-sum-exp: the GPU's iteration k + 1 against the oracle's
    iteration from the GPU's own state after k iterations."""
    prob = _problem(kind, 21)
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0, lam=lam,
                  precision=precision, cert_every=0)
    S.step(k)
    eps_prev = O.eps_schedule(1.0, lam, k - 1)
    st = O.DualState(S.get(P.OT_LOG_ALPHA), S.get(P.OT_LOG_BETA), S.get(P.OT_LOG_BETA_PREV),
                     S.get(P.OT_LOG_ALPHA_HAT), S.get(P.OT_LOG_BETA_HAT), S.get(P.OT_LOG_BETA_TILDE), k, eps_prev)
    a = prob.a / prob.a.sum()
    b = prob.b / prob.b.sum()
    for _ in range(3):
        st = O.dual_obdrs_step(st, np.log(a), np.log(b), C, 1.0, lam)
        S.step(1)
        err = _potential_err(st, S.get(P.OT_LOG_ALPHA_HAT), S.get(P.OT_LOG_BETA_HAT), st.eps, np.log(b))
        assert err <= TOL_POT[precision], (st.k, err)
        # continue the oracle from the GPU's state: each comparison covers one iteration
        st = O.DualState(S.get(P.OT_LOG_ALPHA), S.get(P.OT_LOG_BETA), S.get(P.OT_LOG_BETA_PREV),
                         S.get(P.OT_LOG_ALPHA_HAT), S.get(P.OT_LOG_BETA_HAT), S.get(P.OT_LOG_BETA_TILDE), st.k,
                         st.eps)
    S.close()


def test_cost_scale_from_device_max(ctx):
    """cost_scale = 0: kappa = 1 / max pair cost (App. G) computed on the device."""
    prob = I.rgb_problem(3000, seed=8, m=2500)
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=0.0, omega=0.0, eps0=0.1)
    kappa, omega = S.cost()
    exact = O.max_pair_cost_hull(prob.x, prob.y)
    assert kappa == pytest.approx(1.0 / exact, rel=1e-6)
    mn = float(O.cost_matrix(prob.x, prob.y, 1.0).min())
    assert omega == pytest.approx(kappa * (exact - mn), rel=1e-6)
    S.close()


def test_invalid_inputs_rejected(ctx):
    prob = I.grid_problem(8, seed=1)
    with pytest.raises(P.OTError) as e:
        ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, lam=2.0)
    assert e.value.status == P.OT_EINVAL
    bad = prob.a.copy()
    bad[3] = 0.0
    with pytest.raises(P.OTError) as e:
        ctx.state(prob.x, prob.y, bad, prob.b, cost_scale=prob.kappa)
    assert e.value.status == P.OT_EINVAL
    # the paper's treatment of zero masses: floor them (App. G)
    S = ctx.state(prob.x, prob.y, bad, prob.b, cost_scale=prob.kappa, zero_mass_floor=1e-15)
    S.step(2)
    S.close()
    with pytest.raises(P.OTError):
        ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, eps0=0.0)


def test_full_size_rgb_sampled_rows(ctx):
    """Colour-transfer size (n = m = 2^20, d = 3): the first row sweep on sampled rows."""
    import torch
    n = 1 << 20
    prob = I.rgb_problem(n, seed=21)
    eta = 0.1
    S = ctx.state(torch.from_numpy(prob.x).cuda(), torch.from_numpy(prob.y).cuda(),
                  torch.from_numpy(prob.a).cuda(), torch.from_numpy(prob.b).cuda(),
                  cost_scale=prob.kappa, omega=1.0, eps0=eta, cert_every=0)
    S.step(1)
    lah = S.get(P.OT_LOG_ALPHA_HAT)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(n, size=24, replace=False))
    lse = O.row_lse_sampled(rows, prob.x, prob.y, np.zeros(n), prob.kappa, eta)
    ref = np.log(prob.a[rows]) - lse
    err = np.abs(eta * (lah[rows] - ref)).max() / np.abs(eta * ref).max()
    assert err <= 1e-5, err
    S.close()


def test_non_default_tile_plan_parity_and_server_lanes(ctx):
    """A state created under another tile plan still matches the oracle one step at a time, and a
    server keeps requests of different plans in different lanes (both correct)."""
    prob = _problem("grid32", 5)
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    a = prob.a / prob.a.sum()
    b = prob.b / prob.b.sum()
    try:
        P.set_tile_plan(2, "mufu", 4, 8)
        S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0,
                      precision="mufu", cert_every=0)
        S.step(3)
        st = O.DualState(S.get(P.OT_LOG_ALPHA), S.get(P.OT_LOG_BETA), S.get(P.OT_LOG_BETA_PREV),
                         S.get(P.OT_LOG_ALPHA_HAT), S.get(P.OT_LOG_BETA_HAT), S.get(P.OT_LOG_BETA_TILDE), 3,
                         O.eps_schedule(1.0, 1.0, 2))
        st1 = O.dual_obdrs_step(st, np.log(a), np.log(b), C, 1.0, 1.0)
        S.step(1)
        err = _potential_err(st1, S.get(P.OT_LOG_ALPHA_HAT), S.get(P.OT_LOG_BETA_HAT), st1.eps, np.log(b))
        assert err <= TOL_POT["mufu"], err
        S.close()
        srv = P.Server(ctx, hbm_budget_bytes=1 << 30, max_slots=8)
        r1 = srv.submit(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, max_iters=100,
                        cert_every=50)
        P.set_tile_plan(2, "mufu", 0, 0)
        r2 = srv.submit(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, max_iters=100,
                        cert_every=50)
        f1, g1, res1 = srv.wait(r1, 60.0)
        f2, g2, res2 = srv.wait(r2, 60.0)
        scale = max(np.abs(f2).max(), np.abs(g2).max())
        assert np.abs(f1 - f2).max() / scale <= 1e-4 and abs(res1["U_best"] - res2["U_best"]) <= 1e-6
        srv.close()
    finally:
        P.set_tile_plan(2, "mufu", 0, 0)
